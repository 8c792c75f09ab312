// orca_common.cuh -- shared device-side definitions of the GB300 ORCA step.
//
// Data layout in HBM (one context, n agents, k neighbours):
//   PV[0], PV[1]: float2 pos[n], float2 vel[n].  PV[0] holds the state between steps in
//                 the current cell order; PV[1] receives the cell-sorted copy each step
//                 (the "messages" of Fig. 2: what neighbours read).
//   PR[0], PR[1]: per-agent parameters float2 goal, float radius, max_speed, pref_speed,
//                 time_horizon and uint32 id (agent index of orca_set_agents).  They are
//                 permuted together with the state; the current copy alternates each step.
//   cell keys and in-cell ranks (uint32), per-cell counts and per-tile counts of the
//   counting sort, the cell table cell_start[num_cells + 1], the grid descriptor and
//   counters.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace orca {

constexpr int kMaxNeighbors = 32;
// per-CTA counters of the ORCA kernel: agents, LP3 agents, candidates, half-planes; then
// (operation-counting launches only) LP1 calls, LP1 bounds, violation checks, bisectors;
// then the neighbour search's extra passes, unpredicted starts, rows scanned, and a spare
constexpr int kBlockCounters = 12;
// static obstacles: segments per context (read through L1; each CTA lists the ones its
// tile can reach) and obstacle half-planes per agent
constexpr int kMaxObstacles = 256;
constexpr int kMaxObstacleNeighbors = 4;
// the cell-table scan: tiles of kCellTile cells, kCellsPerThread per thread
constexpr int kCellScanThreads = 256;
constexpr int kCellsPerThread = 16;
constexpr int kCellTile = kCellScanThreads * kCellsPerThread;
// the tile counts sit one per 128-byte line, so that their atomics spread over the L2
// slices instead of queueing in one
constexpr int kTileSumStride = 32;
constexpr int kBboxBlocks = 304;  // 2 x 152 SMs

// device error bits (latched in DeviceMisc::error)
constexpr int kErrNumeric = 1;
constexpr int kErrTimeout = 2;
constexpr int kErrCapacity = 4;
constexpr int kErrBounds = 8;  // an index check of the ORCA_CHECKS build failed

// Index checks.  A build with -DORCA_CHECKS (build.build(checks=True)) tests the indices
// that the kernels compute from data -- cell-table positions, candidate and neighbour
// slots, agent ids, cell keys -- before using them; a failed check latches kErrBounds in
// the device error word (reported by the next synchronising call as ORCA_ERR_BOUNDS) and
// the access is skipped.  The ordinary build compiles the checks away.
__device__ __forceinline__ bool idx_ok(bool ok, int* err) {
#ifdef ORCA_CHECKS
    if (!ok) {
        if (err) atomicOr(err, kErrBounds);
        return false;
    }
#else
    (void)ok;
    (void)err;
#endif
    return true;
}

constexpr int kBoxCopies = 32;
constexpr int kBoxStride = 32;  // ints: one 128-byte line per copy

// Grid of square cells over the crowd's bounding box, computed on the device each step.
struct GridDev {
    float xmin, ymin;  // exact minima over agents
    float s, inv;      // cell edge and fl32(1/s)
    int gx, gy;        // cells per row / column
    int num_cells;     // gx * gy
    float slop;        // conservative bound on cell-assignment rounding, metres
    int pad[4];
};

struct DeviceMisc {
    GridDev grid;              // single scene: the grid; batch: num_cells of all scenes
    unsigned int bbox_ticket;  // last-block-done counter of the bbox reduction
    int error;                 // kErr* bits
    unsigned int tile_counter; // next tile of the persistent ORCA kernel (reset every step)
    unsigned int obs_tiles;    // tiles listed for the obstacle launch (reset every step)
    unsigned long long counters[4];  // agent-steps, LP3 agent-steps, candidates, lines
    // Single scene: the bounding box of the positions a step's ORCA kernel writes, reduced
    // by that kernel (order-preserving integer codes of min x, min y, max x, max y), in
    // the slot of the next step's parity; bbox_ok[s] says slot s holds the complete box
    // of the current positions (cleared whenever positions change outside a step).  Each
    // slot has kBoxCopies copies, one per 128-byte line, which the kernel's warps share
    // out so that their atomics do not queue on one L2 line.
    int bbox_acc[2][kBoxCopies * kBoxStride];
    unsigned int bbox_ok[2];
};

// Order-preserving integer code of a float (a < b iff code(a) < code(b), NaN aside), for
// min / max reductions with integer atomics.
__device__ __forceinline__ int float_order_code(float f) {
    const int k = __float_as_int(f);
    return k >= 0 ? k : k ^ 0x7fffffff;
}
__device__ __forceinline__ float float_from_order_code(int k) {
    return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff);
}

// One scene of a batch: its slot range (fixed: the sort keeps scenes contiguous), its
// parameters and, recomputed every step, its grid and the offset of its cells in the
// global cell table (composite cell id = cell_off + cy * gx + cx).
struct SceneDev {
    GridDev grid;
    int off, cnt;        // agent slots [off, off + cnt)
    int cell_off;        // first global cell id
    int k;               // neighbours kept (<= the context's max_neighbors)
    float nd, dt;        // r_obs, time step
    float cell_size;     // requested cell edge
    int pad_;
    long long cell_budget;  // cells this scene may use (capacity rule)
    // The box of the positions a step's ORCA kernel writes, reduced by that kernel per
    // scene (order codes of min x, min y, max x, max y) into the slot of the next step's
    // parity; box_ok[s]: slot s holds the complete box of the scene's current positions
    // (zero when positions change outside a step).
    int box_acc[2][4];
    unsigned int box_ok[2];
};

struct AgentParams {  // one of PR[0] / PR[1]
    float2* goal;
    float* radius;
    float* max_speed;
    float* pref_speed;
    float* tau;
    uint32_t* id;
    float* hint;  // last step's k-th neighbour d^2 (NaN: none; +inf: fewer than k), or null
};

struct AgentState {  // one of PV[0] / PV[1]
    float2* pos;
    float2* vel;
};

// Cell-sorted message of one agent (Fig. 2: what neighbours observe): position, radius
// and agent index (as bits) in one 16-byte record; velocity is kept apart because only
// the k selected neighbours need it.
struct Sorted {
    float4* msg;    // (x, y, radius, id bits)
    float2* vel;
    uint32_t* slot;  // slot of each agent id (the inverse of msg[].w)
};

struct BinBuffers {
    uint32_t* keys[2];       // keys[0]: cell key of every slot; keys[1]: scratch
    uint32_t* vals[2];       // vals[0]: rank of every slot in its cell; vals[1]: scratch
    uint32_t* hist;          // scratch between steps (agent removal: tile sums)
    uint32_t* digit_totals;  // scratch between steps (agent removal: the count)
    uint32_t* cnt;           // agents per cell, zero between steps (table_cells entries)
    uint32_t* tile_sums;     // agents per kCellTile cells (stride kTileSumStride), zero between steps
    uint32_t* cell_start;    // table_cells + 1 entries
    long long table_cells;   // largest num_cells the table holds
    float4* bbox_partials;
    DeviceMisc* misc;
};

struct MainArgs {
    int n, k;                            // agents; neighbours (single scene)
    float nd, dt;                        // r_obs, time step (single scene)
    const SceneDev* scenes;              // batch: per-scene parameters and grids, else null
    const int* slot_scene;               // batch: scene of each slot, else null
    int rec_stride;                      // row length of rec_nbr (the context's max k)
    uint32_t* tape;                      // rollouts: per-agent LP record (agent order), or null
    const DeviceMisc* misc;
    DeviceMisc* misc_rw;
    const uint32_t* cell_start;
    Sorted in;                           // sorted messages and velocities (read)
    AgentParams prm;                     // sorted parameters (read)
    AgentState out;                      // new state, same slots
    unsigned long long* block_counters;  // kBlockCounters per block, accumulated
    int count_ops;                       // launch the operation-counting instantiation
    const float4* seg;                   // static obstacle segments (x1, y1, x2, y2), or null
    int nseg, kobst;                     // segments; obstacle half-planes kept per agent
    float tau_o;                         // obstacle time horizon
    int32_t* rec_obst;                   // kMaxObstacleNeighbors per agent (agent order), or null
    int row_stride;                      // float4s per shared-memory row (obstacle launches)
    // With obstacles the tiles some agent of which could reach a segment are flagged and
    // listed (obstacle_tiles_kernel); the plain launch skips them, the obstacle launch
    // steps only them.  Null without obstacles.
    unsigned char* tile_near = nullptr;
    int* obs_tiles = nullptr;
    int32_t* rec_nbr;                    // n*k in agent order, or null
    uint32_t* rec_cell;                  // n in agent order, or null
    int* bbox_acc = nullptr;             // single scene: the next step's box slot (copies), or null
    SceneDev* scene_box = nullptr;       // batch: the scenes whose box slot scene_box_slot is filled
    int scene_box_slot = 0;
    // rollouts (TAPE instantiation only), agent order, each may be null: the state the step
    // starts from and the position it ends at
    float2* rec_pos = nullptr;
    float2* rec_vel = nullptr;
    float2* rec_next = nullptr;
};

// host launchers (orca_bin.cu, orca_main.cu)
int main_blocks(int n);
// bounding box and grid, cell keys and counts, cell table (cnt and tile_sums must be zero
// on entry; they are zero again once the step's reorder has run)
// slot: the step's parity (the box slot it reads; its ORCA kernel fills the other one)
cudaError_t launch_binning(int n, float cell_size, long long max_cells, const AgentState& cur,
                           const BinBuffers& b, int slot, cudaStream_t st);
// Positions changed outside a step: every scene's box slots are cleared (the next batched
// step scans).
cudaError_t launch_clear_scene_boxes(int n_scenes, SceneDev* scenes, cudaStream_t st);
// slot: the parity of the step (its scenes' boxes come from box slot `slot` when the
// previous step's ORCA kernel filled it; slot < 0: always scan).
cudaError_t launch_binning_batch(int n, int n_scenes, SceneDev* scenes, const int* slot_scene,
                                 const AgentState& cur, const BinBuffers& b, int slot, cudaStream_t st);
cudaError_t launch_slot_scene(int n, int n_scenes, const SceneDev* scenes, int* slot_scene,
                              cudaStream_t st);
cudaError_t launch_reorder(int n, const BinBuffers& b, const AgentState& src_s,
                           const Sorted& dst_s, const AgentParams& src_p,
                           const AgentParams& dst_p, cudaStream_t st);
cudaError_t launch_unpermute(int n, const AgentState& s, const uint32_t* id, float2* pos_out,
                             float2* vel_out, cudaStream_t st);
cudaError_t launch_permute(int n, const AgentState& s, const uint32_t* id, const float2* pos_in,
                           const float2* vel_in, cudaStream_t st);
// pos / vel: device-mapped pointers of pinned host arrays (agent order, 16-byte aligned);
// slot_of: the agent -> slot map, built from id first when build_map (then n uint32 of
// scratch), else already valid for the current order
cudaError_t launch_host_state(int n, const AgentState& s, const uint32_t* id, uint32_t* slot_of,
                              bool build_map, float2* pos, float2* vel, bool to_host, cudaStream_t st);
cudaError_t launch_iota(int n, uint32_t* id, cudaStream_t st);
// Launch shape of the ORCA kernel: threads per CTA (64, 128 or 256) and lanes per queued
// agent in the least-penetration phase (1 or 4).
struct LaunchShape {
    int tpb;
    int lp3_group;
};
int default_lp3_group(int kmax);
// kmax: template bound (>= every scene's k); grid_blocks > 0: persistent launch
// A second stream and two events for a step with static obstacles: the obstacle launch
// forks onto `st` after the tile flags and joins the step's stream before it continues.
struct SideStream {
    cudaStream_t st;
    cudaEvent_t fork, join;
};
cudaError_t launch_main(const MainArgs& a, int kmax, const LaunchShape& sh, int grid_blocks,
                        cudaStream_t st,
                        const SideStream* side = nullptr);
int main_resident_blocks(int kmax, const LaunchShape& sh);
// orca_population.cu: spawn candidates into the crowd (see there); device arrays, m each
// (pos and goal float2)
struct SpawnIn {
    const float2* pos;
    const float2* goal;
    const float* radius;
    const float* max_speed;
    const float* pref_speed;
    const float* tau;
};
cudaError_t launch_spawn(int n, const AgentState& cur, const AgentParams& cur_p, int m, const SpawnIn& in,
                         float window, uint32_t* blocked, uint32_t* entrants, uint32_t* rank,
                         int32_t* accepted, uint32_t* count, cudaStream_t st);
// orca_population.cu: remove the agents that have reached their goal (see there)
cudaError_t launch_remove_arrived(int n, const AgentState& cur, const AgentParams& cur_p,
                                  const AgentParams& dst_p, float2* pos_tmp, float2* vel_tmp,
                                  uint32_t* keep, uint32_t* new_id, uint32_t* old_id,
                                  uint32_t* tile_sums, uint32_t* total, cudaStream_t st);

cudaError_t launch_unpermute_params(int n, const AgentParams& src, float2* goal, float* radius,
                                    float* vmax, float* pref, float* tau, cudaStream_t st);

// Cell coordinate along one axis in FP32, one rounding per operation:
// floor(fl(fl(v - vmin) * inv)) clamped to [0, g - 1].
// Programmatic dependent launch (sm_90+): the kernels of a step are launched with the
// programmatic-serialisation attribute, so the launch of the next kernel is prepared while
// the current one runs; each step kernel starts with pdl_wait(), which blocks until the
// preceding kernel of the stream has completed and its writes are visible (a no-op without
// such a dependency).  No kernel releases its dependents early: measured on the
// 524,288-agent flow, dependents made resident before their predecessor finished slowed
// the step (0.2111 ms) against the release at completion (0.2072 ms; 0.2086 without the
// attribute).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch with the programmatic-stream-serialisation attribute (see pdl_wait).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

__device__ __forceinline__ int cell_coord(float v, float vmin, float inv, int g) {
    float q = __fmul_rn(__fsub_rn(v, vmin), inv);
    int c = __float2int_rd(q);
    c = c < 0 ? 0 : c;
    return c > g - 1 ? g - 1 : c;
}

}  // namespace orca
