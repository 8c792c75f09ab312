// orca_api.cu -- the C ABI (include/orca_gb300.h): context, workspace layout, step
// orchestration and CUDA-graph capture.  No C++ exception crosses the ABI.
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "../../include/orca_gb300.h"
#include "orca_adjoint.cuh"
#include "orca_common.cuh"

namespace orca {

// An NVTX range over one entry point that enqueues GPU work, so that a profiler's timeline
// shows which library call launched what (header-only NVTX: a no-op without a tool).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Sub-allocation plan of the workspace (256-byte aligned pieces).
struct Layout {
    size_t off[32];
    int count = 0;
    size_t total = 0;
    size_t add(size_t bytes) {
        size_t o = total;
        off[count++] = o;
        total += (bytes + 255) & ~size_t(255);
        return o;
    }
};

struct Plan {
    int N, K, S, max_cells, nmb;
    long long table_cells;  // largest grid (cells over all scenes) the cell table holds
    size_t o_msg, o_sslot, o_pv[2][2], o_goal[2], o_rad[2], o_vmax[2], o_pref[2], o_tau[2], o_id[2], o_hint[2];
    size_t o_keys[2], o_vals[2], o_hist, o_tot, o_cells, o_cnt, o_tsum, o_scenes, o_slot, o_part, o_misc, o_blk, o_rnbr, o_rcell, o_robst, o_seg, o_near, o_otiles,
        o_stage[2];
    size_t total;
};

static int default_max_cells(int N) {
    long long c = 4LL * N;
    if (c < 65536) c = 65536;
    if (c > (1LL << 30)) c = 1LL << 30;
    return (int)c;
}

static bool make_plan(const orca_params& p, Plan& pl) {
    if (p.max_agents < 1 || p.max_neighbors < 1 || p.max_neighbors > kMaxNeighbors) return false;
    if (!(p.neighbor_dist > 0.0f) || !(p.dt > 0.0f) || p.cell_size < 0.0f) return false;
    if (p.max_cells < 0 || p.max_scenes < 0) return false;
    pl.N = p.max_agents;
    pl.K = p.max_neighbors;
    pl.S = p.max_scenes > 1 ? p.max_scenes : 1;
    pl.max_cells = p.max_cells ? p.max_cells : default_max_cells(p.max_agents);
    // a batch gives every scene at least one cell beyond its proportional share
    pl.table_cells = (long long)pl.max_cells + pl.S;
    pl.nmb = main_blocks(pl.N);
    Layout L;
    size_t N = (size_t)pl.N;
    pl.o_msg = L.add(N * sizeof(float4));
    pl.o_sslot = L.add(N * 4);
    for (int b = 0; b < 2; ++b) {
        pl.o_pv[b][0] = L.add(N * sizeof(float2));
        pl.o_pv[b][1] = L.add(N * sizeof(float2));
        pl.o_goal[b] = L.add(N * sizeof(float2));
        pl.o_rad[b] = L.add(N * 4);
        pl.o_vmax[b] = L.add(N * 4);
        pl.o_pref[b] = L.add(N * 4);
        pl.o_tau[b] = L.add(N * 4);
        pl.o_id[b] = L.add(N * 4);
        pl.o_hint[b] = L.add(N * 4);
        pl.o_keys[b] = L.add(N * 4);
        pl.o_vals[b] = L.add(N * 4);
        pl.o_stage[b] = L.add(N * sizeof(float2));
    }
    pl.o_hist = L.add((N / 2048 + 1) * 4);  // removal: tile sums of 2048 agents
    pl.o_tot = L.add(4);
    pl.o_cells = L.add(((size_t)pl.table_cells + 1) * 4);
    pl.o_cnt = L.add((size_t)pl.table_cells * 4);
    pl.o_tsum = L.add(((size_t)pl.table_cells / kCellTile + 1) * kTileSumStride * 4);
    pl.o_scenes = L.add((size_t)pl.S * sizeof(SceneDev));
    pl.o_slot = p.max_scenes > 1 ? L.add(N * 4) : (size_t)-1;
    pl.o_part = L.add(kBboxBlocks * sizeof(float4));
    pl.o_misc = L.add(sizeof(DeviceMisc));
    pl.o_blk = L.add((size_t)pl.nmb * kBlockCounters * sizeof(unsigned long long));
    pl.o_seg = L.add((size_t)kMaxObstacles * sizeof(float4));
    pl.o_near = L.add((size_t)pl.nmb);       // a flag per tile (obstacle steps)
    pl.o_otiles = L.add((size_t)pl.nmb * 4);  // the flagged tiles
    if (p.flags & ORCA_FLAG_RECORD) {
        pl.o_rnbr = L.add(N * pl.K * 4);
        pl.o_rcell = L.add(N * 4);
        pl.o_robst = L.add(N * kMaxObstacleNeighbors * 4);
    } else {
        pl.o_rnbr = pl.o_rcell = pl.o_robst = (size_t)-1;
    }
    pl.total = L.total;
    return true;
}

}  // namespace orca

using namespace orca;

struct orca_ctx {
    orca_params p;
    Plan plan;
    int device = 0;
    char* ws = nullptr;
    bool own_ws = false;
    AgentState PV[2];  // PV[0]: state between steps; PV[1].vel: sorted velocities
    Sorted sorted;     // sorted messages (+ PV[1].vel)
    AgentParams PR[2];
    BinBuffers bins;
    unsigned long long* blk = nullptr;
    int32_t* rec_nbr = nullptr;
    uint32_t* rec_cell = nullptr;
    int32_t* rec_obst = nullptr;
    unsigned char* tile_near = nullptr;  // obstacle steps: tiles near a segment, and their list
    int* obs_tiles = nullptr;
    SideStream side{nullptr, nullptr, nullptr};  // created with the first obstacles
    float4* seg = nullptr;  // static obstacle segments
    int nseg = 0, kobst = 0;
    float tau_o = 1.0f;
    float2* stage[2];
    int n = 0;
    int cur = 0;  // which PR buffer holds the current parameters
    bool stepped = false;
    bool slot_ok = false;  // sorted.slot maps every agent to its slot in the current order
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    int graph_n = -1;
    bool prof = false;
    bool count_ops = false;  // steps launch the operation-counting ORCA kernel
    int n_scenes = 0;  // 0: single scene (orca_set_agents); else a batch
    SceneDev* scenes = nullptr;
    int* slot_scene = nullptr;
    int resident = 0;  // CTAs of the ORCA kernel resident at once (persistent launch)
    LaunchShape shape{128, 1};
    bool shape_auto = true;  // no orca_set_launch yet: small crowds take the agent split
    int roll_T = 0, roll_C = 0;  // last orca_rollout_forward
    void* roll_ws = nullptr;
    cudaEvent_t pev[4] = {nullptr, nullptr, nullptr, nullptr};
    std::string err;
};

// Message of the last failure of an entry point without a context, per host thread: two
// threads failing at once each keep their own message.
static thread_local std::string g_create_err;

static int fail(orca_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    else g_create_err = msg;
    return code;
}

namespace orca {
// Message for orca_last_error(NULL), for entry points that have no context.
void set_context_free_error(const std::string& msg) { g_create_err = msg; }
}  // namespace orca

static int cuda_fail(orca_ctx* c, cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(c, ORCA_ERR_CUDA, m);
}

#define CK(call, what)                                    \
    do {                                                  \
        cudaError_t e_ = (call);                          \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
    } while (0)

static void bind_buffers(orca_ctx* c) {
    const Plan& pl = c->plan;
    char* w = c->ws;
    for (int b = 0; b < 2; ++b) {
        c->PV[b].pos = (float2*)(w + pl.o_pv[b][0]);
        c->PV[b].vel = (float2*)(w + pl.o_pv[b][1]);
        c->PR[b].goal = (float2*)(w + pl.o_goal[b]);
        c->PR[b].radius = (float*)(w + pl.o_rad[b]);
        c->PR[b].max_speed = (float*)(w + pl.o_vmax[b]);
        c->PR[b].pref_speed = (float*)(w + pl.o_pref[b]);
        c->PR[b].tau = (float*)(w + pl.o_tau[b]);
        c->PR[b].id = (uint32_t*)(w + pl.o_id[b]);
        c->PR[b].hint = (float*)(w + pl.o_hint[b]);
        c->bins.keys[b] = (uint32_t*)(w + pl.o_keys[b]);
        c->bins.vals[b] = (uint32_t*)(w + pl.o_vals[b]);
        c->stage[b] = (float2*)(w + pl.o_stage[b]);
    }
    c->sorted.msg = (float4*)(w + pl.o_msg);
    c->sorted.slot = (uint32_t*)(w + pl.o_sslot);
    c->sorted.vel = c->PV[1].vel;
    c->bins.hist = (uint32_t*)(w + pl.o_hist);
    c->bins.digit_totals = (uint32_t*)(w + pl.o_tot);
    c->bins.cell_start = (uint32_t*)(w + pl.o_cells);
    c->bins.cnt = (uint32_t*)(w + pl.o_cnt);
    c->bins.tile_sums = (uint32_t*)(w + pl.o_tsum);
    c->bins.table_cells = pl.table_cells;
    c->bins.bbox_partials = (float4*)(w + pl.o_part);
    c->bins.misc = (DeviceMisc*)(w + pl.o_misc);
    c->blk = (unsigned long long*)(w + pl.o_blk);
    c->scenes = (SceneDev*)(w + pl.o_scenes);
    c->slot_scene = pl.o_slot == (size_t)-1 ? nullptr : (int*)(w + pl.o_slot);
    c->rec_nbr = pl.o_rnbr == (size_t)-1 ? nullptr : (int32_t*)(w + pl.o_rnbr);
    c->rec_cell = pl.o_rcell == (size_t)-1 ? nullptr : (uint32_t*)(w + pl.o_rcell);
    c->rec_obst = pl.o_robst == (size_t)-1 ? nullptr : (int32_t*)(w + pl.o_robst);
    c->seg = (float4*)(w + pl.o_seg);
    c->tile_near = (unsigned char*)(w + pl.o_near);
    c->obs_tiles = (int*)(w + pl.o_otiles);
}

static void drop_graphs(orca_ctx* c) {
    for (int b = 0; b < 2; ++b)
        if (c->exec[b]) {
            cudaGraphExecDestroy(c->exec[b]);
            c->exec[b] = nullptr;
        }
    c->graph_n = -1;
}

// Launch shape of a step: the context's, except that without an orca_set_launch a single
// scene of at most kSplitMaxAgents agents with k <= 16 takes the agent split (four lanes
// per agent; 2-12% faster there, slower above about 20,000 agents).
constexpr int kSplitMaxAgents = 12000;
static LaunchShape step_shape(const orca_ctx* c) {
    if (c->shape_auto && c->n_scenes == 0 && c->nseg == 0 && c->n <= kSplitMaxAgents && c->plan.K <= 16)
        return LaunchShape{64, 4};
    return c->shape;
}

// Enqueue one step whose current parameters live in PR[par].
static cudaError_t enqueue_step(orca_ctx* c, int par, cudaStream_t st) {
    const Plan& pl = c->plan;
    float cs = c->p.cell_size > 0.0f ? c->p.cell_size : c->p.neighbor_dist * 0.25f;
    cudaError_t e = cudaSuccess;
    if (c->prof && (e = cudaEventRecordWithFlags(c->pev[0], st, cudaEventRecordExternal)) != cudaSuccess) return e;
    if (c->n_scenes > 0)
        e = launch_binning_batch(c->n, c->n_scenes, c->scenes, c->slot_scene, c->PV[0], c->bins, par, st);
    else
        e = launch_binning(c->n, cs, pl.max_cells, c->PV[0], c->bins, par, st);
    if (e != cudaSuccess) return e;
    if (c->prof && (e = cudaEventRecordWithFlags(c->pev[1], st, cudaEventRecordExternal)) != cudaSuccess) return e;
    e = launch_reorder(c->n, c->bins, c->PV[0], c->sorted, c->PR[par], c->PR[par ^ 1], st);
    if (e != cudaSuccess) return e;
    if (c->prof && (e = cudaEventRecordWithFlags(c->pev[2], st, cudaEventRecordExternal)) != cudaSuccess) return e;
    MainArgs a{};
    a.n = c->n;
    a.k = pl.K;
    a.nd = c->p.neighbor_dist;
    a.dt = c->p.dt;
    a.misc = c->bins.misc;
    a.misc_rw = c->bins.misc;
    a.cell_start = c->bins.cell_start;
    a.in = c->sorted;
    a.prm = c->PR[par ^ 1];
    a.out = c->PV[0];
    a.block_counters = c->blk;
    a.count_ops = c->count_ops ? 1 : 0;
    a.seg = c->seg;
    a.nseg = c->n_scenes > 0 ? 0 : c->nseg;
    a.kobst = c->kobst;
    a.tau_o = c->tau_o;
    a.rec_obst = c->rec_obst;
    if (a.nseg > 0) {
        a.tile_near = c->tile_near;
        a.obs_tiles = c->obs_tiles;
    }
    a.rec_nbr = c->rec_nbr;
    a.rec_cell = c->rec_cell;
    a.scenes = c->n_scenes > 0 ? c->scenes : nullptr;
    a.slot_scene = c->n_scenes > 0 ? c->slot_scene : nullptr;
    a.rec_stride = pl.K;
    a.tape = nullptr;
    if (c->n_scenes == 0) a.bbox_acc = c->bins.misc->bbox_acc[par ^ 1];
    else {
        a.scene_box = c->scenes;
        a.scene_box_slot = par ^ 1;
    }
    e = launch_main(a, pl.K, step_shape(c), c->n_scenes > 0 ? c->resident : 0, st,
                    a.nseg > 0 && c->side.st ? &c->side : nullptr);
    if (e != cudaSuccess) return e;
    if (c->prof) e = cudaEventRecordWithFlags(c->pev[3], st, cudaEventRecordExternal);
    return e;
}

// kernels per step: bounding box (a batch: the scenes' boxes and cell ranges), keys +
// counts, cell table, reorder, ORCA kernel (with obstacles: tile flags, the plain ORCA
// launch and the obstacle launch)
static int launches_per_step(const orca_ctx* c) {
    const int obstacles = c->n_scenes == 0 && c->nseg > 0 ? 2 : 0;  // tile flags, obstacle launch
    return 5 + obstacles;
}

// One step launched directly with the neighbour lists and LP records written in agent
// order, and (each may be null) the state it starts from and the positions it ends at.
static cudaError_t enqueue_recording_step(orca_ctx* c, int par, int32_t* nbr, uint32_t* tape,
                                          float2* state, float2* next, cudaStream_t st) {
    const Plan& pl = c->plan;
    float cs = c->p.cell_size > 0.0f ? c->p.cell_size : c->p.neighbor_dist * 0.25f;
    cudaError_t e = launch_binning(c->n, cs, pl.max_cells, c->PV[0], c->bins, par, st);
    if (e != cudaSuccess) return e;
    e = launch_reorder(c->n, c->bins, c->PV[0], c->sorted, c->PR[par], c->PR[par ^ 1], st);
    if (e != cudaSuccess) return e;
    MainArgs a{};
    a.n = c->n;
    a.k = pl.K;
    a.nd = c->p.neighbor_dist;
    a.dt = c->p.dt;
    a.misc = c->bins.misc;
    a.misc_rw = c->bins.misc;
    a.cell_start = c->bins.cell_start;
    a.in = c->sorted;
    a.prm = c->PR[par ^ 1];
    a.out = c->PV[0];
    a.block_counters = c->blk;
    a.count_ops = 0;
    a.seg = nullptr;
    a.nseg = 0;
    a.kobst = 0;
    a.tau_o = 1.0f;
    a.rec_obst = nullptr;
    a.rec_nbr = nbr;
    a.rec_cell = nullptr;
    a.scenes = nullptr;
    a.slot_scene = nullptr;
    a.rec_stride = pl.K;
    a.tape = tape;
    a.bbox_acc = c->bins.misc->bbox_acc[par ^ 1];
    a.rec_pos = state;
    a.rec_vel = state ? state + c->n : nullptr;
    a.rec_next = next;
    return launch_main(a, pl.K, c->shape, 0, st);
}

// Capture the two step graphs (one per parity).  When instantiated graphs exist and only
// the number of agents changed since (removal, spawning: the calls that change n without
// dropping the graphs), the new captures update them in place, which costs a fraction of
// a fresh instantiation; a capture whose shape the update does not take is instantiated.
static int build_graphs(orca_ctx* ctx) {
    const bool update = ctx->exec[0] && ctx->exec[1];
    if (!update) drop_graphs(ctx);
    for (int par = 0; par < 2; ++par) {
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(ctx->cap, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
        cudaError_t e = enqueue_step(ctx, par, ctx->cap);
        cudaError_t e2 = cudaStreamEndCapture(ctx->cap, &g);
        if (e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            drop_graphs(ctx);
            return cuda_fail(ctx, e, "kernel launch during capture");
        }
        if (e2 != cudaSuccess) {
            drop_graphs(ctx);
            return cuda_fail(ctx, e2, "cudaStreamEndCapture");
        }
        if (update && ctx->exec[par]) {
            cudaGraphExecUpdateResultInfo info;
            if (cudaGraphExecUpdate(ctx->exec[par], g, &info) == cudaSuccess) {
                cudaGraphDestroy(g);
                continue;
            }
            cudaGetLastError();  // not updatable: instantiate instead
            cudaGraphExecDestroy(ctx->exec[par]);
            ctx->exec[par] = nullptr;
        }
        e = cudaGraphInstantiate(&ctx->exec[par], g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            drop_graphs(ctx);
            return cuda_fail(ctx, e, "cudaGraphInstantiate");
        }
    }
    ctx->graph_n = ctx->n;
    return ORCA_OK;
}

// The device-side address of a pinned (page-locked, mapped) host array of `bytes` bytes
// that starts on a 16-byte boundary, or null for other memory.  Kernels read and write
// such arrays directly over the CPU-GPU link, so its last byte must be pinned too and
// mapped contiguously with the first (one registration); otherwise the caller falls back
// to the staging copy.
static void* mapped_host_ptr(const void* p, size_t bytes) {
    if (!p || bytes == 0) return nullptr;
    cudaPointerAttributes at, end;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();  // clear the (non-sticky) error of an unknown pointer
        return nullptr;
    }
    if (at.type != cudaMemoryTypeHost || ((uintptr_t)at.devicePointer & 15)) return nullptr;
    const char* last = (const char*)p + (bytes - 1);
    if (cudaPointerGetAttributes(&end, last) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (end.type != cudaMemoryTypeHost ||
        (const char*)end.devicePointer != (const char*)at.devicePointer + (bytes - 1))
        return nullptr;
    return at.devicePointer;
}

// The agent -> slot map for pinned transfers: the one the last step's reorder wrote, or
// scratch to build it in (slot_ok false).
static uint32_t* slot_map(orca_ctx* ctx) {
    return ctx->slot_ok ? ctx->sorted.slot : (uint32_t*)ctx->stage[0];
}

static int check_device_error(orca_ctx* ctx, cudaStream_t st) {
    int herr = 0;
    CK(cudaMemcpyAsync(&herr, &ctx->bins.misc->error, sizeof(int), cudaMemcpyDeviceToHost, st),
       "cudaMemcpyAsync(error word)");
    CK(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    if (herr & kErrNumeric) return fail(ctx, ORCA_ERR_NUMERIC, "non-finite velocity or position produced");
    if (herr & kErrTimeout) return fail(ctx, ORCA_ERR_TIMEOUT, "a bounded device-side wait gave up");
    if (herr & kErrCapacity)
        return fail(ctx, ORCA_ERR_CAPACITY, "crowd extent does not fit the cell table (non-finite positions?)");
    if (herr & kErrBounds)
        return fail(ctx, ORCA_ERR_BOUNDS, "a device-side index check failed (ORCA_CHECKS build)");
    return ORCA_OK;
}

// Positions changed outside a step: the box the last step's ORCA kernel reduced no longer
// holds, so the next step's bounding-box kernel scans.
static cudaError_t clear_box(orca_ctx* ctx, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(ctx->bins.misc->bbox_ok, 0, sizeof ctx->bins.misc->bbox_ok, st);
    if (e == cudaSuccess && ctx->n_scenes > 0) e = launch_clear_scene_boxes(ctx->n_scenes, ctx->scenes, st);
    return e;
}

// Enqueue the write of agent-order positions / velocities (either may be null) into the
// current slots, on st, without synchronising.  Pinned host arrays are read by one kernel
// over the CPU-GPU link; other host arrays go through the staging buffers.
static int enqueue_write_state(orca_ctx* ctx, const float* pos_xy, const float* vel_xy, int where,
                               cudaStream_t st) {
    const size_t N = (size_t)ctx->n;
    // new positions: the next step scans for its bounding box
    if (pos_xy) CK(clear_box(ctx, st), "clear box flags");
    const float2* pin = (const float2*)pos_xy;
    const float2* vin = (const float2*)vel_xy;
    if (where == ORCA_HOST) {
        void* mp = mapped_host_ptr(pos_xy, N * 8);
        void* mv = mapped_host_ptr(vel_xy, N * 8);
        if ((mp || !pos_xy) && (mv || !vel_xy)) {
            CK(launch_host_state(ctx->n, ctx->PV[0], ctx->PR[ctx->cur].id, slot_map(ctx), !ctx->slot_ok,
                                 (float2*)mp, (float2*)mv, false, st),
               "host state kernel");
            return ORCA_OK;
        }
        if (pos_xy) CK(cudaMemcpyAsync(ctx->stage[0], pos_xy, N * 8, cudaMemcpyHostToDevice, st), "copy pos");
        if (vel_xy) CK(cudaMemcpyAsync(ctx->stage[1], vel_xy, N * 8, cudaMemcpyHostToDevice, st), "copy vel");
        pin = pos_xy ? ctx->stage[0] : nullptr;
        vin = vel_xy ? ctx->stage[1] : nullptr;
    }
    CK(launch_permute(ctx->n, ctx->PV[0], ctx->PR[ctx->cur].id, pin, vin, st), "permute kernel");
    return ORCA_OK;
}

// Enqueue the read of the state in agent order (either output may be null) on st, without
// synchronising.  Pinned host arrays are written by one kernel over the CPU-GPU link.
static int enqueue_read_state(orca_ctx* ctx, float* pos_xy, float* vel_xy, int where, cudaStream_t st) {
    const size_t N = (size_t)ctx->n;
    void* mp = where == ORCA_HOST ? mapped_host_ptr(pos_xy, N * 8) : nullptr;
    void* mv = where == ORCA_HOST ? mapped_host_ptr(vel_xy, N * 8) : nullptr;
    if (where == ORCA_DEVICE) {
        CK(launch_unpermute(ctx->n, ctx->PV[0], ctx->PR[ctx->cur].id, (float2*)pos_xy, (float2*)vel_xy, st),
           "unpermute kernel");
    } else if ((mp || !pos_xy) && (mv || !vel_xy)) {
        CK(launch_host_state(ctx->n, ctx->PV[0], ctx->PR[ctx->cur].id, slot_map(ctx), !ctx->slot_ok,
                             (float2*)mp, (float2*)mv, true, st),
           "host state kernel");
    } else {
        CK(launch_unpermute(ctx->n, ctx->PV[0], ctx->PR[ctx->cur].id, ctx->stage[0], ctx->stage[1], st),
           "unpermute kernel");
        if (pos_xy) CK(cudaMemcpyAsync(pos_xy, ctx->stage[0], N * 8, cudaMemcpyDeviceToHost, st), "copy pos");
        if (vel_xy) CK(cudaMemcpyAsync(vel_xy, ctx->stage[1], N * 8, cudaMemcpyDeviceToHost, st), "copy vel");
    }
    return ORCA_OK;
}

extern "C" {

ORCA_API int orca_workspace_size(const orca_params* params, size_t* bytes) {
    if (!params || !bytes) return fail(nullptr, ORCA_ERR_ARG, "null argument");
    Plan pl;
    if (!make_plan(*params, pl)) return fail(nullptr, ORCA_ERR_ARG, "invalid orca_params");
    *bytes = pl.total;
    return ORCA_OK;
}

ORCA_API int orca_create(const orca_params* params, void* workspace, size_t workspace_bytes,
                         orca_ctx** out) {
    if (!out) return fail(nullptr, ORCA_ERR_ARG, "null out");
    *out = nullptr;
    if (!params) return fail(nullptr, ORCA_ERR_ARG, "null params");
    Plan pl;
    if (!make_plan(*params, pl)) return fail(nullptr, ORCA_ERR_ARG, "invalid orca_params");
    if (workspace && ((uintptr_t)workspace & 255))
        return fail(nullptr, ORCA_ERR_ARG, "workspace must be 256-byte aligned");
    if (workspace && workspace_bytes < pl.total)
        return fail(nullptr, ORCA_ERR_NOMEM, "workspace smaller than orca_workspace_size()");
    orca_ctx* ctx = new (std::nothrow) orca_ctx();
    if (!ctx) return fail(nullptr, ORCA_ERR_NOMEM, "host allocation failed");
    ctx->p = *params;
    ctx->plan = pl;
    ctx->shape.lp3_group = default_lp3_group(pl.K);
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess && workspace) {
        ctx->ws = (char*)workspace;
    } else if (e == cudaSuccess) {
        e = cudaMalloc((void**)&ctx->ws, pl.total);
        if (e != cudaSuccess) {
            delete ctx;
            return fail(nullptr, ORCA_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        ctx->own_ws = true;
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        bind_buffers(ctx);
        e = cudaMemset(ctx->bins.misc, 0, sizeof(DeviceMisc));
        // the counting sort's cell and tile counts are zero between steps
        if (e == cudaSuccess) e = cudaMemset(ctx->bins.cnt, 0, (size_t)pl.table_cells * 4);
        if (e == cudaSuccess)
            e = cudaMemset(ctx->bins.tile_sums, 0,
                           ((size_t)pl.table_cells / kCellTile + 1) * kTileSumStride * 4);
    }
    if (e != cudaSuccess) {
        std::string m = std::string("context set-up: ") + cudaGetErrorString(e);
        if (ctx->own_ws) cudaFree(ctx->ws);
        if (ctx->cap) cudaStreamDestroy(ctx->cap);
        delete ctx;
        return fail(nullptr, ORCA_ERR_CUDA, m);
    }
    *out = ctx;
    return ORCA_OK;
}

ORCA_API int orca_destroy(orca_ctx* ctx) {
    if (!ctx) return ORCA_ERR_ARG;
    cudaDeviceSynchronize();
    drop_graphs(ctx);
    for (int q = 0; q < 4; ++q)
        if (ctx->pev[q]) cudaEventDestroy(ctx->pev[q]);
    if (ctx->cap) cudaStreamDestroy(ctx->cap);
    if (ctx->side.st) cudaStreamDestroy(ctx->side.st);
    if (ctx->side.fork) cudaEventDestroy(ctx->side.fork);
    if (ctx->side.join) cudaEventDestroy(ctx->side.join);
    if (ctx->own_ws) cudaFree(ctx->ws);
    delete ctx;
    return ORCA_OK;
}

ORCA_API int orca_profile(orca_ctx* ctx, int enable) {
    if (!ctx) return ORCA_ERR_ARG;
    bool on = enable != 0;
    if (on && !ctx->pev[0])
        for (int q = 0; q < 4; ++q) CK(cudaEventCreate(&ctx->pev[q]), "cudaEventCreate");
    if (on != ctx->prof) drop_graphs(ctx);
    ctx->prof = on;
    return ORCA_OK;
}

ORCA_API int orca_profile_read(orca_ctx* ctx, float* ms3) {
    if (!ctx || !ms3) return ORCA_ERR_ARG;
    if (!ctx->prof || !ctx->stepped) return fail(ctx, ORCA_ERR_STATE, "no profiled step yet");
    CK(cudaEventSynchronize(ctx->pev[3]), "cudaEventSynchronize");
    for (int q = 0; q < 3; ++q) CK(cudaEventElapsedTime(&ms3[q], ctx->pev[q], ctx->pev[q + 1]), "cudaEventElapsedTime");
    return ORCA_OK;
}

ORCA_API int orca_set_cell_size(orca_ctx* ctx, float cell_size) {
    if (!ctx) return ORCA_ERR_ARG;
    if (!(cell_size >= 0.0f) || !isfinite(cell_size)) return fail(ctx, ORCA_ERR_ARG, "cell_size must be >= 0");
    if (cell_size != ctx->p.cell_size) {
        ctx->p.cell_size = cell_size;
        drop_graphs(ctx);
    }
    return ORCA_OK;
}

ORCA_API int orca_set_launch(orca_ctx* ctx, int32_t threads_per_block, int32_t lp3_lanes) {
    if (!ctx) return ORCA_ERR_ARG;
    if (threads_per_block != 64 && threads_per_block != 128 && threads_per_block != 256)
        return fail(ctx, ORCA_ERR_ARG, "threads_per_block must be 64, 128 or 256");
    if (lp3_lanes != 0 && lp3_lanes != 1 && lp3_lanes != 4 && lp3_lanes != 32)
        return fail(ctx, ORCA_ERR_ARG, "lp3_lanes must be 0 (default), 1, 4 or 32");
    LaunchShape sh{threads_per_block, lp3_lanes ? lp3_lanes : default_lp3_group(ctx->plan.K)};
    if (ctx->shape_auto || sh.tpb != ctx->shape.tpb || sh.lp3_group != ctx->shape.lp3_group) {
        ctx->shape_auto = false;
        ctx->shape = sh;
        ctx->resident = 0;
        if (ctx->n_scenes > 0) ctx->resident = main_resident_blocks(ctx->plan.K, ctx->shape);
        drop_graphs(ctx);
    }
    return ORCA_OK;
}

ORCA_API int orca_launches_per_step(const orca_ctx* ctx, int32_t* count) {
    if (!ctx || !count) return ORCA_ERR_ARG;
    *count = launches_per_step(ctx);
    return ORCA_OK;
}

ORCA_API int orca_set_agents(orca_ctx* ctx, int32_t n, const float* pos_xy, const float* vel_xy,
                             const float* goal_xy, const float* radius, const float* max_speed,
                             const float* pref_speed, const float* time_horizon, int where,
                             void* stream) {
    NvtxRange nvtx_range("orca_set_agents");
    if (!ctx) return ORCA_ERR_ARG;
    if (n < 0) return fail(ctx, ORCA_ERR_ARG, "n < 0");
    if (n > ctx->plan.N) return fail(ctx, ORCA_ERR_CAPACITY, "n exceeds max_agents");
    if (where != ORCA_HOST && where != ORCA_DEVICE) return fail(ctx, ORCA_ERR_ARG, "bad `where`");
    if (n > 0 && (!pos_xy || !vel_xy || !goal_xy || !radius || !max_speed || !pref_speed || !time_horizon))
        return fail(ctx, ORCA_ERR_ARG, "null array");
    cudaStream_t st = (cudaStream_t)stream;
    cudaMemcpyKind kind = where == ORCA_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    size_t N = (size_t)n;
    if (n > 0) {
        CK(cudaMemcpyAsync(ctx->PV[0].pos, pos_xy, N * 8, kind, st), "copy pos");
        CK(cudaMemcpyAsync(ctx->PV[0].vel, vel_xy, N * 8, kind, st), "copy vel");
        CK(cudaMemcpyAsync(ctx->PR[0].goal, goal_xy, N * 8, kind, st), "copy goal");
        CK(cudaMemcpyAsync(ctx->PR[0].radius, radius, N * 4, kind, st), "copy radius");
        CK(cudaMemcpyAsync(ctx->PR[0].max_speed, max_speed, N * 4, kind, st), "copy max_speed");
        CK(cudaMemcpyAsync(ctx->PR[0].pref_speed, pref_speed, N * 4, kind, st), "copy pref_speed");
        CK(cudaMemcpyAsync(ctx->PR[0].tau, time_horizon, N * 4, kind, st), "copy time_horizon");
        CK(launch_iota(n, ctx->PR[0].id, st), "iota kernel");
        // no neighbour-radius hint yet (NaN bits); it only steers the search's pruning
        CK(cudaMemsetAsync(ctx->PR[0].hint, 0xff, N * 4, st), "reset hint");
    }
    CK(cudaMemsetAsync(ctx->bins.misc, 0, sizeof(DeviceMisc), st), "reset misc");
    CK(cudaMemsetAsync(ctx->blk, 0, (size_t)ctx->plan.nmb * kBlockCounters * sizeof(unsigned long long), st),
       "reset counters");
    if (ctx->rec_nbr && n > 0) CK(cudaMemsetAsync(ctx->rec_nbr, 0xff, N * ctx->plan.K * 4, st), "reset record");
    if (ctx->rec_cell && n > 0) CK(cudaMemsetAsync(ctx->rec_cell, 0, N * 4, st), "reset record");
    if (where == ORCA_HOST) CK(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    ctx->n = n;
    ctx->cur = 0;
    ctx->stepped = false;
    ctx->slot_ok = false;
    if (ctx->n_scenes != 0) {
        ctx->n_scenes = 0;
        drop_graphs(ctx);
    }
    return ORCA_OK;
}

ORCA_API int orca_update_state(orca_ctx* ctx, const float* pos_xy, const float* vel_xy, int where,
                               void* stream) {
    NvtxRange nvtx_range("orca_update_state");
    if (!ctx) return ORCA_ERR_ARG;
    if (where != ORCA_HOST && where != ORCA_DEVICE) return fail(ctx, ORCA_ERR_ARG, "bad `where`");
    if (ctx->n == 0 || (!pos_xy && !vel_xy)) return ORCA_OK;
    cudaStream_t st = (cudaStream_t)stream;
    int r = enqueue_write_state(ctx, pos_xy, vel_xy, where, st);
    if (r != ORCA_OK) return r;
    if (where == ORCA_HOST) CK(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    return ORCA_OK;
}

ORCA_API int orca_set_scenes(orca_ctx* ctx, int32_t n_scenes, const orca_scene* scenes,
                             const float* pos_xy, const float* vel_xy, const float* goal_xy,
                             const float* radius, const float* max_speed, const float* pref_speed,
                             const float* time_horizon, int where, void* stream) {
    NvtxRange nvtx_range("orca_set_scenes");
    if (!ctx) return ORCA_ERR_ARG;
    if (ctx->nseg > 0) return fail(ctx, ORCA_ERR_STATE, "clear the static obstacles before a batch");
    if (!ctx->slot_scene) return fail(ctx, ORCA_ERR_STATE, "context created with max_scenes <= 1");
    if (n_scenes < 1 || !scenes) return fail(ctx, ORCA_ERR_ARG, "need at least one scene");
    if (n_scenes > ctx->plan.S) return fail(ctx, ORCA_ERR_CAPACITY, "n_scenes exceeds max_scenes");
    long long total = 0;
    for (int q = 0; q < n_scenes; ++q) {
        const orca_scene& sc = scenes[q];
        if (sc.count < 0 || sc.max_neighbors < 1 || sc.max_neighbors > ctx->plan.K ||
            !(sc.neighbor_dist > 0.0f) || !(sc.dt > 0.0f) || !(sc.cell_size >= 0.0f))
            return fail(ctx, ORCA_ERR_ARG, "invalid orca_scene " + std::to_string(q));
        total += sc.count;
    }
    if (total > ctx->plan.N) return fail(ctx, ORCA_ERR_CAPACITY, "agents exceed max_agents");
    int n = (int)total;
    int r = orca_set_agents(ctx, n, pos_xy, vel_xy, goal_xy, radius, max_speed, pref_speed,
                            time_horizon, where, stream);
    if (r != ORCA_OK) return r;
    SceneDev* h = new (std::nothrow) SceneDev[n_scenes];
    if (!h) return fail(ctx, ORCA_ERR_NOMEM, "host allocation failed");
    long long off = 0;
    for (int q = 0; q < n_scenes; ++q) {
        SceneDev d;
        memset(&d, 0, sizeof d);
        d.off = (int)off;
        d.cnt = scenes[q].count;
        d.k = scenes[q].max_neighbors;
        d.nd = scenes[q].neighbor_dist;
        d.dt = scenes[q].dt;
        d.cell_size = scenes[q].cell_size;
        long long share = n > 0 ? (long long)ctx->plan.max_cells * scenes[q].count / n : 0;
        d.cell_budget = share < 1 ? 1 : share;
        h[q] = d;
        off += scenes[q].count;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(ctx->scenes, h, sizeof(SceneDev) * n_scenes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_slot_scene(n, n_scenes, ctx->scenes, ctx->slot_scene, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    delete[] h;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "set scenes");
    if (!ctx->resident) ctx->resident = main_resident_blocks(ctx->plan.K, ctx->shape);
    ctx->n_scenes = n_scenes;
    drop_graphs(ctx);
    return ORCA_OK;
}

ORCA_API int orca_get_scene_grids(orca_ctx* ctx, float* grid_f, int32_t* grid_i, void* stream) {
    if (!ctx) return ORCA_ERR_ARG;
    if (ctx->n_scenes < 1) return fail(ctx, ORCA_ERR_STATE, "no batch loaded");
    cudaStream_t st = (cudaStream_t)stream;
    SceneDev* h = new (std::nothrow) SceneDev[ctx->n_scenes];
    if (!h) return fail(ctx, ORCA_ERR_NOMEM, "host allocation failed");
    cudaError_t e = cudaMemcpyAsync(h, ctx->scenes, sizeof(SceneDev) * ctx->n_scenes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        delete[] h;
        return cuda_fail(ctx, e, "copy scene grids");
    }
    for (int q = 0; q < ctx->n_scenes; ++q) {
        if (grid_f) {
            grid_f[4 * q] = h[q].grid.xmin;
            grid_f[4 * q + 1] = h[q].grid.ymin;
            grid_f[4 * q + 2] = h[q].grid.s;
            grid_f[4 * q + 3] = h[q].grid.inv;
        }
        if (grid_i) {
            grid_i[3 * q] = h[q].grid.gx;
            grid_i[3 * q + 1] = h[q].grid.gy;
            grid_i[3 * q + 2] = h[q].cell_off;
        }
    }
    delete[] h;
    return ORCA_OK;
}

ORCA_API int orca_step(orca_ctx* ctx, int32_t nsteps, void* stream) {
    NvtxRange nvtx_range("orca_step");
    if (!ctx) return ORCA_ERR_ARG;
    if (nsteps < 0) return fail(ctx, ORCA_ERR_ARG, "nsteps < 0");
    if (ctx->n == 0 || nsteps == 0) return ORCA_OK;
    cudaStream_t st = (cudaStream_t)stream;
    bool graphs = !(ctx->p.flags & ORCA_FLAG_NO_GRAPH);
    if (graphs && ctx->graph_n != ctx->n) {
        int r = build_graphs(ctx);
        if (r != ORCA_OK) return r;
    }
    for (int s = 0; s < nsteps; ++s) {
        if (graphs) CK(cudaGraphLaunch(ctx->exec[ctx->cur], st), "cudaGraphLaunch");
        else CK(enqueue_step(ctx, ctx->cur, st), "step launch");
        ctx->cur ^= 1;
    }
    ctx->stepped = true;
    ctx->slot_ok = true;  // the last reorder wrote the map of the order the step left
    return ORCA_OK;
}

ORCA_API int orca_get_state(orca_ctx* ctx, float* pos_xy, float* vel_xy, int where, void* stream) {
    NvtxRange nvtx_range("orca_get_state");
    if (!ctx) return ORCA_ERR_ARG;
    if (where != ORCA_HOST && where != ORCA_DEVICE) return fail(ctx, ORCA_ERR_ARG, "bad `where`");
    cudaStream_t st = (cudaStream_t)stream;
    if (ctx->n > 0) {
        int r = enqueue_read_state(ctx, pos_xy, vel_xy, where, st);
        if (r != ORCA_OK) return r;
    }
    if (where == ORCA_HOST) return check_device_error(ctx, st);
    return ORCA_OK;
}

ORCA_API int orca_step_host(orca_ctx* ctx, const float* pos_in, const float* vel_in, int32_t nsteps,
                            float* pos_out, float* vel_out, void* stream) {
    NvtxRange nvtx_range("orca_step_host");
    if (!ctx) return ORCA_ERR_ARG;
    if (nsteps < 0) return fail(ctx, ORCA_ERR_ARG, "nsteps < 0");
    cudaStream_t st = (cudaStream_t)stream;
    if (ctx->n > 0 && (pos_in || vel_in)) {
        int r = enqueue_write_state(ctx, pos_in, vel_in, ORCA_HOST, st);
        if (r != ORCA_OK) return r;
    }
    int r = orca_step(ctx, nsteps, stream);
    if (r != ORCA_OK) return r;
    if (ctx->n > 0 && (pos_out || vel_out)) {
        r = enqueue_read_state(ctx, pos_out, vel_out, ORCA_HOST, st);
        if (r != ORCA_OK) return r;
    }
    return check_device_error(ctx, st);
}

ORCA_API int orca_get_neighbors(orca_ctx* ctx, int32_t* nbr, int where, void* stream) {
    if (!ctx) return ORCA_ERR_ARG;
    if (!ctx->rec_nbr) return fail(ctx, ORCA_ERR_STATE, "context created without ORCA_FLAG_RECORD");
    if (!nbr) return fail(ctx, ORCA_ERR_ARG, "null nbr");
    cudaStream_t st = (cudaStream_t)stream;
    size_t bytes = (size_t)ctx->n * ctx->plan.K * 4;
    if (bytes)
        CK(cudaMemcpyAsync(nbr, ctx->rec_nbr, bytes,
                           where == ORCA_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st),
           "copy neighbours");
    if (where == ORCA_HOST) CK(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    return ORCA_OK;
}

ORCA_API int orca_set_obstacles(orca_ctx* ctx, int32_t n_seg, const float* seg_xyxy,
                                float time_horizon, int32_t max_obstacle_neighbors, int where,
                                void* stream) {
    if (!ctx) return ORCA_ERR_ARG;
    if (where != ORCA_HOST && where != ORCA_DEVICE) return fail(ctx, ORCA_ERR_ARG, "bad `where`");
    if (n_seg < 0 || n_seg > kMaxObstacles)
        return fail(ctx, ORCA_ERR_CAPACITY, "n_seg must be 0.." + std::to_string(kMaxObstacles));
    if (n_seg > 0) {
        if (!seg_xyxy) return fail(ctx, ORCA_ERR_ARG, "null segments");
        if (!(time_horizon > 0.0f)) return fail(ctx, ORCA_ERR_ARG, "time_horizon must be > 0");
        if (max_obstacle_neighbors < 1 || max_obstacle_neighbors > kMaxObstacleNeighbors)
            return fail(ctx, ORCA_ERR_ARG,
                        "max_obstacle_neighbors must be 1.." + std::to_string(kMaxObstacleNeighbors));
        if (ctx->n_scenes > 0) return fail(ctx, ORCA_ERR_STATE, "obstacles need a single-scene context");
        if (ctx->count_ops) return fail(ctx, ORCA_ERR_STATE, "operation counting is on");
        cudaStream_t st = (cudaStream_t)stream;
        CK(cudaMemcpyAsync(ctx->seg, seg_xyxy, (size_t)n_seg * 16,
                           where == ORCA_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st),
           "copy segments");
        if (where == ORCA_HOST) CK(cudaStreamSynchronize(st), "cudaStreamSynchronize");
        if (!ctx->side.st) {
            CK(cudaStreamCreateWithFlags(&ctx->side.st, cudaStreamNonBlocking), "cudaStreamCreateWithFlags");
            CK(cudaEventCreateWithFlags(&ctx->side.fork, cudaEventDisableTiming), "cudaEventCreateWithFlags");
            CK(cudaEventCreateWithFlags(&ctx->side.join, cudaEventDisableTiming), "cudaEventCreateWithFlags");
        }
        ctx->kobst = max_obstacle_neighbors;
        ctx->tau_o = time_horizon;
    }
    ctx->nseg = n_seg;
    drop_graphs(ctx);  // the step graphs capture the obstacle parameters
    return ORCA_OK;
}

ORCA_API int orca_get_obstacle_neighbors(orca_ctx* ctx, int32_t* obst, int where, void* stream) {
    if (!ctx) return ORCA_ERR_ARG;
    if (!ctx->rec_obst) return fail(ctx, ORCA_ERR_STATE, "context created without ORCA_FLAG_RECORD");
    if (!obst) return fail(ctx, ORCA_ERR_ARG, "null obst");
    cudaStream_t st = (cudaStream_t)stream;
    size_t bytes = (size_t)ctx->n * kMaxObstacleNeighbors * 4;
    if (bytes)
        CK(cudaMemcpyAsync(obst, ctx->rec_obst, bytes,
                           where == ORCA_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st),
           "copy obstacle neighbours");
    if (where == ORCA_HOST) CK(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    return ORCA_OK;
}

ORCA_API int orca_get_cells(orca_ctx* ctx, uint32_t* cell, float* grid_f, int32_t* grid_i, int where,
                            void* stream) {
    if (!ctx) return ORCA_ERR_ARG;
    if (!ctx->rec_cell) return fail(ctx, ORCA_ERR_STATE, "context created without ORCA_FLAG_RECORD");
    cudaStream_t st = (cudaStream_t)stream;
    if (cell && ctx->n)
        CK(cudaMemcpyAsync(cell, ctx->rec_cell, (size_t)ctx->n * 4,
                           where == ORCA_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st),
           "copy cells");
    GridDev g;
    CK(cudaMemcpyAsync(&g, &ctx->bins.misc->grid, sizeof g, cudaMemcpyDeviceToHost, st), "copy grid");
    CK(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    if (grid_f) {
        grid_f[0] = g.xmin;
        grid_f[1] = g.ymin;
        grid_f[2] = g.s;
        grid_f[3] = g.inv;
    }
    if (grid_i) {
        grid_i[0] = g.gx;
        grid_i[1] = g.gy;
    }
    return ORCA_OK;
}

// Sum of per-CTA counters first..first+3 over the CTAs.
static int sum_counters(orca_ctx* ctx, int first, int64_t* out4, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    size_t cnt = (size_t)ctx->plan.nmb * kBlockCounters;
    unsigned long long* h = new (std::nothrow) unsigned long long[cnt];
    if (!h) return fail(ctx, ORCA_ERR_NOMEM, "host allocation failed");
    cudaError_t e = cudaMemcpyAsync(h, ctx->blk, cnt * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        delete[] h;
        return cuda_fail(ctx, e, "copy counters");
    }
    for (int q = 0; q < 4; ++q) out4[q] = 0;
    for (size_t b = 0; b < (size_t)ctx->plan.nmb; ++b)
        for (int q = 0; q < 4; ++q) out4[q] += (int64_t)h[kBlockCounters * b + first + q];
    delete[] h;
    return ORCA_OK;
}

ORCA_API int orca_get_counters(orca_ctx* ctx, int64_t* counters4, void* stream) {
    if (!ctx || !counters4) return ORCA_ERR_ARG;
    return sum_counters(ctx, 0, counters4, stream);
}

ORCA_API int orca_remove_arrived(orca_ctx* ctx, int32_t* n_remaining, int32_t* kept_ids, int where,
                                 void* stream) {
    NvtxRange nvtx_range("orca_remove_arrived");
    if (!ctx || !n_remaining) return ORCA_ERR_ARG;
    if (where != ORCA_HOST && where != ORCA_DEVICE) return fail(ctx, ORCA_ERR_ARG, "bad `where`");
    if (ctx->n_scenes > 0) return fail(ctx, ORCA_ERR_STATE, "removal needs a single-scene context");
    cudaStream_t st = (cudaStream_t)stream;
    const int n = ctx->n, par = ctx->cur;
    if (n == 0) {
        *n_remaining = 0;
        return ORCA_OK;
    }
    // scratch between steps: sort keys (keep flags, new indices), sort values (old
    // indices), digit histograms (tile sums), digit totals (the count); the survivors'
    // state goes through the readout staging buffers, their parameters to the other
    // parameter copy, which becomes the current one
    CK(clear_box(ctx, st), "clear box flags");
    CK(launch_remove_arrived(n, ctx->PV[0], ctx->PR[par], ctx->PR[par ^ 1], ctx->stage[0],
                             ctx->stage[1], ctx->bins.keys[0], ctx->bins.keys[1],
                             ctx->bins.vals[0], ctx->bins.hist, ctx->bins.digit_totals, st),
       "removal kernels");
    uint32_t total = 0;
    CK(cudaMemcpyAsync(&total, ctx->bins.digit_totals, 4, cudaMemcpyDeviceToHost, st), "copy count");
    CK(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    const int m = (int)total;
    if (m > 0) {
        CK(cudaMemcpyAsync(ctx->PV[0].pos, ctx->stage[0], (size_t)m * 8, cudaMemcpyDeviceToDevice, st),
           "copy pos");
        CK(cudaMemcpyAsync(ctx->PV[0].vel, ctx->stage[1], (size_t)m * 8, cudaMemcpyDeviceToDevice, st),
           "copy vel");
        if (kept_ids)
            CK(cudaMemcpyAsync(kept_ids, ctx->bins.vals[0], (size_t)m * 4,
                               where == ORCA_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, st),
               "copy kept ids");
    }
    if (where == ORCA_HOST) CK(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    ctx->n = m;
    ctx->cur = par ^ 1;
    ctx->slot_ok = false;  // survivors renumbered
    *n_remaining = m;
    return ORCA_OK;
}

ORCA_API int orca_spawn_agents(orca_ctx* ctx, int32_t m, const float* cand_pos, const float* goal_xy,
                               const float* radius, const float* max_speed, const float* pref_speed,
                               const float* time_horizon, float window, int where, int32_t* accepted,
                               int32_t* n_after, void* stream) {
    NvtxRange nvtx_range("orca_spawn_agents");
    if (!ctx || !n_after) return ORCA_ERR_ARG;
    if (where != ORCA_HOST && where != ORCA_DEVICE) return fail(ctx, ORCA_ERR_ARG, "bad `where`");
    if (ctx->n_scenes > 0) return fail(ctx, ORCA_ERR_STATE, "spawning needs a single-scene context");
    if (m < 0 || !(window >= 0.0f)) return fail(ctx, ORCA_ERR_ARG, "m < 0 or window not >= 0");
    if (m > 0 && (!cand_pos || !goal_xy || !radius || !max_speed || !pref_speed || !time_horizon))
        return fail(ctx, ORCA_ERR_ARG, "null array");
    if ((long long)ctx->n + m > (long long)ctx->plan.N)
        return fail(ctx, ORCA_ERR_CAPACITY, "n + m exceeds max_agents");
    const int n = ctx->n, par = ctx->cur;
    *n_after = n;
    if (m == 0) return ORCA_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t M = (size_t)m;
    SpawnIn in;
    if (where == ORCA_HOST) {
        // candidates staged in scratch that holds nothing between steps: the readout staging
        // buffers and the other parameter copy
        const AgentParams& sp = ctx->PR[par ^ 1];
        CK(cudaMemcpyAsync(ctx->stage[0], cand_pos, M * 8, cudaMemcpyHostToDevice, st), "copy candidates");
        CK(cudaMemcpyAsync(ctx->stage[1], goal_xy, M * 8, cudaMemcpyHostToDevice, st), "copy candidates");
        CK(cudaMemcpyAsync(sp.radius, radius, M * 4, cudaMemcpyHostToDevice, st), "copy candidates");
        CK(cudaMemcpyAsync(sp.max_speed, max_speed, M * 4, cudaMemcpyHostToDevice, st), "copy candidates");
        CK(cudaMemcpyAsync(sp.pref_speed, pref_speed, M * 4, cudaMemcpyHostToDevice, st), "copy candidates");
        CK(cudaMemcpyAsync(sp.tau, time_horizon, M * 4, cudaMemcpyHostToDevice, st), "copy candidates");
        in = SpawnIn{ctx->stage[0], ctx->stage[1], sp.radius, sp.max_speed, sp.pref_speed, sp.tau};
    } else {
        in = SpawnIn{(const float2*)cand_pos, (const float2*)goal_xy, radius, max_speed, pref_speed,
                     time_horizon};
    }
    int32_t* acc_dev = where == ORCA_DEVICE && accepted ? accepted : (int32_t*)ctx->bins.vals[0];
    CK(clear_box(ctx, st), "clear box flags");
    CK(launch_spawn(n, ctx->PV[0], ctx->PR[par], m, in, window, ctx->bins.keys[1], ctx->bins.vals[1],
                    ctx->bins.keys[0], acc_dev, ctx->bins.digit_totals, st),
       "spawn kernels");
    uint32_t count = 0;
    CK(cudaMemcpyAsync(&count, ctx->bins.digit_totals, 4, cudaMemcpyDeviceToHost, st), "copy count");
    if (where == ORCA_HOST && accepted)
        CK(cudaMemcpyAsync(accepted, acc_dev, M * 4, cudaMemcpyDeviceToHost, st), "copy accepted");
    CK(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    ctx->n = n + (int)count;
    ctx->slot_ok = false;  // the entrants have no slot in the map yet
    *n_after = ctx->n;
    return ORCA_OK;
}

ORCA_API int orca_count_ops(orca_ctx* ctx, int32_t on) {
    if (!ctx) return ORCA_ERR_ARG;
    bool want = on != 0;
    if (want && ctx->nseg > 0) return fail(ctx, ORCA_ERR_STATE, "operation counting has no obstacle kernel");
    if (want != ctx->count_ops) {
        ctx->count_ops = want;
        drop_graphs(ctx);
    }
    return ORCA_OK;
}

ORCA_API int orca_get_op_counters(orca_ctx* ctx, int64_t* counters4, void* stream) {
    if (!ctx || !counters4) return ORCA_ERR_ARG;
    return sum_counters(ctx, 4, counters4, stream);
}

ORCA_API int orca_get_search_counters(orca_ctx* ctx, int64_t* counters4, void* stream) {
    if (!ctx || !counters4) return ORCA_ERR_ARG;
    return sum_counters(ctx, 8, counters4, stream);
}

// Rollout workspace: checkpoints, parameters in agent order, one segment's recomputed
// states / neighbour lists / LP records, two pairs of adjoint buffers, and the scratch of
// the deterministic neighbour accumulation (per-slot contributions, transposed lists).
struct RolloutPlan {
    int T, C, nseg;
    size_t ckpt, goal, radius, vmax, pref, tau, seg_state, seg_nbr, seg_tape, adj, gscratch, ent, contrib,
        contrib_r, incnt, inlist, total;
};

// C = 0: one segment of T steps, recorded by the forward pass itself.
static RolloutPlan rollout_plan(const orca_ctx* c, int T, int C) {
    RolloutPlan r;
    r.T = T;
    r.C = C;
    r.nseg = C > 0 ? (T + C - 1) / C : 1;
    const size_t S = (size_t)(C > 0 ? C : T);  // steps recorded at once
    size_t N = (size_t)(c->n > 0 ? c->n : 1), K = (size_t)c->plan.K;
    Layout L;
    r.ckpt = L.add((size_t)(r.nseg + 1) * N * 16);
    r.goal = L.add(N * 8);
    r.radius = L.add(N * 4);
    r.vmax = L.add(N * 4);
    r.pref = L.add(N * 4);
    r.tau = L.add(N * 4);
    r.seg_state = L.add((S + 1) * N * 16);
    r.seg_nbr = L.add(S * N * K * 4);
    r.seg_tape = L.add(S * N * 4);
    r.adj = L.add(4 * N * 8);
    r.gscratch = L.add(3 * N * 4);
    r.ent = L.add(N * kAdjEntries * 4);
    r.contrib = L.add(N * kAdjEntries * 4 * 4);
    r.contrib_r = L.add(N * kAdjEntries * 4);
    r.incnt = L.add(N * 4);
    r.inlist = L.add(N * kInCap * 4);
    r.total = L.total;
    return r;
}

ORCA_API int orca_rollout_workspace_size(const orca_ctx* ctx, int32_t T, int32_t ckpt_every,
                                         size_t* bytes) {
    if (!ctx || !bytes || T < 1 || ckpt_every < 0) return ORCA_ERR_ARG;
    *bytes = rollout_plan(ctx, T, ckpt_every).total;
    return ORCA_OK;
}

ORCA_API int orca_rollout_forward(orca_ctx* ctx, int32_t T, int32_t ckpt_every, float* traj_pos,
                                  void* workspace, size_t workspace_bytes, void* stream) {
    NvtxRange nvtx_range("orca_rollout_forward");
    if (!ctx) return ORCA_ERR_ARG;
    ctx->slot_ok = false;  // rollouts reload and step the state on their own
    if (T < 1 || ckpt_every < 0) return fail(ctx, ORCA_ERR_ARG, "T must be >= 1 and ckpt_every >= 0");
    if (ctx->n_scenes > 0) return fail(ctx, ORCA_ERR_STATE, "rollouts need a single scene");
    if (ctx->nseg > 0) return fail(ctx, ORCA_ERR_STATE, "the adjoint has no static obstacles");
    if (ctx->n < 1) return fail(ctx, ORCA_ERR_STATE, "no agents loaded");
    RolloutPlan r = rollout_plan(ctx, T, ckpt_every);
    if (!workspace || ((uintptr_t)workspace & 255) || workspace_bytes < r.total)
        return fail(ctx, ORCA_ERR_NOMEM, "rollout workspace missing, misaligned or too small");
    cudaStream_t st = (cudaStream_t)stream;
    char* w = (char*)workspace;
    size_t N = (size_t)ctx->n;
    auto ck = [&](int s) { return (float2*)(w + r.ckpt + (size_t)s * N * 16); };
    CK(launch_unpermute_params(ctx->n, ctx->PR[ctx->cur], (float2*)(w + r.goal), (float*)(w + r.radius),
                               (float*)(w + r.vmax), (float*)(w + r.pref), (float*)(w + r.tau), st),
       "unpermute parameters");
    if (ckpt_every == 0) {
        // every step recorded as the backward pass needs it: the state it starts from, the
        // neighbour lists and the LP records
        for (int t = 0; t < T; ++t) {
            float2* sp = (float2*)(w + r.seg_state + (size_t)t * N * 16);
            CK(enqueue_recording_step(ctx, ctx->cur, (int32_t*)(w + r.seg_nbr) + (size_t)t * N * ctx->plan.K,
                                      (uint32_t*)(w + r.seg_tape) + (size_t)t * N, sp,
                                      traj_pos ? (float2*)traj_pos + (size_t)t * N : nullptr, st),
               "recording step");
            ctx->cur ^= 1;
        }
        ctx->roll_T = T;
        ctx->roll_C = 0;
        ctx->roll_ws = workspace;
        return ORCA_OK;
    }
    CK(launch_unpermute(ctx->n, ctx->PV[0], ctx->PR[ctx->cur].id, ck(0), ck(0) + N, st), "checkpoint");
    for (int t = 0; t < T; ++t) {
        int rr = orca_step(ctx, 1, stream);
        if (rr != ORCA_OK) return rr;
        if (traj_pos)
            CK(launch_unpermute(ctx->n, ctx->PV[0], ctx->PR[ctx->cur].id, (float2*)traj_pos + (size_t)t * N,
                                nullptr, st), "trajectory");
        if ((t + 1) % ckpt_every == 0 && t + 1 < T) {
            float2* c = ck((t + 1) / ckpt_every);
            CK(launch_unpermute(ctx->n, ctx->PV[0], ctx->PR[ctx->cur].id, c, c + N, st), "checkpoint");
        }
    }
    ctx->roll_T = T;
    ctx->roll_C = ckpt_every;
    ctx->roll_ws = workspace;
    return ORCA_OK;
}

ORCA_API int orca_rollout_backward(orca_ctx* ctx, const float* dL_dpos, float* g_pref_speed,
                                   float* g_radius, float* g_time_horizon, float* g_pos0,
                                   float* g_vel0, void* workspace, size_t workspace_bytes,
                                   void* stream) {
    NvtxRange nvtx_range("orca_rollout_backward");
    if (!ctx) return ORCA_ERR_ARG;
    ctx->slot_ok = false;  // rollouts reload and step the state on their own
    if (!dL_dpos) return fail(ctx, ORCA_ERR_ARG, "dL_dpos is required");
    if (workspace != ctx->roll_ws || ctx->roll_T < 1)
        return fail(ctx, ORCA_ERR_STATE, "no orca_rollout_forward with this workspace");
    RolloutPlan r = rollout_plan(ctx, ctx->roll_T, ctx->roll_C);
    if (workspace_bytes < r.total) return fail(ctx, ORCA_ERR_NOMEM, "rollout workspace too small");
    cudaStream_t st = (cudaStream_t)stream;
    char* w = (char*)workspace;
    const int n = ctx->n, T = r.T, C = r.C;
    const size_t N = (size_t)n, K = (size_t)ctx->plan.K;
    auto ck = [&](int s) { return (float2*)(w + r.ckpt + (size_t)s * N * 16); };
    auto sstate = [&](int q) { return (float2*)(w + r.seg_state + (size_t)q * N * 16); };
    float2* adj = (float2*)(w + r.adj);
    float2* pnext = adj;
    float2* vnext = adj + N;
    float2* pcur = adj + 2 * N;
    float2* vcur = adj + 3 * N;
    const float2* dLdp = (const float2*)dL_dpos;
    // parameter gradients accumulate into the caller's arrays, or into scratch
    float* gs = (float*)(w + r.gscratch);
    float* gp = g_pref_speed ? g_pref_speed : gs;
    float* gr = g_radius ? g_radius : gs + N;
    float* gt = g_time_horizon ? g_time_horizon : gs + 2 * N;
    CK(cudaMemsetAsync(gp, 0, N * 4, st), "zero");
    CK(cudaMemsetAsync(gr, 0, N * 4, st), "zero");
    CK(cudaMemsetAsync(gt, 0, N * 4, st), "zero");
    CK(cudaMemcpyAsync(pnext, dLdp + (size_t)(T - 1) * N, N * 8, cudaMemcpyDeviceToDevice, st), "seed");
    CK(cudaMemsetAsync(vnext, 0, N * 8, st), "zero");
    CK(cudaMemsetAsync(w + r.incnt, 0, N * 4, st), "zero");
    for (int seg = r.nseg - 1; seg >= 0; --seg) {
        // C = 0: the forward pass recorded all T steps (one segment, nothing to re-run)
        const int t0 = seg * C, t1 = C > 0 && t0 + C < T ? t0 + C : T;
        if (C > 0) {
            int rr = orca_set_agents(ctx, n, (const float*)ck(seg), (const float*)(ck(seg) + N),
                                     (const float*)(w + r.goal), (const float*)(w + r.radius),
                                     (const float*)(w + r.vmax), (const float*)(w + r.pref),
                                     (const float*)(w + r.tau), ORCA_DEVICE, stream);
            if (rr != ORCA_OK) return rr;
        }
        for (int t = t0; C > 0 && t < t1; ++t) {
            CK(enqueue_recording_step(ctx, ctx->cur, (int32_t*)(w + r.seg_nbr) + (size_t)(t - t0) * N * K,
                                      (uint32_t*)(w + r.seg_tape) + (size_t)(t - t0) * N, sstate(t - t0),
                                      nullptr, st),
               "recording step");
            ctx->cur ^= 1;
        }
        for (int t = t1 - 1; t >= t0; --t) {
            const float2* sp = sstate(t - t0);
            AdjArgs<float> A;
            A.n = n;
            A.kstride = (int)K;
            A.dt = ctx->p.dt;
            A.pos = sp;
            A.vel = sp + N;
            A.goal = (const float2*)(w + r.goal);
            A.radius = (const float*)(w + r.radius);
            A.max_speed = (const float*)(w + r.vmax);
            A.pref_speed = (const float*)(w + r.pref);
            A.tau = (const float*)(w + r.tau);
            A.nbr = (const int32_t*)(w + r.seg_nbr) + (size_t)(t - t0) * N * K;
            A.tape = (const uint32_t*)(w + r.seg_tape) + (size_t)(t - t0) * N;
            A.pbar_next = pnext;
            A.vbar_next = vnext;
            // p(t) for t >= 1 is a trajectory point of the loss: its own gradient joins
            A.dl_dp = t >= 1 ? dLdp + (size_t)(t - 1) * N : nullptr;
            A.pbar = pcur;
            A.vbar = vcur;
            A.g_pref = gp;
            A.g_radius = gr;
            A.g_tau = gt;
            A.ent = (int32_t*)(w + r.ent);
            A.contrib = (float*)(w + r.contrib);
            A.contrib_r = (float*)(w + r.contrib_r);
            A.incnt = (uint32_t*)(w + r.incnt);
            A.inlist = (uint32_t*)(w + r.inlist);
            A.err = &ctx->bins.misc->error;
            CK(launch_adjoint_step(A, (int)K, st), "adjoint kernels");
            float2* tmp = pnext;
            pnext = pcur;
            pcur = tmp;
            tmp = vnext;
            vnext = vcur;
            vcur = tmp;
        }
    }
    if (g_pos0) CK(cudaMemcpyAsync(g_pos0, pnext, N * 8, cudaMemcpyDeviceToDevice, st), "copy");
    if (g_vel0) CK(cudaMemcpyAsync(g_vel0, vnext, N * 8, cudaMemcpyDeviceToDevice, st), "copy");
    ctx->roll_T = 0;
    return ORCA_OK;
}

ORCA_API int orca_sync(orca_ctx* ctx, void* stream) {
    if (!ctx) return ORCA_ERR_ARG;
    return check_device_error(ctx, (cudaStream_t)stream);
}

ORCA_API int orca_num_agents(const orca_ctx* ctx, int32_t* n) {
    if (!ctx || !n) return ORCA_ERR_ARG;
    *n = ctx->n;
    return ORCA_OK;
}

ORCA_API const char* orca_last_error(const orca_ctx* ctx) {
    return ctx ? ctx->err.c_str() : g_create_err.c_str();
}

ORCA_API const char* orca_status_string(int status) {
    switch (status) {
        case ORCA_OK: return "ok";
        case ORCA_ERR_ARG: return "invalid argument";
        case ORCA_ERR_NOMEM: return "out of memory";
        case ORCA_ERR_CUDA: return "CUDA error";
        case ORCA_ERR_STATE: return "invalid state";
        case ORCA_ERR_NUMERIC: return "non-finite result";
        case ORCA_ERR_TIMEOUT: return "device wait timed out";
        case ORCA_ERR_CAPACITY: return "capacity exceeded";
        case ORCA_ERR_BOUNDS: return "device index check failed";
        default: return "unknown status";
    }
}

}  // extern "C"
