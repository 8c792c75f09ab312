// orca_static.cu -- one ORCA step that allocates no memory (orca_step_static).
//
// Some callers cannot allocate GPU memory at all: code running inside a host framework
// that owns every device allocation through its own pool, plugins loaded into a process
// whose allocator must not be bypassed, or call sites where cudaMalloc's implicit device
// synchronisation is not allowed.  For them this file keeps all scratch space of one step
// in a fixed, file-scope device array, sized for at most kStaticMaxAgents agents and
// kStaticMaxCells grid cells (about 7 MiB, held on every GPU that loads the library until
// the process exits).  The caller passes only its inputs and outputs.
//
// The step itself is the library's ordinary one (same kernels, same arithmetic): bounding
// box and grid, cell keys and counts, cell table, reorder into cell order, the per-agent
// ORCA kernel, and a scatter back to the caller's agent order.
#include <string>

#include "../../include/orca_gb300.h"
#include "orca_common.cuh"

namespace orca {

void set_context_free_error(const std::string& msg);

constexpr int kStaticMaxAgents = 65536;
constexpr int kStaticMaxCells = 262144;

// Scratch layout (bytes), every piece 256-byte aligned.  The pieces from misc to the end
// are cleared by every call (grid, counters, and the counting sort's cell and tile counts).
struct StaticLayout {
    size_t id, keys, ranks, cells, part, msg, sslot, svel, goal, radius, vmax, pref, tau, sid, opos,
        ovel, misc, cnt, tsum, blk, total;
};

constexpr size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

constexpr StaticLayout static_layout() {
    StaticLayout L{};
    size_t N = kStaticMaxAgents, o = 0;
    int nmb = (kStaticMaxAgents + 63) / 64;
    L.id = o; o += al256(N * 4);
    L.keys = o; o += al256(N * 4);
    L.ranks = o; o += al256(N * 4);
    L.cells = o; o += al256(((size_t)kStaticMaxCells + 1) * 4);
    L.part = o; o += al256(kBboxBlocks * 16);
    L.msg = o; o += al256(N * 16);
    L.sslot = o; o += al256(N * 4);
    L.svel = o; o += al256(N * 8);
    L.goal = o; o += al256(N * 8);
    L.radius = o; o += al256(N * 4);
    L.vmax = o; o += al256(N * 4);
    L.pref = o; o += al256(N * 4);
    L.tau = o; o += al256(N * 4);
    L.sid = o; o += al256(N * 4);
    L.opos = o; o += al256(N * 8);
    L.ovel = o; o += al256(N * 8);
    L.misc = o; o += al256(sizeof(DeviceMisc));
    L.cnt = o; o += al256((size_t)kStaticMaxCells * 4);
    L.tsum = o; o += al256(((size_t)kStaticMaxCells / kCellTile + 1) * kTileSumStride * 4);
    L.blk = o; o += al256((size_t)nmb * kBlockCounters * 8);
    L.total = o;
    return L;
}

constexpr StaticLayout kStatic = static_layout();

// The scratch space.  Host code must not use this name as an address: it obtains the
// device address with cudaGetSymbolAddress and passes pointers on.
static __device__ __align__(256) unsigned char g_orca_static_scratch[kStatic.total];

static int static_fail(int code, const std::string& msg) {
    set_context_free_error(msg);
    return code;
}

// Device address of the scratch array in the current context, looked up on every call (a
// host-side table lookup once the module is loaded): a cached address would outlive a
// reset of the device's primary context, after which the array lives elsewhere.
static int static_scratch(char** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_orca_static_scratch);
    if (e != cudaSuccess || !p)
        return static_fail(ORCA_ERR_CUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    *out = (char*)p;
    return ORCA_OK;
}

}  // namespace orca

using namespace orca;

extern "C" ORCA_API int orca_step_static(int32_t n, const float* pos_xy, const float* vel_xy,
                                         const float* goal_xy, const float* radius,
                                         const float* max_speed, const float* pref_speed,
                                         const float* time_horizon, float neighbor_dist,
                                         int32_t max_neighbors, float dt, float cell_size,
                                         float* pos_out_xy, float* vel_out_xy, void* stream) {
    if (n < 0) return static_fail(ORCA_ERR_ARG, "orca_step_static: n < 0");
    if (n > kStaticMaxAgents)
        return static_fail(ORCA_ERR_CAPACITY, "orca_step_static: n exceeds the fixed scratch capacity of "
                                                  "65536 agents; use orca_create/orca_step");
    if (max_neighbors < 1 || max_neighbors > kMaxNeighbors)
        return static_fail(ORCA_ERR_ARG, "orca_step_static: max_neighbors must be 1..32");
    if (!(neighbor_dist > 0.0f) || !(dt > 0.0f) || cell_size < 0.0f)
        return static_fail(ORCA_ERR_ARG, "orca_step_static: neighbor_dist and dt must be > 0, cell_size >= 0");
    if (n == 0) return ORCA_OK;
    if (!pos_xy || !vel_xy || !goal_xy || !radius || !max_speed || !pref_speed || !time_horizon ||
        !pos_out_xy || !vel_out_xy)
        return static_fail(ORCA_ERR_ARG, "orca_step_static: null array");
    char* base = nullptr;
    int r = static_scratch(&base);
    if (r != ORCA_OK) return r;
    cudaStream_t st = (cudaStream_t)stream;
    const StaticLayout& L = kStatic;

    AgentState src{(float2*)pos_xy, (float2*)vel_xy};
    AgentParams src_p{(float2*)goal_xy, (float*)radius, (float*)max_speed, (float*)pref_speed,
                      (float*)time_horizon, (uint32_t*)(base + L.id), nullptr};
    Sorted sorted{(float4*)(base + L.msg), (float2*)(base + L.svel), (uint32_t*)(base + L.sslot)};
    AgentParams dst_p{(float2*)(base + L.goal), (float*)(base + L.radius), (float*)(base + L.vmax),
                      (float*)(base + L.pref), (float*)(base + L.tau), (uint32_t*)(base + L.sid),
                      nullptr};
    AgentState out{(float2*)(base + L.opos), (float2*)(base + L.ovel)};
    BinBuffers bins{};
    bins.keys[0] = (uint32_t*)(base + L.keys);
    bins.vals[0] = (uint32_t*)(base + L.ranks);
    bins.cnt = (uint32_t*)(base + L.cnt);
    bins.tile_sums = (uint32_t*)(base + L.tsum);
    bins.cell_start = (uint32_t*)(base + L.cells);
    bins.table_cells = kStaticMaxCells;
    bins.bbox_partials = (float4*)(base + L.part);
    bins.misc = (DeviceMisc*)(base + L.misc);

    float cs = cell_size > 0.0f ? cell_size : neighbor_dist * 0.25f;
    // start from zero: the grid, ticket and counters of the previous call, and the cell and
    // tile counts (zero after every completed call, cleared anyway)
    cudaError_t e = cudaMemsetAsync(base + L.misc, 0, kStatic.total - L.misc, st);
    if (e == cudaSuccess) e = launch_iota(n, src_p.id, st);
    if (e == cudaSuccess) e = launch_binning(n, cs, kStaticMaxCells, src, bins, -1, st);
    if (e == cudaSuccess) e = launch_reorder(n, bins, src, sorted, src_p, dst_p, st);
    if (e == cudaSuccess) {
        MainArgs a{};
        a.n = n;
        a.k = max_neighbors;
        a.nd = neighbor_dist;
        a.dt = dt;
        a.misc = bins.misc;
        a.misc_rw = bins.misc;
        a.cell_start = bins.cell_start;
        a.in = sorted;
        a.prm = dst_p;
        a.out = out;
        a.block_counters = (unsigned long long*)(base + L.blk);
        a.count_ops = 0;
        a.seg = nullptr;  // no static obstacles here
        a.nseg = 0;
        a.rec_obst = nullptr;
        a.rec_nbr = nullptr;
        a.rec_cell = nullptr;
        a.scenes = nullptr;
        a.slot_scene = nullptr;
        a.rec_stride = max_neighbors;
        a.tape = nullptr;
        LaunchShape sh{128, default_lp3_group(max_neighbors)};
        e = launch_main(a, max_neighbors, sh, 0, st);
    }
    if (e == cudaSuccess) e = launch_unpermute(n, out, dst_p.id, (float2*)pos_out_xy, (float2*)vel_out_xy, st);
    if (e != cudaSuccess)
        return static_fail(ORCA_ERR_CUDA, std::string("orca_step_static: ") + cudaGetErrorString(e));
    return ORCA_OK;
}
