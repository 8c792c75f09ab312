// orca_population.cu -- agents leave the simulation at their goal (Section 4: "once a
// person reaches the goal location they are removed").
//
// After a step the state sits in cell order.  Removal decides arrival per slot, numbers
// the survivors 0..n'-1 in increasing old index (an exclusive scan over a per-index keep
// flag), and scatters each survivor's state, parameters and radius prediction to its new
// index, so the compacted crowd is in index order with dense indices (the next step sorts
// it into cells again).
#include "orca_common.cuh"

namespace orca {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

// Arrival, in FP32 with one rounding per operation: |goal - p|^2 <= r^2.
__global__ void __launch_bounds__(256) keep_flags_kernel(int n, const float2* __restrict__ pos,
                                                         const float2* __restrict__ goal,
                                                         const float* __restrict__ radius,
                                                         const uint32_t* __restrict__ id,
                                                         uint32_t* __restrict__ keep_by_id) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    float2 p = pos[t], g = goal[t];
    float dx = __fsub_rn(g.x, p.x), dy = __fsub_rn(g.y, p.y);
    float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
    float r = radius[t];
    keep_by_id[id[t]] = d2 <= __fmul_rn(r, r) ? 0u : 1u;
}

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t& excl) {
    __shared__ uint32_t s_warp[kScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    uint32_t base = 0, total = 0;
#pragma unroll
    for (int w = 0; w < kScanThreads / 32; ++w) {
        uint32_t sw = s_warp[w];
        if (w < warp) base += sw;
        total += sw;
    }
    __syncthreads();
    excl = base + inc - v;
    return total;
}

// Number of kept agents in each tile of kScanTile indices.
__global__ void __launch_bounds__(kScanThreads) tile_sums_kernel(int n, const uint32_t* __restrict__ keep,
                                                                 uint32_t* __restrict__ tile_sums) {
    const int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    uint32_t c = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q)
        if (base + q < n) c += keep[base + q];
    uint32_t excl;
    uint32_t total = block_exclusive_scan(c, excl);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = total;
}

// Exclusive scan of the tile sums in place (one CTA), and the grand total.
__global__ void __launch_bounds__(kScanThreads) tile_offsets_kernel(int tiles, uint32_t* __restrict__ tile_sums,
                                                                    uint32_t* __restrict__ total) {
    uint32_t carry = 0;
    for (int b0 = 0; b0 < tiles; b0 += kScanThreads) {
        int b = b0 + threadIdx.x;
        uint32_t v = b < tiles ? tile_sums[b] : 0u;
        uint32_t excl;
        uint32_t sum = block_exclusive_scan(v, excl);
        if (b < tiles) tile_sums[b] = carry + excl;
        carry += sum;
    }
    if (threadIdx.x == 0) *total = carry;
}

// New index of every kept agent (kept agents in increasing old index), and the old index
// of every new index.
__global__ void __launch_bounds__(kScanThreads) new_index_kernel(int n, const uint32_t* __restrict__ keep,
                                                                 const uint32_t* __restrict__ tile_offsets,
                                                                 uint32_t* __restrict__ new_id,
                                                                 uint32_t* __restrict__ old_id) {
    const int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    uint32_t f[kScanItems], c = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        f[q] = base + q < n ? keep[base + q] : 0u;
        c += f[q];
    }
    uint32_t excl;
    block_exclusive_scan(c, excl);
    uint32_t j = tile_offsets[blockIdx.x] + excl;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        if (base + q >= n) break;
        if (f[q]) {
            new_id[base + q] = j;
            old_id[j] = (uint32_t)(base + q);
            ++j;
        } else {
            new_id[base + q] = 0xffffffffu;
        }
    }
}

// Scatter every survivor (sorted slot t) to its new index.
__global__ void __launch_bounds__(256) compact_kernel(int n, AgentState src, AgentParams sp,
                                                      const uint32_t* __restrict__ new_id,
                                                      float2* __restrict__ pos_out,
                                                      float2* __restrict__ vel_out, AgentParams dp) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    uint32_t j = new_id[sp.id[t]];
    if (j == 0xffffffffu) return;
    pos_out[j] = src.pos[t];
    vel_out[j] = src.vel[t];
    dp.goal[j] = sp.goal[t];
    dp.radius[j] = sp.radius[t];
    dp.max_speed[j] = sp.max_speed[t];
    dp.pref_speed[j] = sp.pref_speed[t];
    dp.tau[j] = sp.tau[t];
    dp.id[j] = j;
    if (dp.hint) dp.hint[j] = sp.hint[t];
}

int scan_tiles(int n) { return (n + kScanTile - 1) / kScanTile; }

cudaError_t launch_remove_arrived(int n, const AgentState& cur, const AgentParams& cur_p,
                                  const AgentParams& dst_p, float2* pos_tmp, float2* vel_tmp,
                                  uint32_t* keep, uint32_t* new_id, uint32_t* old_id,
                                  uint32_t* tile_sums, uint32_t* total, cudaStream_t st) {
    int tiles = scan_tiles(n);
    keep_flags_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, cur.pos, cur_p.goal, cur_p.radius,
                                                        cur_p.id, keep);
    tile_sums_kernel<<<tiles, kScanThreads, 0, st>>>(n, keep, tile_sums);
    tile_offsets_kernel<<<1, kScanThreads, 0, st>>>(tiles, tile_sums, total);
    new_index_kernel<<<tiles, kScanThreads, 0, st>>>(n, keep, tile_sums, new_id, old_id);
    compact_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, cur, cur_p, new_id, pos_tmp, vel_tmp, dst_p);
    return cudaGetLastError();
}

}  // namespace orca
