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

// ---------------------------------------------------------------------------------
// Spawning during a run (Section 4: new people are placed where they overlap nobody
// within a time period based on their size and speed).  A candidate enters at rest; it
// conflicts with a present agent j when the two could touch within the window T moving
// straight at each other, |p_c - p_j| <= r_c + r_j + (V_c + |v_j|) T, and with a
// candidate accepted before it (index order) likewise with that candidate's V in place of
// |v_j|.  Decided in FP32, one rounding per operation (the oracle decides it the same way).
// ---------------------------------------------------------------------------------
__device__ __forceinline__ bool spawn_conflict(float xc, float yc, float rc, float vc, float xj, float yj,
                                               float rj, float sj, float window) {
    const float dx = __fsub_rn(xc, xj), dy = __fsub_rn(yc, yj);
    const float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
    const float reach = __fadd_rn(__fadd_rn(rc, rj), __fmul_rn(__fadd_rn(vc, sj), window));
    return d2 <= __fmul_rn(reach, reach);
}

// Candidate c (one CTA each) against every present agent: blocked[c] = 1 on a conflict.
__global__ void __launch_bounds__(256) spawn_crowd_kernel(int n, AgentState cur, const float* __restrict__ radius,
                                                          int m, const float2* __restrict__ cpos,
                                                          const float* __restrict__ crad,
                                                          const float* __restrict__ cvmax, float window,
                                                          uint32_t* __restrict__ blocked) {
    const int c = blockIdx.x;
    if (c >= m) return;
    const float2 pc = cpos[c];
    const float rc = crad[c], vc = cvmax[c];
    bool hit = false;
    for (int j = threadIdx.x; j < n && !hit; j += blockDim.x) {
        const float2 pj = cur.pos[j], vj = cur.vel[j];
        const float sj = __fsqrt_rn(__fadd_rn(__fmul_rn(vj.x, vj.x), __fmul_rn(vj.y, vj.y)));
        hit = spawn_conflict(pc.x, pc.y, rc, vc, pj.x, pj.y, radius[j], sj, window);
    }
    hit = __syncthreads_or(hit);
    if (threadIdx.x == 0) blocked[c] = hit ? 1u : 0u;
}

// In candidate order (one CTA): a candidate not blocked by the crowd enters unless it
// conflicts with one that entered before it.  rank[c] receives its place among the
// entrants (or ~0), accepted[c] 1 or 0; *count the number of entrants.
__global__ void __launch_bounds__(256) spawn_accept_kernel(int m, const float2* __restrict__ cpos,
                                                           const float* __restrict__ crad,
                                                           const float* __restrict__ cvmax, float window,
                                                           const uint32_t* __restrict__ blocked,
                                                           uint32_t* __restrict__ entrants,
                                                           uint32_t* __restrict__ rank,
                                                           int32_t* __restrict__ accepted,
                                                           uint32_t* __restrict__ count) {
    int na = 0;  // entrants so far (their candidate indices in entrants[0..na))
    for (int c = 0; c < m; ++c) {
        bool hit = blocked[c] != 0u;
        if (!hit) {
            const float2 pc = cpos[c];
            const float rc = crad[c], vc = cvmax[c];
            for (int q = threadIdx.x; q < na && !hit; q += blockDim.x) {
                const uint32_t e = entrants[q];
                const float2 pe = cpos[e];
                hit = spawn_conflict(pc.x, pc.y, rc, vc, pe.x, pe.y, crad[e], cvmax[e], window);
            }
        }
        hit = __syncthreads_or(hit);
        if (threadIdx.x == 0) {
            accepted[c] = hit ? 0 : 1;
            rank[c] = hit ? 0xffffffffu : (uint32_t)na;
            if (!hit) entrants[na] = (uint32_t)c;
        }
        if (!hit) ++na;
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = (uint32_t)na;
}

// The entrants appended at rest after the n present agents, with agent indices n, n+1, ...
// in candidate order and no search-radius prediction.
__global__ void __launch_bounds__(256) spawn_append_kernel(int n, int m, const float2* __restrict__ cpos,
                                                           const float2* __restrict__ cgoal,
                                                           const float* __restrict__ crad,
                                                           const float* __restrict__ cvmax,
                                                           const float* __restrict__ cpref,
                                                           const float* __restrict__ ctau,
                                                           const uint32_t* __restrict__ rank,
                                                           AgentState cur, AgentParams cp) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m || rank[c] == 0xffffffffu) return;
    const uint32_t j = (uint32_t)n + rank[c];
    cur.pos[j] = cpos[c];
    cur.vel[j] = make_float2(0.0f, 0.0f);
    cp.goal[j] = cgoal[c];
    cp.radius[j] = crad[c];
    cp.max_speed[j] = cvmax[c];
    cp.pref_speed[j] = cpref[c];
    cp.tau[j] = ctau[c];
    cp.id[j] = j;
    if (cp.hint) cp.hint[j] = __int_as_float(0x7fffffff);
}

cudaError_t launch_spawn(int n, const AgentState& cur, const AgentParams& cur_p, int m, const SpawnIn& in,
                         float window, uint32_t* blocked, uint32_t* entrants, uint32_t* rank,
                         int32_t* accepted, uint32_t* count, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    spawn_crowd_kernel<<<m, 256, 0, st>>>(n, cur, cur_p.radius, m, in.pos, in.radius, in.max_speed, window,
                                          blocked);
    spawn_accept_kernel<<<1, 256, 0, st>>>(m, in.pos, in.radius, in.max_speed, window, blocked, entrants,
                                           rank, accepted, count);
    spawn_append_kernel<<<(m + 255) / 256, 256, 0, st>>>(n, m, in.pos, in.goal, in.radius, in.max_speed,
                                                         in.pref_speed, in.tau, rank, cur, cur_p);
    return cudaGetLastError();
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
