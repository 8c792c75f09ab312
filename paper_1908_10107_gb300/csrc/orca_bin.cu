// orca_bin.cu -- spatial binning of the crowd (Fig. 2: "messages organised into bins").
//
// Per step, on one stream, with no host round trip:
//   bbox_grid       exact min/max of positions -> grid descriptor (cell edge, gx, gy).
//   keys_hist       cell key of every agent + digit histogram of radix pass 0.
//   radix_upsweep / radix_scan / radix_downsweep   stable LSD radix sort of
//                   (cell key, slot) with 9-bit digits; only ceil(bits(num_cells)/9)
//                   passes do work, the rest return at once.
//   reorder         gathers state and parameters into the new cell order, writes the
//                   id -> slot map, and the cell table: cell_start[c] = first sorted slot
//                   of cell c for every c in [0, num_cells] (empty cells included, no
//                   memset needed).
//
// The sort is stable with respect to the previous step's cell order, so the layout is
// deterministic; nothing downstream depends on the order inside a cell (neighbours are
// ranked by (distance, agent index)).
#include "orca_common.cuh"

namespace orca {

// Grid over a bounding box r = (xmin, ymin, xmax, ymax), all in FP32:
// inv = fl(1/s), g = floor(fl(fl(max - min) * inv)) + 1, doubling s while gx*gy exceeds
// max_cells.  A non-finite or absurd extent puts everything in one cell and sets *err.
__device__ GridDev derive_grid(float4 r, float cell_size, long long max_cells, int max_passes,
                               int* err) {
    GridDev g;
    g.xmin = r.x;
    g.ymin = r.y;
    float ex = __fsub_rn(r.z, r.x), ey = __fsub_rn(r.w, r.y);
    float s = cell_size, inv = 1.0f, fx = 0.0f, fy = 0.0f;
    bool fits = false;
    for (int it = 0; it < 200 && !fits; ++it) {
        inv = __fdiv_rn(1.0f, s);
        fx = floorf(__fmul_rn(ex, inv));
        fy = floorf(__fmul_rn(ey, inv));
        double cells = ((double)fx + 1.0) * ((double)fy + 1.0);
        if (cells <= (double)max_cells) fits = true;
        else s = __fmul_rn(s, 2.0f);
    }
    if (!fits || !(ex >= 0.0f) || !(ey >= 0.0f)) {
        *err |= kErrCapacity;
        fx = fy = 0.0f;
        s = 1.0f;
        inv = 1.0f;
        if (!(g.xmin == g.xmin) || isinf(g.xmin)) g.xmin = 0.0f;
        if (!(g.ymin == g.ymin) || isinf(g.ymin)) g.ymin = 0.0f;
    }
    g.s = s;
    g.inv = inv;
    g.gx = (int)fx + 1;
    g.gy = (int)fy + 1;
    g.num_cells = g.gx * g.gy;
    int bits = 0;
    while (bits < 31 && (1u << bits) < (unsigned)g.num_cells) ++bits;
    int passes = (bits + kRadixBits - 1) / kRadixBits;
    g.passes = passes < 1 ? 1 : (passes > max_passes ? max_passes : passes);
    // rounding of fl(fl(x - xmin) * inv) moves a cell boundary by at most a few ulps of
    // the extent; 1e-5 relative is a wide margin
    g.slop = 1e-5f * (fabsf(g.xmin) + fabsf(g.ymin) + ex + ey + 2.0f * s) + 1e-6f;
    return g;
}

// ---------------------------------------------------------------------------------
// Bounding box and grid.  Each block reduces a grid-stride share; the last block to
// finish (ticket counter, no waiting) folds the partials and derives the grid in FP32:
// inv = fl(1/s), g = floor(fl(fl(max - min) * inv)) + 1, doubling s while gx*gy exceeds
// the table capacity.
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) bbox_grid_kernel(int n, const float2* __restrict__ pos,
                                                        float cell_size, long long max_cells,
                                                        int max_passes, float4* partials,
                                                        DeviceMisc* misc) {
    pdl_wait();
    float xmin = INFINITY, ymin = INFINITY, xmax = -INFINITY, ymax = -INFINITY;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float2 p = pos[i];
        xmin = fminf(xmin, p.x);
        xmax = fmaxf(xmax, p.x);
        ymin = fminf(ymin, p.y);
        ymax = fmaxf(ymax, p.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        xmin = fminf(xmin, __shfl_xor_sync(0xffffffffu, xmin, o));
        xmax = fmaxf(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
        ymin = fminf(ymin, __shfl_xor_sync(0xffffffffu, ymin, o));
        ymax = fmaxf(ymax, __shfl_xor_sync(0xffffffffu, ymax, o));
    }
    __shared__ float4 s_part[8];
    __shared__ bool s_last;
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) s_part[warp] = make_float4(xmin, ymin, xmax, ymax);
    __syncthreads();
    if (threadIdx.x == 0) {
        float4 r = s_part[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            r.x = fminf(r.x, s_part[w].x);
            r.y = fminf(r.y, s_part[w].y);
            r.z = fmaxf(r.z, s_part[w].z);
            r.w = fmaxf(r.w, s_part[w].w);
        }
        partials[blockIdx.x] = r;
        __threadfence();
        unsigned int ticket = atomicAdd(&misc->bbox_ticket, 1u);
        s_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;
    // last block: fold the partials with every thread, then one thread derives the grid
    __threadfence();
    float4 r = make_float4(INFINITY, INFINITY, -INFINITY, -INFINITY);
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
        float4 q = __ldcg(&partials[b]);
        r.x = fminf(r.x, q.x);
        r.y = fminf(r.y, q.y);
        r.z = fmaxf(r.z, q.z);
        r.w = fmaxf(r.w, q.w);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        r.x = fminf(r.x, __shfl_xor_sync(0xffffffffu, r.x, o));
        r.y = fminf(r.y, __shfl_xor_sync(0xffffffffu, r.y, o));
        r.z = fmaxf(r.z, __shfl_xor_sync(0xffffffffu, r.z, o));
        r.w = fmaxf(r.w, __shfl_xor_sync(0xffffffffu, r.w, o));
    }
    __syncthreads();
    if (lane == 0) s_part[warp] = r;
    __syncthreads();
    if (threadIdx.x != 0) return;
    r = s_part[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
        r.x = fminf(r.x, s_part[w].x);
        r.y = fminf(r.y, s_part[w].y);
        r.z = fmaxf(r.z, s_part[w].z);
        r.w = fmaxf(r.w, s_part[w].w);
    }
    misc->bbox_ticket = 0;
    misc->tile_counter = 0;
    misc->obs_tiles = 0;
    int err = 0;
    misc->grid = derive_grid(r, cell_size, max_cells, max_passes, &err);
    if (err) atomicOr(&misc->error, err);
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Cell key of each agent and the digit-0 histogram of this block's tile.
// Batch mode (scenes != null): the key is the scene's cell offset plus its local cell.
__global__ void __launch_bounds__(kSortThreads) keys_hist_kernel(int n, const float2* __restrict__ pos,
                                                                 const DeviceMisc* __restrict__ misc,
                                                                 const SceneDev* __restrict__ scenes,
                                                                 const int* __restrict__ slot_scene,
                                                                 uint32_t* __restrict__ keys,
                                                                 uint32_t* __restrict__ hist) {
    pdl_wait();
    __shared__ uint32_t s_hist[kRadixBuckets];
    for (int d = threadIdx.x; d < kRadixBuckets; d += blockDim.x) s_hist[d] = 0;
    __syncthreads();
    int base = blockIdx.x * kSortTile;
#pragma unroll
    for (int c = 0; c < kSortItems; ++c) {
        int i = base + c * kSortThreads + threadIdx.x;
        if (i < n) {
            float2 p = pos[i];
            uint32_t off = 0;
            const GridDev* gp = &misc->grid;
            if (scenes) {
                const SceneDev* sc = scenes + slot_scene[i];
                gp = &sc->grid;
                off = (uint32_t)sc->cell_off;
            }
            const GridDev g = *gp;
            int cx = cell_coord(p.x, g.xmin, g.inv, g.gx);
            int cy = cell_coord(p.y, g.ymin, g.inv, g.gy);
            uint32_t key = off + (uint32_t)cy * (uint32_t)g.gx + (uint32_t)cx;
            keys[i] = key;
            atomicAdd(&s_hist[key & (kRadixBuckets - 1)], 1u);
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadixBuckets; d += blockDim.x)
        hist[d * gridDim.x + blockIdx.x] = s_hist[d];
}

__global__ void __launch_bounds__(kSortThreads) radix_upsweep_kernel(int n, int pass,
                                                                     const DeviceMisc* __restrict__ misc,
                                                                     const uint32_t* __restrict__ keys,
                                                                     uint32_t* __restrict__ hist) {
    pdl_wait();
    if (pass >= misc->grid.passes) return;
    __shared__ uint32_t s_hist[kRadixBuckets];
    for (int d = threadIdx.x; d < kRadixBuckets; d += blockDim.x) s_hist[d] = 0;
    __syncthreads();
    int shift = pass * kRadixBits;
    int base = blockIdx.x * kSortTile;
#pragma unroll
    for (int c = 0; c < kSortItems; ++c) {
        int i = base + c * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&s_hist[(keys[i] >> shift) & (kRadixBuckets - 1)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadixBuckets; d += blockDim.x)
        hist[d * gridDim.x + blockIdx.x] = s_hist[d];
}

// Exclusive scan, in place, of each digit's row hist[d * nblocks + 0..nblocks-1] (one
// warp per digit, kScanWarps digits per CTA), and the digit's total into totals[d].  The
// scan across digits is done by every downsweep block from the 256 totals.
constexpr int kScanWarps = 8;
__global__ void __launch_bounds__(kScanWarps * 32) radix_scan_kernel(int nblocks, int pass,
                                                                     const DeviceMisc* __restrict__ misc,
                                                                     uint32_t* __restrict__ hist,
                                                                     uint32_t* __restrict__ totals) {
    pdl_wait();
    if (pass >= misc->grid.passes) return;
    int lane = threadIdx.x & 31;
    int d = blockIdx.x * kScanWarps + (threadIdx.x >> 5);
    uint32_t run = 0;
    uint32_t* row = hist + (size_t)d * nblocks;
    for (int b0 = 0; b0 < nblocks; b0 += 32) {
        int b = b0 + lane;
        uint32_t v = b < nblocks ? row[b] : 0u;
        uint32_t inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (b < nblocks) row[b] = run + inc - v;
        run += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) totals[d] = run;
}

// Stable scatter of one radix pass.  The tile is walked in order in chunks of one item
// per thread; inside a warp, lanes with equal digits rank themselves with match.any, and
// per-warp digit counts in shared memory order the warps.  vals == nullptr means the
// identity (slot index).
__global__ void __launch_bounds__(kSortThreads) radix_downsweep_kernel(
    int n, int pass, const DeviceMisc* __restrict__ misc, const uint32_t* __restrict__ keys_in,
    const uint32_t* __restrict__ vals_in, uint32_t* __restrict__ keys_out,
    uint32_t* __restrict__ vals_out, const uint32_t* __restrict__ offsets,
    const uint32_t* __restrict__ totals) {
    pdl_wait();
    if (pass >= misc->grid.passes) return;
    constexpr int kWarps = kSortThreads / 32;
    constexpr int kPer = kRadixBuckets / kSortThreads;  // digits per thread below
    static_assert(kRadixBuckets % kSortThreads == 0, "whole digits per thread");
    __shared__ uint32_t s_run[kRadixBuckets];
    __shared__ uint32_t s_wcnt[kWarps][kRadixBuckets];
    __shared__ uint32_t s_wsum[kWarps];
    int warp = threadIdx.x >> 5;
    {
        // base of each digit: exclusive scan of the digit totals (kPer consecutive digits
        // per thread)
        int lane0 = threadIdx.x & 31;
        uint32_t v[kPer], sum = 0;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            v[q] = totals[threadIdx.x * kPer + q];
            sum += v[q];
        }
        uint32_t inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane0 >= o) inc += y;
        }
        if (lane0 == 31) s_wsum[warp] = inc;
        __syncthreads();
        uint32_t base = inc - sum;
        for (int w = 0; w < warp; ++w) base += s_wsum[w];
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            int d = threadIdx.x * kPer + q;
            s_run[d] = base + offsets[d * gridDim.x + blockIdx.x];
            base += v[q];
#pragma unroll
            for (int w = 0; w < kWarps; ++w) s_wcnt[w][d] = 0;
        }
    }
    __syncthreads();
    int shift = pass * kRadixBits;
    int base = blockIdx.x * kSortTile;
    unsigned lt = lanemask_lt();
    for (int c = 0; c < kSortItems; ++c) {
        int i = base + c * kSortThreads + threadIdx.x;
        bool valid = i < n;
        uint32_t key = valid ? keys_in[i] : 0u;
        uint32_t val = valid ? (vals_in ? vals_in[i] : (uint32_t)i) : 0u;
        uint32_t d = (key >> shift) & (kRadixBuckets - 1);
        unsigned vmask = __ballot_sync(0xffffffffu, valid);
        unsigned rank = 0;
        if (valid) {
            unsigned peers = __match_any_sync(vmask, d);
            rank = __popc(peers & lt);
            if ((peers & lt) == 0) s_wcnt[warp][d] = __popc(peers);
        }
        __syncthreads();
        if (valid) {
            uint32_t dst = s_run[d] + rank;
            for (int w = 0; w < warp; ++w) dst += s_wcnt[w][d];
            keys_out[dst] = key;
            vals_out[dst] = val;
        }
        __syncthreads();
        for (int dd = threadIdx.x; dd < kRadixBuckets; dd += blockDim.x) {
            uint32_t tot = 0;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                tot += s_wcnt[w][dd];
                s_wcnt[w][dd] = 0;
            }
            s_run[dd] += tot;
        }
        __syncthreads();
    }
}

// Gather state and parameters into the sorted order; build the message records, the
// id -> slot map and the cell table.  Each thread takes kReorderR slots (blockDim apart)
// and issues all their loads before any store, so that more gathers are in flight.
constexpr int kReorderR = 2;
__global__ void __launch_bounds__(256) reorder_kernel(int n, const uint32_t* __restrict__ vals_a,
                                                      const uint32_t* __restrict__ vals_b,
                                                      const uint32_t* __restrict__ keys_a,
                                                      const uint32_t* __restrict__ keys_b,
                                                      const DeviceMisc* __restrict__ misc,
                                                      uint32_t* __restrict__ cell_start,
                                                      AgentState src_s, Sorted dst_s,
                                                      AgentParams src_p, AgentParams dst_p) {
    pdl_wait();
    const GridDev& g = misc->grid;
    const uint32_t* vals = (g.passes & 1) ? vals_b : vals_a;
    const uint32_t* keys = (g.passes & 1) ? keys_b : keys_a;
    const int t0 = blockIdx.x * blockDim.x * kReorderR + threadIdx.x;
    uint32_t s[kReorderR];
    int prev[kReorderR], cur[kReorderR];
#pragma unroll
    for (int r = 0; r < kReorderR; ++r) {
        int t = t0 + r * blockDim.x;
        bool ok = t < n;
        s[r] = ok ? vals[t] : 0u;
        cur[r] = ok ? (int)keys[t] : 0;
        prev[r] = (ok && t > 0) ? (int)keys[t - 1] : -1;
    }
    float2 p[kReorderR], v[kReorderR], goal[kReorderR];
    float rad[kReorderR], vmax[kReorderR], pref[kReorderR], tau[kReorderR], hint[kReorderR];
    uint32_t id[kReorderR];
#pragma unroll
    for (int r = 0; r < kReorderR; ++r) {
        if (t0 + r * (int)blockDim.x >= n) continue;
        uint32_t q = s[r];
        p[r] = src_s.pos[q];
        v[r] = src_s.vel[q];
        goal[r] = src_p.goal[q];
        rad[r] = src_p.radius[q];
        vmax[r] = src_p.max_speed[q];
        pref[r] = src_p.pref_speed[q];
        tau[r] = src_p.tau[q];
        id[r] = src_p.id[q];
        hint[r] = dst_p.hint ? src_p.hint[q] : 0.0f;
    }
#pragma unroll
    for (int r = 0; r < kReorderR; ++r) {
        int t = t0 + r * blockDim.x;
        if (t >= n) continue;
        dst_s.msg[t] = make_float4(p[r].x, p[r].y, rad[r], __uint_as_float(id[r]));
        dst_s.slot[id[r]] = (uint32_t)t;
        dst_s.vel[t] = v[r];
        dst_p.goal[t] = goal[r];
        dst_p.radius[t] = rad[r];
        dst_p.max_speed[t] = vmax[r];
        dst_p.pref_speed[t] = pref[r];
        dst_p.tau[t] = tau[r];
        dst_p.id[t] = id[r];
        if (dst_p.hint) dst_p.hint[t] = hint[r];
        // cell table: slot t starts every cell in (key[t-1], key[t]]; the last slot also
        // closes the cells after its own with cell_start = n
        for (int c = prev[r] + 1; c <= cur[r]; ++c) cell_start[c] = (uint32_t)t;
        if (t == n - 1)
            for (int c = cur[r] + 1; c <= g.num_cells; ++c) cell_start[c] = (uint32_t)n;
    }
}

// State back to agent order (readout).
__global__ void __launch_bounds__(256) unpermute_kernel(int n, AgentState s, const uint32_t* __restrict__ id,
                                                        float2* __restrict__ pos_out,
                                                        float2* __restrict__ vel_out) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    uint32_t i = id[t];
    if (pos_out) pos_out[i] = s.pos[t];
    if (vel_out) vel_out[i] = s.vel[t];
}

// The inverse of unpermute: agent-order arrays into the current slots (either may be null).
__global__ void __launch_bounds__(256) permute_kernel(int n, AgentState s, const uint32_t* __restrict__ id,
                                                      const float2* __restrict__ pos_in,
                                                      const float2* __restrict__ vel_in) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    uint32_t i = id[t];
    if (pos_in) s.pos[t] = pos_in[i];
    if (vel_in) s.vel[t] = vel_in[i];
}

// Agent -> slot map from the slot -> agent ids.
__global__ void __launch_bounds__(256) slot_map_kernel(int n, const uint32_t* __restrict__ id,
                                                       uint32_t* __restrict__ slot_of) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) slot_of[id[t]] = (uint32_t)t;
}

// State to or from agent-order arrays that live in pinned host memory, read or written by
// the kernel over the CPU-GPU link: two agents per thread, so the host side moves in
// contiguous 16-byte pieces (arrays 16-byte aligned) and the scattered side is device
// memory.  to_host: agent arrays <- slots, else slots <- agent arrays.  Null arrays are
// skipped.
__global__ void __launch_bounds__(256) host_state_kernel(int n, AgentState s,
                                                         const uint32_t* __restrict__ slot_of,
                                                         float2* pos, float2* vel, int to_host) {
    const int i = 2 * (int)(blockIdx.x * blockDim.x + threadIdx.x);
    if (i >= n) return;
    if (i + 1 < n) {
        const uint2 t = *reinterpret_cast<const uint2*>(slot_of + i);
        if (to_host) {
            if (pos) {
                const float2 a = s.pos[t.x], b = s.pos[t.y];
                *reinterpret_cast<float4*>(pos + i) = make_float4(a.x, a.y, b.x, b.y);
            }
            if (vel) {
                const float2 a = s.vel[t.x], b = s.vel[t.y];
                *reinterpret_cast<float4*>(vel + i) = make_float4(a.x, a.y, b.x, b.y);
            }
        } else {
            if (pos) {
                const float4 q = *reinterpret_cast<const float4*>(pos + i);
                s.pos[t.x] = make_float2(q.x, q.y);
                s.pos[t.y] = make_float2(q.z, q.w);
            }
            if (vel) {
                const float4 q = *reinterpret_cast<const float4*>(vel + i);
                s.vel[t.x] = make_float2(q.x, q.y);
                s.vel[t.y] = make_float2(q.z, q.w);
            }
        }
        return;
    }
    const uint32_t t = slot_of[i];  // the last agent of an odd count
    if (to_host) {
        if (pos) pos[i] = s.pos[t];
        if (vel) vel[i] = s.vel[t];
    } else {
        if (pos) s.pos[t] = pos[i];
        if (vel) s.vel[t] = vel[i];
    }
}

__global__ void __launch_bounds__(256) iota_kernel(int n, uint32_t* __restrict__ id) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < n) id[t] = (uint32_t)t;
}

// ---------------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------------
int sort_blocks(int n) { return (n + kSortTile - 1) / kSortTile; }

cudaError_t launch_radix_passes(int n, int nsb, int max_passes, const BinBuffers& b, cudaStream_t st);

cudaError_t launch_binning(int n, float cell_size, long long max_cells, int max_passes,
                           const AgentState& cur, const BinBuffers& b, cudaStream_t st) {
    int nb_bbox = (n + 255) / 256;
    if (nb_bbox > kBboxBlocks) nb_bbox = kBboxBlocks;
    bbox_grid_kernel<<<nb_bbox, 256, 0, st>>>(n, cur.pos, cell_size, max_cells, max_passes,
                                              b.bbox_partials, b.misc);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int nsb = sort_blocks(n);
    e = launch_pdl(keys_hist_kernel, nsb, kSortThreads, 0, st, n, (const float2*)cur.pos,
                   (const DeviceMisc*)b.misc, (const SceneDev*)nullptr, (const int*)nullptr,
                   b.keys[0], b.hist);
    if (e != cudaSuccess) return e;
    return launch_radix_passes(n, nsb, max_passes, b, st);
}

// Radix passes over the keys written by keys_hist (the reorder kernel builds the cell table).
cudaError_t launch_radix_passes(int n, int nsb, int max_passes, const BinBuffers& b, cudaStream_t st) {
    const DeviceMisc* misc = b.misc;
    for (int pass = 0; pass < max_passes; ++pass) {
        int src = pass & 1, dst = src ^ 1;
        cudaError_t e = cudaSuccess;
        if (pass > 0)
            e = launch_pdl(radix_upsweep_kernel, nsb, kSortThreads, 0, st, n, pass, misc,
                           (const uint32_t*)b.keys[src], b.hist);
        if (e == cudaSuccess)
            e = launch_pdl(radix_scan_kernel, kRadixBuckets / kScanWarps, kScanWarps * 32, 0, st, nsb,
                           pass, misc, b.hist, b.digit_totals);
        if (e == cudaSuccess)
            e = launch_pdl(radix_downsweep_kernel, nsb, kSortThreads, 0, st, n, pass, misc,
                           (const uint32_t*)b.keys[src],
                           (const uint32_t*)(pass == 0 ? nullptr : b.vals[src]), b.keys[dst],
                           b.vals[dst], (const uint32_t*)b.hist, (const uint32_t*)b.digit_totals);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_reorder(int n, const BinBuffers& b, const AgentState& src_s,
                           const Sorted& dst_s, const AgentParams& src_p,
                           const AgentParams& dst_p, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    return launch_pdl(reorder_kernel, (n + 256 * kReorderR - 1) / (256 * kReorderR), 256, 0, st, n,
                      (const uint32_t*)b.vals[0], (const uint32_t*)b.vals[1],
                      (const uint32_t*)b.keys[0], (const uint32_t*)b.keys[1],
                      (const DeviceMisc*)b.misc, b.cell_start, src_s, dst_s, src_p, dst_p);
}

cudaError_t launch_unpermute(int n, const AgentState& s, const uint32_t* id, float2* pos_out,
                             float2* vel_out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    unpermute_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, s, id, pos_out, vel_out);
    return cudaGetLastError();
}

cudaError_t launch_permute(int n, const AgentState& s, const uint32_t* id, const float2* pos_in,
                           const float2* vel_in, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    permute_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, s, id, pos_in, vel_in);
    return cudaGetLastError();
}

cudaError_t launch_host_state(int n, const AgentState& s, const uint32_t* id, uint32_t* slot_of,
                              bool build_map, float2* pos, float2* vel, bool to_host, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    if (build_map) slot_map_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, id, slot_of);
    const int pairs = (n + 1) / 2;
    host_state_kernel<<<(pairs + 255) / 256, 256, 0, st>>>(n, s, slot_of, pos, vel, to_host ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_iota(int n, uint32_t* id, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    iota_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, id);
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------------
// Batch of independent scenes
// ---------------------------------------------------------------------------------
// Bounding box and grid of each scene: one CTA per scene over its slot range.
__global__ void __launch_bounds__(1024) scene_bbox_grid_kernel(const float2* __restrict__ pos,
                                                               SceneDev* scenes, int max_passes,
                                                               DeviceMisc* misc) {
    pdl_wait();
    SceneDev* sc = scenes + blockIdx.x;
    const int off = sc->off, cnt = sc->cnt;
    float4 r = make_float4(INFINITY, INFINITY, -INFINITY, -INFINITY);
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        float2 p = pos[off + i];
        r.x = fminf(r.x, p.x);
        r.y = fminf(r.y, p.y);
        r.z = fmaxf(r.z, p.x);
        r.w = fmaxf(r.w, p.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        r.x = fminf(r.x, __shfl_xor_sync(0xffffffffu, r.x, o));
        r.y = fminf(r.y, __shfl_xor_sync(0xffffffffu, r.y, o));
        r.z = fmaxf(r.z, __shfl_xor_sync(0xffffffffu, r.z, o));
        r.w = fmaxf(r.w, __shfl_xor_sync(0xffffffffu, r.w, o));
    }
    __shared__ float4 s_part[32];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) s_part[warp] = r;
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
        r.x = fminf(r.x, s_part[w].x);
        r.y = fminf(r.y, s_part[w].y);
        r.z = fmaxf(r.z, s_part[w].z);
        r.w = fmaxf(r.w, s_part[w].w);
    }
    if (cnt == 0) r = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    float cs = sc->cell_size > 0.0f ? sc->cell_size : sc->nd * 0.25f;
    int err = 0;
    sc->grid = derive_grid(r, cs, sc->cell_budget, max_passes, &err);
    if (err) atomicOr(&misc->error, err);
}

// Cell offsets of the scenes (exclusive scan of their cell counts), the total and the
// radix passes it needs; resets the persistent kernel's tile counter.
__global__ void __launch_bounds__(1024) scene_prefix_kernel(int n_scenes, SceneDev* scenes,
                                                            int max_passes, DeviceMisc* misc) {
    pdl_wait();
    __shared__ long long s_sum[1024];
    int per = (n_scenes + blockDim.x - 1) / blockDim.x;
    int s0 = threadIdx.x * per, s1 = min(s0 + per, n_scenes);
    long long sum = 0;
    for (int q = s0; q < s1; ++q) sum += scenes[q].grid.num_cells;
    s_sum[threadIdx.x] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long run = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            long long v = s_sum[t];
            s_sum[t] = run;
            run += v;
        }
        int bits = 0;
        while (bits < 31 && (1LL << bits) < run) ++bits;
        int passes = (bits + kRadixBits - 1) / kRadixBits;
        misc->grid.num_cells = (int)run;
        misc->grid.passes = passes < 1 ? 1 : (passes > max_passes ? max_passes : passes);
        misc->tile_counter = 0;
    }
    __syncthreads();
    long long run = s_sum[threadIdx.x];
    for (int q = s0; q < s1; ++q) {
        scenes[q].cell_off = (int)run;
        run += scenes[q].grid.num_cells;
    }
}

// Scene of every slot: the first scene whose slot range ends after it (binary search;
// the ends are non-decreasing, and empty scenes own no slot).
__global__ void __launch_bounds__(256) slot_scene_kernel(int n, int n_scenes,
                                                         const SceneDev* __restrict__ scenes,
                                                         int* __restrict__ slot_scene) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int lo = 0, hi = n_scenes - 1;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (scenes[mid].off + scenes[mid].cnt > t) hi = mid;
        else lo = mid + 1;
    }
    slot_scene[t] = lo;
}

cudaError_t launch_slot_scene(int n, int n_scenes, const SceneDev* scenes, int* slot_scene,
                              cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    slot_scene_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, n_scenes, scenes, slot_scene);
    return cudaGetLastError();
}

cudaError_t launch_binning_batch(int n, int n_scenes, SceneDev* scenes, const int* slot_scene,
                                 int max_passes, const AgentState& cur, const BinBuffers& b,
                                 cudaStream_t st) {
    scene_bbox_grid_kernel<<<n_scenes, 1024, 0, st>>>(cur.pos, scenes, max_passes, b.misc);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
        e = launch_pdl(scene_prefix_kernel, 1, 1024, 0, st, n_scenes, scenes, max_passes, b.misc);
    int nsb = sort_blocks(n);
    if (e == cudaSuccess)
        e = launch_pdl(keys_hist_kernel, nsb, kSortThreads, 0, st, n, (const float2*)cur.pos,
                       (const DeviceMisc*)b.misc, (const SceneDev*)scenes, slot_scene, b.keys[0],
                       b.hist);
    if (e != cudaSuccess) return e;
    return launch_radix_passes(n, nsb, max_passes, b, st);
}

}  // namespace orca
