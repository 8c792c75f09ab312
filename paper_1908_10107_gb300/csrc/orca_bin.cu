// orca_bin.cu -- spatial binning of the crowd (Fig. 2: "messages organised into bins").
//
// Per step, on one stream, with no host round trip, four kernels:
//   bbox_grid    exact min/max of positions -> grid descriptor (cell edge, gx, gy).
//   keys_count   cell key of every agent, and its rank among the agents of its cell: one
//                atomic increment of the cell's count per group of warp lanes that share
//                the cell; the count of every tile of kCellTile cells likewise.
//   cell_scan    the cell table cell_start[c] = agents in cells before c, for every c in
//                [0, num_cells] (empty cells included): an exclusive scan of the counts in
//                tiles of kCellTile cells, each CTA starting from the sum of the earlier
//                tiles' counts; it clears the counts for the next step.
//   reorder      every agent goes to slot cell_start[key] + rank: state and parameters
//                are read in the previous order (coalesced) and written to the new slot
//                with the message record and the id -> slot map.
//
// This is a counting sort by cell (one pass over the agents, one over the cells).  The
// order inside a cell follows the atomic increments and so varies from run to run;
// nothing computed depends on it: neighbours are ranked by (distance, agent index), and
// every agent's result is a function of its own neighbour list alone.
#include "orca_common.cuh"

namespace orca {

// Grid over a bounding box r = (xmin, ymin, xmax, ymax), all in FP32:
// inv = fl(1/s), g = floor(fl(fl(max - min) * inv)) + 1, doubling s while gx*gy exceeds
// max_cells.  A non-finite or absurd extent puts everything in one cell and sets *err.
__device__ GridDev derive_grid(float4 r, float cell_size, long long max_cells, int* err) {
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
// Reset the box slot the step's ORCA kernel will fill and mark it as coming; called by
// the first warp of one block (lane q resets copy q).
__device__ __forceinline__ void open_next_box(DeviceMisc* misc, int slot, int lane) {
    for (int q = lane; q < kBoxCopies; q += 32) {
        int* acc = misc->bbox_acc[slot ^ 1] + q * kBoxStride;
        acc[0] = acc[1] = float_order_code(INFINITY);
        acc[2] = acc[3] = float_order_code(-INFINITY);
    }
    if (lane == 0) misc->bbox_ok[slot ^ 1] = 1u;
}

__global__ void __launch_bounds__(256) bbox_grid_kernel(int n, const float2* __restrict__ pos,
                                                        float cell_size, long long max_cells,
                                                        float4* partials, DeviceMisc* misc,
                                                        int slot) {
    pdl_wait();
    // The previous step's ORCA kernel reduced the box of the positions it wrote: use it
    // (the min / max are exact, so the grid is the one a scan would give).
    if (slot >= 0 && misc->bbox_ok[slot]) {
        if (blockIdx.x == 0 && threadIdx.x < 32) {
            const int lane = threadIdx.x;
            int c0 = float_order_code(INFINITY), c1 = c0, c2 = float_order_code(-INFINITY), c3 = c2;
            for (int q = lane; q < kBoxCopies; q += 32) {
                const int* acc = misc->bbox_acc[slot] + q * kBoxStride;
                c0 = min(c0, acc[0]);
                c1 = min(c1, acc[1]);
                c2 = max(c2, acc[2]);
                c3 = max(c3, acc[3]);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                c0 = min(c0, __shfl_xor_sync(0xffffffffu, c0, o));
                c1 = min(c1, __shfl_xor_sync(0xffffffffu, c1, o));
                c2 = max(c2, __shfl_xor_sync(0xffffffffu, c2, o));
                c3 = max(c3, __shfl_xor_sync(0xffffffffu, c3, o));
            }
            open_next_box(misc, slot, lane);
            if (lane == 0) {
                const float4 r = make_float4(float_from_order_code(c0), float_from_order_code(c1),
                                             float_from_order_code(c2), float_from_order_code(c3));
                misc->bbox_ticket = 0;
                misc->tile_counter = 0;
                misc->obs_tiles = 0;
                int err = 0;
                misc->grid = derive_grid(r, cell_size, max_cells, &err);
                if (err) atomicOr(&misc->error, err);
            }
        }
        return;
    }
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
    if (slot >= 0 && threadIdx.x < 32) open_next_box(misc, slot, threadIdx.x);
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
    misc->grid = derive_grid(r, cell_size, max_cells, &err);
    if (err) atomicOr(&misc->error, err);
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Cell key of every agent and its rank among the agents of its cell.  Lanes of a warp
// that share a cell (agents arrive in the previous step's cell order, so neighbouring
// lanes mostly do) take one atomic on the cell's count: the leader adds the group's size
// and every lane's rank is the leader's old count plus the group's lanes below it.  The
// tile counts for the scan are gathered the same way.  Lanes past the crowd carry an
// impossible key, so every lane of a warp takes part in the warp primitives.
// Batch mode (scenes != null): the key is the scene's cell offset plus its local cell.
__global__ void __launch_bounds__(256) keys_count_kernel(int n, const float2* __restrict__ pos,
                                                         const DeviceMisc* __restrict__ misc,
                                                         const SceneDev* __restrict__ scenes,
                                                         const int* __restrict__ slot_scene,
                                                         uint32_t* __restrict__ keys,
                                                         uint32_t* __restrict__ ranks,
                                                         uint32_t* cnt, uint32_t* tile_sums,
                                                         long long table_cells) {
    pdl_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = i < n;
    uint32_t key = 0xffffffffu;
    if (valid) {
        const float2 p = pos[i];
        uint32_t off = 0;
        const GridDev* gp = &misc->grid;
        if (scenes) {
            const SceneDev* sc = scenes + slot_scene[i];
            gp = &sc->grid;
            off = (uint32_t)sc->cell_off;
        }
        const GridDev g = *gp;
        const int cx = cell_coord(p.x, g.xmin, g.inv, g.gx);
        const int cy = cell_coord(p.y, g.ymin, g.inv, g.gy);
        key = off + (uint32_t)cy * (uint32_t)g.gx + (uint32_t)cx;
        if (!idx_ok((long long)key < table_cells, const_cast<int*>(&misc->error))) key = 0u;
        keys[i] = key;
    }
    const int lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (valid && lane == leader) base = atomicAdd(cnt + key, (uint32_t)__popc(peers));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (valid) ranks[i] = base + (uint32_t)__popc(peers & lt);
    // tile counts: the block's agents come in the previous step's cell order, so their
    // keys mostly fall in a few consecutive tiles from the tile of the block's first agent;
    // those are counted in shared memory and added with one atomic each, the rest directly
    constexpr int kSlots = 4;
    __shared__ uint32_t s_tc[kSlots];
    __shared__ uint32_t s_t0;
    if (threadIdx.x < kSlots) s_tc[threadIdx.x] = 0u;
    if (threadIdx.x == 0) s_t0 = valid ? key / (uint32_t)kCellTile : 0u;
    __syncthreads();
    const uint32_t tile = valid ? key / (uint32_t)kCellTile : 0xffffffffu;
    const unsigned tp = __match_any_sync(0xffffffffu, tile);
    if (valid && lane == __ffs(tp) - 1) {
        const uint32_t slot = tile - s_t0;  // wraps to a large value below the first tile
        if (slot < (uint32_t)kSlots) atomicAdd(s_tc + slot, (uint32_t)__popc(tp));
        else atomicAdd(tile_sums + (size_t)tile * kTileSumStride, (uint32_t)__popc(tp));
    }
    __syncthreads();
    if (threadIdx.x < kSlots && s_tc[threadIdx.x])
        atomicAdd(tile_sums + (size_t)(s_t0 + threadIdx.x) * kTileSumStride, s_tc[threadIdx.x]);
}

// Block-wide exclusive scan (kCellScanThreads threads) of one value per thread; also
// returns the block total through `total`.
__device__ __forceinline__ uint32_t cell_block_scan(uint32_t v, uint32_t& total) {
    __shared__ uint32_t s_warp[kCellScanThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    uint32_t base = 0;
    total = 0;
#pragma unroll
    for (int w = 0; w < kCellScanThreads / 32; ++w) {
        const uint32_t sw = s_warp[w];
        if (w < warp) base += sw;
        total += sw;
    }
    __syncthreads();
    return base + inc - v;
}

// The cell table from the counts, tiles of kCellTile cells (kCellsPerThread consecutive
// cells per thread, read and written as 16-byte vectors): a tile starts at the sum of the
// earlier tiles' counts (keys_count gathered them), then an exclusive scan inside the
// tile.  The counts are cleared on the way for the next step, and the thread whose range
// holds num_cells closes the table with cell_start[num_cells] = n.  CTA b takes tiles b,
// b + gridDim.x, ... up to the grid's last one (the launch is sized for the table's
// capacity, capped at two CTAs per SM, so a small grid costs few idle CTAs).
__global__ void __launch_bounds__(kCellScanThreads) cell_scan_kernel(int n, const DeviceMisc* __restrict__ misc,
                                                                     uint32_t* __restrict__ cnt,
                                                                     const uint32_t* __restrict__ tile_sums,
                                                                     uint32_t* __restrict__ cell_start) {
    pdl_wait();
    const long long nc = misc->grid.num_cells;
#pragma unroll 1
    for (int tile = blockIdx.x; (long long)tile * kCellTile <= nc; tile += gridDim.x) {
        uint32_t pre = 0, tot = 0;
        for (int b = threadIdx.x; b < tile; b += kCellScanThreads) pre += tile_sums[(size_t)b * kTileSumStride];
        (void)cell_block_scan(pre, tot);  // every thread gets the sum of the earlier tiles
        pre = tot;
        const long long c0 = (long long)tile * kCellTile + (long long)threadIdx.x * kCellsPerThread;
        const bool full = c0 + kCellsPerThread <= nc;
        uint32_t v[kCellsPerThread];
        if (full) {
            const uint4* src = reinterpret_cast<const uint4*>(cnt + c0);
#pragma unroll
            for (int q = 0; q < kCellsPerThread / 4; ++q) {
                const uint4 w = src[q];
                v[4 * q] = w.x;
                v[4 * q + 1] = w.y;
                v[4 * q + 2] = w.z;
                v[4 * q + 3] = w.w;
            }
        } else {
#pragma unroll
            for (int q = 0; q < kCellsPerThread; ++q) v[q] = c0 + q < nc ? cnt[c0 + q] : 0u;
        }
        uint32_t sum = 0;
#pragma unroll
        for (int q = 0; q < kCellsPerThread; ++q) sum += v[q];
        uint32_t run = pre + cell_block_scan(sum, tot);
#pragma unroll
        for (int q = 0; q < kCellsPerThread; ++q) {
            const uint32_t c = v[q];
            v[q] = run;
            run += c;
        }
        if (full) {
            uint4* dst = reinterpret_cast<uint4*>(cell_start + c0);
            uint4* clr = reinterpret_cast<uint4*>(cnt + c0);
#pragma unroll
            for (int q = 0; q < kCellsPerThread / 4; ++q) {
                dst[q] = make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                clr[q] = make_uint4(0u, 0u, 0u, 0u);
            }
        } else {
#pragma unroll
            for (int q = 0; q < kCellsPerThread; ++q)
                if (c0 + q < nc) {
                    cell_start[c0 + q] = v[q];
                    cnt[c0 + q] = 0u;
                }
        }
        if (c0 <= nc && nc < c0 + kCellsPerThread) cell_start[nc] = (uint32_t)n;
    }
}

// Every agent to its slot cell_start[key] + rank: state and parameters read at the old
// slot (coalesced), written to the new one with the message record and the id -> slot
// map.  Each thread takes kReorderR agents (blockDim apart) and issues all their loads
// before any store, so that more loads are in flight.  Block 0 first clears the tile
// counts, which the cell scan (complete before this kernel starts) no longer needs.
constexpr int kReorderR = 2;
__global__ void __launch_bounds__(256) reorder_kernel(int n, const uint32_t* __restrict__ keys,
                                                      const uint32_t* __restrict__ ranks,
                                                      DeviceMisc* misc,
                                                      const uint32_t* __restrict__ cell_start,
                                                      uint32_t* __restrict__ tile_sums,
                                                      AgentState src_s, Sorted dst_s,
                                                      AgentParams src_p, AgentParams dst_p) {
    pdl_wait();
    if (blockIdx.x == 0) {
        const int tiles = misc->grid.num_cells / kCellTile + 1;
        for (int b = threadIdx.x; b < tiles; b += blockDim.x) tile_sums[(size_t)b * kTileSumStride] = 0u;
    }
    const int i0 = blockIdx.x * blockDim.x * kReorderR + threadIdx.x;
    uint32_t t[kReorderR];
    float2 p[kReorderR], v[kReorderR], goal[kReorderR];
    float rad[kReorderR], vmax[kReorderR], pref[kReorderR], tau[kReorderR], hint[kReorderR];
    uint32_t id[kReorderR];
#pragma unroll
    for (int r = 0; r < kReorderR; ++r) {
        const int i = i0 + r * blockDim.x;
        if (i >= n) continue;
        t[r] = cell_start[keys[i]] + ranks[i];
        p[r] = src_s.pos[i];
        v[r] = src_s.vel[i];
        goal[r] = src_p.goal[i];
        rad[r] = src_p.radius[i];
        vmax[r] = src_p.max_speed[i];
        pref[r] = src_p.pref_speed[i];
        tau[r] = src_p.tau[i];
        id[r] = src_p.id[i];
        hint[r] = dst_p.hint ? src_p.hint[i] : 0.0f;
    }
#pragma unroll
    for (int r = 0; r < kReorderR; ++r) {
        if (i0 + r * (int)blockDim.x >= n) continue;
        const uint32_t q = t[r];
        if (q >= (uint32_t)n) {  // counts that do not add up (never in a consistent step)
            atomicOr(&misc->error, kErrCapacity);
            continue;
        }
        dst_s.msg[q] = make_float4(p[r].x, p[r].y, rad[r], __uint_as_float(id[r]));
        dst_s.slot[id[r]] = q;
        dst_s.vel[q] = v[r];
        dst_p.goal[q] = goal[r];
        dst_p.radius[q] = rad[r];
        dst_p.max_speed[q] = vmax[r];
        dst_p.pref_speed[q] = pref[r];
        dst_p.tau[q] = tau[r];
        dst_p.id[q] = id[r];
        if (dst_p.hint) dst_p.hint[q] = hint[r];
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
// CTAs of the cell scan: one per tile of the largest grid the table holds, at most two per
// SM (152 SMs; each CTA loops over its tiles).
static int scan_blocks(long long table_cells) {
    const long long tiles = table_cells / kCellTile + 1;
    return (int)(tiles < 304 ? tiles : 304);
}

// keys_count, cell_scan (the grid and the bounding box are already in misc).
static cudaError_t launch_counting_sort(int n, const SceneDev* scenes, const int* slot_scene,
                                       const AgentState& cur, const BinBuffers& b, cudaStream_t st) {
    cudaError_t e = launch_pdl(keys_count_kernel, (n + 255) / 256, 256, 0, st, n, (const float2*)cur.pos,
                               (const DeviceMisc*)b.misc, scenes, slot_scene, b.keys[0], b.vals[0],
                               b.cnt, b.tile_sums, b.table_cells);
    if (e != cudaSuccess) return e;
    return launch_pdl(cell_scan_kernel, scan_blocks(b.table_cells), kCellScanThreads, 0, st, n,
                      (const DeviceMisc*)b.misc, b.cnt, (const uint32_t*)b.tile_sums, b.cell_start);
}

cudaError_t launch_binning(int n, float cell_size, long long max_cells, const AgentState& cur,
                           const BinBuffers& b, int slot, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int nb_bbox = (n + 255) / 256;
    if (nb_bbox > kBboxBlocks) nb_bbox = kBboxBlocks;
    bbox_grid_kernel<<<nb_bbox, 256, 0, st>>>(n, cur.pos, cell_size, max_cells, b.bbox_partials, b.misc,
                                              slot);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_counting_sort(n, nullptr, nullptr, cur, b, st);
}

cudaError_t launch_reorder(int n, const BinBuffers& b, const AgentState& src_s,
                           const Sorted& dst_s, const AgentParams& src_p,
                           const AgentParams& dst_p, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    return launch_pdl(reorder_kernel, (n + 256 * kReorderR - 1) / (256 * kReorderR), 256, 0, st, n,
                      (const uint32_t*)b.keys[0], (const uint32_t*)b.vals[0], b.misc,
                      (const uint32_t*)b.cell_start, b.tile_sums, src_s, dst_s, src_p, dst_p);
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
// Bounding box and grid of each scene, one CTA per scene: from the box the previous
// step's ORCA kernel reduced into the scene's slot `slot` when that slot is complete, else
// a min / max scan of the scene's positions.  The CTA opens the other slot for this step's
// ORCA kernel.  The last CTA to finish (ticket counter, no waiting) then lays the scenes'
// cell ranges end to end: cell_off of every scene and the table's total.
constexpr int kSceneThreads = 1024;
__global__ void __launch_bounds__(kSceneThreads) scene_bbox_grid_kernel(const float2* __restrict__ pos,
                                                                        int n_scenes, SceneDev* scenes,
                                                                        DeviceMisc* misc, int slot) {
    pdl_wait();
    SceneDev* sc = scenes + blockIdx.x;
    const int off = sc->off, cnt = sc->cnt;
    __shared__ float4 s_part[kSceneThreads / 32];
    __shared__ bool s_last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4 r = make_float4(INFINITY, INFINITY, -INFINITY, -INFINITY);
    if (slot >= 0 && sc->box_ok[slot]) {
        if (threadIdx.x == 0) {
            const int* c = sc->box_acc[slot];
            r = make_float4(float_from_order_code(c[0]), float_from_order_code(c[1]),
                            float_from_order_code(c[2]), float_from_order_code(c[3]));
        }
    } else {
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
        if (lane == 0) s_part[warp] = r;
        __syncthreads();
        if (threadIdx.x == 0)
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
                r.x = fminf(r.x, s_part[w].x);
                r.y = fminf(r.y, s_part[w].y);
                r.z = fmaxf(r.z, s_part[w].z);
                r.w = fmaxf(r.w, s_part[w].w);
            }
    }
    if (threadIdx.x == 0) {
        if (cnt == 0) r = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        float cs = sc->cell_size > 0.0f ? sc->cell_size : sc->nd * 0.25f;
        int err = 0;
        sc->grid = derive_grid(r, cs, sc->cell_budget, &err);
        if (err) atomicOr(&misc->error, err);
        if (slot >= 0) {  // the slot this step's ORCA kernel fills
            int* c = sc->box_acc[slot ^ 1];
            c[0] = c[1] = float_order_code(INFINITY);
            c[2] = c[3] = float_order_code(-INFINITY);
            sc->box_ok[slot ^ 1] = 1u;
        }
        __threadfence();
        s_last = atomicAdd(&misc->bbox_ticket, 1u) == (unsigned)gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    // last CTA: exclusive scan of the scenes' cell counts (kSceneThreads-wide, in rounds)
    __threadfence();
    __shared__ long long s_w[kSceneThreads / 32];
    __shared__ long long s_base;
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    for (int q0 = 0; q0 < n_scenes; q0 += kSceneThreads) {
        const int q = q0 + threadIdx.x;
        const long long v = q < n_scenes ? (long long)__ldcg(&scenes[q].grid.num_cells) : 0;
        long long inc = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) s_w[warp] = inc;
        __syncthreads();
        long long wb = 0, tot = 0;
        for (int w = 0; w < kSceneThreads / 32; ++w) {
            if (w < warp) wb += s_w[w];
            tot += s_w[w];
        }
        if (q < n_scenes) scenes[q].cell_off = (int)(s_base + wb + inc - v);
        __syncthreads();
        if (threadIdx.x == 0) s_base += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        misc->grid.num_cells = (int)s_base;
        misc->tile_counter = 0;
        misc->bbox_ticket = 0;
    }
}

__global__ void __launch_bounds__(256) clear_scene_boxes_kernel(int n_scenes, SceneDev* scenes) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n_scenes) scenes[q].box_ok[0] = scenes[q].box_ok[1] = 0u;
}

cudaError_t launch_clear_scene_boxes(int n_scenes, SceneDev* scenes, cudaStream_t st) {
    if (n_scenes <= 0) return cudaSuccess;
    clear_scene_boxes_kernel<<<(n_scenes + 255) / 256, 256, 0, st>>>(n_scenes, scenes);
    return cudaGetLastError();
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
                                 const AgentState& cur, const BinBuffers& b, int slot, cudaStream_t st) {
    scene_bbox_grid_kernel<<<n_scenes, kSceneThreads, 0, st>>>(cur.pos, n_scenes, scenes, b.misc, slot);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || n <= 0) return e;
    return launch_counting_sort(n, scenes, slot_scene, cur, b, st);
}

}  // namespace orca
