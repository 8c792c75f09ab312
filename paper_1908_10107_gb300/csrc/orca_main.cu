// orca_main.cu -- per-agent ORCA velocity selection and integration (Sections 2-3).
//
// One CTA of TPB threads (64 to 256) takes TPB consecutive agents of the cell order, so its agents
// are spatial neighbours and their candidate reads overlap in L1/L2.  Phases:
//   1. (thread per agent) exact k nearest neighbours by (fl32 d^2, agent index) among
//      agents strictly inside r_obs (Fig. 2), by a ring search over grid cells with
//      conservative per-cell and per-ring distance bounds; then one ORCA half-plane per
//      neighbour (Fig. 1) written to the agent's row of shared memory;
//   2. (thread per agent) LP2 -- incremental 2-D LP over the disc and the half-planes in
//      neighbour order; agents whose LP2 fails are appended to a per-CTA queue;
//   3. LP3 -- least penetration (Section 3) -- for the queued agents, a group of G lanes
//      per agent, so the whole CTA works on the queue instead of idling the lanes whose
//      LP2 succeeded;
//   4. vel <- x, pos <- pos + x*dt into the same sorted slot of the state buffer.
// Half-planes never leave the SM (the paper stores them in global memory, Section 5).
#include "orca_geom.cuh"

namespace orca {

// A half-plane in normal form: the valid side is {x : n.x >= c}, |n| = 1.  In the
// paper's point-and-direction form (boundary through P with direction d, valid side on
// the left of d) this is n = (-d.y, d.x) and c = n.P.  The normal form keeps every LP1
// computation at the scale of the speed disc: the boundary point nearest the origin is
// c*n, and a line with |c| > V misses the disc before any large number is formed; the
// least-penetration bisectors need no intersection points (which can lie far away).
// Stored as float4 (nx, ny, c, unused).


// Algorithmic operation counts of the LP (operation-counting launches only): LP1 calls,
// LP1 bounds evaluated, violation checks (LP2 and LP3 scans), LP3 bisectors formed -- the
// quantities the oracle counts, for the kernel's arithmetic roofline.
struct OpCount {
    unsigned lp1, bounds, checks, bis;
};

// What the neighbour searches cost (every launch): passes beyond the first (a start radius
// that held fewer than k agents inside r_obs, grown 1.5x), searches that started without a
// prediction, grid rows scanned.
struct SearchCount {
    unsigned retries, cold, rows;
};

struct LpTape {
    int mode, i, f, bound, j, side;
    __device__ __forceinline__ unsigned pack() const {
        return (unsigned)mode | (unsigned)i << 3 | (unsigned)f << 9 | (unsigned)bound << 15 |
               (unsigned)j << 17 | (unsigned)side << 23;
    }
};

// The LP's arithmetic with every rounding spelled out (explicit fused and unfused
// operations, no contraction left to the compiler), so that the one-lane and the
// lane-group LP3 -- different code around the same formulas -- round identically and
// take the same decisions.
__device__ __forceinline__ float lp_dot(float ax, float ay, float bx, float by) {
    return __fmaf_rn(ax, bx, __fmul_rn(ay, by));
}
__device__ __forceinline__ float lp_det(float ax, float ay, float bx, float by) {
    return __fmaf_rn(ax, by, -__fmul_rn(ay, bx));
}
// Violation of half-plane l at x: c - n.x (> 0: x is outside).
__device__ __forceinline__ float lp_viol(float4 l, float x, float y) {
    return __fsub_rn(l.z, lp_dot(l.x, l.y, x, y));
}
// c_j - c_i (n_i.n_j): LP1's right-hand side for bounding line j on base line i.
__device__ __forceinline__ float lp_rhs(float4 li, float4 lj) {
    return __fmaf_rn(-li.z, lp_dot(li.x, li.y, lj.x, lj.y), lj.z);
}
// The point c n + t d of a unit line (d = (n.y, -n.x)).
__device__ __forceinline__ float2 lp_point(float4 l, float t) {
    return make_float2(__fmaf_rn(t, l.y, __fmul_rn(l.z, l.x)),
                       __fmaf_rn(t, -l.x, __fmul_rn(l.z, l.y)));
}

// Line j is (nearly) parallel to the unit line it bounds: |det| <= eps |n_j| (|n_j| = 1
// for unit lines; squares otherwise, no root).
template <bool kUnit>
__device__ __forceinline__ bool parallel_to(float den, float4 lj) {
    if (kUnit) return fabsf(den) <= kEps;
    return __fmul_rn(den, den) <= __fmul_rn(kEps * kEps, lp_dot(lj.x, lj.y, lj.x, lj.y));
}

// The same half-plane with a unit normal.
__device__ __forceinline__ float4 unit_line(float4 l) {
    float inv = rsqrtf(lp_dot(l.x, l.y, l.x, l.y));
    return make_float4(__fmul_rn(l.x, inv), __fmul_rn(l.y, inv), __fmul_rn(l.z, inv), l.w);
}

// LP1: best point on the boundary of line i inside the disc |x| <= V and the half-planes
// 0..i-1.  x(t) = c_i n_i + t d_i with d_i = (n_i.y, -n_i.x).  The disc gives
// |t| <= sqrt(V^2 - c_i^2); half-plane j gives -det(n_i, n_j) t >= c_j - c_i (n_i.n_j),
// an upper bound on t when det(n_i, n_j) > 0, a lower one when < 0; a (nearly) parallel
// j (|det| <= eps) is infeasible iff its right-hand side is positive.
// rec (may be null) receives which bound fixed t.
template <class LineAt>
__device__ __forceinline__ bool lp1_dev(const LineAt& line, int i, float4 li, float V, float ox,
                                        float oy, bool dir_opt, float& xx, float& xy,
                                        LpTape* rec = nullptr, OpCount* oc = nullptr) {
    float D = __fmaf_rn(-li.z, li.z, __fmul_rn(V, V));
    if (D < 0.0f) return false;
    float sq = sqrtf(D);
    float tL = -sq, tR = sq;
    int srcL = -1, srcR = -1;  // -1: the disc, else the bounding line
#pragma unroll 1
    for (int j = 0; j < i; ++j) {
        float4 lj;
        if (!line(j, lj)) continue;
        if (oc) ++oc->bounds;
        float den = lp_det(li.x, li.y, lj.x, lj.y);
        float rhs = lp_rhs(li, lj);
        if (parallel_to<LineAt::kUnit>(den, lj)) {
            if (rhs > 0.0f) return false;
            continue;
        }
        float t = __fdividef(-rhs, den);
        if (den >= 0.0f) {
            if (rec && t < tR) srcR = j;
            tR = fminf(tR, t);
        } else {
            if (rec && t > tL) srcL = j;
            tL = fmaxf(tL, t);
        }
        if (tL > tR) return false;
    }
    float t = lp_dot(ox, oy, li.y, -li.x);
    if (rec) {
        int side = -1;
        if (dir_opt) side = t > 0.0f ? 1 : 0;
        else if (t < tL) side = 0;
        else if (t > tR) side = 1;
        rec->side = side < 0 ? 0 : side;
        int src = side == 0 ? srcL : srcR;
        rec->bound = side < 0 ? kBoundFree : (src < 0 ? kBoundDisc : kBoundLine);
        rec->j = src < 0 ? 0 : src;
    }
    if (dir_opt) t = t > 0.0f ? tR : tL;
    else t = fminf(fmaxf(t, tL), tR);
    float2 x = lp_point(li, t);
    xx = x.x;
    xy = x.y;
    return true;
}

// LP2: incremental 2-D LP over lines 0..n-1 in order (Section 3).  Returns n on success,
// else the index of the line where LP1 failed (x keeps its last value).
// rec (may be null) receives what fixed the returned x: the start point (mode kTapePref,
// kTapePrefClip, or kTapeLp3Dir in direction mode) or the last LP1 (kTapeLine, line i).
template <class LineAt>
__device__ __forceinline__ int lp2_dev(const LineAt& line, int n, float V, float ox, float oy,
                                       bool dir_opt, float& xx, float& xy, LpTape* rec = nullptr,
                                       OpCount* oc = nullptr) {
    if (dir_opt) {
        xx = __fmul_rn(ox, V);
        xy = __fmul_rn(oy, V);
        if (rec) rec->mode = kTapeLp3Dir;
    } else {
        float o2 = lp_dot(ox, oy, ox, oy);
        if (o2 > __fmul_rn(V, V)) {
            float s = __fmul_rn(V, rsqrtf(o2));
            xx = __fmul_rn(ox, s);
            xy = __fmul_rn(oy, s);
            if (rec) rec->mode = kTapePrefClip;
        } else {
            xx = ox;
            xy = oy;
            if (rec) rec->mode = kTapePref;
        }
    }
    // Each pass scans ahead to the next violated line and then runs LP1 on it.  The lanes
    // of a warp meet again after the scan, so LP1 runs for all of them together even when
    // their violated lines have different indices (a loop over i with LP1 inside would
    // run it once for every index at which any lane needs it).
    int i = 0;
#pragma unroll 1
    for (;;) {
        float4 li = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        bool hit = false;
#pragma unroll 1
        for (; i < n; ++i) {
            if (!line(i, li)) continue;
            if (oc) ++oc->checks;
            if (lp_viol(li, xx, xy) > 0.0f) {
                hit = true;
                break;
            }
        }
        if (!hit) return n;
        if (oc) ++oc->lp1;
        if (!LineAt::kUnit) li = unit_line(li);
        float sx = xx, sy = xy;
        LpTape r1;
        if (!lp1_dev(line, i, li, V, ox, oy, dir_opt, xx, xy, rec ? &r1 : nullptr, oc)) {
            xx = sx;
            xy = sy;
            return i;
        }
        if (rec) {
            r1.mode = kTapeLine;
            r1.i = i;
            r1.f = 0;
            *rec = r1;
        }
        ++i;
    }
}

// Lines of one agent: its shared-memory row (unit normals).
struct RowLines {
    static constexpr bool kUnit = true;
    const float4* row;
    __device__ __forceinline__ bool operator()(int j, float4& l) const {
        l = row[j];
        return true;
    }
};

// Bisectors of line i with lines j < i (LP3's projected problem), formed on demand:
// (n_j - n_i).x >= c_j - c_i, NOT normalised; same-direction parallel lines give none.
// Every use is scale-free -- the side of a point, an LP1 bound t = -rhs/den -- except the
// parallel test, which compares |den| with eps |n| (parallel_to), and the line LP1 runs
// on, which unit_line normalises.
// With static obstacles the first nobst lines of the row are hard constraints: they enter
// the projected problem unchanged (Bisectors returns them as they are).
struct Bisectors {
    static constexpr bool kUnit = false;
    const float4* row;
    float4 li;
    int nobst = 0;
    __device__ __forceinline__ bool operator()(int j, float4& q) const {
        float4 lj = row[j];
        if (j < nobst) {
            q = lj;
            return true;
        }
        float den = lp_det(li.x, li.y, lj.x, lj.y);
        if (fabsf(den) <= kEps && lp_dot(li.x, li.y, lj.x, lj.y) > 0.0f) return false;
        q = make_float4(__fsub_rn(lj.x, li.x), __fsub_rn(lj.y, li.y), __fsub_rn(lj.z, li.z), 0.0f);
        return true;
    }
};

// LP3: least penetration (Section 3), one thread per queued agent.  Penetration of line
// i at x: c_i - n_i.x.  When line i is violated by more than the current penetration, LP2
// in direction mode maximises n_i.x over the bisectors of i with the earlier lines; a
// numerically failed LP2 keeps x.
// rec (may be null) keeps the record of the LP2 phase until an LP3 solve succeeds.
// Returns the lines of the projected problems solved: a problem for line i takes that
// line and the i lines before it, i + 1 in all (the search counters report the sum).
__device__ __forceinline__ int lp3_dev(const float4* row, int n, int begin, float V, float& xx,
                                       float& xy, LpTape* rec = nullptr, OpCount* oc = nullptr,
                                       int nobst = 0) {
    float dist = 0.0f;
    int i = begin, problems = 0;
    // scan ahead to the next line violated by more than dist, then solve for it (the
    // lanes meet again after the scan, as in lp2_dev)
#pragma unroll 1
    for (;;) {
        float4 li = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        bool hit = false;
#pragma unroll 1
        for (; i < n; ++i) {
            li = row[i];
            if (oc) ++oc->checks;
            if (lp_viol(li, xx, xy) > dist) {
                hit = true;
                break;
            }
        }
        if (!hit) return problems;
        problems += i + 1;
        if (oc) oc->bis += i > nobst ? i - nobst : 0;
        Bisectors bis{row, li, nobst};
        // the projected problem: every obstacle line, then the bisectors with the lines
        // from nobst to i-1
        const int m = i > nobst ? i : nobst;
        float sx = xx, sy = xy;
        LpTape r2;
        if (lp2_dev(bis, m, V, li.x, li.y, true, xx, xy, rec ? &r2 : nullptr, oc) < m) {
            xx = sx;
            xy = sy;
        } else if (rec) {
            if (r2.mode == kTapeLine) {  // LP1 on the bisector of lines i and r2.i
                r2.f = r2.i;
                r2.mode = kTapeLp3Line;
            } else {
                r2.f = 0;
                r2.bound = kBoundFree;
                r2.j = 0;
                r2.side = 0;
            }
            r2.i = i;
            *rec = r2;
        }
        dist = lp_viol(li, xx, xy);
        ++i;
    }
}

// LP3: least penetration (Section 3), by a group of G lanes (G a power of two, lanes
// aligned in the warp) on one queued agent.  Penetration of line i at x: c_i - n_i.x.
// When line i is violated by more than the current penetration, LP2 in direction mode
// maximises n_i.x over the bisectors of i with the earlier lines; a numerically failed
// LP2 keeps x.  The group takes the sequential algorithm's decisions in the same order:
//   * LP2's scan for the first violated bisector checks G bisectors at a time and takes
//     the lowest violated index of the first chunk that has one (a ballot);
//   * LP1's bounds over the earlier bisectors are split over the lanes and combined with
//     min / max shuffles (exact, order-free); the sequential early exits (tL > tR, an
//     infeasible parallel bisector) become "any lane failed" / "final tL > tR", which
//     fail exactly when some prefix fails because the bounds only tighten.
// Returns the lines of the projected problems solved, as lp3_dev does (the same in every
// lane of the group).
template <int G>
__device__ __forceinline__ int lp3_group_dev(const float4* row, int n, int begin, float V,
                                             float& xx, float& xy) {
    const int lane = threadIdx.x & 31;
    const int g = lane & (G - 1);
    const int base = lane & ~(G - 1);
    const unsigned mask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << base);
    float dist = 0.0f;
    int problems = 0;
#pragma unroll 1
    for (int i = begin; i < n; ++i) {
        const float4 li = row[i];
        if (!(lp_viol(li, xx, xy) > dist)) continue;
        problems += i + 1;
        Bisectors bis{row, li};
        float nx = __fmul_rn(li.x, V), ny = __fmul_rn(li.y, V);  // direction mode starts at V n_i
        bool ok = true;
        int start = 0;
#pragma unroll 1
        for (;;) {
            int f = -1;
#pragma unroll 1
            for (int c0 = start; c0 < i; c0 += G) {
                int j = c0 + g;
                bool viol = false;
                float4 q;
                if (j < i && bis(j, q)) viol = lp_viol(q, nx, ny) > 0.0f;
                unsigned bal = (__ballot_sync(mask, viol) >> base) & (G == 32 ? 0xffffffffu : ((1u << G) - 1u));
                if (bal) {
                    f = c0 + __ffs(bal) - 1;
                    break;
                }
            }
            if (f < 0) break;  // every bisector holds: LP2 succeeded
            float4 qf;
            bis(f, qf);
            qf = unit_line(qf);
            float D = __fmaf_rn(-qf.z, qf.z, __fmul_rn(V, V));
            if (D < 0.0f) {
                ok = false;
                break;
            }
            float sq = sqrtf(D);
            float tL = -sq, tR = sq;
            bool fail = false;
#pragma unroll 1
            for (int j = g; j < f; j += G) {
                float4 qj;
                if (!bis(j, qj)) continue;
                float den = lp_det(qf.x, qf.y, qj.x, qj.y);
                float rhs = lp_rhs(qf, qj);
                if (parallel_to<false>(den, qj)) {
                    fail |= rhs > 0.0f;
                    continue;
                }
                float t = __fdividef(-rhs, den);
                if (den >= 0.0f) tR = fminf(tR, t);
                else tL = fmaxf(tL, t);
            }
#pragma unroll
            for (int o = 1; o < G; o <<= 1) {
                tR = fminf(tR, __shfl_xor_sync(mask, tR, o));
                tL = fmaxf(tL, __shfl_xor_sync(mask, tL, o));
            }
            if (__any_sync(mask, fail) || tL > tR) {
                ok = false;
                break;
            }
            float t = lp_dot(li.x, li.y, qf.y, -qf.x) > 0.0f ? tR : tL;
            float2 x = lp_point(qf, t);
            nx = x.x;
            ny = x.y;
            start = f + 1;
        }
        if (ok) {
            xx = nx;
            xy = ny;
        }
        dist = lp_viol(li, xx, xy);
    }
    return problems;
}

// ---------------------------------------------------------------------------------
// Work-unit LP: the paper's load-balanced LP (Section 3: the new-velocity computations
// are cut into equal work units that idle threads take over), built warp-cooperatively.
// Every lane keeps its own agent's incremental LP.  In each round every lane scans ahead
// to the next line on which it must run LP1 (or finishes); then the bound evaluations of
// all those LP1s -- one per earlier line of each -- are dealt out as work units over the
// warp's 32 lanes, and each LP1's interval is the min / max of its units' bounds
// (shared-memory atomics on order-preserving integer codes).  The bounds, intervals and
// every decision are the one-lane solve's, so the results are bitwise equal.  All 32
// lanes of a warp must call these routines; lanes without a problem only help.
// ---------------------------------------------------------------------------------
struct WarpLpShared {  // one per warp
    int tl[32], tr[32];     // LP1 interval ends, order-preserving integer codes
    int bad[32];            // LP1 infeasible (empty disc chord or parallel bound)
    int pre[32];            // exclusive prefix of the lanes' unit counts
    int base[32];           // LP2: the line LP1 runs on
    int row[32];            // the owner's half-plane row (float4 offset into s_lines)
    float4 li[32], qf[32];  // LP3: the line i and the unit bisector LP1 runs on
};

__device__ __forceinline__ int ord_key(float f) {
    int k = __float_as_int(f);
    return k >= 0 ? k : k ^ 0x7fffffff;
}
__device__ __forceinline__ float ord_val(int k) { return __int_as_float(k >= 0 ? k : k ^ 0x7fffffff); }

// Exclusive prefix of cnt over the warp into S.pre; returns the warp total.
__device__ __forceinline__ int units_prefix(WarpLpShared& S, int cnt) {
    const int lane = threadIdx.x & 31;
    int inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    S.pre[lane] = inc - cnt;
    return __shfl_sync(0xffffffffu, inc, 31);
}

// The lane owning unit u: the last lane whose prefix is <= u (it has units).
__device__ __forceinline__ int unit_owner(const WarpLpShared& S, int u) {
    int lo = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1)
        if (S.pre[lo + step] <= u) lo += step;
    return lo;
}

// One LP1 bound of line lj on the unit line lb, merged into the owner's interval.
template <bool kUnit>
__device__ __forceinline__ void unit_bound(WarpLpShared& S, int o, float4 lb, float4 lj) {
    float den = lp_det(lb.x, lb.y, lj.x, lj.y);
    float rhs = lp_rhs(lb, lj);
    if (parallel_to<kUnit>(den, lj)) {
        if (rhs > 0.0f) S.bad[o] = 1;
        return;
    }
    float t = __fdividef(-rhs, den);
    if (den >= 0.0f) atomicMin(&S.tr[o], ord_key(t));
    else atomicMax(&S.tl[o], ord_key(t));
}

// The disc's chord on unit line l: opens the lane's interval (or marks it empty).
__device__ __forceinline__ void open_interval(WarpLpShared& S, int lane, float4 l, float V) {
    float D = __fmaf_rn(-l.z, l.z, __fmul_rn(V, V));
    float sq = D < 0.0f ? 0.0f : sqrtf(D);
    S.tl[lane] = ord_key(-sq);
    S.tr[lane] = ord_key(sq);
    S.bad[lane] = D < 0.0f;
}

// LP2 (objective: closest to o) over the n half-planes of the lane's row; returns n, or
// the line where LP1 failed (x keeps its last value).  The lp2_dev of one lane, with the
// LP1 bounds shared out.
__device__ __forceinline__ int warp_lp2_units(WarpLpShared& S, const float4* s_lines, int row_off,
                                              bool active, int n, float V, float ox, float oy,
                                              float& xx, float& xy) {
    const int lane = threadIdx.x & 31;
    const float4* row = s_lines + row_off;
    if (active) {
        float o2 = lp_dot(ox, oy, ox, oy);
        if (o2 > __fmul_rn(V, V)) {
            float sc = __fmul_rn(V, rsqrtf(o2));
            xx = __fmul_rn(ox, sc);
            xy = __fmul_rn(oy, sc);
        } else {
            xx = ox;
            xy = oy;
        }
    }
    int i = 0, result = n;
    bool done = !active;
#pragma unroll 1
    for (;;) {
        bool need = false;
        float4 li = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        if (!done) {
#pragma unroll 1
            for (; i < n; ++i) {
                li = row[i];
                if (lp_viol(li, xx, xy) > 0.0f) {
                    need = true;
                    break;
                }
            }
            if (!need) {
                done = true;
                result = n;
            }
        }
        if (__ballot_sync(0xffffffffu, need) == 0u) break;
        const int total = units_prefix(S, need ? i : 0);
        if (need) {
            open_interval(S, lane, li, V);
            S.base[lane] = i;
            S.row[lane] = row_off;
        }
        __syncwarp();
#pragma unroll 1
        for (int u = lane; u < total; u += 32) {
            const int o = unit_owner(S, u);
            const float4* ro = s_lines + S.row[o];
            unit_bound<true>(S, o, ro[S.base[o]], ro[u - S.pre[o]]);
        }
        __syncwarp();
        if (need) {
            float tL = ord_val(S.tl[lane]), tR = ord_val(S.tr[lane]);
            if (S.bad[lane] || tL > tR) {
                done = true;
                result = i;
            } else {
                float t = fminf(fmaxf(lp_dot(ox, oy, li.y, -li.x), tL), tR);
                float2 x = lp_point(li, t);
                xx = x.x;
                xy = x.y;
                ++i;
            }
        }
        __syncwarp();
    }
    return result;
}

// LP3 (least penetration) of the lane's queued agent, if it has one: the lp3_dev of one
// lane (outer scan over the lines, inner direction-mode LP2 over the bisectors), with the
// bounds of every bisector LP1 shared out.
// Returns the lines of the projected problems of the lane's agent, as lp3_dev does.
__device__ __forceinline__ int warp_lp3_units(WarpLpShared& S, const float4* s_lines, int row_off,
                                              bool has, int n, int begin, float V, float& xx,
                                              float& xy) {
    const int lane = threadIdx.x & 31;
    const float4* row = s_lines + row_off;
    float dist = 0.0f, sx = 0.0f, sy = 0.0f;
    int i = begin, f = 0, problems = 0;
    bool done = !has, inner = false;
    float4 li = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll 1
    for (;;) {
        bool need = false;
        float4 qraw = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll 1
        while (!done) {
            if (!inner) {
                bool hit = false;
#pragma unroll 1
                for (; i < n; ++i) {
                    li = row[i];
                    if (lp_viol(li, xx, xy) > dist) {
                        hit = true;
                        break;
                    }
                }
                if (!hit) {
                    done = true;
                    break;
                }
                inner = true;
                problems += i + 1;
                f = 0;
                sx = xx;
                sy = xy;
                xx = __fmul_rn(li.x, V);  // direction mode starts at V n_i
                xy = __fmul_rn(li.y, V);
            }
            Bisectors bis{row, li};
#pragma unroll 1
            for (; f < i; ++f) {
                float4 q;
                if (!bis(f, q)) continue;
                if (lp_viol(q, xx, xy) > 0.0f) {
                    need = true;
                    qraw = q;
                    break;
                }
            }
            if (need) break;
            dist = lp_viol(li, xx, xy);  // every bisector holds: the inner LP2 succeeded
            inner = false;
            ++i;
        }
        if (__ballot_sync(0xffffffffu, need) == 0u) break;
        const int total = units_prefix(S, need ? f : 0);
        if (need) {
            float4 qf = unit_line(qraw);
            open_interval(S, lane, qf, V);
            S.li[lane] = li;
            S.qf[lane] = qf;
            S.row[lane] = row_off;
        }
        __syncwarp();
#pragma unroll 1
        for (int u = lane; u < total; u += 32) {
            const int o = unit_owner(S, u);
            Bisectors bo{s_lines + S.row[o], S.li[o]};
            float4 qj;
            if (bo(u - S.pre[o], qj)) unit_bound<false>(S, o, S.qf[o], qj);
        }
        __syncwarp();
        if (need) {
            float tL = ord_val(S.tl[lane]), tR = ord_val(S.tr[lane]);
            if (S.bad[lane] || tL > tR) {  // the inner LP2 failed: keep the point from before it
                xx = sx;
                xy = sy;
                dist = lp_viol(li, xx, xy);
                inner = false;
                ++i;
            } else {
                float4 qf = S.qf[lane];
                float t = lp_dot(li.x, li.y, qf.y, -qf.x) > 0.0f ? tR : tL;
                float2 x = lp_point(qf, t);
                xx = x.x;
                xy = x.y;
                ++f;
            }
        }
        __syncwarp();
    }
    return problems;
}

// Insert key into the ascending list kk; its largest entry drops out, and a key not below
// kk[KMAX-1] leaves the list unchanged.  With c_l = (key < kk[l]) (all independent, and
// monotone in l because kk is sorted) the new entry l is kk[l-1] if c_{l-1}, else key if
// c_l, else kk[l]: no chain of dependent decisions.
template <int KMAX>
__device__ __forceinline__ void insert_key(unsigned long long key, unsigned long long (&kk)[KMAX]) {
    bool c[KMAX];
#pragma unroll
    for (int l = 0; l < KMAX; ++l) c[l] = key < kk[l];
#pragma unroll
    for (int l = KMAX - 1; l > 0; --l) kk[l] = c[l - 1] ? kk[l - 1] : (c[l] ? key : kk[l]);
    if (c[0]) kk[0] = key;
}

// ---------------------------------------------------------------------------------
// Static obstacles (segments; the ORCA obstacle rule): optimisation velocity 0 and full
// responsibility, so with q the segment's nearest point relative to the agent and d = |q|
// the permitted velocities are v.q/d <= (d - r)/tau_o (dt in place of tau_o when d <= r;
// an agent exactly on the segment takes its left normal).  Normal form n = -q/d,
// c = -(d - r)/tau_o.  An agent takes the kobst nearest segments it could reach within
// tau_o -- FP32 squared distance (clamped projection, one rounding per operation) strictly
// below fl(fl(V tau_o) + r)^2 -- ordered by (d^2, segment index).
// ---------------------------------------------------------------------------------
__device__ __forceinline__ float seg_dist2(float4 sg, float2 p) {
    const float ex = __fsub_rn(sg.z, sg.x), ey = __fsub_rn(sg.w, sg.y);
    const float wx = __fsub_rn(p.x, sg.x), wy = __fsub_rn(p.y, sg.y);
    const float l2 = __fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey));
    float t = 0.0f;
    if (l2 > 0.0f) {
        t = __fdiv_rn(__fadd_rn(__fmul_rn(wx, ex), __fmul_rn(wy, ey)), l2);
        t = t < 0.0f ? 0.0f : (t > 1.0f ? 1.0f : t);
    }
    const float qx = __fsub_rn(__fadd_rn(sg.x, __fmul_rn(t, ex)), p.x);
    const float qy = __fsub_rn(__fadd_rn(sg.y, __fmul_rn(t, ey)), p.y);
    return __fadd_rn(__fmul_rn(qx, qx), __fmul_rn(qy, qy));
}

// a - b as an unevaluated pair hi + lo, exactly (Knuth's TwoSum on a and -b).
__device__ __forceinline__ float2 two_diff(float a, float b) {
    const float s = __fsub_rn(a, b);
    const float bv = __fsub_rn(s, a);        // the part of -b that made it into s
    const float av = __fsub_rn(s, bv);
    const float e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(__fsub_rn(0.0f, b), bv));
    return make_float2(s, e);
}

// The obstacle half-plane of an agent at p, radius r, against segment sg (the ORCA obstacle
// rule: the obstacle does not move and takes no share of the avoidance).  With q the
// closest point of the segment and d = |q - p|: n = (p - q)/d, c = -(d - r)/tau_o, or
// -(d - r)/dt when the agent overlaps the segment (d <= r).  d = 0 takes the segment's
// left normal, a point segment (1, 0).
// The distance is formed from exact differences: p - a, p - b and b - a as TwoSum pairs and,
// for a closest point inside the segment, the cross product det(b - a, p - a) with its
// products' rounding errors (FMA) carried.  Its error is then a few ulps of d, where the
// closest point written in absolute coordinates would carry ulp(|p|) -- which the 1/dt of
// an overlapping agent turns into a velocity error of order 1e-4 m/s at 100 m from the origin.
__device__ __forceinline__ float4 obstacle_line(float4 sg, float2 p, float r, float dt,
                                                float tau_o) {
    const float2 wx = two_diff(p.x, sg.x), wy = two_diff(p.y, sg.y);  // p - a
    const float2 ex = two_diff(sg.z, sg.x), ey = two_diff(sg.w, sg.y); // b - a
    const float l2 = __fadd_rn(__fmul_rn(ex.x, ex.x), __fmul_rn(ey.x, ey.x));
    float t = 0.0f;
    if (l2 > 0.0f) t = __fdiv_rn(__fadd_rn(__fmul_rn(wx.x, ex.x), __fmul_rn(wy.x, ey.x)), l2);
    float d, nx = 1.0f, ny = 0.0f;
    const float il = l2 > 0.0f ? __fdiv_rn(1.0f, sqrtf(l2)) : 0.0f;
    if (t > 0.0f && t < 1.0f) {
        // interior: d = |det(e, w)| / |e|, n = sign(det) (-e_y, e_x) / |e|
        const float p1 = __fmul_rn(ex.x, wy.x), e1 = __fmaf_rn(ex.x, wy.x, -p1);
        const float p2 = __fmul_rn(ey.x, wx.x), e2 = __fmaf_rn(ey.x, wx.x, -p2);
        const float cross = __fsub_rn(__fadd_rn(__fmul_rn(ex.x, wy.y), __fmul_rn(ex.y, wy.x)),
                                      __fadd_rn(__fmul_rn(ey.x, wx.y), __fmul_rn(ey.y, wx.x)));
        const float det = __fadd_rn(__fsub_rn(p1, p2), __fadd_rn(__fsub_rn(e1, e2), cross));
        d = __fmul_rn(fabsf(det), il);
        const float s = det < 0.0f ? -il : il;
        nx = -__fmul_rn(ey.x, s);
        ny = __fmul_rn(ex.x, s);
    } else {
        // an end point is nearest: the agent's offset from it, p - a or p - b
        float vx = wx.x, vy = wy.x;
        if (t >= 1.0f) {
            vx = two_diff(p.x, sg.z).x;
            vy = two_diff(p.y, sg.w).x;
        }
        d = sqrtf(__fadd_rn(__fmul_rn(vx, vx), __fmul_rn(vy, vy)));
        if (d > 0.0f) {
            nx = __fdiv_rn(vx, d);
            ny = __fdiv_rn(vy, d);
        } else if (l2 > 0.0f) {
            nx = -__fmul_rn(ey.x, il);
            ny = __fmul_rn(ex.x, il);
        }
    }
    const float c = -__fdiv_rn(__fsub_rn(d, r), d > r ? tau_o : dt);
    return make_float4(nx, ny, c, 0.0f);
}

// Whether segment sg could be within reach R of some point of the box [x0, x1] x [y0, y1]:
// its own box against the box widened by R and a margin well above the FP32 rounding of
// the distance test (a few ulps of the largest coordinate involved).  False means the
// segment is farther than R from every point of the box.
__device__ __forceinline__ bool segment_in_reach(float4 sg, float x0, float y0, float x1, float y1,
                                                 float R) {
    const float M = fmaxf(fmaxf(fabsf(x0), fabsf(x1)), fmaxf(fabsf(y0), fabsf(y1)));
    const float ms = fmaxf(fmaxf(fabsf(sg.x), fabsf(sg.z)), fmaxf(fabsf(sg.y), fabsf(sg.w)));
    const float g = R + 1e-4f * (1.0f + fmaxf(M, ms) + R);
    return fminf(sg.x, sg.z) <= x1 + g && fmaxf(sg.x, sg.z) >= x0 - g &&
           fminf(sg.y, sg.w) <= y1 + g && fmaxf(sg.y, sg.w) >= y0 - g;
}

// Segments some agent of the tile could select.  The tile's agents are neighbours in the
// cell order, so their bounding box is small; each segment is tested against it and the
// tile's largest reach fl(fl(V tau_o) + r) (segment_in_reach).  The selection keys
// carry the segment index, so the kept subset, in any order, selects what a scan of all
// segments selects.  Ends with a barrier; nsel must be 0 on entry.
template <int TPB>
__device__ __forceinline__ void cull_segments(const MainArgs& a, int t, bool active,
                                              unsigned short* sel, int* nsel, float (*box)[5]) {
    float x0 = INFINITY, y0 = INFINITY, x1 = -INFINITY, y1 = -INFINITY, R = 0.0f;
    if (active) {
        const float4 m = a.in.msg[t];
        x0 = x1 = m.x;
        y0 = y1 = m.y;
        R = __fadd_rn(__fmul_rn(a.prm.max_speed[t], a.tau_o), m.z);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x0 = fminf(x0, __shfl_xor_sync(0xffffffffu, x0, o));
        y0 = fminf(y0, __shfl_xor_sync(0xffffffffu, y0, o));
        x1 = fmaxf(x1, __shfl_xor_sync(0xffffffffu, x1, o));
        y1 = fmaxf(y1, __shfl_xor_sync(0xffffffffu, y1, o));
        R = fmaxf(R, __shfl_xor_sync(0xffffffffu, R, o));
    }
    if ((threadIdx.x & 31) == 0) {
        float* b = box[threadIdx.x >> 5];
        b[0] = x0;
        b[1] = y0;
        b[2] = x1;
        b[3] = y1;
        b[4] = R;
    }
    __syncthreads();
#pragma unroll
    for (int w = 0; w < TPB / 32; ++w) {
        x0 = fminf(x0, box[w][0]);
        y0 = fminf(y0, box[w][1]);
        x1 = fmaxf(x1, box[w][2]);
        y1 = fmaxf(y1, box[w][3]);
        R = fmaxf(R, box[w][4]);
    }
#pragma unroll 1
    for (int j = threadIdx.x; j < a.nseg; j += TPB)
        if (segment_in_reach(__ldg(a.seg + j), x0, y0, x1, y1, R))
            sel[atomicAdd(nsel, 1)] = (unsigned short)j;
    __syncthreads();
}

// Writes the agent's obstacle half-planes to row[0..] (nearest first) and returns how many;
// rec (may be null) receives the segments' indices, -1 padded to kMaxObstacleNeighbors.
// Only the segments sel[0..nsel) are scanned (cull_segments keeps every one that an agent
// of the tile could select).
template <int KO>
__device__ __forceinline__ int obstacle_lines(const float4* __restrict__ segs,
                                              const unsigned short* sel,
                                              int nsel, int kobst, float2 p, float r, float V,
                                              float dt, float tau_o, float4* row, int32_t* rec) {
    const float rng = __fadd_rn(__fmul_rn(V, tau_o), r);
    const float rng2 = __fmul_rn(rng, rng);
    unsigned long long ok[KO];
#pragma unroll
    for (int l = 0; l < KO; ++l) ok[l] = (l < KO - kobst) ? 0ull : ~0ull;
#pragma unroll 1
    for (int q = 0; q < nsel; ++q) {
        const int j = sel[q];
        const float d2 = seg_dist2(__ldg(segs + j), p);
        if (d2 < rng2) insert_key<KO>(((unsigned long long)__float_as_uint(d2) << 32) | (unsigned)j, ok);
    }
    int nob = 0;
#pragma unroll
    for (int l = 0; l < KO; ++l) {
        if (l < KO - kobst || ok[l] == ~0ull) continue;
        const int j = (int)(ok[l] & 0xffffffffu);
        if (rec) rec[nob] = j;
        row[nob++] = obstacle_line(__ldg(segs + j), p, r, dt, tau_o);
    }
    if (rec)
        for (int l = nob; l < kMaxObstacleNeighbors; ++l) rec[l] = -1;
    return nob;
}

// Insert the nb parked keys into kk; once the list is full, lim becomes its k-th d^2.
template <int KMAX>
__device__ __forceinline__ void drain(const unsigned long long* buf, int nb,
                                      unsigned long long (&kk)[KMAX], float& lim) {
#pragma unroll 1
    for (int i = 0; i < nb; ++i) insert_key<KMAX>(buf[i], kk);
    if (kk[KMAX - 1] != ~0ull) lim = fminf(lim, __uint_as_float((unsigned)(kk[KMAX - 1] >> 32)));
}

// Candidates q0..q1-1 (sorted slots) offered to the top-k list of the agent at slot t,
// kU at a time (their loads in flight together).  A candidate enters when its fl32 d^2
// <= lim; entrants are parked in buf (shared memory) and inserted in bulk -- when fewer
// than kU free places are left, and after the search -- which keeps the divergent
// insertion out of the candidate loop.  Equal d^2 is settled by the 64-bit key.
// kU: three candidates at a time for k <= 10, whose row ranges are short (fewer wasted
// slots at a row's end), four above (measured: 1% faster on the 524,288-agent flow at
// k = 10, 1% slower on the dense crowd at k = 20 with three).
template <int KMAX>
constexpr int candidates_per_round() { return KMAX <= 10 ? 3 : 4; }
template <int KMAX, int CAP>
__device__ __forceinline__ void offer_range(const float4* __restrict__ msg, uint32_t q0, uint32_t q1,
                                            int t, float2 p, unsigned long long (&kk)[KMAX],
                                            unsigned long long* buf, int& nb, float& lim) {
    constexpr int kU = candidates_per_round<KMAX>();
    static_assert(CAP > kU, "parking space for one batch");
#pragma unroll 1
    for (uint32_t q = q0; q < q1; q += kU) {
        float d2[kU];
        unsigned id[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const uint32_t qu = q + u;
            float4 mj = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            if (qu < q1) mj = msg[qu];
            float ddx = __fsub_rn(mj.x, p.x), ddy = __fsub_rn(mj.y, p.y);
            d2[u] = __fadd_rn(__fmul_rn(ddx, ddx), __fmul_rn(ddy, ddy));
            id[u] = __float_as_uint(mj.w);
            if (qu >= q1 || (int)qu == t) d2[u] = INFINITY;
        }
#pragma unroll
        for (int u = 0; u < kU; ++u)
            if (d2[u] <= lim)
                buf[nb++] = ((unsigned long long)__float_as_uint(d2[u]) << 32) | id[u];
        if (nb > CAP - kU) {
            drain<KMAX>(buf, nb, kk, lim);
            nb = 0;
        }
    }
}

// Start radius (squared) of a search with no prediction, the first step after a load:
// the radius that holds about k + sqrt(k) + 2 other agents at the density of the 3 x 3
// cells around the agent (counted from the cell table; near the crowd's edge the block's
// empty part lowers the estimate, so the start errs wider there).  A start that misses
// costs its agent a second pass, a start too wide costs every agent of the warp the
// drains of the extra candidates; on the 524,288-agent scenes the margin of one standard
// deviation (sqrt(k)) gave the fastest first step (0.28-0.34 ms against 0.44-0.50 ms for
// 3 sqrt(k) + 3), with about one agent in forty searching twice.  One cell edge when the
// block holds nobody else.
__device__ __forceinline__ float density_lim(const MainArgs& a, const GridDev& g, int cell_off,
                                             float2 p, int k) {
    const int cx = cell_coord(p.x, g.xmin, g.inv, g.gx);
    const int cy = cell_coord(p.y, g.ymin, g.inv, g.gy);
    const int x0 = cx > 0 ? cx - 1 : 0, x1 = cx + 1 < g.gx ? cx + 1 : g.gx - 1;
    const int y0 = cy > 0 ? cy - 1 : 0, y1 = cy + 1 < g.gy ? cy + 1 : g.gy - 1;
    uint32_t cnt = 0;
#pragma unroll 1
    for (int y = y0; y <= y1; ++y) {
        const int c = cell_off + y * g.gx;
        if (!idx_ok(c + x0 >= 0 && c + x1 + 1 <= a.misc->grid.num_cells, &a.misc_rw->error)) continue;
        cnt += a.cell_start[c + x1 + 1] - a.cell_start[c + x0];
    }
    if (cnt <= 1) return g.s * g.s;
    const float area = (float)((x1 - x0 + 1) * (y1 - y0 + 1)) * g.s * g.s;
    const float want = (float)k + sqrtf((float)k) + 2.0f;
    return want * area / (3.14159265f * (float)(cnt - 1));
}

// Exact k nearest neighbours of the agent at sorted slot t: keys (d2 bits << 32 | id)
// kept ascending in kk; the first KMAX-k entries are permanent zero sentinels so that
// the live window is the last k entries.
//
// The search goes row by row: the agent's row of cells first, then always the nearer of
// the next rows above and below.  Cells are numbered row-major, so the cells of one row
// that can hold a candidate form one contiguous slot range, read in one pass.  In a row
// whose vertical gap to the agent is at least h, a candidate with fl32 d^2 <= lim lies
// within w = sqrt(lim (1 + 1e-5) - h^2) horizontally (the factor covers the rounding of
// d^2); the range runs from the cell of p.x - w to the cell of p.x + w, widened by twice
// the cell-assignment slop (the cell map is monotone in x, so no such candidate is
// outside it).  h is the row's distance minus the slop; the search stops when the next
// row's h^2 exceeds lim.  lim shrinks as the list fills, narrowing later rows.
//
// lim starts at lim0 (a predicted radius capped below r_obs^2; NaN: from the density).
// Every candidate with d^2 <= lim0 is offered, and all others have larger d^2, so when at
// least k candidates were offered the list is exact; when fewer were and lim0 was below
// the r_obs bound, the search is repeated with 1.5 x the radius (capped at the r_obs
// bound).  buf holds CAP parked keys.
template <int KMAX, int CAP>
__device__ __forceinline__ unsigned knn_dev(const MainArgs& a, const GridDev& g, int cell_off,
                                            float nd, int t, float2 p, int k, float lim0,
                                            unsigned long long* buf,
                                            unsigned long long (&kk)[KMAX], SearchCount& sc) {
    const int cy = cell_coord(p.y, g.ymin, g.inv, g.gy);
    float nd2 = __fmul_rn(nd, nd);
    const float lim_max = __int_as_float(__float_as_int(nd2) - 1);  // largest float below r_obs^2
    // no prediction: from the local density
    if (lim0 != lim0) {
        lim0 = density_lim(a, g, cell_off, p, k);
        ++sc.cold;
    }
    lim0 = fminf(lim0, lim_max);
    unsigned cand = 0;
#pragma unroll 1
    for (;;) {
#pragma unroll
        for (int l = 0; l < KMAX; ++l) kk[l] = (l < KMAX - k) ? 0ull : ~0ull;
        float lim = lim0;
        int nb = 0, y = cy, up = cy + 1, dn = cy - 1;
        float h = 0.0f;
#pragma unroll 1
        for (;;) {
            float w = sqrtf(fmaxf(lim * (1.0f + 1e-5f) - h * h, 0.0f)) + 2.0f * g.slop;
            int x0 = cell_coord(p.x - w, g.xmin, g.inv, g.gx);
            int x1 = cell_coord(p.x + w, g.xmin, g.inv, g.gx);
            int c = cell_off + y * g.gx;
            uint32_t q0 = 0u, q1 = 0u;
            if (idx_ok(c + x0 >= 0 && c + x1 + 1 <= a.misc->grid.num_cells, &a.misc_rw->error)) {
                q0 = a.cell_start[c + x0];
                q1 = a.cell_start[c + x1 + 1];
                if (!idx_ok(q0 <= q1 && q1 <= (uint32_t)a.n, &a.misc_rw->error)) q1 = q0;
            }
            cand += q1 - q0;
            ++sc.rows;
            offer_range<KMAX, CAP>(a.in.msg, q0, q1, t, p, kk, buf, nb, lim);
            // the nearer of the next rows above and below (none left: infinite gaps)
            float hu = up < g.gy ? (g.ymin + (float)up * g.s) - p.y : INFINITY;
            float hd = dn >= 0 ? p.y - (g.ymin + (float)(dn + 1) * g.s) : INFINITY;
            if (hu <= hd) {
                y = up++;
                h = hu;
            } else {
                y = dn--;
                h = hd;
            }
            if (h == INFINITY) break;
            h = fmaxf(0.0f, h - g.slop);
            if (h * h * (1.0f - 1e-5f) > lim) break;
        }
        drain<KMAX>(buf, nb, kk, lim);  // the parked keys, all lanes together
        if (kk[KMAX - 1] != ~0ull || !(lim0 < lim_max)) break;
        // fewer than k inside: 1.5 x the radius (from at least 1e-3 r_obs, so the bound
        // reaches r_obs within 18 passes whatever the prediction was)
        lim0 = fminf(fmaxf(2.25f * lim0, 1e-6f * lim_max), lim_max);
        ++sc.retries;
    }
    return cand;
}

// Minimum resident CTAs for __launch_bounds__: a register budget per thread that keeps
// 28 warps per SM at k <= 10, 16 at k <= 20 and 8 at k = 32 without heavy spilling.
template <int KMAX, int TPB>
constexpr int main_min_blocks() {
    return ((KMAX <= 10 ? 28 : (KMAX <= 20 ? 16 : 8)) * 32 + TPB - 1) / TPB;
}

// Default LP mode: each lane solves alone for k <= 16, warp work units above.  Measured on
// the 524,288-agent flow (k = 10): one lane 0.135 ms, 4-lane LP3 groups 0.160, work units
// 0.167; on the 2,097,152-agent dense crowd (k = 20): one lane 1.89 ms, groups 2.00, work
// units 1.70 -- with 20 half-planes an LP1 has enough bounds to share (the autotuner
// checks every mode).
int default_lp3_group(int kmax) { return kmax <= 16 ? 1 : 32; }

// Row of one agent: KMAX neighbour half-planes and one float4 of padding (an odd stride in
// float4s: conflict-free float4 rows).  With static obstacles the row also holds the
// kobst obstacle half-planes; its stride is set per launch (obs_row_len), so a few
// obstacle lines cost a few float4s of shared memory per agent, not the maximum.
template <int KMAX>
constexpr int row_len() { return KMAX + 1; }
template <int KMAX, int TPB>
constexpr size_t main_smem_bytes() { return sizeof(float4) * TPB * row_len<KMAX>(); }
constexpr int obs_row_len(int kmax, int kobst) { return (kmax + kobst) | 1; }

// Parameters of the scene an agent belongs to (the one scene, or its scene of a batch).
struct SceneView {
    GridDev g;
    int cell_off, k;
    float nd, dt;
};

__device__ __forceinline__ void scene_view(const MainArgs& a, int t, SceneView& v) {
    if (a.scenes) {
        const SceneDev& sc = a.scenes[a.slot_scene[t]];
        v.g = sc.grid;
        v.cell_off = sc.cell_off;
        v.k = sc.k;
        v.nd = sc.nd;
        v.dt = sc.dt;
    } else {
        v.g = a.misc->grid;
        v.cell_off = 0;
        v.k = a.k;
        v.nd = a.nd;
        v.dt = a.dt;
    }
}

// Tiles (TPB consecutive sorted slots, the ORCA kernel's CTAs) with a segment within reach
// of some agent: one warp per tile, the same reach test as cull_segments.  Flags them for
// the plain launch to skip and lists them for the obstacle launch, so a crowd pays for the
// obstacle instantiation (wider rows, culling) only near obstacles.  The list's order
// varies between runs; each tile's results do not depend on it.
__global__ void __launch_bounds__(256) obstacle_tiles_kernel(MainArgs a, int tpb) {
    pdl_wait();
    const int ntiles = (a.n + tpb - 1) / tpb;
    const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (w >= ntiles) return;  // whole warps
    float x0 = INFINITY, y0 = INFINITY, x1 = -INFINITY, y1 = -INFINITY, R = 0.0f;
    for (int i = lane; i < tpb; i += 32) {
        const int t = w * tpb + i;
        if (t >= a.n) break;
        const float4 m = a.in.msg[t];
        x0 = fminf(x0, m.x);
        y0 = fminf(y0, m.y);
        x1 = fmaxf(x1, m.x);
        y1 = fmaxf(y1, m.y);
        R = fmaxf(R, __fadd_rn(__fmul_rn(a.prm.max_speed[t], a.tau_o), m.z));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        x0 = fminf(x0, __shfl_xor_sync(0xffffffffu, x0, o));
        y0 = fminf(y0, __shfl_xor_sync(0xffffffffu, y0, o));
        x1 = fmaxf(x1, __shfl_xor_sync(0xffffffffu, x1, o));
        y1 = fmaxf(y1, __shfl_xor_sync(0xffffffffu, y1, o));
        R = fmaxf(R, __shfl_xor_sync(0xffffffffu, R, o));
    }
    bool near = false;
    for (int j = lane; j < a.nseg && !near; j += 32)
        near = segment_in_reach(__ldg(a.seg + j), x0, y0, x1, y1, R);
    near = __any_sync(0xffffffffu, near);
    if (lane == 0) {
        a.tile_near[w] = near ? 1 : 0;
        if (near) a.obs_tiles[atomicAdd(&a.misc_rw->obs_tiles, 1u)] = w;
    }
}

// Persistent over tiles of TPB consecutive agents: tile blockIdx.x first, then
// tiles taken from a per-step counter (with one CTA per tile this loop runs once).  The
// obstacle instantiation (OBS) steps the tiles obstacle_tiles_kernel listed instead,
// entries blockIdx.x, blockIdx.x + gridDim.x, ...
template <int KMAX, int TPB, int G, bool TAPE = false, bool COUNT = false, bool OBS = false>
__global__ void __launch_bounds__(TPB, main_min_blocks<KMAX, TPB>()) orca_main_kernel(MainArgs a) {
    pdl_wait();
    // padded rows: conflict-free float4 accesses; KP float4s always (the kNN parking space)
    constexpr int KP = row_len<KMAX>();
    const int kp = OBS ? a.row_stride : KP;
    extern __shared__ float4 s_lines[];  // TPB * kp half-planes
    __shared__ float2 s_x[TPB];
    __shared__ float s_V[TPB];
    __shared__ unsigned char s_b[TPB];
    __shared__ unsigned char s_cnt[TPB];
    __shared__ unsigned char s_queued[TPB];
    __shared__ unsigned char s_queue[TPB];
    __shared__ LpTape s_tape[TAPE ? TPB : 1];
    __shared__ int s_qn, s_tile;
    __shared__ unsigned long long s_cand, s_lines_n, s_act, s_lp3, s_proj;
    __shared__ unsigned long long s_search[3];
    __shared__ unsigned long long s_ops[COUNT ? 4 : 1];
    constexpr bool WU = G == 32;  // work-unit LP (warp-cooperative) instead of per-lane LP
    __shared__ WarpLpShared s_wlp[WU ? TPB / 32 : 1];
    __shared__ unsigned char s_nob[OBS ? TPB : 1];         // obstacle lines in each row
    __shared__ unsigned short s_sel[OBS ? kMaxObstacles : 1];  // segments the tile can reach
    __shared__ float s_box[OBS ? TPB / 32 : 1][5];
    __shared__ int s_nsel;
    const int tid = threadIdx.x;
    if (tid == 0) {
        s_cand = 0;
        s_lines_n = 0;
        s_act = 0;
        s_lp3 = 0;
        s_proj = 0;
        s_search[0] = s_search[1] = s_search[2] = 0;
        for (int q = 0; q < (COUNT ? 4 : 1); ++q) s_ops[q] = 0;
    }
    OpCount oc{0u, 0u, 0u, 0u};
    SearchCount sc{0u, 0u, 0u};
    unsigned proj = 0;  // lines of the least-penetration projected problems this lane solved
    const int ntiles = (a.n + TPB - 1) / TPB;
    float4* row = s_lines + tid * kp;
    // the obstacle launch steps the listed tiles li = blockIdx.x, + gridDim.x, ...
    const int nlist = OBS ? (int)a.misc->obs_tiles : 0;
    int li = blockIdx.x;
    int tile = OBS ? (li < nlist ? a.obs_tiles[li] : ntiles) : (int)blockIdx.x;
#pragma unroll 1
    while (tile < ntiles) {
        // with obstacles the plain launch (one CTA per tile) leaves flagged tiles to the
        // obstacle launch
        if (!OBS && a.tile_near != nullptr && a.tile_near[tile]) break;
        if (tid == 0) {
            s_qn = 0;
            s_nsel = 0;
        }
        s_queued[tid] = 0;
        __syncthreads();
        const int t = tile * TPB + tid;
        const bool active = t < a.n;
        if (OBS) cull_segments<TPB>(a, t, active, s_sel, &s_nsel, s_box);
        float2 p = make_float2(0.0f, 0.0f);
        float xx = 0.0f, xy = 0.0f, dt = 1.0f, V = 0.0f, ox = 0.0f, oy = 0.0f;
        uint32_t me = 0;
        int cnt = 0;
        unsigned cand = 0;
        int nob = 0;  // obstacle half-planes at the front of the row
        // an agent whose LP2 failed at line b joins the CTA's least-penetration queue
        auto enqueue = [&](int b) {
            int slot = atomicAdd(&s_qn, 1);
            s_queue[slot] = (unsigned char)tid;
            s_queued[tid] = 1;
            s_x[tid] = make_float2(xx, xy);
            s_b[tid] = (unsigned char)b;
            s_cnt[tid] = (unsigned char)(nob + cnt);
            s_V[tid] = V;
            if (OBS) s_nob[OBS ? tid : 0] = (unsigned char)nob;
        };
        if (active) {
            SceneView sv;
            scene_view(a, t, sv);
            dt = sv.dt;
            // ---- phase 1: neighbours and half-planes
            float4 me4 = a.in.msg[t];
            p = make_float2(me4.x, me4.y);
            me = __float_as_uint(me4.w);
            // search radius predicted from the previous step's k-th neighbour distance
            // (no distance grows by more than the two agents' displacements, about 2 V dt);
            // +inf (fewer than k inside r_obs last time) starts at the r_obs bound, NaN (no
            // prediction) from the density of the cells around the agent
            V = a.prm.max_speed[t];
            float lim0 = __int_as_float(0x7fffffff);
            if (a.prm.hint) {
                float hd = sqrtf(a.prm.hint[t]) * (1.0f + 1e-3f) + 2.5f * V * dt + 1e-3f;
                lim0 = hd * hd;
            }
            unsigned long long kk[KMAX];
            cand = knn_dev<KMAX, 2 * KP>(a, sv.g, sv.cell_off, sv.nd, t, p, sv.k, lim0,
                                         reinterpret_cast<unsigned long long*>(row), kk, sc);
            if (a.prm.hint)
                a.prm.hint[t] = kk[KMAX - 1] != ~0ull
                                    ? __uint_as_float((unsigned)(kk[KMAX - 1] >> 32))
                                    : INFINITY;
            // static obstacles first: their half-planes open the row (a plain launch records
            // none)
            if (!OBS && a.rec_obst)
                for (int l = 0; l < kMaxObstacleNeighbors; ++l)
                    a.rec_obst[(size_t)me * kMaxObstacleNeighbors + l] = -1;
            if (OBS)
                nob = obstacle_lines<kMaxObstacleNeighbors>(
                    a.seg, s_sel, s_nsel, a.kobst, p, me4.z, V, dt, a.tau_o, row,
                    a.rec_obst ? a.rec_obst + (size_t)me * kMaxObstacleNeighbors : nullptr);
            // park the neighbours' slots in the row (one unrolled store each), then build
            // the half-planes in a rolled loop: one copy of the line code keeps the kernel
            // small enough for the instruction cache.  The next neighbour's record and
            // velocity are loaded while the current half-plane is built.
#pragma unroll
            for (int l = 0; l < KMAX; ++l) {
                if (l >= KMAX - sv.k && kk[l] != ~0ull) {
                    const uint32_t nid = (uint32_t)kk[l];
                    if (!idx_ok(nid < (uint32_t)a.n, &a.misc_rw->error)) continue;
                    const uint32_t q = a.in.slot[nid];
                    if (!idx_ok(q < (uint32_t)a.n, &a.misc_rw->error)) continue;
                    row[nob + cnt++].w = __uint_as_float(q);
                }
            }
            float2 v = a.in.vel[t];
            float itau = __fdividef(1.0f, a.prm.tau[t]);
            float idt = __fdividef(1.0f, dt);
            float half_idt = 0.5f * idt;
            {
                const int lend = nob + cnt;
                float4 nm = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                float2 nv = make_float2(0.0f, 0.0f);
                if (nob < lend) {
                    const int q = __float_as_int(row[nob].w);
                    nm = a.in.msg[q];
                    nv = a.in.vel[q];
                }
#pragma unroll 1
                for (int l = nob; l < lend; ++l) {
                    const float4 cm = nm;
                    const float2 cv = nv;
                    if (l + 1 < lend) {
                        const int q = __float_as_int(row[l + 1].w);
                        nm = a.in.msg[q];
                        nv = a.in.vel[q];
                    }
                    row[l] = orca_line_dev(p, v, me4.z, itau, dt, half_idt, me, cm, cv);
                }
            }
            if (a.rec_nbr) {
                int w = 0;
#pragma unroll
                for (int l = 0; l < KMAX; ++l)
                    if (l >= KMAX - sv.k)
                        a.rec_nbr[(size_t)me * a.rec_stride + (w++)] =
                            kk[l] != ~0ull ? (int32_t)(kk[l] & 0xffffffffu) : -1;
                for (; w < a.rec_stride; ++w) a.rec_nbr[(size_t)me * a.rec_stride + w] = -1;
            }
            if (a.rec_cell) {
                int cx = cell_coord(p.x, sv.g.xmin, sv.g.inv, sv.g.gx);
                int cy = cell_coord(p.y, sv.g.ymin, sv.g.inv, sv.g.gy);
                a.rec_cell[me] = (uint32_t)sv.cell_off + (uint32_t)cy * (uint32_t)sv.g.gx + (uint32_t)cx;
            }
            // ---- phase 2: preferred velocity (towards the goal at the preferred speed, or
            // onto the goal within one step) and LP2
            float2 o = pref_velocity_dev(p, a.prm.goal[t], a.prm.pref_speed[t], dt, idt);
            ox = o.x;
            oy = o.y;
            if (!WU) {
                RowLines rl{row};
                LpTape tape;
                tape.i = tape.f = tape.bound = tape.j = tape.side = 0;
                int b = lp2_dev(rl, nob + cnt, V, ox, oy, false, xx, xy, TAPE ? &tape : nullptr,
                                COUNT ? &oc : nullptr);
                if (TAPE) s_tape[tid] = tape;
                if (b < nob + cnt) enqueue(b);
            }
        }
        if (WU) {
            // the whole warp runs its LP2s together (lanes past the crowd's end only help)
            int b = warp_lp2_units(s_wlp[WU ? tid >> 5 : 0], s_lines, tid * kp, active, cnt, V, ox,
                                   oy, xx, xy);
            if (active && b < cnt) enqueue(b);
        }
        __syncthreads();
        // ---- phase 3: least penetration for the queued agents, G lanes each.  Queue
        // entries are dealt round-robin over the warps (entry q to warp q % warps), so a
        // short queue keeps every warp busy instead of filling the first warp and leaving
        // the others waiting at the barrier.
        const int nq = s_qn;
        constexpr int GL = WU ? 1 : G;  // lanes per queue entry
        constexpr int kGroupsPerWarp = 32 / GL, kWarps = TPB / 32;
        const int gi = tid / GL;
        const int q0 = (gi % kGroupsPerWarp) * kWarps + gi / kGroupsPerWarp;
        if (WU) {
            // every lane of every warp takes part in each round (warp-uniform trip count)
#pragma unroll 1
            for (int q1 = 0; q1 < nq; q1 += TPB) {
                const int q = q1 + q0;
                const bool has = q < nq;
                const int ag = has ? s_queue[q] : 0;
                float2 x = has ? s_x[ag] : make_float2(0.0f, 0.0f);
                proj += (unsigned)warp_lp3_units(s_wlp[WU ? tid >> 5 : 0], s_lines, ag * kp, has,
                                                 has ? s_cnt[ag] : 0, has ? s_b[ag] : 0,
                                                 has ? s_V[ag] : 0.0f, x.x, x.y);
                if (has) s_x[ag] = x;
            }
        }
        for (int q = q0; !WU && q < nq; q += TPB / GL) {
            int ag = s_queue[q];
            float2 x = s_x[ag];
            int np;
            if (G == 1) np = lp3_dev(s_lines + ag * kp, s_cnt[ag], s_b[ag], s_V[ag], x.x, x.y,
                                     TAPE ? &s_tape[TAPE ? ag : 0] : nullptr, COUNT ? &oc : nullptr,
                                     OBS ? s_nob[OBS ? ag : 0] : 0);
            else np = lp3_group_dev<WU ? 4 : G>(s_lines + ag * kp, s_cnt[ag], s_b[ag], s_V[ag], x.x, x.y);
            if ((tid & (G - 1)) == 0) {
                s_x[ag] = x;
                proj += (unsigned)np;
            }
        }
        __syncthreads();
        // ---- phase 4: integrate
        float bx0 = INFINITY, by0 = INFINITY, bx1 = -INFINITY, by1 = -INFINITY;
        if (active) {
            if (s_queued[tid]) {
                float2 x = s_x[tid];
                xx = x.x;
                xy = x.y;
            }
            const float nx = __fmaf_rn(xx, dt, p.x), ny = __fmaf_rn(xy, dt, p.y);
            if (!isfinite(xx) || !isfinite(xy) || !isfinite(nx) || !isfinite(ny))
                atomicOr(&a.misc_rw->error, kErrNumeric);
            a.out.vel[t] = make_float2(xx, xy);
            a.out.pos[t] = make_float2(nx, ny);
            if (TAPE) {
                a.tape[me] = s_tape[TAPE ? tid : 0].pack();
                if (a.rec_pos) a.rec_pos[me] = p;
                if (a.rec_vel) a.rec_vel[me] = a.in.vel[t];
                if (a.rec_next) a.rec_next[me] = make_float2(nx, ny);
            }
            bx0 = bx1 = nx;
            by0 = by1 = ny;
        }
        // the box of the positions written, for the next step's grid (single scene): a
        // warp reduction (fminf / fmaxf skip NaN, as the bounding-box scan does), then one
        // atomic per bound on the warp's copy of the accumulator
        if (a.bbox_acc) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                bx0 = fminf(bx0, __shfl_xor_sync(0xffffffffu, bx0, o));
                by0 = fminf(by0, __shfl_xor_sync(0xffffffffu, by0, o));
                bx1 = fmaxf(bx1, __shfl_xor_sync(0xffffffffu, bx1, o));
                by1 = fmaxf(by1, __shfl_xor_sync(0xffffffffu, by1, o));
            }
            if ((tid & 31) == 0 && bx0 <= bx1) {
                int* acc = a.bbox_acc + ((blockIdx.x * (TPB / 32) + (tid >> 5)) % kBoxCopies) * kBoxStride;
                atomicMin(acc + 0, float_order_code(bx0));
                atomicMin(acc + 1, float_order_code(by0));
                atomicMax(acc + 2, float_order_code(bx1));
                atomicMax(acc + 3, float_order_code(by1));
            }
        }
        // batch: the box of each scene's written positions, for the scene's next grid -- the
        // warp's lanes grouped by scene (a warp straddles at most a few), a min / max
        // reduction per group, one atomic per bound per group
        if (a.scene_box) {
            const int sid = active ? a.slot_scene[t] : -1;
            const unsigned grp = __match_any_sync(0xffffffffu, sid);
            const int c0 = __reduce_min_sync(grp, float_order_code(bx0));
            const int c1 = __reduce_min_sync(grp, float_order_code(by0));
            const int c2 = __reduce_max_sync(grp, float_order_code(bx1));
            const int c3 = __reduce_max_sync(grp, float_order_code(by1));
            if (sid >= 0 && (tid & 31) == __ffs(grp) - 1) {
                int* acc = a.scene_box[sid].box_acc[a.scene_box_slot];
                atomicMin(acc + 0, c0);
                atomicMin(acc + 1, c1);
                atomicMax(acc + 2, c2);
                atomicMax(acc + 3, c3);
            }
        }
        // ---- counters: one shared-memory atomic per warp
        unsigned wc = __reduce_add_sync(0xffffffffu, cand);
        unsigned wl = __reduce_add_sync(0xffffffffu, (unsigned)cnt);
        unsigned wa = __reduce_add_sync(0xffffffffu, active ? 1u : 0u);
        if ((tid & 31) == 0) {
            atomicAdd(&s_cand, (unsigned long long)wc);
            atomicAdd(&s_lines_n, (unsigned long long)wl);
            atomicAdd(&s_act, (unsigned long long)wa);
        }
        if (tid == 0) s_lp3 += (unsigned long long)nq;
        {
            const unsigned v3[3] = {sc.retries, sc.cold, sc.rows};
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const unsigned w = __reduce_add_sync(0xffffffffu, v3[q]);
                if ((tid & 31) == 0 && w) atomicAdd(&s_search[q], (unsigned long long)w);
            }
            sc = SearchCount{0u, 0u, 0u};
            const unsigned wp = __reduce_add_sync(0xffffffffu, proj);
            if ((tid & 31) == 0 && wp) atomicAdd(&s_proj, (unsigned long long)wp);
            proj = 0;
        }
        if (COUNT) {
            unsigned v[4] = {oc.lp1, oc.bounds, oc.checks, oc.bis};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                unsigned w = __reduce_add_sync(0xffffffffu, v[q]);
                if ((tid & 31) == 0) atomicAdd(&s_ops[q], (unsigned long long)w);
            }
            oc = OpCount{0u, 0u, 0u, 0u};
        }
        if (OBS) {
            li += gridDim.x;
            tile = li < nlist ? a.obs_tiles[li] : ntiles;
            __syncthreads();
            continue;
        }
        if ((int)gridDim.x >= ntiles) break;  // one CTA per tile: no work queue
        if (tid == 0) s_tile = (int)atomicAdd(&a.misc_rw->tile_counter, 1u) + (int)gridDim.x;
        __syncthreads();
        tile = s_tile;
    }
    __syncthreads();
    // atomic: with obstacles the plain and the obstacle launch run side by side and their
    // CTAs share rows
    if (tid == 0) {
        unsigned long long* c = a.block_counters + kBlockCounters * (size_t)blockIdx.x;
        atomicAdd(c + 0, s_act);
        atomicAdd(c + 1, s_lp3);
        atomicAdd(c + 2, s_cand);
        atomicAdd(c + 3, s_lines_n);
        for (int q = 0; q < 3; ++q) atomicAdd(c + 8 + q, s_search[q]);
        atomicAdd(c + 11, s_proj);
        if (COUNT)
            for (int q = 0; q < 4; ++q) atomicAdd(c + 4 + q, s_ops[COUNT ? q : 0]);
    }
}

// ---------------------------------------------------------------------------------
// Agent split (lanes = 4): each agent is stepped by a quad of lanes (lanes 4j..4j+3 of a
// warp), for crowds too small to fill the GPU, where a step is as long as one agent's
// chain of dependent instructions.  The quad scans the candidate rows together (lane q
// takes every fourth candidate and parks its entrants in its own shared-memory row; the
// quad's leader inserts them all), builds the half-planes four at a time, and solves the
// least-penetration LP with the 4-lane group LP3; LP2 stays on the leader.  Every decision
// is the one-lane kernel's (the same exact neighbour list, the same half-plane arithmetic,
// the same LP decisions), so the results are bitwise those of the other modes.  Single
// scene, no obstacles, no record of the LP (those launches use one lane per agent).
// ---------------------------------------------------------------------------------
// candidates per lane per round, sixteen per quad: at these crowd sizes a search waits on
// its loads, and more of them in flight shorten it (measured on the 2,500- and 10,000-agent
// crossings: 2-4% faster per step than eight per quad, twenty no better)
constexpr int kSplitU = 4;

template <int KMAX, int CAP>
__device__ __forceinline__ unsigned knn_split_dev(const MainArgs& a, const GridDev& g, int cell_off, float nd,
                                                  int t, float2 p, int k, float lim0,
                                                  unsigned long long* quad_buf, int stride, int gq,
                                                  unsigned qmask, int lead, unsigned long long (&kk)[KMAX],
                                                  SearchCount& sc) {
    static_assert(CAP > kSplitU, "parking space for one round");
    const int cy = cell_coord(p.y, g.ymin, g.inv, g.gy);
    const float nd2 = __fmul_rn(nd, nd);
    const float lim_max = __int_as_float(__float_as_int(nd2) - 1);
    if (lim0 != lim0) {
        lim0 = density_lim(a, g, cell_off, p, k);
        if (gq == 0) ++sc.cold;
    }
    lim0 = fminf(lim0, lim_max);
    unsigned long long* buf = quad_buf + gq * stride;
    unsigned cand = 0;
    int nb = 0;
    float lim = lim0;
    // the leader inserts every lane's parked keys (the sorted list is the same in any
    // insertion order); lim is then its list's k-th d^2 for the whole quad
    auto drain_quad = [&]() {
        int n4[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) n4[j] = __shfl_sync(qmask, nb, lead + j);
        __syncwarp(qmask);  // the parked keys are visible to the leader
        if (gq == 0) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const unsigned long long* bj = quad_buf + j * stride;
#pragma unroll 1
                for (int i = 0; i < n4[j]; ++i) insert_key<KMAX>(bj[i], kk);
            }
            if (kk[KMAX - 1] != ~0ull) lim = fminf(lim, __uint_as_float((unsigned)(kk[KMAX - 1] >> 32)));
        }
        lim = __shfl_sync(qmask, lim, lead);
        nb = 0;
        __syncwarp(qmask);  // the leader has read the rows before they are refilled
    };
#pragma unroll 1
    for (;;) {
#pragma unroll
        for (int l = 0; l < KMAX; ++l) kk[l] = (l < KMAX - k) ? 0ull : ~0ull;
        lim = lim0;
        nb = 0;
        int y = cy, up = cy + 1, dn = cy - 1;
        float h = 0.0f;
#pragma unroll 1
        for (;;) {
            const float w = sqrtf(fmaxf(lim * (1.0f + 1e-5f) - h * h, 0.0f)) + 2.0f * g.slop;
            const int x0 = cell_coord(p.x - w, g.xmin, g.inv, g.gx);
            const int x1 = cell_coord(p.x + w, g.xmin, g.inv, g.gx);
            const int c = cell_off + y * g.gx;
            uint32_t q0 = 0u, q1 = 0u;
            if (idx_ok(c + x0 >= 0 && c + x1 + 1 <= a.misc->grid.num_cells, &a.misc_rw->error)) {
                q0 = a.cell_start[c + x0];
                q1 = a.cell_start[c + x1 + 1];
                if (!idx_ok(q0 <= q1 && q1 <= (uint32_t)a.n, &a.misc_rw->error)) q1 = q0;
            }
            if (gq == 0) {
                cand += q1 - q0;
                ++sc.rows;
            }
            // rounds of 4 x kSplitU candidates, the same count in every lane of the quad
#pragma unroll 1
            for (uint32_t base = q0; base < q1; base += 4 * kSplitU) {
                float d2[kSplitU];
                unsigned id[kSplitU];
#pragma unroll
                for (int u = 0; u < kSplitU; ++u) {
                    const uint32_t qu = base + (uint32_t)(gq + 4 * u);
                    float4 mj = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    if (qu < q1) mj = a.in.msg[qu];
                    const float ddx = __fsub_rn(mj.x, p.x), ddy = __fsub_rn(mj.y, p.y);
                    d2[u] = __fadd_rn(__fmul_rn(ddx, ddx), __fmul_rn(ddy, ddy));
                    id[u] = __float_as_uint(mj.w);
                    if (qu >= q1 || (int)qu == t) d2[u] = INFINITY;
                }
#pragma unroll
                for (int u = 0; u < kSplitU; ++u)
                    if (d2[u] <= lim) buf[nb++] = ((unsigned long long)__float_as_uint(d2[u]) << 32) | id[u];
                if (__any_sync(qmask, nb > CAP - kSplitU)) drain_quad();
            }
            const float hu = up < g.gy ? (g.ymin + (float)up * g.s) - p.y : INFINITY;
            const float hd = dn >= 0 ? p.y - (g.ymin + (float)(dn + 1) * g.s) : INFINITY;
            if (hu <= hd) {
                y = up++;
                h = hu;
            } else {
                y = dn--;
                h = hd;
            }
            if (h == INFINITY) break;
            h = fmaxf(0.0f, h - g.slop);
            if (h * h * (1.0f - 1e-5f) > lim) break;
        }
        drain_quad();
        const int full = __shfl_sync(qmask, kk[KMAX - 1] != ~0ull ? 1 : 0, lead);
        if (full || !(lim0 < lim_max)) break;
        lim0 = fminf(fmaxf(2.25f * lim0, 1e-6f * lim_max), lim_max);
        if (gq == 0) ++sc.retries;
    }
    return cand;
}

template <int KMAX, int TPB>
__global__ void __launch_bounds__(TPB, main_min_blocks<KMAX, TPB>()) orca_split_kernel(MainArgs a) {
    pdl_wait();
    constexpr int KP = row_len<KMAX>();
    extern __shared__ float4 s_lines[];  // TPB rows: each lane's parking row; the leader's holds the lines
    __shared__ unsigned long long s_cand, s_lines_n, s_act, s_lp3, s_proj;
    __shared__ unsigned long long s_search[3];
    const int tid = threadIdx.x, lane = tid & 31, gq = tid & 3;
    const int lead = lane & ~3;
    const unsigned qmask = 0xfu << lead;
    if (tid == 0) {
        s_cand = s_lines_n = s_act = s_lp3 = s_proj = 0;
        s_search[0] = s_search[1] = s_search[2] = 0;
    }
    __syncthreads();
    SearchCount sc{0u, 0u, 0u};
    const int t = blockIdx.x * (TPB / 4) + (tid >> 2);
    const bool active = t < a.n;  // the same for the four lanes of a quad
    float4* row = s_lines + (tid & ~3) * KP;  // the agent's half-planes (the leader's row)
    unsigned cand = 0;
    int cnt = 0, lp3 = 0, proj = 0;
    float bx0 = INFINITY, by0 = INFINITY, bx1 = -INFINITY, by1 = -INFINITY;
    if (active) {
        SceneView sv;
        scene_view(a, t, sv);
        const float dt = sv.dt;
        const float4 me4 = a.in.msg[t];
        const float2 p = make_float2(me4.x, me4.y);
        const uint32_t me = __float_as_uint(me4.w);
        const float V = a.prm.max_speed[t];
        float lim0 = __int_as_float(0x7fffffff);
        if (a.prm.hint) {
            const float hd = sqrtf(a.prm.hint[t]) * (1.0f + 1e-3f) + 2.5f * V * dt + 1e-3f;
            lim0 = hd * hd;
        }
        unsigned long long kk[KMAX];
        cand = knn_split_dev<KMAX, 2 * KP>(a, sv.g, sv.cell_off, sv.nd, t, p, sv.k, lim0,
                                           reinterpret_cast<unsigned long long*>(row), 2 * KP, gq, qmask,
                                           lead, kk, sc);
        if (gq == 0) {
            if (a.prm.hint)
                a.prm.hint[t] = kk[KMAX - 1] != ~0ull ? __uint_as_float((unsigned)(kk[KMAX - 1] >> 32)) : INFINITY;
            // the neighbours' slots, in rank order, parked in the row
#pragma unroll
            for (int l = 0; l < KMAX; ++l) {
                if (l >= KMAX - sv.k && kk[l] != ~0ull) {
                    const uint32_t nid = (uint32_t)kk[l];
                    if (!idx_ok(nid < (uint32_t)a.n, &a.misc_rw->error)) continue;
                    const uint32_t q = a.in.slot[nid];
                    if (!idx_ok(q < (uint32_t)a.n, &a.misc_rw->error)) continue;
                    row[cnt++].w = __uint_as_float(q);
                }
            }
            if (a.rec_nbr) {
                int w = 0;
#pragma unroll
                for (int l = 0; l < KMAX; ++l)
                    if (l >= KMAX - sv.k)
                        a.rec_nbr[(size_t)me * a.rec_stride + (w++)] =
                            kk[l] != ~0ull ? (int32_t)(kk[l] & 0xffffffffu) : -1;
                for (; w < a.rec_stride; ++w) a.rec_nbr[(size_t)me * a.rec_stride + w] = -1;
            }
            if (a.rec_cell) {
                const int cx = cell_coord(p.x, sv.g.xmin, sv.g.inv, sv.g.gx);
                const int cyy = cell_coord(p.y, sv.g.ymin, sv.g.inv, sv.g.gy);
                a.rec_cell[me] = (uint32_t)sv.cell_off + (uint32_t)cyy * (uint32_t)sv.g.gx + (uint32_t)cx;
            }
        }
        cnt = __shfl_sync(qmask, cnt, lead);
        __syncwarp(qmask);
        // half-planes l = gq, gq + 4, ... (each lane overwrites only its own entries' slots)
        const float2 v = a.in.vel[t];
        const float itau = __fdividef(1.0f, a.prm.tau[t]);
        const float idt = __fdividef(1.0f, dt);
        const float half_idt = 0.5f * idt;
#pragma unroll 1
        for (int l = gq; l < cnt; l += 4) {
            const int q = __float_as_int(row[l].w);
            row[l] = orca_line_dev(p, v, me4.z, itau, dt, half_idt, me, a.in.msg[q], a.in.vel[q]);
        }
        __syncwarp(qmask);
        float xx = 0.0f, xy = 0.0f;
        int b = cnt;
        if (gq == 0) {
            const float2 o = pref_velocity_dev(p, a.prm.goal[t], a.prm.pref_speed[t], dt, idt);
            RowLines rl{row};
            b = lp2_dev(rl, cnt, V, o.x, o.y, false, xx, xy);
        }
        b = __shfl_sync(qmask, b, lead);
        xx = __shfl_sync(qmask, xx, lead);
        xy = __shfl_sync(qmask, xy, lead);
        if (b < cnt) {
            proj = lp3_group_dev<4>(row, cnt, b, V, xx, xy);
            lp3 = 1;
        }
        if (gq == 0) {
            const float nx = __fmaf_rn(xx, dt, p.x), ny = __fmaf_rn(xy, dt, p.y);
            if (!isfinite(xx) || !isfinite(xy) || !isfinite(nx) || !isfinite(ny))
                atomicOr(&a.misc_rw->error, kErrNumeric);
            a.out.vel[t] = make_float2(xx, xy);
            a.out.pos[t] = make_float2(nx, ny);
            bx0 = bx1 = nx;
            by0 = by1 = ny;
        }
    }
    if (a.bbox_acc) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            bx0 = fminf(bx0, __shfl_xor_sync(0xffffffffu, bx0, o));
            by0 = fminf(by0, __shfl_xor_sync(0xffffffffu, by0, o));
            bx1 = fmaxf(bx1, __shfl_xor_sync(0xffffffffu, bx1, o));
            by1 = fmaxf(by1, __shfl_xor_sync(0xffffffffu, by1, o));
        }
        if (lane == 0 && bx0 <= bx1) {
            int* acc = a.bbox_acc + ((blockIdx.x * (TPB / 32) + (tid >> 5)) % kBoxCopies) * kBoxStride;
            atomicMin(acc + 0, float_order_code(bx0));
            atomicMin(acc + 1, float_order_code(by0));
            atomicMax(acc + 2, float_order_code(bx1));
            atomicMax(acc + 3, float_order_code(by1));
        }
    }
    // counters: the leaders' counts (one shared-memory atomic per warp)
    const bool leader = active && gq == 0;
    const unsigned wc = __reduce_add_sync(0xffffffffu, leader ? cand : 0u);
    const unsigned wl = __reduce_add_sync(0xffffffffu, leader ? (unsigned)cnt : 0u);
    const unsigned wa = __reduce_add_sync(0xffffffffu, leader ? 1u : 0u);
    const unsigned w3 = __reduce_add_sync(0xffffffffu, leader ? (unsigned)lp3 : 0u);
    const unsigned wp = __reduce_add_sync(0xffffffffu, leader ? (unsigned)proj : 0u);
    const unsigned v3[3] = {sc.retries, sc.cold, sc.rows};
    unsigned ws[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) ws[q] = __reduce_add_sync(0xffffffffu, v3[q]);
    if (lane == 0) {
        atomicAdd(&s_cand, (unsigned long long)wc);
        atomicAdd(&s_lines_n, (unsigned long long)wl);
        atomicAdd(&s_act, (unsigned long long)wa);
        atomicAdd(&s_lp3, (unsigned long long)w3);
        if (wp) atomicAdd(&s_proj, (unsigned long long)wp);
        for (int q = 0; q < 3; ++q)
            if (ws[q]) atomicAdd(&s_search[q], (unsigned long long)ws[q]);
    }
    __syncthreads();
    if (tid == 0) {
        // four split CTAs (at least 64 agents) share one block's counters
        unsigned long long* c = a.block_counters + kBlockCounters * (size_t)(blockIdx.x >> 2);
        atomicAdd(c + 0, s_act);
        atomicAdd(c + 1, s_lp3);
        atomicAdd(c + 2, s_cand);
        atomicAdd(c + 3, s_lines_n);
        for (int q = 0; q < 3; ++q) atomicAdd(c + 8 + q, s_search[q]);
        atomicAdd(c + 11, s_proj);
    }
}

// at most one CTA per 64 agents (the smallest CTA; the agent split's CTAs share counters)
int main_blocks(int n) { return (n + 63) / 64; }

// CTAs of the ORCA kernel that fit on the GPU at once (for the persistent launch).
template <int KMAX, int TPB, int G>
static int resident_blocks_k() {
    constexpr size_t smem = main_smem_bytes<KMAX, TPB>();
    if (cudaFuncSetAttribute(orca_main_kernel<KMAX, TPB, G>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return 0;
    int per_sm = 0, dev = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, orca_main_kernel<KMAX, TPB, G>, TPB, smem) !=
        cudaSuccess)
        return 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return per_sm * sms;
}

template <int KMAX, int TPB, int G>
static cudaError_t launch_main_k(const MainArgs& a, int grid_blocks, cudaStream_t st) {
    constexpr size_t smem = main_smem_bytes<KMAX, TPB>();
    cudaError_t e = cudaFuncSetAttribute(orca_main_kernel<KMAX, TPB, G>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int nb = (a.n + TPB - 1) / TPB;
    if (grid_blocks > 0 && grid_blocks < nb) nb = grid_blocks;
    return launch_pdl(orca_main_kernel<KMAX, TPB, G>, nb, TPB, smem, st, a);
}

// Dispatch over (k bound, threads per CTA, LP3 lanes per agent).  resident != null:
// return the resident CTA count instead of launching.
template <int KMAX, int TPB>
static cudaError_t dispatch_g(const MainArgs& a, int g, int grid_blocks, cudaStream_t st, int* resident) {
    if (g == 32) {
        if (resident) { *resident = resident_blocks_k<KMAX, TPB, 32>(); return cudaSuccess; }
        return launch_main_k<KMAX, TPB, 32>(a, grid_blocks, st);
    }
    // agent split: a single scene without obstacles (the plain launch of an obstacle step
    // skips the flagged tiles of TPB agents, which only the one-lane kernel knows)
    if (g == 4 && !resident && !a.scenes && !a.tile_near && grid_blocks <= 0) {
        constexpr size_t smem = main_smem_bytes<KMAX, TPB>();
        cudaError_t e = cudaFuncSetAttribute(orca_split_kernel<KMAX, TPB>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        return launch_pdl(orca_split_kernel<KMAX, TPB>, (a.n + TPB / 4 - 1) / (TPB / 4), TPB, smem, st, a);
    }
    if (resident) { *resident = resident_blocks_k<KMAX, TPB, 1>(); return cudaSuccess; }
    return launch_main_k<KMAX, TPB, 1>(a, grid_blocks, st);
}

template <int KMAX>
static cudaError_t dispatch_tpb(const MainArgs& a, const LaunchShape& sh, int grid_blocks, cudaStream_t st,
                                int* resident) {
    if (sh.tpb == 64) return dispatch_g<KMAX, 64>(a, sh.lp3_group, grid_blocks, st, resident);
    if (sh.tpb == 256) return dispatch_g<KMAX, 256>(a, sh.lp3_group, grid_blocks, st, resident);
    return dispatch_g<KMAX, 128>(a, sh.lp3_group, grid_blocks, st, resident);
}

// Obstacle launch: one lane per solve, 64 or 128 threads; the listed tiles are dealt over
// at most 2048 CTAs (one pass each when fewer tiles are listed).
template <int KMAX, int TPB>
static cudaError_t launch_obs_k(const MainArgs& a, cudaStream_t st) {
    constexpr size_t smem_max = sizeof(float4) * TPB * obs_row_len(KMAX, kMaxObstacleNeighbors);
    cudaError_t e = cudaFuncSetAttribute(orca_main_kernel<KMAX, TPB, 1, false, false, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_max);
    if (e != cudaSuccess) return e;
    MainArgs b = a;
    b.row_stride = obs_row_len(KMAX, a.kobst);
    const int ntiles = (a.n + TPB - 1) / TPB;
    return launch_pdl(orca_main_kernel<KMAX, TPB, 1, false, false, true>, ntiles < 2048 ? ntiles : 2048,
                      TPB, sizeof(float4) * TPB * b.row_stride, st, b);
}

// A step with static obstacles: flag and list the tiles near a segment, then the plain
// launch over the other tiles and the obstacle launch over the listed ones.  The two
// touch disjoint tiles, so with a side stream they run concurrently (a fork after the
// flags, a join before the step goes on): the few obstacle tiles, often the slowest
// (agents pressed into walls need least penetration), then overlap the bulk instead of
// trailing it.  Tiles are 64 or 128 agents in both (a 256-thread shape runs as 128).
template <int KMAX>
static cudaError_t dispatch_obs(const MainArgs& a, const LaunchShape& sh, cudaStream_t st,
                                const SideStream* side) {
    if (a.n == 0) return cudaSuccess;
    const int tpb = sh.tpb == 64 ? 64 : 128;
    const int ntiles = (a.n + tpb - 1) / tpb;
    cudaError_t e = launch_pdl(obstacle_tiles_kernel, (ntiles * 32 + 255) / 256, 256, 0, st, a, tpb);
    if (e != cudaSuccess) return e;
    MainArgs b = a;
    b.tile_near = nullptr;
    cudaStream_t obs_st = st;
    if (side) {
        if ((e = cudaEventRecord(side->fork, st)) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(side->st, side->fork, 0)) != cudaSuccess) return e;
        obs_st = side->st;
        e = tpb == 64 ? launch_obs_k<KMAX, 64>(b, obs_st) : launch_obs_k<KMAX, 128>(b, obs_st);
        if (e != cudaSuccess) return e;
    }
    e = dispatch_tpb<KMAX>(a, LaunchShape{tpb, sh.lp3_group}, 0, st, nullptr);
    if (e != cudaSuccess) return e;
    if (side) {
        if ((e = cudaEventRecord(side->join, side->st)) != cudaSuccess) return e;
        return cudaStreamWaitEvent(st, side->join, 0);
    }
    return tpb == 64 ? launch_obs_k<KMAX, 64>(b, st) : launch_obs_k<KMAX, 128>(b, st);
}

// Operation-counting launch: 128 threads, serial LP3, one CTA per tile (the counts are
// algorithmic, so any launch shape gives the same numbers).
template <int KMAX>
static cudaError_t launch_count_k(const MainArgs& a, cudaStream_t st) {
    constexpr size_t smem = main_smem_bytes<KMAX, 128>();
    cudaError_t e = cudaFuncSetAttribute(orca_main_kernel<KMAX, 128, 1, false, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(orca_main_kernel<KMAX, 128, 1, false, true>, (a.n + 127) / 128, 128, smem, st, a);
}

template <int KMAX>
static cudaError_t launch_tape_k(const MainArgs& a, cudaStream_t st) {
    constexpr size_t smem = main_smem_bytes<KMAX, 128>();
    cudaError_t e = cudaFuncSetAttribute(orca_main_kernel<KMAX, 128, 1, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(orca_main_kernel<KMAX, 128, 1, true>, (a.n + 127) / 128, 128, smem, st, a);
}

static cudaError_t dispatch(const MainArgs& a, int kmax, const LaunchShape& sh, int grid_blocks,
                            cudaStream_t st, int* resident, const SideStream* side = nullptr) {
    if (a.tape && !resident) {  // recording step of a rollout: 128 threads, serial LP3
        if (kmax <= 10) return launch_tape_k<10>(a, st);
        if (kmax <= 16) return launch_tape_k<16>(a, st);
        if (kmax <= 20) return launch_tape_k<20>(a, st);
        return launch_tape_k<32>(a, st);
    }
    if (a.nseg > 0 && !resident) {  // static obstacles (single scene, no tape, no counting)
        if (kmax <= 10) return dispatch_obs<10>(a, sh, st, side);
        if (kmax <= 16) return dispatch_obs<16>(a, sh, st, side);
        if (kmax <= 20) return dispatch_obs<20>(a, sh, st, side);
        return dispatch_obs<32>(a, sh, st, side);
    }
    if (a.count_ops && !resident) {
        if (kmax <= 10) return launch_count_k<10>(a, st);
        if (kmax <= 16) return launch_count_k<16>(a, st);
        if (kmax <= 20) return launch_count_k<20>(a, st);
        return launch_count_k<32>(a, st);
    }
    if (kmax <= 10) return dispatch_tpb<10>(a, sh, grid_blocks, st, resident);
    if (kmax <= 16) return dispatch_tpb<16>(a, sh, grid_blocks, st, resident);
    if (kmax <= 20) return dispatch_tpb<20>(a, sh, grid_blocks, st, resident);
    return dispatch_tpb<32>(a, sh, grid_blocks, st, resident);
}

int main_resident_blocks(int kmax, const LaunchShape& sh) {
    int r = 0;
    MainArgs dummy{};
    dispatch(dummy, kmax, sh, 0, nullptr, &r);
    return r;
}

cudaError_t launch_main(const MainArgs& a, int kmax, const LaunchShape& sh, int grid_blocks,
                        cudaStream_t st, const SideStream* side) {
    return dispatch(a, kmax, sh, grid_blocks, st, nullptr, side);
}

}  // namespace orca
