// orca_main.cu -- per-agent ORCA velocity selection and integration (Sections 2-3).
//
// One thread per agent, agents in cell order (so a warp's neighbourhoods overlap and its
// candidate reads hit L1/L2).  Per agent:
//   1. exact k nearest neighbours by (fl32 d^2, agent index) among agents strictly
//      inside r_obs (Fig. 2), found by a ring search over grid cells with conservative
//      per-cell and per-ring distance bounds;
//   2. one ORCA half-plane per neighbour (Fig. 1), kept on chip, never stored;
//   3. LP2 (incremental 2-D LP over the disc and the half-planes, in neighbour order) and,
//      if it fails, LP3 (least penetration, Section 3);
//   4. vel <- x, pos <- pos + x*dt, written in the same sorted slot of the other buffer.
#include "orca_common.cuh"

namespace orca {

// A half-plane in normal form: the valid side is {x : n.x >= c}, |n| = 1.  In the
// paper's point-and-direction form (boundary through P with direction d, valid side on
// the left of d) this is n = (-d.y, d.x) and c = n.P.  The normal form keeps every LP1
// computation at the scale of the speed disc: the boundary point nearest the origin is
// c*n, and a line with |c| > V misses the disc before any large number is formed; the
// least-penetration bisectors need no intersection points (which can lie far away).
struct Ln {
    float nx, ny, c;
};

constexpr float kEps = 1e-5f;

__device__ __forceinline__ float det2f(float ax, float ay, float bx, float by) {
    return ax * by - ay * bx;
}

// LP1: best point on the boundary of line i inside the disc |x| <= V and half-planes
// 0..i-1.  x(t) = c_i n_i + t d_i with d_i = (n_i.y, -n_i.x).  The disc gives
// |t| <= sqrt(V^2 - c_i^2); half-plane j gives -det(n_i, n_j) t >= c_j - c_i (n_i.n_j),
// an upper bound on t when det(n_i, n_j) > 0, a lower one when < 0; a (nearly) parallel
// j (|det| <= eps) is infeasible iff its right-hand side is positive.
__device__ bool lp1_dev(const Ln* L, int i, float V, float ox, float oy, bool dir_opt, float& xx,
                        float& xy) {
    const Ln li = L[i];
    float D = V * V - li.c * li.c;
    if (D < 0.0f) return false;
    float sq = sqrtf(D);
    float tL = -sq, tR = sq;
    for (int j = 0; j < i; ++j) {
        const Ln lj = L[j];
        float den = det2f(li.nx, li.ny, lj.nx, lj.ny);
        float rhs = lj.c - li.c * (li.nx * lj.nx + li.ny * lj.ny);
        if (fabsf(den) <= kEps) {
            if (rhs > 0.0f) return false;
            continue;
        }
        float t = -rhs / den;
        if (den >= 0.0f) tR = fminf(tR, t);
        else tL = fmaxf(tL, t);
        if (tL > tR) return false;
    }
    float dx = li.ny, dy = -li.nx;
    float t;
    if (dir_opt) {
        t = (ox * dx + oy * dy > 0.0f) ? tR : tL;
    } else {
        t = fminf(fmaxf(ox * dx + oy * dy, tL), tR);
    }
    xx = li.c * li.nx + t * dx;
    xy = li.c * li.ny + t * dy;
    return true;
}

// LP2: incremental 2-D LP over lines 0..n-1 in neighbour order (Section 3).  Returns n on
// success, else the index of the line where LP1 failed (x keeps its last value).
__device__ int lp2_dev(const Ln* L, int n, float V, float ox, float oy, bool dir_opt, float& xx,
                       float& xy) {
    if (dir_opt) {
        xx = ox * V;
        xy = oy * V;
    } else {
        float o2 = ox * ox + oy * oy;
        if (o2 > V * V) {
            float s = V / sqrtf(o2);
            xx = ox * s;
            xy = oy * s;
        } else {
            xx = ox;
            xy = oy;
        }
    }
    for (int i = 0; i < n; ++i) {
        if (L[i].c - (L[i].nx * xx + L[i].ny * xy) > 0.0f) {
            float sx = xx, sy = xy;
            if (!lp1_dev(L, i, V, ox, oy, dir_opt, xx, xy)) {
                xx = sx;
                xy = sy;
                return i;
            }
        }
    }
    return n;
}

// LP3: least penetration (Section 3).  Penetration of line i at x: c_i - n_i.x.  For a
// line violated by more than the current penetration, the bisector of lines i and j
// (equal penetration) is the half-plane (n_j - n_i).x >= c_j - c_i, normalised; same-
// direction parallel lines give none.  LP2 in direction mode maximises n_i.x over the
// bisectors; a numerically failed LP2 keeps x.
template <int KMAX>
__device__ void lp3_dev(const Ln* L, int n, int begin, float V, float& xx, float& xy) {
    Ln proj[KMAX];
    float dist = 0.0f;
    for (int i = begin; i < n; ++i) {
        const Ln li = L[i];
        if (li.c - (li.nx * xx + li.ny * xy) > dist) {
            int m = 0;
            for (int j = 0; j < i; ++j) {
                const Ln lj = L[j];
                float den = det2f(li.nx, li.ny, lj.nx, lj.ny);
                if (fabsf(den) <= kEps && li.nx * lj.nx + li.ny * lj.ny > 0.0f) continue;
                float mx = lj.nx - li.nx, my = lj.ny - li.ny;
                float inv = rsqrtf(mx * mx + my * my);
                Ln q;
                q.nx = mx * inv;
                q.ny = my * inv;
                q.c = (lj.c - li.c) * inv;
                proj[m++] = q;
            }
            float sx = xx, sy = xy;
            if (lp2_dev(proj, m, V, li.nx, li.ny, true, xx, xy) < m) {
                xx = sx;
                xy = sy;
            }
            dist = li.c - (li.nx * xx + li.ny * xy);
        }
    }
}

// Half-plane of agent (p, v, r, tau) induced by neighbour (pj, vj, rj) -- Fig. 1.
// u runs from the relative velocity to the nearest boundary point of VO^tau; the
// boundary passes through v + u/2 with the valid side along the VO's outward normal.
//   cut-off circle / overlap: n = w/|w| (w = v_rel - p/tau, or p/dt when overlapping),
//     c = n.v + (R/tau - |w|)/2;
//   legs: n is the leg's outward normal and c = n.(v + v_j)/2.
// When overlapping, R/dt - |w| is formed as (R - |q|)/dt with q = p - v_rel dt (both
// O(1) metres), which keeps more of the offset's FP32 precision.
__device__ __forceinline__ Ln orca_line_dev(float2 p, float2 v, float r, float tau, float dt,
                                            uint32_t me, float2 pj, float2 vj, float rj,
                                            uint32_t jid) {
    float px = pj.x - p.x, py = pj.y - p.y;
    float vx = v.x - vj.x, vy = v.y - vj.y;
    float R = r + rj;
    float p2 = px * px + py * py, R2 = R * R;
    Ln L;
    if (p2 > R2) {
        float itau = 1.0f / tau;
        float wx = vx - px * itau, wy = vy - py * itau;
        float w2 = wx * wx + wy * wy, wp = wx * px + wy * py;
        if (wp < 0.0f && wp * wp > R2 * w2) {
            float wl = sqrtf(w2);
            L.nx = wx / wl;
            L.ny = wy / wl;
            L.c = L.nx * v.x + L.ny * v.y + 0.5f * (R * itau - wl);
        } else {
            float leg = sqrtf(p2 - R2);
            if (det2f(px, py, wx, wy) > 0.0f) {  // left leg
                L.nx = -(px * R + py * leg) / p2;
                L.ny = (px * leg - py * R) / p2;
            } else {  // right leg
                L.nx = (py * leg - px * R) / p2;
                L.ny = -(px * leg + py * R) / p2;
            }
            L.c = 0.5f * (L.nx * (v.x + vj.x) + L.ny * (v.y + vj.y));
        }
    } else {
        float qx = px - vx * dt, qy = py - vy * dt;  // = -w dt
        float ql = sqrtf(qx * qx + qy * qy);
        float nx, ny;
        if (ql > 0.0f) {
            nx = -qx / ql;
            ny = -qy / ql;
        } else if (p2 > 0.0f) {
            float ip = 1.0f / sqrtf(p2);
            nx = -px * ip;
            ny = -py * ip;
        } else {
            nx = me < jid ? 1.0f : -1.0f;
            ny = 0.0f;
        }
        L.nx = nx;
        L.ny = ny;
        L.c = nx * v.x + ny * v.y + 0.5f * (R - ql) / dt;
    }
    return L;
}

template <int KMAX>
__global__ void __launch_bounds__(128) orca_main_v0_kernel(MainArgs a) {
    __shared__ unsigned long long s_cand, s_lines;
    if (threadIdx.x == 0) {
        s_cand = 0;
        s_lines = 0;
    }
    __syncthreads();
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    bool active = t < a.n;
    bool used3 = false;
    if (active) {
        const GridDev g = a.misc->grid;
        const float2* __restrict__ spos = a.in.pos;
        const uint32_t* __restrict__ sid = a.prm.id;
        const int k = a.k;
        float2 p = spos[t];
        uint32_t me = sid[t];
        int cx = cell_coord(p.x, g.xmin, g.inv, g.gx);
        int cy = cell_coord(p.y, g.ymin, g.inv, g.gy);
        float nd2 = __fmul_rn(a.nd, a.nd);

        // top-k keys (d2 bits << 32 | agent index), ascending; the first KMAX-k entries are
        // permanent zero sentinels so that the live window is the last k entries
        unsigned long long kk[KMAX];
        int ks[KMAX];
#pragma unroll
        for (int l = 0; l < KMAX; ++l) {
            kk[l] = (l < KMAX - k) ? 0ull : ~0ull;
            ks[l] = -1;
        }
        unsigned long long cand = 0;
        const float s = g.s, slop = g.slop;
        for (int r = 0;; ++r) {
            for (int dyc = -r; dyc <= r; ++dyc) {
                int yy = cy + dyc;
                if (yy < 0 || yy >= g.gy) continue;
                bool full_row = (dyc == -r || dyc == r);
                for (int part = 0; part < (full_row ? 1 : 2); ++part) {
                    int x0, x1;
                    if (full_row) {
                        x0 = cx - r;
                        x1 = cx + r;
                    } else {
                        x0 = x1 = part == 0 ? cx - r : cx + r;
                    }
                    x0 = max(x0, 0);
                    x1 = min(x1, g.gx - 1);
                    if (x0 > x1) continue;
                    // conservative lower bound of fl32 d^2 to any agent of these cells
                    float bx0 = g.xmin + (float)x0 * s, bx1 = g.xmin + (float)(x1 + 1) * s;
                    float by0 = g.ymin + (float)yy * s, by1 = by0 + s;
                    float ddx = fmaxf(0.0f, fmaxf(bx0 - p.x, p.x - bx1) - slop);
                    float ddy = fmaxf(0.0f, fmaxf(by0 - p.y, p.y - by1) - slop);
                    float lb2 = (ddx * ddx + ddy * ddy) * (1.0f - 1e-5f);
                    bool full = kk[KMAX - 1] != ~0ull;
                    float kth = full ? __uint_as_float((unsigned)(kk[KMAX - 1] >> 32)) : nd2;
                    if (full ? (lb2 > kth) : (lb2 >= nd2)) continue;
                    int c0 = yy * g.gx + x0;
                    uint32_t q0 = a.cell_start[c0], q1 = a.cell_start[c0 + (x1 - x0) + 1];
                    for (uint32_t q = q0; q < q1; ++q) {
                        if ((int)q == t) continue;
                        ++cand;
                        float2 pj = spos[q];
                        float ddx2 = __fsub_rn(pj.x, p.x), ddy2 = __fsub_rn(pj.y, p.y);
                        float d2 = __fadd_rn(__fmul_rn(ddx2, ddx2), __fmul_rn(ddy2, ddy2));
                        if (!(d2 < nd2)) continue;
                        unsigned long long key =
                            ((unsigned long long)__float_as_uint(d2) << 32) | sid[q];
                        if (key >= kk[KMAX - 1]) continue;
                        bool done = false;
#pragma unroll
                        for (int l = KMAX - 1; l > 0; --l) {
                            if (!done) {
                                if (key < kk[l - 1]) {
                                    kk[l] = kk[l - 1];
                                    ks[l] = ks[l - 1];
                                } else {
                                    kk[l] = key;
                                    ks[l] = (int)q;
                                    done = true;
                                }
                            }
                        }
                        if (!done) {
                            kk[0] = key;
                            ks[0] = (int)q;
                        }
                    }
                }
            }
            // stop when ring r+1 cannot hold a better candidate (or does not exist)
            float lb = INFINITY;
            if (cx - r - 1 >= 0) lb = fminf(lb, p.x - (g.xmin + (float)(cx - r) * s));
            if (cx + r + 1 <= g.gx - 1) lb = fminf(lb, (g.xmin + (float)(cx + r + 1) * s) - p.x);
            if (cy - r - 1 >= 0) lb = fminf(lb, p.y - (g.ymin + (float)(cy - r) * s));
            if (cy + r + 1 <= g.gy - 1) lb = fminf(lb, (g.ymin + (float)(cy + r + 1) * s) - p.y);
            if (lb == INFINITY) break;
            lb = fmaxf(0.0f, lb - slop);
            float lb2 = lb * lb * (1.0f - 1e-5f);
            bool full = kk[KMAX - 1] != ~0ull;
            float kth = full ? __uint_as_float((unsigned)(kk[KMAX - 1] >> 32)) : nd2;
            if (full ? (lb2 > kth) : (lb2 >= nd2)) break;
        }

        // half-planes in neighbour order
        float2 v = a.in.vel[t];
        float ri = a.prm.radius[t], tau = a.prm.tau[t];
        Ln L[KMAX];
        int cnt = 0;
#pragma unroll
        for (int l = 0; l < KMAX; ++l) {
            if (l >= KMAX - k && kk[l] != ~0ull) {
                int q = ks[l];
                L[cnt++] = orca_line_dev(p, v, ri, tau, a.dt, me, spos[q], a.in.vel[q],
                                         a.prm.radius[q], (uint32_t)(kk[l] & 0xffffffffu));
            }
        }
        if (a.rec_nbr) {
            int w = 0;
#pragma unroll
            for (int l = 0; l < KMAX; ++l)
                if (l >= KMAX - k) a.rec_nbr[(size_t)me * k + (w++)] =
                    kk[l] != ~0ull ? (int32_t)(kk[l] & 0xffffffffu) : -1;
        }
        if (a.rec_cell) a.rec_cell[me] = (uint32_t)cy * (uint32_t)g.gx + (uint32_t)cx;

        // preferred velocity: towards the goal at the preferred speed, or onto the goal
        float2 goal = a.prm.goal[t];
        float pref = a.prm.pref_speed[t], V = a.prm.max_speed[t];
        float gx_ = goal.x - p.x, gy_ = goal.y - p.y;
        float gd = sqrtf(gx_ * gx_ + gy_ * gy_);
        float ox, oy;
        if (gd > pref * a.dt) {
            ox = gx_ * (pref / gd);
            oy = gy_ * (pref / gd);
        } else {
            ox = gx_ / a.dt;
            oy = gy_ / a.dt;
        }
        float xx, xy;
        int b = lp2_dev(L, cnt, V, ox, oy, false, xx, xy);
        if (b < cnt) {
            used3 = true;
            lp3_dev<KMAX>(L, cnt, b, V, xx, xy);
        }
        float nx = p.x + xx * a.dt, ny = p.y + xy * a.dt;
        if (!isfinite(xx) || !isfinite(xy) || !isfinite(nx) || !isfinite(ny))
            atomicOr(&a.misc_rw->error, kErrNumeric);
        a.out.vel[t] = make_float2(xx, xy);
        a.out.pos[t] = make_float2(nx, ny);
        atomicAdd(&s_cand, cand);
        atomicAdd(&s_lines, (unsigned long long)cnt);
    }
    int n_act = __syncthreads_count(active);
    int n_lp3 = __syncthreads_count(used3);
    if (threadIdx.x == 0) {
        unsigned long long* c = a.block_counters + 4 * (size_t)blockIdx.x;
        c[0] += (unsigned long long)n_act;
        c[1] += (unsigned long long)n_lp3;
        c[2] += s_cand;
        c[3] += s_lines;
    }
}

constexpr int kMainThreads = 128;

int main_blocks(int n) { return (n + kMainThreads - 1) / kMainThreads; }

cudaError_t launch_main(const MainArgs& a, cudaStream_t st) {
    int nb = main_blocks(a.n);
    if (a.k <= 10) orca_main_v0_kernel<10><<<nb, kMainThreads, 0, st>>>(a);
    else if (a.k <= 16) orca_main_v0_kernel<16><<<nb, kMainThreads, 0, st>>>(a);
    else if (a.k <= 20) orca_main_v0_kernel<20><<<nb, kMainThreads, 0, st>>>(a);
    else orca_main_v0_kernel<32><<<nb, kMainThreads, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace orca
