// orca_adjoint.cuh -- the adjoint of one ORCA step (orca_adjoint.cu), its arguments, and
// the FP64 counterparts of the half-plane and preferred-velocity construction used by the
// FP64 validation rollout (orca_validate.cu) and the FP64 instantiation of the adjoint.
#pragma once

#include "orca_geom.cuh"

namespace orca {

// A half-plane in normal form: the valid side is {x : n.x >= c}, |n| = 1.
template <class T>
struct Line {
    T nx, ny, c;
};

template <class T>
struct Vec2Of;
template <>
struct Vec2Of<float> {
    using type = float2;
};
template <>
struct Vec2Of<double> {
    using type = double2;
};

constexpr int kAdjEntries = 3;
// Entries one agent's list holds; an agent that receives more is summed by a scan of all
// agents' entries (exact, same order, slow).  The index-checked build keeps two, so that
// its tests run the scan on ordinary crowds.
#ifdef ORCA_CHECKS
constexpr int kInCap = 2;
#else
constexpr int kInCap = 24;
#endif

// One reverse step; everything in agent order.
template <class T>
struct AdjArgs {
    using T2 = typename Vec2Of<T>::type;
    int n, kstride;
    T dt;
    const T2* pos;          // state at step t
    const T2* vel;
    const T2* goal;         // parameters
    const T* radius;
    const T* max_speed;
    const T* pref_speed;
    const T* tau;
    const int32_t* nbr;     // n * kstride, -1 padded
    const uint32_t* tape;   // n LP records
    const T2* pbar_next;    // dL/dp(t+1), dL/dv(t+1) (total derivatives)
    const T2* vbar_next;
    const T2* dl_dp;        // partial dL/dp(t) of the loss itself, or null
    T2* pbar;               // written: dL/dp(t), dL/dv(t)
    T2* vbar;
    T* g_pref;              // parameter gradients (accumulated over the steps)
    T* g_radius;
    T* g_tau;
    // At most kAdjEntries half-planes of an agent carry an adjoint (the line or bisector
    // its velocity lies on, the one that bounds it, line i of a least-penetration solve):
    // entry a * kAdjEntries + q is one of them, with the neighbour it came from (ent, -1:
    // none) and its contribution to that neighbour (contrib: pbar x, y, vbar x, y;
    // contrib_r: radius)
    int32_t* ent;           // n * kAdjEntries
    T* contrib;             // n * kAdjEntries * 4
    T* contrib_r;           // n * kAdjEntries
    uint32_t* incnt;        // n: entries each agent receives; zero on entry and on exit
    uint32_t* inlist;       // n * kInCap: the entries agent b receives, in arrival order
    int* err;               // the device error word (index checks of the ORCA_CHECKS build)
};

// adj_agent, adj_gather on st (T = float or double).
template <class T>
cudaError_t launch_adjoint_step(const AdjArgs<T>& A, int kmax, cudaStream_t st);

// FP64 half-plane of agent (p, v, r, 1/tau) induced by neighbour (pj, rj, vj): the same
// construction as orca_line_dev (Fig. 1; normal form, the reciprocal half u/2, dt in place
// of tau for overlapping agents) in plain double arithmetic.
__device__ __forceinline__ Line<double> orca_line_fp64(double2 p, double2 v, double r, double itau,
                                                       double dt, double half_idt, uint32_t me,
                                                       double2 pj, double rj, uint32_t j, double2 vj,
                                                       int* branch) {
    const double px = pj.x - p.x, py = pj.y - p.y;
    const double vx = v.x - vj.x, vy = v.y - vj.y;
    const double R = r + rj;
    const double p2 = px * px + py * py, R2 = R * R;
    Line<double> L;
    if (p2 > R2) {
        const double wx = vx - px * itau, wy = vy - py * itau;
        const double w2 = wx * wx + wy * wy;
        const double wp = wx * px + wy * py;
        if (wp < 0.0 && wp * wp > R2 * w2) {
            *branch = kLineCutoff;
            const double wl = sqrt(w2);
            L.nx = wx / wl;
            L.ny = wy / wl;
            L.c = L.nx * v.x + L.ny * v.y + 0.5 * (R * itau - wl);
        } else {
            const double leg = sqrt(p2 - R2);
            if (px * wy - py * wx > 0.0) {  // left leg
                *branch = kLineLeftLeg;
                L.nx = -(px * R + py * leg) / p2;
                L.ny = (px * leg - py * R) / p2;
            } else {  // right leg
                *branch = kLineRightLeg;
                L.nx = (py * leg - px * R) / p2;
                L.ny = -(px * leg + py * R) / p2;
            }
            L.c = 0.5 * (L.nx * (v.x + vj.x) + L.ny * (v.y + vj.y));
        }
    } else {
        const double qx = px - vx * dt, qy = py - vy * dt;
        const double ql = sqrt(qx * qx + qy * qy);
        double nx, ny;
        *branch = ql > 0.0 ? kLineOverlap : kLineOverlapFixed;
        if (ql > 0.0) {
            nx = -qx / ql;
            ny = -qy / ql;
        } else if (p2 > 0.0) {
            const double pl = sqrt(p2);
            nx = -px / pl;
            ny = -py / pl;
        } else {
            nx = me < j ? 1.0 : -1.0;
            ny = 0.0;
        }
        L.nx = nx;
        L.ny = ny;
        L.c = nx * v.x + ny * v.y + (R - ql) * half_idt;
    }
    return L;
}

// FP64 preferred velocity: towards the goal at the preferred speed, or, within one step of
// the goal, the velocity that reaches it (far = 1 for the first case).
__device__ __forceinline__ double2 pref_velocity_fp64(double2 p, double2 goal, double pref, double dt,
                                                      double idt, int* far) {
    const double gx = goal.x - p.x, gy = goal.y - p.y;
    const double gl = sqrt(gx * gx + gy * gy);
    if (gl > pref * dt) {
        *far = 1;
        return make_double2(gx * (pref / gl), gy * (pref / gl));
    }
    *far = 0;
    return make_double2(gx * idt, gy * idt);
}

}  // namespace orca
