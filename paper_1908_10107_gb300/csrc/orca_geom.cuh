// orca_geom.cuh -- half-plane construction and preferred velocity shared by the forward
// step (orca_main.cu) and its adjoint (orca_adjoint.cu): both must take identical branch
// decisions from identical FP32 arithmetic.
#pragma once

#include "orca_common.cuh"

namespace orca {

constexpr float kEps = 1e-5f;

// half-plane construction branches (Fig. 1)
constexpr int kLineCutoff = 0;        // cut-off circle of VO^tau
constexpr int kLineLeftLeg = 1;
constexpr int kLineRightLeg = 2;
constexpr int kLineOverlap = 3;       // agents overlap: one-step disc
constexpr int kLineOverlapFixed = 4;  // overlap with q = 0: direction fixed by a rule

// What fixes an agent's final velocity, recorded for the adjoint (rollouts only):
//   kTapePref      x = preferred velocity o;          kTapePrefClip  x = V o / |o|;
//   kTapeLine      x from LP1 on line i (LP2 phase);
//   kTapeLp3Dir    x = V n_i (LP3, no bisector was violated);
//   kTapeLp3Line   x from LP1 on the bisector of lines i and f (LP3).
// For the LP1 cases: t was free (projection of o), or the disc's or line / bisector j's
// bound on the tL (side 0) or tR (side 1) end.  Packed in 32 bits: mode | i << 3 | f << 9 |
// bound << 15 | j << 17 | side << 23.
constexpr int kTapePref = 0, kTapePrefClip = 1, kTapeLine = 2, kTapeLp3Dir = 3, kTapeLp3Line = 4;
constexpr int kBoundFree = 0, kBoundDisc = 1, kBoundLine = 2;

// Every formula below is written with explicit FP32 operations (fused where a product
// feeds a sum), none left to the compiler's contraction: each kernel that builds a
// half-plane -- the plain and the obstacle instantiations of the step, the adjoint --
// then rounds it identically, whatever code surrounds the call.
__device__ __forceinline__ float det2f(float ax, float ay, float bx, float by) {
    return __fmaf_rn(ax, by, -__fmul_rn(ay, bx));
}

// Half-plane of agent (p, v, r, 1/tau) induced by neighbour message mj = (x, y, r, id)
// with velocity vj -- Fig. 1.  u runs from the relative velocity to the nearest
// boundary point of VO^tau; the boundary passes through v + u/2 with the valid side
// along the VO's outward normal.
//   cut-off circle / overlap: n = w/|w| (w = v_rel - p/tau, or p/dt when overlapping),
//     c = n.v + (R/tau - |w|)/2;
//   legs: n is the leg's outward normal and c = n.(v + v_j)/2.
// When overlapping, R/dt - |w| is formed as (R - |q|)/dt with q = p - v_rel dt (both
// O(1) metres), which keeps more of the offset's FP32 precision.
__device__ __forceinline__ float4 orca_line_dev(float2 p, float2 v, float r, float itau,
                                                float dt, float half_idt, uint32_t me,
                                                float4 mj, float2 vj, int* branch = nullptr) {
    const float px = __fsub_rn(mj.x, p.x), py = __fsub_rn(mj.y, p.y);
    const float vx = __fsub_rn(v.x, vj.x), vy = __fsub_rn(v.y, vj.y);
    const float R = __fadd_rn(r, mj.z);
    const float p2 = __fmaf_rn(px, px, __fmul_rn(py, py)), R2 = __fmul_rn(R, R);
    float4 L;
    L.w = 0.0f;
    if (p2 > R2) {
        const float wx = __fmaf_rn(-px, itau, vx), wy = __fmaf_rn(-py, itau, vy);
        const float w2 = __fmaf_rn(wx, wx, __fmul_rn(wy, wy));
        const float wp = __fmaf_rn(wx, px, __fmul_rn(wy, py));
        if (wp < 0.0f && __fmul_rn(wp, wp) > __fmul_rn(R2, w2)) {
            if (branch) *branch = kLineCutoff;
            const float iw = rsqrtf(w2);
            L.x = __fmul_rn(wx, iw);
            L.y = __fmul_rn(wy, iw);
            const float half_gap = __fmul_rn(0.5f, __fmaf_rn(R, itau, -__fmul_rn(w2, iw)));
            L.z = __fmaf_rn(L.x, v.x, __fmaf_rn(L.y, v.y, half_gap));
        } else {
            const float l2 = __fsub_rn(p2, R2);
            const float leg = __fmul_rn(l2, rsqrtf(l2));
            const float ip2 = __fdividef(1.0f, p2);
            if (det2f(px, py, wx, wy) > 0.0f) {  // left leg
                if (branch) *branch = kLineLeftLeg;
                L.x = -__fmul_rn(__fmaf_rn(px, R, __fmul_rn(py, leg)), ip2);
                L.y = __fmul_rn(__fmaf_rn(px, leg, -__fmul_rn(py, R)), ip2);
            } else {  // right leg
                if (branch) *branch = kLineRightLeg;
                L.x = __fmul_rn(__fmaf_rn(py, leg, -__fmul_rn(px, R)), ip2);
                L.y = -__fmul_rn(__fmaf_rn(px, leg, __fmul_rn(py, R)), ip2);
            }
            L.z = __fmul_rn(0.5f, __fmaf_rn(L.x, __fadd_rn(v.x, vj.x),
                                            __fmul_rn(L.y, __fadd_rn(v.y, vj.y))));
        }
    } else {
        const float qx = __fmaf_rn(-vx, dt, px), qy = __fmaf_rn(-vy, dt, py);  // = -w dt
        const float ql = sqrtf(__fmaf_rn(qx, qx, __fmul_rn(qy, qy)));
        float nx, ny;
        if (branch) *branch = ql > 0.0f ? kLineOverlap : kLineOverlapFixed;
        if (ql > 0.0f) {
            const float iq = __fdividef(1.0f, ql);
            nx = -__fmul_rn(qx, iq);
            ny = -__fmul_rn(qy, iq);
        } else if (p2 > 0.0f) {
            const float ip = rsqrtf(p2);
            nx = -__fmul_rn(px, ip);
            ny = -__fmul_rn(py, ip);
        } else {
            nx = me < __float_as_uint(mj.w) ? 1.0f : -1.0f;
            ny = 0.0f;
        }
        L.x = nx;
        L.y = ny;
        L.z = __fmaf_rn(nx, v.x, __fmaf_rn(ny, v.y, __fmul_rn(__fsub_rn(R, ql), half_idt)));
    }
    return L;
}

// Preferred velocity (Section 3; Section 4 set-up): towards the goal at the preferred
// speed, or, within one step of the goal, the velocity that reaches it.  far = 1 for the
// first case.
__device__ __forceinline__ float2 pref_velocity_dev(float2 p, float2 goal, float pref, float dt,
                                                    float idt, int* far = nullptr) {
    const float gx_ = __fsub_rn(goal.x, p.x), gy_ = __fsub_rn(goal.y, p.y);
    const float g2 = __fmaf_rn(gx_, gx_, __fmul_rn(gy_, gy_));
    const float ig = rsqrtf(g2);
    if (__fmul_rn(g2, ig) > __fmul_rn(pref, dt)) {
        if (far) *far = 1;
        const float s = __fmul_rn(pref, ig);
        return make_float2(__fmul_rn(gx_, s), __fmul_rn(gy_, s));
    }
    if (far) *far = 0;
    return make_float2(__fmul_rn(gx_, idt), __fmul_rn(gy_, idt));
}

}  // namespace orca
