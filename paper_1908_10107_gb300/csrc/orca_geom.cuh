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

__device__ __forceinline__ float det2f(float ax, float ay, float bx, float by) {
    return ax * by - ay * bx;
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
    float px = mj.x - p.x, py = mj.y - p.y;
    float vx = v.x - vj.x, vy = v.y - vj.y;
    float R = r + mj.z;
    float p2 = px * px + py * py, R2 = R * R;
    float4 L;
    L.w = 0.0f;
    if (p2 > R2) {
        float wx = vx - px * itau, wy = vy - py * itau;
        float w2 = wx * wx + wy * wy, wp = wx * px + wy * py;
        if (wp < 0.0f && wp * wp > R2 * w2) {
            if (branch) *branch = kLineCutoff;
            float iw = rsqrtf(w2);
            L.x = wx * iw;
            L.y = wy * iw;
            L.z = L.x * v.x + L.y * v.y + 0.5f * (R * itau - w2 * iw);
        } else {
            float l2 = p2 - R2;
            float leg = l2 * rsqrtf(l2);
            float ip2 = __fdividef(1.0f, p2);
            if (det2f(px, py, wx, wy) > 0.0f) {  // left leg
                if (branch) *branch = kLineLeftLeg;
                L.x = -(px * R + py * leg) * ip2;
                L.y = (px * leg - py * R) * ip2;
            } else {  // right leg
                if (branch) *branch = kLineRightLeg;
                L.x = (py * leg - px * R) * ip2;
                L.y = -(px * leg + py * R) * ip2;
            }
            L.z = 0.5f * (L.x * (v.x + vj.x) + L.y * (v.y + vj.y));
        }
    } else {
        float qx = px - vx * dt, qy = py - vy * dt;  // = -w dt
        float ql = sqrtf(qx * qx + qy * qy);
        float nx, ny;
        if (branch) *branch = ql > 0.0f ? kLineOverlap : kLineOverlapFixed;
        if (ql > 0.0f) {
            float iq = __fdividef(1.0f, ql);
            nx = -qx * iq;
            ny = -qy * iq;
        } else if (p2 > 0.0f) {
            float ip = rsqrtf(p2);
            nx = -px * ip;
            ny = -py * ip;
        } else {
            nx = me < __float_as_uint(mj.w) ? 1.0f : -1.0f;
            ny = 0.0f;
        }
        L.x = nx;
        L.y = ny;
        L.z = nx * v.x + ny * v.y + (R - ql) * half_idt;
    }
    return L;
}

// Preferred velocity (Section 3; Section 4 set-up): towards the goal at the preferred
// speed, or, within one step of the goal, the velocity that reaches it.  far = 1 for the
// first case.
__device__ __forceinline__ float2 pref_velocity_dev(float2 p, float2 goal, float pref, float dt,
                                                    float idt, int* far = nullptr) {
    float gx_ = goal.x - p.x, gy_ = goal.y - p.y;
    float g2 = gx_ * gx_ + gy_ * gy_;
    float ig = rsqrtf(g2);
    if (g2 * ig > pref * dt) {
        if (far) *far = 1;
        return make_float2(gx_ * (pref * ig), gy_ * (pref * ig));
    }
    if (far) *far = 0;
    return make_float2(gx_ * idt, gy_ * idt);
}

}  // namespace orca
