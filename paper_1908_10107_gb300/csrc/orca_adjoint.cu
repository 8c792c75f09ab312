// orca_adjoint.cu -- reverse-mode derivative of one ORCA step (adjoint of Sections 2-3).
//
// One step maps the state (p, v) and the per-agent parameters (radius r, preferred speed
// s, time horizon tau) to p' = p + x dt, v' = x, where x is the velocity the LP selects.
// With the neighbour sets and every discrete decision of the step held fixed -- which
// constraints fix x (recorded on the forward pass as the "tape"), which branch built each
// half-plane, which branch built the preferred velocity -- x is a smooth function of the
// half-planes (n_l, c_l) and of the preferred velocity o, and those are smooth functions of
// the state and parameters.  This kernel pushes the adjoints (dL/dp', dL/dv') of one agent
// back through that chain:
//   x -> (n, c) of at most three half-planes (the line or bisector x lies on, the one that
//        bounds it, and line i of a least-penetration solve) and o;
//   (n, c) -> p, v, r of the agent and of the neighbour, tau of the agent;
//   o -> p and s of the agent.
// Contributions to neighbours are added with atomics.
#include "orca_geom.cuh"

namespace orca {

constexpr int kTapePref = 0, kTapePrefClip = 1, kTapeLine = 2, kTapeLp3Dir = 3, kTapeLp3Line = 4;
constexpr int kBoundFree = 0, kBoundDisc = 1;

__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }
__device__ __forceinline__ float dot2(float2 a, float2 b) { return a.x * b.x + a.y * b.y; }
__device__ __forceinline__ void add2(float2* p, float2 v) {
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
}

// Adjoint of x = e*m + t*d(m), d(m) = (m.y, -m.x), given xbar: returns tbar and adds to
// ebar, mbar.
__device__ __forceinline__ float point_on_line_bar(float2 m, float e, float t, float2 xbar,
                                                   float& ebar, float2& mbar) {
    ebar += dot2(m, xbar);
    // dx/dm = e I + t Q with Q m = d(m); Q^T xbar = (-xbar.y, xbar.x)
    mbar.x += e * xbar.x - t * xbar.y;
    mbar.y += e * xbar.y + t * xbar.x;
    return dot2(f2(m.y, -m.x), xbar);
}

// t from a bounding line j on line i: t = -rhs/den, rhs = e_j - e_i (m_i.m_j),
// den = det(m_i, m_j).  Adds the adjoints of (m_i, e_i, m_j, e_j) for tbar.
__device__ __forceinline__ float bound_t(float2 mi, float ei, float2 mj, float ej) {
    float den = det2f(mi.x, mi.y, mj.x, mj.y);
    float rhs = ej - ei * dot2(mi, mj);
    return -rhs / den;
}

__device__ __forceinline__ void bound_bar(float2 mi, float ei, float2 mj, float ej, float tbar,
                                          float2& mibar, float& eibar, float2& mjbar, float& ejbar) {
    float den = det2f(mi.x, mi.y, mj.x, mj.y);
    float rhs = ej - ei * dot2(mi, mj);
    float t = -rhs / den;
    float rbar = -tbar / den;
    float dbar = -tbar * t / den;
    ejbar += rbar;
    eibar -= rbar * dot2(mi, mj);
    mibar.x -= rbar * ei * mj.x;
    mibar.y -= rbar * ei * mj.y;
    mjbar.x -= rbar * ei * mi.x;
    mjbar.y -= rbar * ei * mi.y;
    mibar.x += dbar * mj.y;
    mibar.y -= dbar * mj.x;
    mjbar.x -= dbar * mi.y;
    mjbar.y += dbar * mi.x;
}

// Bisector of lines i and f: m = (n_f - n_i)/|n_f - n_i|, e = (c_f - c_i)/|n_f - n_i|.
__device__ __forceinline__ void bisector(float4 li, float4 lf, float2& m, float& e) {
    float ux = lf.x - li.x, uy = lf.y - li.y;
    float inv = rsqrtf(ux * ux + uy * uy);
    m = f2(ux * inv, uy * inv);
    e = (lf.z - li.z) * inv;
}

__device__ __forceinline__ void bisector_bar(float4 li, float4 lf, float2 mbar, float ebar,
                                             float2& nibar, float& cibar, float2& nfbar, float& cfbar) {
    float ux = lf.x - li.x, uy = lf.y - li.y;
    float ul = sqrtf(ux * ux + uy * uy);
    float2 m = f2(ux / ul, uy / ul);
    float e = (lf.z - li.z) / ul;
    float mm = dot2(m, mbar);
    float2 ubar = f2((mbar.x - m.x * mm - e * ebar * m.x) / ul, (mbar.y - m.y * mm - e * ebar * m.y) / ul);
    nfbar.x += ubar.x;
    nfbar.y += ubar.y;
    nibar.x -= ubar.x;
    nibar.y -= ubar.y;
    cfbar += ebar / ul;
    cibar -= ebar / ul;
}

// Adjoint of the half-plane of agent a (p, v, r, 1/tau) induced by neighbour b (pb, vb, rb)
// for (nbar, cbar), branch as in the forward step.  Outputs the adjoints of the agent's
// and the neighbour's position, velocity, radius, and of 1/tau.
__device__ __forceinline__ void line_bar(float2 pa, float2 va, float ra, float itau, float dt,
                                         float half_idt, float2 pb, float2 vb, float rb, int branch,
                                         float4 L, float2 nbar, float cbar, float2& pabar,
                                         float2& vabar, float& rbar_ab, float& itaubar,
                                         float2& pbbar, float2& vbbar) {
    float2 p = f2(pb.x - pa.x, pb.y - pa.y);
    float2 v = f2(va.x - vb.x, va.y - vb.y);
    float R = ra + rb;
    float2 n = f2(L.x, L.y);
    float2 pbar = f2(0.f, 0.f), vbar = f2(0.f, 0.f);
    float Rbar = 0.f;
    if (branch == kLineCutoff) {
        float2 w = f2(v.x - p.x * itau, v.y - p.y * itau);
        float wl = sqrtf(dot2(w, w));
        vabar.x += cbar * n.x;
        vabar.y += cbar * n.y;
        float2 nt = f2(nbar.x + cbar * va.x, nbar.y + cbar * va.y);
        float nn = dot2(n, nt);
        float2 wbar = f2((nt.x - n.x * nn) / wl - 0.5f * cbar * n.x, (nt.y - n.y * nn) / wl - 0.5f * cbar * n.y);
        Rbar += 0.5f * cbar * itau;
        itaubar += 0.5f * cbar * R - dot2(p, wbar);
        vbar.x += wbar.x;
        vbar.y += wbar.y;
        pbar.x -= itau * wbar.x;
        pbar.y -= itau * wbar.y;
    } else if (branch == kLineLeftLeg || branch == kLineRightLeg) {
        float s = branch == kLineLeftLeg ? 1.0f : -1.0f;
        float p2 = dot2(p, p);
        float l = sqrtf(p2 - R * R);
        float2 vs = f2(va.x + vb.x, va.y + vb.y);
        vabar.x += 0.5f * cbar * n.x;
        vabar.y += 0.5f * cbar * n.y;
        vbbar.x += 0.5f * cbar * n.x;
        vbbar.y += 0.5f * cbar * n.y;
        float2 nt = f2(nbar.x + 0.5f * cbar * vs.x, nbar.y + 0.5f * cbar * vs.y);
        float2 Jp = f2(-p.y, p.x);  // J = rotation by +90 degrees
        float ntJp = dot2(nt, Jp);
        // n = (-R p + s l J p) / p2;  M^T nt = -R nt + s l J^T nt, J^T nt = (nt.y, -nt.x)
        float2 MTn = f2(-R * nt.x + s * l * nt.y, -R * nt.y - s * l * nt.x);
        float nnt = dot2(n, nt);
        pbar.x += MTn.x / p2 + s * ntJp * p.x / (l * p2) - 2.0f * nnt * p.x / p2;
        pbar.y += MTn.y / p2 + s * ntJp * p.y / (l * p2) - 2.0f * nnt * p.y / p2;
        Rbar += (-dot2(nt, p) - s * ntJp * R / l) / p2;
    } else {  // overlap: q = p - v dt, n = -q/|q|, c = n.v_a + (R - |q|)/(2 dt)
        vabar.x += cbar * n.x;
        vabar.y += cbar * n.y;
        Rbar += cbar * half_idt;
        if (branch == kLineOverlap) {
            float2 q = f2(p.x - v.x * dt, p.y - v.y * dt);
            float ql = sqrtf(dot2(q, q));
            float2 nt = f2(nbar.x + cbar * va.x, nbar.y + cbar * va.y);
            float nn = dot2(n, nt);
            float2 qbar = f2(-(nt.x - n.x * nn) / ql + cbar * half_idt * n.x,
                             -(nt.y - n.y * nn) / ql + cbar * half_idt * n.y);
            pbar.x += qbar.x;
            pbar.y += qbar.y;
            vbar.x -= dt * qbar.x;
            vbar.y -= dt * qbar.y;
        }
    }
    // p = p_b - p_a, v = v_a - v_b, R = r_a + r_b
    pbbar.x += pbar.x;
    pbbar.y += pbar.y;
    pabar.x -= pbar.x;
    pabar.y -= pbar.y;
    vabar.x += vbar.x;
    vabar.y += vbar.y;
    vbbar.x -= vbar.x;
    vbbar.y -= vbar.y;
    rbar_ab += Rbar;
}

template <int KMAX>
__global__ void __launch_bounds__(128) orca_adjoint_kernel(AdjointArgs A) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= A.n) return;
    const float2 pbn = A.pbar_next[a], vbn = A.vbar_next[a];
    // p' = p + x dt, v' = x
    add2(&A.pbar[a], pbn);
    float2 xbar = f2(vbn.x + A.dt * pbn.x, vbn.y + A.dt * pbn.y);
    if (xbar.x == 0.0f && xbar.y == 0.0f) return;

    const float dt = A.dt;
    const float2 pa = A.pos[a], va = A.vel[a];
    const float ra = A.radius[a], V = A.max_speed[a];
    const float itau = __fdividef(1.0f, A.tau[a]);
    const float idt = __fdividef(1.0f, dt);
    const float half_idt = 0.5f * idt;
    // half-planes and preferred velocity exactly as the forward step built them
    float4 L[KMAX];
    int br[KMAX], nb[KMAX];
    int cnt = 0;
    for (int l = 0; l < KMAX && l < A.kstride; ++l) {
        int j = A.nbr[(size_t)a * A.kstride + l];
        if (j < 0) break;
        nb[cnt] = j;
        L[cnt] = orca_line_dev(pa, va, ra, itau, dt, half_idt, (uint32_t)a,
                               make_float4(A.pos[j].x, A.pos[j].y, A.radius[j], __uint_as_float((uint32_t)j)),
                               A.vel[j], &br[cnt]);
        ++cnt;
    }
    int far = 0;
    const float2 o = pref_velocity_dev(pa, A.goal[a], A.pref_speed[a], dt, idt, &far);

    const uint32_t tp = A.tape[a];
    const int mode = tp & 7, i = (tp >> 3) & 63, f = (tp >> 9) & 63, bound = (tp >> 15) & 3,
              j = (tp >> 17) & 63, side = (tp >> 23) & 1;
    float2 nbar[KMAX];
    float cbar[KMAX];
    for (int l = 0; l < cnt; ++l) {
        nbar[l] = f2(0.f, 0.f);
        cbar[l] = 0.f;
    }
    float2 obar = f2(0.f, 0.f);

    if (mode == kTapePref) {
        obar = xbar;
    } else if (mode == kTapePrefClip) {
        float ol = sqrtf(dot2(o, o));
        float2 oh = f2(o.x / ol, o.y / ol);
        float k = dot2(oh, xbar);
        obar = f2(V / ol * (xbar.x - oh.x * k), V / ol * (xbar.y - oh.y * k));
    } else if (mode == kTapeLine) {
        const float4 li = L[i];
        const float2 mi = f2(li.x, li.y);
        const float2 di = f2(li.y, -li.x);
        float t;
        if (bound == kBoundFree) t = dot2(di, o);
        else if (bound == kBoundDisc) t = (side ? 1.f : -1.f) * sqrtf(fmaxf(V * V - li.z * li.z, 0.f));
        else t = bound_t(mi, li.z, f2(L[j].x, L[j].y), L[j].z);
        float2 mibar = f2(0.f, 0.f);
        float eibar = 0.f;
        float tbar = point_on_line_bar(mi, li.z, t, xbar, eibar, mibar);
        if (bound == kBoundFree) {  // t = d(n_i).o
            mibar.x += -tbar * o.y;
            mibar.y += tbar * o.x;
            obar = f2(tbar * di.x, tbar * di.y);
        } else if (bound == kBoundDisc) {
            if (t != 0.f) eibar += -tbar * li.z / t;
        } else {
            float2 mjbar = f2(0.f, 0.f);
            float ejbar = 0.f;
            bound_bar(mi, li.z, f2(L[j].x, L[j].y), L[j].z, tbar, mibar, eibar, mjbar, ejbar);
            nbar[j].x += mjbar.x;
            nbar[j].y += mjbar.y;
            cbar[j] += ejbar;
        }
        nbar[i].x += mibar.x;
        nbar[i].y += mibar.y;
        cbar[i] += eibar;
    } else if (mode == kTapeLp3Dir) {  // x = V n_i
        nbar[i].x += V * xbar.x;
        nbar[i].y += V * xbar.y;
    } else {  // kTapeLp3Line: LP1 on the bisector of lines i and f
        const float4 li = L[i];
        float2 m;
        float e;
        bisector(li, L[f], m, e);
        float t;
        float2 mj;
        float ej = 0.f;
        if (bound == kBoundDisc) {
            t = (side ? 1.f : -1.f) * sqrtf(fmaxf(V * V - e * e, 0.f));
        } else {
            bisector(li, L[j], mj, ej);
            t = bound_t(m, e, mj, ej);
        }
        float2 mbar = f2(0.f, 0.f);
        float ebar = 0.f;
        float tbar = point_on_line_bar(m, e, t, xbar, ebar, mbar);
        if (bound == kBoundDisc) {
            if (t != 0.f) ebar += -tbar * e / t;
        } else {
            float2 mjbar = f2(0.f, 0.f);
            float ejbar = 0.f;
            bound_bar(m, e, mj, ej, tbar, mbar, ebar, mjbar, ejbar);
            bisector_bar(li, L[j], mjbar, ejbar, nbar[i], cbar[i], nbar[j], cbar[j]);
        }
        bisector_bar(li, L[f], mbar, ebar, nbar[i], cbar[i], nbar[f], cbar[f]);
    }

    // half-planes -> state and parameters of the agent and its neighbours
    float2 pabar = f2(0.f, 0.f), vabar = f2(0.f, 0.f);
    float rabar = 0.f, itaubar = 0.f;
    for (int l = 0; l < cnt; ++l) {
        if (nbar[l].x == 0.f && nbar[l].y == 0.f && cbar[l] == 0.f) continue;
        const int b = nb[l];
        float2 pbbar = f2(0.f, 0.f), vbbar = f2(0.f, 0.f);
        float Rbar = 0.f;
        line_bar(pa, va, ra, itau, dt, half_idt, A.pos[b], A.vel[b], A.radius[b], br[l], L[l], nbar[l],
                 cbar[l], pabar, vabar, Rbar, itaubar, pbbar, vbbar);
        rabar += Rbar;
        add2(&A.pbar[b], pbbar);
        add2(&A.vbar[b], vbbar);
        atomicAdd(&A.g_radius[b], Rbar);
    }
    // preferred velocity -> position and preferred speed of the agent
    if (obar.x != 0.f || obar.y != 0.f) {
        float2 g = f2(A.goal[a].x - pa.x, A.goal[a].y - pa.y);
        if (far) {
            float gl = sqrtf(dot2(g, g));
            float2 gh = f2(g.x / gl, g.y / gl);
            float k = dot2(gh, obar);
            float s = A.pref_speed[a];
            atomicAdd(&A.g_pref[a], k);
            pabar.x -= s / gl * (obar.x - gh.x * k);
            pabar.y -= s / gl * (obar.y - gh.y * k);
        } else {
            pabar.x -= obar.x * idt;
            pabar.y -= obar.y * idt;
        }
    }
    add2(&A.pbar[a], pabar);
    add2(&A.vbar[a], vabar);
    atomicAdd(&A.g_radius[a], rabar);
    // d(1/tau)/dtau = -1/tau^2
    atomicAdd(&A.g_tau[a], -itaubar * itau * itau);
}

cudaError_t launch_adjoint(const AdjointArgs& A, int kmax, cudaStream_t st) {
    int nb = (A.n + 127) / 128;
    if (A.n <= 0) return cudaSuccess;
    if (kmax <= 10) orca_adjoint_kernel<10><<<nb, 128, 0, st>>>(A);
    else if (kmax <= 16) orca_adjoint_kernel<16><<<nb, 128, 0, st>>>(A);
    else if (kmax <= 20) orca_adjoint_kernel<20><<<nb, 128, 0, st>>>(A);
    else orca_adjoint_kernel<32><<<nb, 128, 0, st>>>(A);
    return cudaGetLastError();
}

// rollout helpers ------------------------------------------------------------------
// Parameters back to agent order.
__global__ void __launch_bounds__(256) unpermute_params_kernel(int n, AgentParams src, float2* goal,
                                                               float* radius, float* vmax,
                                                               float* pref, float* tau) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    uint32_t i = src.id[t];
    goal[i] = src.goal[t];
    radius[i] = src.radius[t];
    vmax[i] = src.max_speed[t];
    pref[i] = src.pref_speed[t];
    tau[i] = src.tau[t];
}

__global__ void __launch_bounds__(256) axpy2_kernel(int n, float2* y, const float2* x) {
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    float2 a = y[t], b = x[t];
    y[t] = make_float2(a.x + b.x, a.y + b.y);
}

cudaError_t launch_unpermute_params(int n, const AgentParams& src, float2* goal, float* radius,
                                    float* vmax, float* pref, float* tau, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    unpermute_params_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, src, goal, radius, vmax, pref, tau);
    return cudaGetLastError();
}

cudaError_t launch_axpy2(int n, float2* y, const float2* x, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    axpy2_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, y, x);
    return cudaGetLastError();
}

}  // namespace orca
