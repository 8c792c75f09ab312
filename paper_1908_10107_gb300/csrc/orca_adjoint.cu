// orca_adjoint.cu -- reverse-mode derivative of one ORCA step (adjoint of Sections 2-3).
//
// One step maps the state (p, v) and the per-agent parameters (radius r, preferred speed
// s, time horizon tau) to p' = p + x dt, v' = x, where x is the velocity the LP selects.
// With the neighbour sets and every discrete decision of the step held fixed -- which
// constraints fix x (recorded on the forward pass as the "tape"), which branch built each
// half-plane, which branch built the preferred velocity -- x is a smooth function of the
// half-planes (n_l, c_l) and of the preferred velocity o, and those are smooth functions of
// the state and parameters.  The adjoint of one agent pushes (dL/dp', dL/dv') back
// through that chain:
//   x -> (n, c) of at most three half-planes (the line or bisector x lies on, the one that
//        bounds it, and line i of a least-penetration solve) and o;
//   (n, c) -> p, v, r of the agent and of the neighbour, tau of the agent;
//   o -> p and s of the agent.
//
// Deterministic accumulation.  What an agent's half-planes contribute to its neighbours
// is not added with atomics (whose order, and so whose rounding, varies between runs):
//   adj_agent   one thread per agent a writes its own adjoints and, for each of the (at
//               most three) half-planes that fix its velocity, the contribution to that
//               half-plane's neighbour in an entry of its own, whose index it appends to
//               the neighbour's list (an atomic counter gives the place; up to kInCap
//               places per agent);
//   adj_gather  one thread per agent b sorts its list by entry (agent, then line) and adds
//               the contributions in that order (and the loss gradient of its position);
//               an agent that received more than kInCap entries finds them all by a scan
//               of every agent's entries, which meets them in the same order.
// Every sum is then taken in a fixed order and the gradients are bitwise reproducible.
//
// The kernels are templates on the scalar type: float for rollouts of the FP32 step, and
// double for the validation rollout (orca_validate.cu), which runs the same adjoint code
// along an FP64 trajectory so that the adjoint can be checked against FP64 finite
// differences without FP32 trajectory drift in the way.
#include "orca_adjoint.cuh"

namespace orca {

// ---- scalar-generic helpers --------------------------------------------------------
template <class T>
struct V2 {
    T x, y;
};
template <class T>
__device__ __forceinline__ V2<T> mk2(T x, T y) { return V2<T>{x, y}; }
template <class T>
__device__ __forceinline__ T dot2(V2<T> a, V2<T> b) { return a.x * b.x + a.y * b.y; }
template <class T>
__device__ __forceinline__ T det2(V2<T> a, V2<T> b) { return a.x * b.y - a.y * b.x; }
__device__ __forceinline__ V2<float> v2of(float2 a) { return V2<float>{a.x, a.y}; }
__device__ __forceinline__ V2<double> v2of(double2 a) { return V2<double>{a.x, a.y}; }
__device__ __forceinline__ float sqrt_t(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt_t(double x) { return sqrt(x); }

// Adjoint of x = e*m + t*d(m), d(m) = (m.y, -m.x), given xbar: returns tbar and adds to
// ebar, mbar.
template <class T>
__device__ __forceinline__ T point_on_line_bar(V2<T> m, T e, T t, V2<T> xbar, T& ebar, V2<T>& mbar) {
    ebar += dot2(m, xbar);
    // dx/dm = e I + t Q with Q m = d(m); Q^T xbar = (-xbar.y, xbar.x)
    mbar.x += e * xbar.x - t * xbar.y;
    mbar.y += e * xbar.y + t * xbar.x;
    return dot2(mk2<T>(m.y, -m.x), xbar);
}

// t from a bounding line j on line i: t = -rhs/den, rhs = e_j - e_i (m_i.m_j),
// den = det(m_i, m_j).
template <class T>
__device__ __forceinline__ T bound_t(V2<T> mi, T ei, V2<T> mj, T ej) {
    T den = det2(mi, mj);
    T rhs = ej - ei * dot2(mi, mj);
    return -rhs / den;
}

// Adds the adjoints of (m_i, e_i, m_j, e_j) for tbar.
template <class T>
__device__ __forceinline__ void bound_bar(V2<T> mi, T ei, V2<T> mj, T ej, T tbar, V2<T>& mibar, T& eibar,
                                          V2<T>& mjbar, T& ejbar) {
    T den = det2(mi, mj);
    T rhs = ej - ei * dot2(mi, mj);
    T t = -rhs / den;
    T rbar = -tbar / den;
    T dbar = -tbar * t / den;
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
template <class T>
__device__ __forceinline__ void bisector(Line<T> li, Line<T> lf, V2<T>& m, T& e) {
    T ux = lf.nx - li.nx, uy = lf.ny - li.ny;
    T ul = sqrt_t(ux * ux + uy * uy);
    m = mk2<T>(ux / ul, uy / ul);
    e = (lf.c - li.c) / ul;
}

template <class T>
__device__ __forceinline__ void bisector_bar(Line<T> li, Line<T> lf, V2<T> mbar, T ebar, V2<T>& nibar,
                                             T& cibar, V2<T>& nfbar, T& cfbar) {
    T ux = lf.nx - li.nx, uy = lf.ny - li.ny;
    T ul = sqrt_t(ux * ux + uy * uy);
    V2<T> m = mk2<T>(ux / ul, uy / ul);
    T e = (lf.c - li.c) / ul;
    T mm = dot2(m, mbar);
    V2<T> ubar = mk2<T>((mbar.x - m.x * mm - e * ebar * m.x) / ul, (mbar.y - m.y * mm - e * ebar * m.y) / ul);
    nfbar.x += ubar.x;
    nfbar.y += ubar.y;
    nibar.x -= ubar.x;
    nibar.y -= ubar.y;
    cfbar += ebar / ul;
    cibar -= ebar / ul;
}

// Adjoint of the half-plane of agent a (p, v, r, 1/tau) induced by neighbour b (pb, vb, rb)
// for (nbar, cbar), branch as in the forward step.  Adds the adjoints of the agent's and
// the neighbour's position, velocity, radius sum, and of 1/tau.
template <class T>
__device__ __forceinline__ void line_bar(V2<T> pa, V2<T> va, T ra, T itau, T dt, T half_idt, V2<T> pb,
                                         V2<T> vb, T rb, int branch, Line<T> L, V2<T> nbar, T cbar,
                                         V2<T>& pabar, V2<T>& vabar, T& rbar_ab, T& itaubar,
                                         V2<T>& pbbar, V2<T>& vbbar) {
    V2<T> p = mk2<T>(pb.x - pa.x, pb.y - pa.y);
    V2<T> v = mk2<T>(va.x - vb.x, va.y - vb.y);
    T R = ra + rb;
    V2<T> n = mk2<T>(L.nx, L.ny);
    V2<T> pbar = mk2<T>(0, 0), vbar = mk2<T>(0, 0);
    T Rbar = 0;
    if (branch == kLineCutoff) {
        V2<T> w = mk2<T>(v.x - p.x * itau, v.y - p.y * itau);
        T wl = sqrt_t(dot2(w, w));
        vabar.x += cbar * n.x;
        vabar.y += cbar * n.y;
        V2<T> nt = mk2<T>(nbar.x + cbar * va.x, nbar.y + cbar * va.y);
        T nn = dot2(n, nt);
        V2<T> wbar = mk2<T>((nt.x - n.x * nn) / wl - T(0.5) * cbar * n.x,
                            (nt.y - n.y * nn) / wl - T(0.5) * cbar * n.y);
        Rbar += T(0.5) * cbar * itau;
        itaubar += T(0.5) * cbar * R - dot2(p, wbar);
        vbar.x += wbar.x;
        vbar.y += wbar.y;
        pbar.x -= itau * wbar.x;
        pbar.y -= itau * wbar.y;
    } else if (branch == kLineLeftLeg || branch == kLineRightLeg) {
        T s = branch == kLineLeftLeg ? T(1) : T(-1);
        T p2 = dot2(p, p);
        T l = sqrt_t(p2 - R * R);
        V2<T> vs = mk2<T>(va.x + vb.x, va.y + vb.y);
        vabar.x += T(0.5) * cbar * n.x;
        vabar.y += T(0.5) * cbar * n.y;
        vbbar.x += T(0.5) * cbar * n.x;
        vbbar.y += T(0.5) * cbar * n.y;
        V2<T> nt = mk2<T>(nbar.x + T(0.5) * cbar * vs.x, nbar.y + T(0.5) * cbar * vs.y);
        V2<T> Jp = mk2<T>(-p.y, p.x);  // J = rotation by +90 degrees
        T ntJp = dot2(nt, Jp);
        // n = (-R p + s l J p) / p2;  M^T nt = -R nt + s l J^T nt, J^T nt = (nt.y, -nt.x)
        V2<T> MTn = mk2<T>(-R * nt.x + s * l * nt.y, -R * nt.y - s * l * nt.x);
        T nnt = dot2(n, nt);
        pbar.x += MTn.x / p2 + s * ntJp * p.x / (l * p2) - T(2) * nnt * p.x / p2;
        pbar.y += MTn.y / p2 + s * ntJp * p.y / (l * p2) - T(2) * nnt * p.y / p2;
        Rbar += (-dot2(nt, p) - s * ntJp * R / l) / p2;
    } else {  // overlap: q = p - v dt, n = -q/|q|, c = n.v_a + (R - |q|)/(2 dt)
        vabar.x += cbar * n.x;
        vabar.y += cbar * n.y;
        Rbar += cbar * half_idt;
        if (branch == kLineOverlap) {
            V2<T> q = mk2<T>(p.x - v.x * dt, p.y - v.y * dt);
            T ql = sqrt_t(dot2(q, q));
            V2<T> nt = mk2<T>(nbar.x + cbar * va.x, nbar.y + cbar * va.y);
            T nn = dot2(n, nt);
            V2<T> qbar = mk2<T>(-(nt.x - n.x * nn) / ql + cbar * half_idt * n.x,
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

// The half-plane and preferred velocity exactly as the forward step built them: the FP32
// step's own functions for float, their FP64 counterparts for double.
__device__ __forceinline__ Line<float> forward_line(const AdjArgs<float>& A, int a, int b, float2 pa,
                                                    float2 va, float ra, float itau, float dt,
                                                    float half_idt, int* br) {
    const float2 pb = A.pos[b];
    const float4 L = orca_line_dev(pa, va, ra, itau, dt, half_idt, (uint32_t)a,
                                   make_float4(pb.x, pb.y, A.radius[b], __uint_as_float((uint32_t)b)),
                                   A.vel[b], br);
    return Line<float>{L.x, L.y, L.z};
}
__device__ __forceinline__ Line<double> forward_line(const AdjArgs<double>& A, int a, int b, double2 pa,
                                                     double2 va, double ra, double itau, double dt,
                                                     double half_idt, int* br) {
    return orca_line_fp64(pa, va, ra, itau, dt, half_idt, (uint32_t)a, A.pos[b], A.radius[b],
                          (uint32_t)b, A.vel[b], br);
}
__device__ __forceinline__ float2 forward_pref(float2 p, float2 goal, float s, float dt, float idt, int* far) {
    return pref_velocity_dev(p, goal, s, dt, idt, far);
}
__device__ __forceinline__ double2 forward_pref(double2 p, double2 goal, double s, double dt, double idt,
                                                int* far) {
    return pref_velocity_fp64(p, goal, s, dt, idt, far);
}
__device__ __forceinline__ float recip(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }

// ---- per-agent adjoint ---------------------------------------------------------------
// Own adjoints of agent a: pbar[a] = dL/dp'(a) + what its half-planes and preferred
// velocity give its position, vbar[a] likewise for its velocity; its parameter gradients
// accumulate (one thread per agent, so without atomics).  Only the half-planes that fix
// the selected velocity -- at most three, named by the LP record -- carry an adjoint; they
// alone are rebuilt, and what each gives its neighbour goes to the agent's entry q
// (entries in increasing line order), whose neighbour's in-degree is counted.
template <class T, int KMAX>
__global__ void __launch_bounds__(128) adj_agent_kernel(AdjArgs<T> A) {
    pdl_wait();  // launched as a dependent of the previous reverse step's gather
    using T2 = typename AdjArgs<T>::T2;
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= A.n) return;
    const int K = A.kstride;
    const uint32_t tp = A.tape[a];
    const int mode = tp & 7, i = (tp >> 3) & 63, f = (tp >> 9) & 63, bound = (tp >> 15) & 3,
              j = (tp >> 17) & 63, side = (tp >> 23) & 1;
    // the lines that fix x, in increasing order (j and f lie below i; in a least-penetration
    // solve the bounding bisector j lies below f)
    int used[kAdjEntries];
    int nu = 0;
    if (mode == kTapeLine) {
        if (bound == kBoundLine) used[nu++] = j;
        used[nu++] = i;
    } else if (mode == kTapeLp3Dir) {
        used[nu++] = i;
    } else if (mode == kTapeLp3Line) {
        if (bound != kBoundDisc) used[nu++] = j;
        used[nu++] = f;
        used[nu++] = i;
    }
    int32_t* my_ent = A.ent + (size_t)a * kAdjEntries;
#pragma unroll
    for (int q = 0; q < kAdjEntries; ++q) my_ent[q] = -1;
    const T2 pbn = A.pbar_next[a], vbn = A.vbar_next[a];
    // p' = p + x dt, v' = x
    const V2<T> xbar = mk2<T>(vbn.x + A.dt * pbn.x, vbn.y + A.dt * pbn.y);
    if (xbar.x == T(0) && xbar.y == T(0)) {
        A.pbar[a] = pbn;
        T2 z;
        z.x = T(0);
        z.y = T(0);
        A.vbar[a] = z;
        return;
    }

    const T dt = A.dt;
    const T2 pa2 = A.pos[a], va2 = A.vel[a];
    const V2<T> pa = v2of(pa2), va = v2of(va2);
    const T ra = A.radius[a], V = A.max_speed[a];
    const T itau = recip(A.tau[a]);
    const T idt = recip(dt);
    const T half_idt = T(0.5) * idt;
    // the used half-planes exactly as the forward step built them
    Line<T> L[KMAX];
    int br[KMAX], nb[KMAX];
    V2<T> nbar[KMAX];
    T cbar[KMAX];
    for (int l = 0; l < KMAX; ++l) {
        nbar[l] = mk2<T>(0, 0);
        cbar[l] = T(0);
    }
    for (int q = 0; q < nu; ++q) {
        const int l = used[q];
        int b = l < K ? A.nbr[(size_t)a * K + l] : -1;
        if (!idx_ok(b >= 0 && b < A.n, A.err)) b = a;
        nb[l] = b;
        L[l] = forward_line(A, a, b, pa2, va2, ra, itau, dt, half_idt, &br[l]);
    }
    int far = 0;
    const T2 o2 = forward_pref(pa2, A.goal[a], A.pref_speed[a], dt, idt, &far);
    const V2<T> o = v2of(o2);
    V2<T> obar = mk2<T>(0, 0);

    if (mode == kTapePref) {
        obar = xbar;
    } else if (mode == kTapePrefClip) {
        T ol = sqrt_t(dot2(o, o));
        V2<T> oh = mk2<T>(o.x / ol, o.y / ol);
        T k = dot2(oh, xbar);
        obar = mk2<T>(V / ol * (xbar.x - oh.x * k), V / ol * (xbar.y - oh.y * k));
    } else if (mode == kTapeLine) {
        const Line<T> li = L[i];
        const V2<T> mi = mk2<T>(li.nx, li.ny);
        const V2<T> di = mk2<T>(li.ny, -li.nx);
        T t;
        if (bound == kBoundFree) t = dot2(di, o);
        else if (bound == kBoundDisc) {
            T D = V * V - li.c * li.c;
            t = (side ? T(1) : T(-1)) * sqrt_t(D > T(0) ? D : T(0));
        } else t = bound_t(mi, li.c, mk2<T>(L[j].nx, L[j].ny), L[j].c);
        V2<T> mibar = mk2<T>(0, 0);
        T eibar = 0;
        T tbar = point_on_line_bar(mi, li.c, t, xbar, eibar, mibar);
        if (bound == kBoundFree) {  // t = d(n_i).o
            mibar.x += -tbar * o.y;
            mibar.y += tbar * o.x;
            obar = mk2<T>(tbar * di.x, tbar * di.y);
        } else if (bound == kBoundDisc) {
            if (t != T(0)) eibar += -tbar * li.c / t;
        } else {
            V2<T> mjbar = mk2<T>(0, 0);
            T ejbar = 0;
            bound_bar(mi, li.c, mk2<T>(L[j].nx, L[j].ny), L[j].c, tbar, mibar, eibar, mjbar, ejbar);
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
        const Line<T> li = L[i];
        V2<T> m;
        T e;
        bisector(li, L[f], m, e);
        T t;
        V2<T> mj = mk2<T>(0, 0);
        T ej = 0;
        if (bound == kBoundDisc) {
            T D = V * V - e * e;
            t = (side ? T(1) : T(-1)) * sqrt_t(D > T(0) ? D : T(0));
        } else {
            bisector(li, L[j], mj, ej);
            t = bound_t(m, e, mj, ej);
        }
        V2<T> mbar = mk2<T>(0, 0);
        T ebar = 0;
        T tbar = point_on_line_bar(m, e, t, xbar, ebar, mbar);
        if (bound == kBoundDisc) {
            if (t != T(0)) ebar += -tbar * e / t;
        } else {
            V2<T> mjbar = mk2<T>(0, 0);
            T ejbar = 0;
            bound_bar(m, e, mj, ej, tbar, mbar, ebar, mjbar, ejbar);
            bisector_bar(li, L[j], mjbar, ejbar, nbar[i], cbar[i], nbar[j], cbar[j]);
        }
        bisector_bar(li, L[f], mbar, ebar, nbar[i], cbar[i], nbar[f], cbar[f]);
    }

    // half-planes -> state and parameters of the agent and its neighbours
    V2<T> pabar = v2of(pbn), vabar = mk2<T>(0, 0);
    T rabar = 0, itaubar = 0;
    for (int q = 0; q < nu; ++q) {
        const int l = used[q];
        if (nbar[l].x == T(0) && nbar[l].y == T(0) && cbar[l] == T(0)) continue;
        const int b = nb[l];
        V2<T> pbbar = mk2<T>(0, 0), vbbar = mk2<T>(0, 0);
        T Rbar = 0;
        line_bar(pa, va, ra, itau, dt, half_idt, v2of(A.pos[b]), v2of(A.vel[b]), A.radius[b], br[l], L[l],
                 nbar[l], cbar[l], pabar, vabar, Rbar, itaubar, pbbar, vbbar);
        rabar += Rbar;
        const size_t e = (size_t)a * kAdjEntries + q;
        T* c = A.contrib + 4 * e;
        c[0] = pbbar.x;
        c[1] = pbbar.y;
        c[2] = vbbar.x;
        c[3] = vbbar.y;
        A.contrib_r[e] = Rbar;
        my_ent[q] = b;
        const uint32_t at = atomicAdd(A.incnt + b, 1u);  // integer: exact in any order
        if (at < (uint32_t)kInCap) A.inlist[(size_t)b * kInCap + at] = (uint32_t)e;
    }
    // preferred velocity -> position and preferred speed of the agent
    if (obar.x != T(0) || obar.y != T(0)) {
        V2<T> g = mk2<T>(A.goal[a].x - pa.x, A.goal[a].y - pa.y);
        if (far) {
            T gl = sqrt_t(dot2(g, g));
            V2<T> gh = mk2<T>(g.x / gl, g.y / gl);
            T k = dot2(gh, obar);
            T s = A.pref_speed[a];
            A.g_pref[a] += k;
            pabar.x -= s / gl * (obar.x - gh.x * k);
            pabar.y -= s / gl * (obar.y - gh.y * k);
        } else {
            pabar.x -= obar.x * idt;
            pabar.y -= obar.y * idt;
        }
    }
    T2 pw, vw;
    pw.x = pabar.x;
    pw.y = pabar.y;
    vw.x = vabar.x;
    vw.y = vabar.y;
    A.pbar[a] = pw;
    A.vbar[a] = vw;
    A.g_radius[a] += rabar;
    // d(1/tau)/dtau = -1/tau^2
    A.g_tau[a] += -itaubar * itau * itau;
}

// Agent b: its list sorted by entry index (agent, then line order) in shared memory, then
// the contributions summed in that order into its adjoints and radius gradient, plus the
// loss gradient of its position at this step (dl_dp, may be null).  An agent that
// received more than kInCap entries takes them from a scan of all agents' entries in
// index order instead (the same order, so the same sums).  Clears its count for the next
// step.
constexpr int kGatherThreads = 128;
template <class T>
__global__ void __launch_bounds__(kGatherThreads) adj_gather_kernel(AdjArgs<T> A) {
    pdl_wait();  // every entry of this step is placed before any list is read
    using T2 = typename AdjArgs<T>::T2;
    __shared__ uint32_t s_l[kInCap * kGatherThreads];
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= A.n) return;
    const uint32_t deg = A.incnt[b];
    T px = 0, py = 0, vx = 0, vy = 0, rr = 0;
    auto add = [&](uint32_t e) {
        const T* c = A.contrib + 4 * (size_t)e;
        px += c[0];
        py += c[1];
        vx += c[2];
        vy += c[3];
        rr += A.contrib_r[e];
    };
    if (deg <= (uint32_t)kInCap) {
        uint32_t* sl = s_l + threadIdx.x;  // element k at sl[k * kGatherThreads]
        const uint32_t* lst = A.inlist + (size_t)b * kInCap;
        for (uint32_t q = 0; q < deg; ++q) sl[q * kGatherThreads] = lst[q];
        for (uint32_t q = 1; q < deg; ++q) {
            const uint32_t key = sl[q * kGatherThreads];
            uint32_t r = q;
            while (r > 0 && sl[(r - 1) * kGatherThreads] > key) {
                sl[r * kGatherThreads] = sl[(r - 1) * kGatherThreads];
                --r;
            }
            sl[r * kGatherThreads] = key;
        }
        for (uint32_t q = 0; q < deg; ++q) add(sl[q * kGatherThreads]);
    } else {
        const uint32_t ne = (uint32_t)A.n * kAdjEntries;
        for (uint32_t e = 0; e < ne; ++e)
            if (A.ent[e] == b) add(e);
    }
    T2 p = A.pbar[b], v = A.vbar[b];
    p.x += px;
    p.y += py;
    if (A.dl_dp) {
        p.x += A.dl_dp[b].x;
        p.y += A.dl_dp[b].y;
    }
    v.x += vx;
    v.y += vy;
    A.pbar[b] = p;
    A.vbar[b] = v;
    A.g_radius[b] += rr;
    A.incnt[b] = 0u;
}

template <class T>
cudaError_t launch_adjoint_step(const AdjArgs<T>& A, int kmax, cudaStream_t st) {
    if (A.n <= 0) return cudaSuccess;
    const int nb = (A.n + 127) / 128;
    // both kernels launched as programmatic dependents: each waits at entry (pdl_wait) for
    // the kernel before it, and its launch overlaps that kernel's tail
    cudaError_t e;
    if (kmax <= 10) e = launch_pdl(adj_agent_kernel<T, 10>, nb, 128, 0, st, A);
    else if (kmax <= 16) e = launch_pdl(adj_agent_kernel<T, 16>, nb, 128, 0, st, A);
    else if (kmax <= 20) e = launch_pdl(adj_agent_kernel<T, 20>, nb, 128, 0, st, A);
    else e = launch_pdl(adj_agent_kernel<T, 32>, nb, 128, 0, st, A);
    if (e != cudaSuccess) return e;
    return launch_pdl(adj_gather_kernel<T>, (A.n + kGatherThreads - 1) / kGatherThreads, kGatherThreads, 0, st, A);
}

template cudaError_t launch_adjoint_step<float>(const AdjArgs<float>&, int, cudaStream_t);
template cudaError_t launch_adjoint_step<double>(const AdjArgs<double>&, int, cudaStream_t);

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

cudaError_t launch_unpermute_params(int n, const AgentParams& src, float2* goal, float* radius,
                                    float* vmax, float* pref, float* tau, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    unpermute_params_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, src, goal, radius, vmax, pref, tau);
    return cudaGetLastError();
}

}  // namespace orca
