// orca_validate.cu -- an FP64 rollout of the ORCA step and its FP64 adjoint, for
// validating the adjoint only (the paper has no counterpart; no step or rollout of the
// library runs this code).
//
// The adjoint of the FP32 rollouts (orca_adjoint.cu) differentiates each step along the
// FP32 trajectory.  Checked against FP64 finite differences of the oracle, a mismatch at
// a long horizon could be an adjoint error or the FP32 trajectory drifting from the FP64
// one.  This file separates the two: it runs the same step in FP64 -- neighbours decided
// in FP32 on the FP32-rounded positions, as the FP32 step and the oracle decide them;
// half-planes, preferred velocity, LP2 and LP3 in double, with the same record of what
// fixed each selected velocity -- and then the double instantiation of the very adjoint
// kernels the FP32 rollouts use.  Its trajectory follows the oracle's to rounding, so
// its gradients can be held to FP64 finite differences at any horizon.
//
// Small crowds only: the neighbour search is a brute-force scan of all agents (one thread
// per agent), every state of the rollout is kept (no checkpoints), and scratch is
// allocated per call with cudaMalloc.
#include <string>

#include "../../include/orca_gb300.h"
#include "orca_adjoint.cuh"

namespace orca {

void set_context_free_error(const std::string& msg);

constexpr int kValidateMaxAgents = 65536;
constexpr double kEps64 = 1e-5;  // the parallel-line tolerance of both precisions

struct Tape64 {
    int mode, i, f, bound, j, side;
    __device__ unsigned pack() const {
        return (unsigned)mode | (unsigned)i << 3 | (unsigned)f << 9 | (unsigned)bound << 15 |
               (unsigned)j << 17 | (unsigned)side << 23;
    }
};

__device__ __forceinline__ double ddot(double ax, double ay, double bx, double by) { return ax * bx + ay * by; }
__device__ __forceinline__ double ddet(double ax, double ay, double bx, double by) { return ax * by - ay * bx; }

// Lines of one agent: its own half-planes (unit normals).
struct Rows64 {
    static constexpr bool kUnit = true;
    const Line<double>* row;
    __device__ bool operator()(int j, Line<double>& l) const {
        l = row[j];
        return true;
    }
};

// Bisectors of line i with lines j < i (least penetration's projected problem), not
// normalised; same-direction parallel lines give none.
struct Bis64 {
    static constexpr bool kUnit = false;
    const Line<double>* row;
    Line<double> li;
    __device__ bool operator()(int j, Line<double>& q) const {
        const Line<double> lj = row[j];
        const double den = ddet(li.nx, li.ny, lj.nx, lj.ny);
        if (fabs(den) <= kEps64 && ddot(li.nx, li.ny, lj.nx, lj.ny) > 0.0) return false;
        q = Line<double>{lj.nx - li.nx, lj.ny - li.ny, lj.c - li.c};
        return true;
    }
};

__device__ __forceinline__ Line<double> unit64(Line<double> l) {
    const double s = sqrt(l.nx * l.nx + l.ny * l.ny);
    return Line<double>{l.nx / s, l.ny / s, l.c / s};
}

// LP1 on unit line li over lines 0..i-1 and the disc |x| <= V (the FP32 step's lp1_dev in
// double): x = c n + t d, d = (n.y, -n.x).
template <class Acc>
__device__ bool lp1_64(const Acc& line, int i, Line<double> li, double V, double ox, double oy, bool dir_opt,
                       double& xx, double& xy, Tape64* rec) {
    const double D = V * V - li.c * li.c;
    if (D < 0.0) return false;
    const double sq = sqrt(D);
    double tL = -sq, tR = sq;
    int srcL = -1, srcR = -1;
    for (int j = 0; j < i; ++j) {
        Line<double> lj;
        if (!line(j, lj)) continue;
        const double den = ddet(li.nx, li.ny, lj.nx, lj.ny);
        const double rhs = lj.c - li.c * ddot(li.nx, li.ny, lj.nx, lj.ny);
        const bool par = Acc::kUnit ? fabs(den) <= kEps64
                                    : den * den <= kEps64 * kEps64 * ddot(lj.nx, lj.ny, lj.nx, lj.ny);
        if (par) {
            if (rhs > 0.0) return false;
            continue;
        }
        const double t = -rhs / den;
        if (den >= 0.0) {
            if (t < tR) srcR = j;
            tR = fmin(tR, t);
        } else {
            if (t > tL) srcL = j;
            tL = fmax(tL, t);
        }
        if (tL > tR) return false;
    }
    double t = ddot(ox, oy, li.ny, -li.nx);
    int side = -1;
    if (dir_opt) side = t > 0.0 ? 1 : 0;
    else if (t < tL) side = 0;
    else if (t > tR) side = 1;
    rec->side = side < 0 ? 0 : side;
    const int src = side == 0 ? srcL : srcR;
    rec->bound = side < 0 ? kBoundFree : (src < 0 ? kBoundDisc : kBoundLine);
    rec->j = src < 0 ? 0 : src;
    if (dir_opt) t = t > 0.0 ? tR : tL;
    else t = fmin(fmax(t, tL), tR);
    xx = li.c * li.nx + t * li.ny;
    xy = li.c * li.ny - t * li.nx;
    return true;
}

// LP2 over lines 0..n-1 in order; returns n, or the line where LP1 failed (x kept).
template <class Acc>
__device__ int lp2_64(const Acc& line, int n, double V, double ox, double oy, bool dir_opt, double& xx,
                      double& xy, Tape64* rec) {
    if (dir_opt) {
        xx = ox * V;
        xy = oy * V;
        rec->mode = kTapeLp3Dir;
    } else {
        const double o2 = ox * ox + oy * oy;
        if (o2 > V * V) {
            const double s = V / sqrt(o2);
            xx = ox * s;
            xy = oy * s;
            rec->mode = kTapePrefClip;
        } else {
            xx = ox;
            xy = oy;
            rec->mode = kTapePref;
        }
    }
    for (int i = 0; i < n; ++i) {
        Line<double> li;
        if (!line(i, li)) continue;
        if (!(li.c - ddot(li.nx, li.ny, xx, xy) > 0.0)) continue;
        if (!Acc::kUnit) li = unit64(li);
        const double sx = xx, sy = xy;
        Tape64 r1 = *rec;
        if (!lp1_64(line, i, li, V, ox, oy, dir_opt, xx, xy, &r1)) {
            xx = sx;
            xy = sy;
            return i;
        }
        r1.mode = kTapeLine;
        r1.i = i;
        r1.f = 0;
        *rec = r1;
    }
    return n;
}

// LP3 (least penetration) from line `begin` on.
__device__ void lp3_64(const Line<double>* row, int n, int begin, double V, double& xx, double& xy,
                       Tape64* rec) {
    double dist = 0.0;
    for (int i = begin; i < n; ++i) {
        const Line<double> li = row[i];
        if (!(li.c - ddot(li.nx, li.ny, xx, xy) > dist)) continue;
        Bis64 bis{row, li};
        const double sx = xx, sy = xy;
        Tape64 r2{0, 0, 0, 0, 0, 0};
        if (lp2_64(bis, i, V, li.nx, li.ny, true, xx, xy, &r2) < i) {
            xx = sx;
            xy = sy;
        } else {
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
        dist = li.c - ddot(li.nx, li.ny, xx, xy);
    }
}

struct Step64 {
    int n, k;
    float nd;
    double dt;
    const double2 *pos, *vel, *goal;
    const double *radius, *vmax, *pref, *tau;
    double2 *pos_out, *vel_out;
    int32_t* nbr;    // n * k, -1 padded
    uint32_t* tape;  // n
};

// One FP64 step, one thread per agent: the k nearest by (fl32 d^2, index) among all
// agents strictly inside r_obs on the FP32-rounded positions; half-planes, preferred
// velocity and the LP in double; the record of what fixed the velocity.
template <int KMAX>
__global__ void __launch_bounds__(128) fp64_step_kernel(Step64 S) {
    const int a = blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= S.n) return;
    const double2 p = S.pos[a], v = S.vel[a];
    const float pxf = (float)p.x, pyf = (float)p.y;
    const float nd2 = __fmul_rn(S.nd, S.nd);
    unsigned long long kk[KMAX];
    int cnt = 0;
    for (int j = 0; j < S.n; ++j) {
        if (j == a) continue;
        const double2 q = S.pos[j];
        const float dx = __fsub_rn((float)q.x, pxf), dy = __fsub_rn((float)q.y, pyf);
        const float d2 = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
        if (!(d2 < nd2)) continue;
        const unsigned long long key = ((unsigned long long)__float_as_uint(d2) << 32) | (unsigned)j;
        if (cnt == S.k && key >= kk[cnt - 1]) continue;
        int r = cnt < S.k ? cnt++ : cnt - 1;
        while (r > 0 && kk[r - 1] > key) {
            kk[r] = kk[r - 1];
            --r;
        }
        kk[r] = key;
    }
    const double dt = S.dt, idt = 1.0 / dt, half_idt = 0.5 * idt;
    const double ra = S.radius[a], V = S.vmax[a], itau = 1.0 / S.tau[a];
    Line<double> row[KMAX];
    for (int l = 0; l < cnt; ++l) {
        const int j = (int)(kk[l] & 0xffffffffu);
        int br = 0;
        row[l] = orca_line_fp64(p, v, ra, itau, dt, half_idt, (uint32_t)a, S.pos[j], S.radius[j], (uint32_t)j,
                                S.vel[j], &br);
        S.nbr[(size_t)a * S.k + l] = j;
    }
    for (int l = cnt; l < S.k; ++l) S.nbr[(size_t)a * S.k + l] = -1;
    int far = 0;
    const double2 o = pref_velocity_fp64(p, S.goal[a], S.pref[a], dt, idt, &far);
    double xx = 0.0, xy = 0.0;
    Tape64 tape{0, 0, 0, 0, 0, 0};
    Rows64 rl{row};
    const int b = lp2_64(rl, cnt, V, o.x, o.y, false, xx, xy, &tape);
    if (b < cnt) lp3_64(row, cnt, b, V, xx, xy, &tape);
    S.tape[a] = tape.pack();
    S.vel_out[a] = make_double2(xx, xy);
    S.pos_out[a] = make_double2(p.x + xx * dt, p.y + xy * dt);
}

static cudaError_t launch_step64(const Step64& S, cudaStream_t st) {
    const int nb = (S.n + 127) / 128;
    if (S.k <= 10) fp64_step_kernel<10><<<nb, 128, 0, st>>>(S);
    else if (S.k <= 16) fp64_step_kernel<16><<<nb, 128, 0, st>>>(S);
    else if (S.k <= 20) fp64_step_kernel<20><<<nb, 128, 0, st>>>(S);
    else fp64_step_kernel<32><<<nb, 128, 0, st>>>(S);
    return cudaGetLastError();
}

static int validate_fail(int code, const std::string& msg) {
    set_context_free_error(msg);
    return code;
}

}  // namespace orca

using namespace orca;

extern "C" ORCA_API int orca_validate_rollout_fp64(
    int32_t n, int32_t max_neighbors, float neighbor_dist, double dt, int32_t T, const double* pos0,
    const double* vel0, const double* goal, const double* radius, const double* max_speed,
    const double* pref_speed, const double* time_horizon, const double* dL_dpos, double* traj_pos,
    double* g_pref_speed, double* g_radius, double* g_time_horizon, double* g_pos0, double* g_vel0,
    void* stream) {
    if (n < 1 || n > kValidateMaxAgents)
        return validate_fail(ORCA_ERR_ARG, "orca_validate_rollout_fp64: n must be 1..65536");
    if (max_neighbors < 1 || max_neighbors > kMaxNeighbors || !(neighbor_dist > 0.0f) || !(dt > 0.0) || T < 1)
        return validate_fail(ORCA_ERR_ARG, "orca_validate_rollout_fp64: bad k, r_obs, dt or T");
    if (!pos0 || !vel0 || !goal || !radius || !max_speed || !pref_speed || !time_horizon || !traj_pos)
        return validate_fail(ORCA_ERR_ARG, "orca_validate_rollout_fp64: null array");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t N = (size_t)n, K = (size_t)max_neighbors;
    // every state of the rollout, its neighbour lists and LP records, the adjoint buffers
    const size_t b_state = 2 * N * sizeof(double2), b_nbr = N * K * 4, b_tape = N * 4;
    size_t off[10], total = 0;
    const size_t E = N * kAdjEntries;
    const size_t sizes[10] = {(size_t)(T + 1) * b_state, (size_t)T * b_nbr, (size_t)T * b_tape,
                              4 * N * sizeof(double2), 3 * N * sizeof(double), E * 4 * sizeof(double),
                              N * 4, N * kInCap * 4, E * 4, E * sizeof(double)};
    for (int q = 0; q < 10; ++q) {
        off[q] = total;
        total += (sizes[q] + 255) & ~size_t(255);
    }
    char* w = nullptr;
    cudaError_t e = cudaMalloc((void**)&w, total);
    if (e != cudaSuccess)
        return validate_fail(ORCA_ERR_NOMEM, std::string("orca_validate_rollout_fp64: ") + cudaGetErrorString(e));
    auto state = [&](int t) { return (double2*)(w + off[0] + (size_t)t * b_state); };
    int32_t* nbr = (int32_t*)(w + off[1]);
    uint32_t* tape = (uint32_t*)(w + off[2]);
    double2* adj = (double2*)(w + off[3]);
    double* gs = (double*)(w + off[4]);
    e = cudaMemcpyAsync(state(0), pos0, N * sizeof(double2), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(state(0) + N, vel0, N * sizeof(double2), cudaMemcpyDeviceToDevice, st);
    for (int t = 0; t < T && e == cudaSuccess; ++t) {
        Step64 S;
        S.n = n;
        S.k = max_neighbors;
        S.nd = neighbor_dist;
        S.dt = dt;
        S.pos = state(t);
        S.vel = state(t) + N;
        S.goal = (const double2*)goal;
        S.radius = radius;
        S.vmax = max_speed;
        S.pref = pref_speed;
        S.tau = time_horizon;
        S.pos_out = state(t + 1);
        S.vel_out = state(t + 1) + N;
        S.nbr = nbr + (size_t)t * N * K;
        S.tape = tape + (size_t)t * N;
        e = launch_step64(S, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(traj_pos + (size_t)t * N * 2, state(t + 1), N * sizeof(double2),
                                cudaMemcpyDeviceToDevice, st);
    }
    if (e == cudaSuccess && dL_dpos) {
        double2* pnext = adj;
        double2* vnext = adj + N;
        double2* pcur = adj + 2 * N;
        double2* vcur = adj + 3 * N;
        double* gp = g_pref_speed ? g_pref_speed : gs;
        double* gr = g_radius ? g_radius : gs + N;
        double* gt = g_time_horizon ? g_time_horizon : gs + 2 * N;
        const double2* dLdp = (const double2*)dL_dpos;
        e = cudaMemsetAsync(gp, 0, N * 8, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(gr, 0, N * 8, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(gt, 0, N * 8, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(w + off[6], 0, N * 4, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(pnext, dLdp + (size_t)(T - 1) * N, N * sizeof(double2), cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(vnext, 0, N * sizeof(double2), st);
        for (int t = T - 1; t >= 0 && e == cudaSuccess; --t) {
            AdjArgs<double> A;
            A.n = n;
            A.kstride = max_neighbors;
            A.dt = dt;
            A.pos = state(t);
            A.vel = state(t) + N;
            A.goal = (const double2*)goal;
            A.radius = radius;
            A.max_speed = max_speed;
            A.pref_speed = pref_speed;
            A.tau = time_horizon;
            A.nbr = nbr + (size_t)t * N * K;
            A.tape = tape + (size_t)t * N;
            A.pbar_next = pnext;
            A.vbar_next = vnext;
            A.dl_dp = t >= 1 ? dLdp + (size_t)(t - 1) * N : nullptr;
            A.pbar = pcur;
            A.vbar = vcur;
            A.g_pref = gp;
            A.g_radius = gr;
            A.g_tau = gt;
            A.contrib = (double*)(w + off[5]);
            A.ent = (int32_t*)(w + off[8]);
            A.contrib_r = (double*)(w + off[9]);
            A.incnt = (uint32_t*)(w + off[6]);
            A.inlist = (uint32_t*)(w + off[7]);
            A.err = nullptr;  // the validation rollout is built without index checks
            e = launch_adjoint_step(A, max_neighbors, st);
            double2* tmp = pnext;
            pnext = pcur;
            pcur = tmp;
            tmp = vnext;
            vnext = vcur;
            vcur = tmp;
        }
        if (e == cudaSuccess && g_pos0) e = cudaMemcpyAsync(g_pos0, pnext, N * sizeof(double2), cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess && g_vel0) e = cudaMemcpyAsync(g_vel0, vnext, N * sizeof(double2), cudaMemcpyDeviceToDevice, st);
    }
    cudaError_t e2 = cudaStreamSynchronize(st);
    cudaFree(w);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess)
        return validate_fail(ORCA_ERR_CUDA, std::string("orca_validate_rollout_fp64: ") + cudaGetErrorString(e));
    return ORCA_OK;
}
