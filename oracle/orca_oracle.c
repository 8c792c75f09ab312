/*
 * orca_oracle.c -- plain, slow, FP64 CPU oracle for one ORCA crowd-simulation step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  The GPU library never includes, links or
 * calls anything from here, and this file includes nothing from the GPU library.
 *
 * What one step computes (Section 3 of "Fast Simulation of Crowd Collision Avoidance",
 * which defers the ORCA mathematics to van den Berg et al., "Reciprocal n-body
 * collision avoidance"):
 *   1. preferred velocity towards the goal at the agent's preferred speed (Section 3,
 *      first paragraph after Fig. 1; Section 4, test set-up);
 *   2. spatial bins over the crowd and the observation filter r_obs (Fig. 2);
 *   3. one ORCA half-plane per observed neighbour: the vector u from the relative
 *      velocity to the nearest point of the boundary of the truncated velocity
 *      obstacle VO^tau, and the half-plane through v + u/2 whose normal follows u
 *      (Fig. 1 a-c);
 *   4. the 2-D linear program: the velocity closest to the preferred one inside the
 *      maximum-speed disc and every half-plane (Section 3, batch LP paragraphs),
 *      solved by an incremental LP (Seidel's method, Section 2, in a fixed order);
 *   5. when the half-planes have no common point, the velocity that least penetrates
 *      them (Section 3, "least penetrates"), i.e. the minimum over the disc of the
 *      largest violation, by the incremental 3-D LP;
 *   6. all agents adopt their new velocity and move simultaneously (Section 2).
 *
 * Precision: every geometric quantity is FP64.  The two integer-valued decisions that
 * must agree bit for bit with the GPU -- the grid cell of an agent and its neighbour
 * set -- are taken in FP32 (float operands, one rounding per operation, no FMA: build
 * with -ffp-contract=off), exactly as the GPU takes them.  In rollout mode (fp64_knn=1)
 * the neighbour search runs in FP64 instead.
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - neighbours: the max_neighbors nearest with squared distance strictly below r_obs^2,
 *     ordered by (d^2, index); this order is also the LP's constraint order;
 *   - the half-plane passes through v_a + u/2 (reciprocal share; the Fig. 1 caption's
 *     "v + u" is the non-reciprocal form);
 *   - overlapping agents (|p| <= R) use the time step dt in place of tau;
 *   - |w| = 0 in the overlap case: n = -p/|p|, or (+1,0)/(-1,0) by index order when the
 *     agents coincide;
 *   - det(p, w) = 0 in the leg case selects the right leg;
 *   - "clamped near the goal": if |goal - p| <= pref_speed*dt the preferred velocity is
 *     (goal - p)/dt;
 *   - parallel-line tolerance eps = 1e-5.
 *
 * Ill-conditioning (for parity tests against an FP32 implementation):
 *   - margin: the half-plane construction's discontinuous decisions (overlap or not,
 *     left or right leg) record their normalised distance to the threshold; the
 *     per-agent minimum is reported;
 *   - sens (optional): the LP is re-solved with each half-plane shifted by +-4 FP32 ulps
 *     of its offset and turned by +-2^-22 rad about its nearest point to the origin, one
 *     at a time -- the rounding any FP32 construction of the half-planes carries -- and
 *     the largest move of the chosen velocity is reported.  An agent whose velocity moves
 *     by more than half the parity tolerance is not determined to that tolerance by FP32
 *     half-planes.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_EPS 1e-5
#define OR_MAXK 64

typedef struct { double x, y; } v2;
typedef struct { v2 P, d; } line2;          /* point P, unit direction d; valid side: left of d */
typedef struct { double m; } tags;            /* running minimum of normalised margins */

static v2 mk(double x, double y) { v2 r; r.x = x; r.y = y; return r; }
static v2 add(v2 a, v2 b) { return mk(a.x + b.x, a.y + b.y); }
static v2 sub(v2 a, v2 b) { return mk(a.x - b.x, a.y - b.y); }
static v2 scl(v2 a, double s) { return mk(a.x * s, a.y * s); }
static double dot(v2 a, v2 b) { return a.x * b.x + a.y * b.y; }
static double det2(v2 a, v2 b) { return a.x * b.y - a.y * b.x; }
static double len(v2 a) { return sqrt(dot(a, a)); }

static void note(tags* t, double value, double threshold, double scale) {
    if (!t) return;
    double s = fabs(scale) > 1e-300 ? fabs(scale) : 1e-300;
    double m = fabs(value - threshold) / s;
    if (m < t->m) t->m = m;
}

/* ----------------------------------------------------------------------------------
 * Uniform grid of spatial bins (Fig. 2).  All arithmetic in FP32.
 *   xmin/ymin: exact minimum over agents; s: cell edge; inv = fl(1/s);
 *   gx = floor(fl(fl(xmax - xmin) * inv)) + 1 (same for gy);
 *   capacity rule: while gx*gy > max_cells, s doubles (exact in FP32).
 *   cell of (x, y): cx = floor(fl(fl(x - xmin) * inv)) clamped to [0, gx-1], likewise
 *   cy; cell = cy*gx + cx.
 * grid_f = {xmin, ymin, s, inv}, grid_i = {gx, gy}.
 * -------------------------------------------------------------------------------- */
int oracle_grid(const float* pos, int n, float cell_size, long long max_cells,
                float* grid_f, int* grid_i) {
    if (n <= 0 || !(cell_size > 0.0f) || max_cells < 1) return -1;
    float xmin = pos[0], xmax = pos[0], ymin = pos[1], ymax = pos[1];
    for (int i = 1; i < n; ++i) {
        float x = pos[2 * i], y = pos[2 * i + 1];
        if (x < xmin) xmin = x;
        if (x > xmax) xmax = x;
        if (y < ymin) ymin = y;
        if (y > ymax) ymax = y;
    }
    float ex = xmax - xmin, ey = ymax - ymin;
    float s = cell_size;
    for (int it = 0; it < 200; ++it) {
        float inv = 1.0f / s;
        float fx = floorf(ex * inv), fy = floorf(ey * inv);
        double cells = ((double)fx + 1.0) * ((double)fy + 1.0);
        if (cells <= (double)max_cells) {
            grid_f[0] = xmin; grid_f[1] = ymin; grid_f[2] = s; grid_f[3] = inv;
            grid_i[0] = (int)fx + 1; grid_i[1] = (int)fy + 1;
            return 0;
        }
        s = s * 2.0f;
    }
    return -2;
}

static int cell_coord(float v, float vmin, float inv, int g) {
    float q = (v - vmin) * inv;
    int c = (int)floorf(q);
    if (c < 0) c = 0;
    if (c > g - 1) c = g - 1;
    return c;
}

void oracle_cells(const float* pos, int n, const float* grid_f, const int* grid_i,
                  uint32_t* cell) {
    for (int i = 0; i < n; ++i) {
        int cx = cell_coord(pos[2 * i], grid_f[0], grid_f[3], grid_i[0]);
        int cy = cell_coord(pos[2 * i + 1], grid_f[1], grid_f[3], grid_i[1]);
        cell[i] = (uint32_t)cy * (uint32_t)grid_i[0] + (uint32_t)cx;
    }
}

/* ----------------------------------------------------------------------------------
 * Neighbour sets: for agent i, the k smallest (d^2, j) over j != i with d^2 < r_obs^2.
 * FP32 mode: dx = fl(xj - xi), dy = fl(yj - yi), d^2 = fl(fl(dx*dx) + fl(dy*dy)),
 * threshold fl(r_obs*r_obs).  FP64 mode: the same formula in double.
 * -------------------------------------------------------------------------------- */
typedef struct { double d2; int j; float d2f; } cand;

static int cand_less(double d2a, int ja, double d2b, int jb) {
    return d2a < d2b || (d2a == d2b && ja < jb);
}

static void cand_insert(cand* list, int* cnt, int k, double d2, float d2f, int j) {
    if (*cnt == k && !cand_less(d2, j, list[k - 1].d2, list[k - 1].j)) return;
    int p = (*cnt < k) ? (*cnt)++ : k - 1;
    while (p > 0 && cand_less(d2, j, list[p - 1].d2, list[p - 1].j)) {
        list[p] = list[p - 1];
        --p;
    }
    list[p].d2 = d2; list[p].j = j; list[p].d2f = d2f;
}

static void consider(const float* pf, const double* pd, int fp64, int i, int j,
                     float nd2f, double nd2d, cand* list, int* cnt, int k) {
    if (j == i) return;
    if (fp64) {
        double dx = pd[2 * j] - pd[2 * i], dy = pd[2 * j + 1] - pd[2 * i + 1];
        double d2 = dx * dx + dy * dy;
        if (d2 < nd2d) cand_insert(list, cnt, k, d2, (float)d2, j);
    } else {
        float dx = pf[2 * j] - pf[2 * i];
        float dy = pf[2 * j + 1] - pf[2 * i + 1];
        float dxx = dx * dx;
        float dyy = dy * dy;
        float d2 = dxx + dyy;
        if (d2 < nd2f) cand_insert(list, cnt, k, (double)d2, d2, j);
    }
}

/* Cell lists for the grid mode: agents of each cell in ascending index order. */
typedef struct { int gx, gy; float xmin, ymin, inv; int* start; int* items; } bins;

static int bins_build(bins* b, const float* pf, int n, const float* grid_f, const int* grid_i) {
    b->gx = grid_i[0]; b->gy = grid_i[1];
    b->xmin = grid_f[0]; b->ymin = grid_f[1]; b->inv = grid_f[3];
    long long nc = (long long)b->gx * b->gy;
    b->start = (int*)calloc((size_t)nc + 1, sizeof(int));
    b->items = (int*)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    uint32_t* cell = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    if (!b->start || !b->items || !cell) { free(cell); return -1; }
    oracle_cells(pf, n, grid_f, grid_i, cell);
    for (int i = 0; i < n; ++i) b->start[cell[i] + 1]++;
    for (long long c = 0; c < nc; ++c) b->start[c + 1] += b->start[c];
    int* fill = (int*)malloc(sizeof(int) * (size_t)nc);
    if (!fill) { free(cell); return -1; }
    memcpy(fill, b->start, sizeof(int) * (size_t)nc);
    for (int i = 0; i < n; ++i) b->items[fill[cell[i]]++] = i;
    free(fill);
    free(cell);
    return 0;
}

static void bins_free(bins* b) { free(b->start); free(b->items); }

/* Grid-mode search: every cell overlapping [x - r_obs, x + r_obs] x [y - r_obs, y + r_obs],
 * widened by one cell on each side to absorb the FP32 rounding of cell indices. */
static long long knn_grid_one(const bins* b, const float* pf, const double* pd, int fp64,
                              int i, float ndf, double ndd, cand* list, int* cnt, int k) {
    float nd2f = ndf * ndf;
    double nd2d = ndd * ndd;
    double xi = fp64 ? pd[2 * i] : pf[2 * i], yi = fp64 ? pd[2 * i + 1] : pf[2 * i + 1];
    double s = 1.0 / (double)b->inv;
    double rx = (fp64 ? ndd : (double)ndf);
    long long cx0 = (long long)floor((xi - rx - b->xmin) / s) - 1;
    long long cx1 = (long long)floor((xi + rx - b->xmin) / s) + 1;
    long long cy0 = (long long)floor((yi - rx - b->ymin) / s) - 1;
    long long cy1 = (long long)floor((yi + rx - b->ymin) / s) + 1;
    if (cx0 < 0) cx0 = 0;
    if (cy0 < 0) cy0 = 0;
    if (cx1 > b->gx - 1) cx1 = b->gx - 1;
    if (cy1 > b->gy - 1) cy1 = b->gy - 1;
    long long scanned = 0;
    for (long long cy = cy0; cy <= cy1; ++cy)
        for (long long cx = cx0; cx <= cx1; ++cx) {
            long long c = cy * b->gx + cx;
            for (int q = b->start[c]; q < b->start[c + 1]; ++q) {
                consider(pf, pd, fp64, i, b->items[q], nd2f, nd2d, list, cnt, k);
                ++scanned;
            }
        }
    return scanned;
}

static void knn_brute_one(const float* pf, const double* pd, int fp64, int n, int i,
                          float ndf, double ndd, cand* list, int* cnt, int k) {
    float nd2f = ndf * ndf;
    double nd2d = ndd * ndd;
    for (int j = 0; j < n; ++j) consider(pf, pd, fp64, i, j, nd2f, nd2d, list, cnt, k);
}

/* Exported neighbour search (mode 0 brute force, 1 grid).  nbr: n*k, -1 padded;
 * nbr_d2: the FP32 d^2 of each kept neighbour (0 for padding).  Returns candidates
 * scanned. */
long long oracle_knn(const float* pos, int n, float neighbor_dist, int k, int mode,
                     const float* grid_f, const int* grid_i, int32_t* nbr, float* nbr_d2) {
    if (k < 1 || k > OR_MAXK) return -1;
    bins b;
    long long scanned = 0;
    if (mode == 1 && bins_build(&b, pos, n, grid_f, grid_i) != 0) return -1;
    for (int i = 0; i < n; ++i) {
        cand list[OR_MAXK];
        int cnt = 0;
        if (mode == 1) scanned += knn_grid_one(&b, pos, NULL, 0, i, neighbor_dist, 0, list, &cnt, k);
        else { knn_brute_one(pos, NULL, 0, n, i, neighbor_dist, 0, list, &cnt, k); scanned += n - 1; }
        for (int q = 0; q < k; ++q) {
            nbr[(size_t)i * k + q] = q < cnt ? list[q].j : -1;
            if (nbr_d2) nbr_d2[(size_t)i * k + q] = q < cnt ? list[q].d2f : 0.0f;
        }
    }
    if (mode == 1) bins_free(&b);
    return scanned;
}

/* ----------------------------------------------------------------------------------
 * ORCA half-plane of agent a induced by neighbour b (Fig. 1).
 *   p = p_b - p_a, v = v_a - v_b, R = r_a + r_b.
 *   |p|^2 > R^2 (apart): w = v - p/tau.
 *     cutoff circle when w.p < 0 and (w.p)^2 > R^2 |w|^2: n = w/|w|,
 *       u = (R/tau - |w|) n, d = (n_y, -n_x);
 *     otherwise a leg, l = sqrt(|p|^2 - R^2): left leg if det(p, w) > 0,
 *       d = (p_x l - p_y R, p_x R + p_y l)/|p|^2; right leg otherwise,
 *       d = -(p_x l + p_y R, -p_x R + p_y l)/|p|^2; u = (v.d) d - v.
 *   |p|^2 <= R^2 (overlap): the same cutoff construction with dt in place of tau.
 *   P = v_a + u/2.  Branch codes: 0 cutoff, 1 left leg, 2 right leg, 3 overlap.
 * -------------------------------------------------------------------------------- */
static line2 orca_line(v2 pa, v2 va, double ra, v2 pb, v2 vb, double rb, double tau,
                       double dt, int ia, int ib, tags* tg, int* branch, v2* u_out) {
    v2 p = sub(pb, pa), v = sub(va, vb);
    double R = ra + rb, p2 = dot(p, p), R2 = R * R;
    line2 L;
    v2 u;
    int br;
    note(tg, p2, R2, R2);
    if (p2 > R2) {
        v2 w = sub(v, scl(p, 1.0 / tau));
        double w2 = dot(w, w), wp = dot(w, p);
        if (wp < 0.0 && wp * wp > R2 * w2) {
            double wl = sqrt(w2);
            v2 nrm = scl(w, 1.0 / wl);
            L.d = mk(nrm.y, -nrm.x);
            u = scl(nrm, R / tau - wl);
            br = 0;
        } else {
            double leg = sqrt(p2 - R2);
            double side = det2(p, w);
            note(tg, side, 0.0, sqrt(p2 * w2));
            if (side > 0.0) {
                L.d = scl(mk(p.x * leg - p.y * R, p.x * R + p.y * leg), 1.0 / p2);
                br = 1;
            } else {
                L.d = scl(mk(p.x * leg + p.y * R, -p.x * R + p.y * leg), -1.0 / p2);
                br = 2;
            }
            u = sub(scl(L.d, dot(v, L.d)), v);
        }
    } else {
        v2 w = sub(v, scl(p, 1.0 / dt));
        double wl = len(w);
        v2 nrm;
        if (wl > 0.0) nrm = scl(w, 1.0 / wl);
        else if (p2 > 0.0) nrm = scl(p, -1.0 / sqrt(p2));
        else nrm = mk(ia < ib ? 1.0 : -1.0, 0.0);
        L.d = mk(nrm.y, -nrm.x);
        u = scl(nrm, R / dt - wl);
        br = 3;
    }
    L.P = add(va, scl(u, 0.5));
    if (branch) *branch = br;
    if (u_out) *u_out = u;
    return L;
}

/* ----------------------------------------------------------------------------------
 * LP1: best point on line i inside the disc |x| <= V and the half-planes 0..i-1.
 * Parametrise x(t) = P_i + t d_i.  The disc gives t in [-a - sqrt(D), -a + sqrt(D)],
 * a = P_i.d_i, D = a^2 + V^2 - |P_i|^2.  Half-plane j bounds t by num/den with
 * den = det(d_i, d_j), num = det(d_j, P_i - P_j): an upper bound when den > 0, a lower
 * one when den < 0; a (nearly) parallel j (|den| <= eps) is infeasible iff num < 0.
 * Objective: direction mode (maximise o.x) picks the end of the interval along o;
 * otherwise the projection of o onto the line, clamped to the interval.
 * Returns 1 and writes *x on success, 0 when the interval is empty.
 * -------------------------------------------------------------------------------- */
/* Operation counts of the LP (for the flop model of a step; no effect on results).
 * problem_lines: over LP3's projected problems, the lines each involves -- a problem for
 * line i (0-based) takes that line and the i lines before it, i + 1 in all. */
typedef struct {
    long long lp1, bounds, checks, bisectors, problem_lines;
} lpcount;

static int lp1(const line2* L, int i, double V, v2 o, int dir_opt, v2* x, tags* tg,
               lpcount* work) {
    (void)tg;
    double a = dot(L[i].P, L[i].d);
    double D = a * a + V * V - dot(L[i].P, L[i].P);
    if (D < 0.0) return 0;
    double sq = sqrt(D);
    double tL = -a - sq, tR = -a + sq;
    for (int j = 0; j < i; ++j) {
        double den = det2(L[i].d, L[j].d);
        double num = det2(L[j].d, sub(L[i].P, L[j].P));
        if (work) ++work->bounds;
        if (fabs(den) <= OR_EPS) {
            if (num < 0.0) return 0;
            continue;
        }
        double t = num / den;
        if (den >= 0.0) { if (t < tR) tR = t; }
        else { if (t > tL) tL = t; }
        if (tL > tR) return 0;
    }
    if (dir_opt) {
        double od = dot(o, L[i].d);
        *x = add(L[i].P, scl(L[i].d, od > 0.0 ? tR : tL));
    } else {
        double t = dot(L[i].d, sub(o, L[i].P));
        if (t < tL) t = tL;
        if (t > tR) t = tR;
        *x = add(L[i].P, scl(L[i].d, t));
    }
    return 1;
}

/* LP2: incremental 2-D LP over lines 0..n-1 in order.  Start point: V*o in direction
 * mode (o a unit vector), else o pulled onto the disc if outside it.  A line whose valid
 * side does not contain x (det(d_i, P_i - x) > 0) moves x onto it by LP1.  Returns n on
 * success, else the index of the line where LP1 found no point (x keeps its last
 * feasible value). */
static int lp2(const line2* L, int n, double V, v2 o, int dir_opt, v2* x, tags* tg,
               lpcount* work) {
    (void)tg;
    if (dir_opt) *x = scl(o, V);
    else if (dot(o, o) > V * V) *x = scl(o, V / len(o));
    else *x = o;
    for (int i = 0; i < n; ++i) {
        double viol = det2(L[i].d, sub(L[i].P, *x));
        if (work) ++work->checks;
        if (viol > 0.0) {
            v2 keep = *x;
            if (work) ++work->lp1;
            if (!lp1(L, i, V, o, dir_opt, x, tg, work)) { *x = keep; return i; }
        }
    }
    return n;
}

/* LP3: least-penetration fallback (Section 3).  Minimises, over the disc, the largest
 * violation max_i det(d_i, P_i - x), starting from line `begin` with penetration 0.
 * The first nobst lines (static obstacles) are hard constraints: they are copied into
 * every projected problem unchanged, and only the other lines get bisectors.
 * When line i is violated by more than the current penetration, the optimum lies on
 * the set where line i's violation equals the others'; each earlier line j gives the
 * bisecting half-plane (through the intersection of lines i and j, direction
 * normalise(d_j - d_i); parallel lines of opposite direction give the midline, parallel
 * lines of the same direction give no constraint), and LP2 in direction mode maximises
 * progress along the normal (-d_i.y, d_i.x).  A numerically failed LP2 keeps x. */
static void lp3(const line2* L, int n, int nobst, int begin, double V, v2* x, tags* tg,
                lpcount* work) {
    (void)tg;
    line2 proj[OR_MAXK];
    double dist = 0.0;
    for (int i = begin; i < n; ++i) {
        double pen = det2(L[i].d, sub(L[i].P, *x));
        if (work) ++work->checks;
        if (pen > dist) {
            /* the first nobst lines (static obstacles) stay hard constraints: they enter
               the projected problem unchanged; bisectors come from the others */
            int m = 0;
            for (int j = 0; j < nobst && j < OR_MAXK; ++j) proj[m++] = L[j];
            for (int j = nobst; j < i; ++j) {
                line2 q;
                double den = det2(L[i].d, L[j].d);
                if (fabs(den) <= OR_EPS) {
                    if (dot(L[i].d, L[j].d) > 0.0) continue;
                    q.P = scl(add(L[i].P, L[j].P), 0.5);
                } else {
                    q.P = add(L[i].P, scl(L[i].d, det2(L[j].d, sub(L[i].P, L[j].P)) / den));
                }
                v2 dd = sub(L[j].d, L[i].d);
                q.d = scl(dd, 1.0 / len(dd));
                proj[m++] = q;
            }
            v2 keep = *x;
            if (work) work->bisectors += i > nobst ? i - nobst : 0;
            if (work) work->problem_lines += i + 1;
            if (lp2(proj, m, V, mk(-L[i].d.y, L[i].d.x), 1, x, tg, work) < m) *x = keep;
            dist = det2(L[i].d, sub(L[i].P, *x));
        }
    }
}

/* ----------------------------------------------------------------------------------
 * Exported building blocks (for pins).  lines: n*4 doubles {Px, Py, dx, dy}.
 * -------------------------------------------------------------------------------- */
int oracle_orca_line(const double* a /* px,py,vx,vy,r */, const double* b, double tau,
                     double dt, int ia, int ib, double* line4, double* u2, double* margin) {
    tags tg = {1e300};
    int br;
    v2 u;
    line2 L = orca_line(mk(a[0], a[1]), mk(a[2], a[3]), a[4], mk(b[0], b[1]), mk(b[2], b[3]),
                        b[4], tau, dt, ia, ib, &tg, &br, &u);
    line4[0] = L.P.x; line4[1] = L.P.y; line4[2] = L.d.x; line4[3] = L.d.y;
    if (u2) { u2[0] = u.x; u2[1] = u.y; }
    if (margin) *margin = tg.m;
    return br;
}

static void unpack(const double* lines, int n, line2* L) {
    for (int i = 0; i < n; ++i) {
        L[i].P = mk(lines[4 * i], lines[4 * i + 1]);
        L[i].d = mk(lines[4 * i + 2], lines[4 * i + 3]);
    }
}

int oracle_lp2(const double* lines, int n, double V, const double* o, int dir_opt,
               double* x2) {
    line2 L[OR_MAXK];
    if (n < 0 || n > OR_MAXK) return -1;
    unpack(lines, n, L);
    v2 x;
    int r = lp2(L, n, V, mk(o[0], o[1]), dir_opt, &x, NULL, NULL);
    x2[0] = x.x; x2[1] = x.y;
    return r;
}

int oracle_solve_fixed(const double* lines, int n, int nobst, double V, const double* o,
                       double* x2);

/* Obstacle half-plane of an agent at p (px, py) with radius r against a segment
 * (x1, y1, x2, y2): line4 = {Px, Py, dx, dy}; returns 1 if the agent overlaps it. */
int oracle_obstacle_line(const double* p, double r, const double* seg, double tau_o, double dt,
                         double* line4);

/* Full velocity selection: LP2, then LP3 from the failing line.  Returns 1 if LP3 ran. */
int oracle_solve(const double* lines, int n, double V, const double* o, double* x2) {
    return oracle_solve_fixed(lines, n, 0, V, o, x2);
}

/* As oracle_solve, also returning the LP's operation counts: counts[5] = {LP1 calls, LP1
 * bounds, violation checks, LP3 bisectors formed, LP3 problem lines} (see lpcount). */
int oracle_solve_counted(const double* lines, int n, double V, const double* o, double* x2,
                         long long* counts) {
    line2 L[OR_MAXK];
    if (n < 0 || n > OR_MAXK) return -1;
    unpack(lines, n, L);
    lpcount w = {0, 0, 0, 0, 0};
    v2 x;
    int b = lp2(L, n, V, mk(o[0], o[1]), 0, &x, NULL, &w);
    if (b < n) lp3(L, n, 0, b, V, &x, NULL, &w);
    x2[0] = x.x; x2[1] = x.y;
    counts[0] = w.lp1; counts[1] = w.bounds; counts[2] = w.checks; counts[3] = w.bisectors;
    counts[4] = w.problem_lines;
    return b < n;
}

/* As oracle_solve, with the first nobst lines hard (static obstacles) in LP3. */
int oracle_solve_fixed(const double* lines, int n, int nobst, double V, const double* o,
                       double* x2) {
    line2 L[OR_MAXK];
    if (n < 0 || n > OR_MAXK || nobst < 0 || nobst > n) return -1;
    unpack(lines, n, L);
    v2 x;
    int b = lp2(L, n, V, mk(o[0], o[1]), 0, &x, NULL, NULL);
    if (b < n) lp3(L, n, nobst, b, V, &x, NULL, NULL);
    x2[0] = x.x; x2[1] = x.y;
    return b < n;
}

/* Preferred velocity: towards the goal at pref_speed; within one step of the goal,
 * the velocity that reaches it in one step. */
static v2 pref_velocity(v2 p, v2 goal, double pref_speed, double dt) {
    v2 g = sub(goal, p);
    double dist = len(g);
    if (dist > pref_speed * dt) return scl(g, pref_speed / dist);
    return scl(g, 1.0 / dt);
}

/* ----------------------------------------------------------------------------------
 * Static obstacles (line segments; not in the paper's experiments -- the ORCA rule for
 * obstacles of van den Berg et al., which the paper defers to).  The optimisation
 * velocity for an obstacle is 0 and the agent takes full responsibility, so the half-plane
 * follows from the point of the truncated velocity obstacle nearest the origin.  With q
 * the point of the segment nearest the agent (relative to it) and d = |q|, that point is
 * (d - r) q / (d tau_o), and the permitted velocities are v.q/d <= (d - r)/tau_o: along
 * the direction to the segment the agent may close at most d - r within tau_o.  (The
 * segment lies beyond the supporting line through its nearest point, so such a velocity
 * keeps the agent at least r from it for tau_o.)  An agent already closer than r uses dt
 * in place of tau_o (it must open the gap within one step), like overlapping agents; an
 * agent exactly on the segment takes the segment's left normal.  In normal form:
 * n = -q/d, c = -(d - r)/tau_o (or -(d - r)/dt).
 *
 * Which segments: those whose FP32 squared distance (nearest point by the clamped
 * projection, one rounding per operation) is strictly below fl(fl(V tau_o) + r)^2, the
 * segments the agent could reach within tau_o; the kobst nearest by (d^2, segment index).
 * -------------------------------------------------------------------------------- */
static float seg_dist2_f32(const float* sg, float px, float py) {
    float ex = sg[2] - sg[0], ey = sg[3] - sg[1];
    float wx = px - sg[0], wy = py - sg[1];
    float exx = ex * ex, eyy = ey * ey;
    float l2 = exx + eyy;
    float t = 0.0f;
    if (l2 > 0.0f) {
        float wex = wx * ex, wey = wy * ey;
        float pr = wex + wey;
        t = pr / l2;
        t = t < 0.0f ? 0.0f : (t > 1.0f ? 1.0f : t);
    }
    float tex = t * ex, tey = t * ey;
    float cx = sg[0] + tex, cy = sg[1] + tey;
    float qx = cx - px, qy = cy - py;
    float qxx = qx * qx, qyy = qy * qy;
    return qxx + qyy;
}

static line2 obstacle_line(v2 pa, double ra, const double* sg, double tau_o, double dt,
                           tags* tg) {
    v2 a = mk(sg[0], sg[1]), e = mk(sg[2] - sg[0], sg[3] - sg[1]);
    double l2 = dot(e, e), t = 0.0;
    if (l2 > 0.0) {
        t = dot(sub(pa, a), e) / l2;
        t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
    }
    v2 q = sub(add(a, scl(e, t)), pa);
    double d = len(q);
    v2 n;
    double c;
    note(tg, d, ra, ra);  /* overlap or not */
    if (d > 0.0) n = scl(q, -1.0 / d);
    else n = l2 > 0.0 ? scl(mk(-e.y, e.x), 1.0 / sqrt(l2)) : mk(1.0, 0.0);
    c = d > ra ? -(d - ra) / tau_o : -(d - ra) / dt;
    line2 L;
    L.d = mk(n.y, -n.x);
    L.P = scl(n, c);
    return L;
}

int oracle_obstacle_line(const double* p, double r, const double* seg, double tau_o, double dt,
                         double* line4) {
    line2 L = obstacle_line(mk(p[0], p[1]), r, seg, tau_o, dt, NULL);
    line4[0] = L.P.x; line4[1] = L.P.y; line4[2] = L.d.x; line4[3] = L.d.y;
    v2 a = mk(seg[0], seg[1]), e = mk(seg[2] - seg[0], seg[3] - seg[1]);
    double l2 = dot(e, e), t = 0.0;
    if (l2 > 0.0) {
        t = dot(sub(mk(p[0], p[1]), a), e) / l2;
        t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
    }
    return len(sub(add(a, scl(e, t)), mk(p[0], p[1]))) <= r;
}

/* ----------------------------------------------------------------------------------
 * One synchronous step for n agents.
 * Inputs (length n or 2n, FP64; promote FP32 state for parity runs):
 *   pos, vel, goal (x,y interleaved), radius, max_speed, pref_speed, time_horizon.
 * Scene parameters: neighbor_dist (r_obs), k = max_neighbors, dt.
 * knn_mode: 0 brute force, 1 grid (grid_f/grid_i from oracle_grid; NULL -> cell = r_obs).
 * fp64_knn: 0 -> neighbour search in FP32 on (float)pos; 1 -> in FP64.
 * subset/n_subset: if subset is non-NULL, only agents subset[0..n_subset-1] are stepped
 *   (their neighbours are still searched among all n agents) and output row q belongs to
 *   agent subset[q]; otherwise every agent is stepped and row i is agent i.
 * Outputs: pos_out, vel_out (2 per row), nbr (k per row, -1 padded, may be NULL), status
 * (1 per row: 1 if LP3 ran, may be NULL), margin (1 per row, may be NULL), counters[8] =
 * {candidates scanned, lines built, LP1 calls (incl. inside LP3), agents needing LP3,
 * LP1 bounds evaluated, LP2/LP3 violation checks, LP3 bisectors formed, LP3 problem lines}
 * (may be NULL), sens (1 per row, may be NULL; filled when cond_check != 0, see the
 * header).  Returns 0, or a negative value on bad arguments / allocation failure.
 * -------------------------------------------------------------------------------- */
/* Velocity selection (LP2, then LP3 if needed) on given lines. */
static v2 select_velocity(const line2* L, int n, int nobst, double V, v2 o) {
    v2 x;
    int b = lp2(L, n, V, o, 0, &x, NULL, NULL);
    if (b < n) lp3(L, n, nobst, b, V, &x, NULL, NULL);
    return x;
}

/* Largest move of the selected velocity when one half-plane at a time is shifted along
 * its normal by +-eta_c (4 FP32 ulps of max(|offset|, V)) or turned by +-2^-22 rad about
 * its point nearest the origin. */
static double lp_sensitivity(const line2* L, int n, int nobst, double V, v2 o, v2 x) {
    line2 Q[OR_MAXK];
    double worst = 0.0;
    const double eta_r = ldexp(1.0, -22);
    for (int q = 0; q < n; ++q) {
        v2 nq = mk(-L[q].d.y, L[q].d.x);
        double c = dot(nq, L[q].P);
        double mag = fabs(c) > V ? fabs(c) : V;
        int e2;
        frexp(mag, &e2);
        double eta_c = ldexp(1.0, e2 - 22); /* 4 ulps of a float in [2^(e2-1), 2^e2) */
        for (int k = 0; k < 4; ++k) {
            memcpy(Q, L, sizeof(line2) * (size_t)n);
            v2 nn = nq;
            double cc = c;
            if (k == 0) cc = c + eta_c;
            else if (k == 1) cc = c - eta_c;
            else {
                double a = k == 2 ? eta_r : -eta_r;
                nn = mk(nq.x * cos(a) - nq.y * sin(a), nq.x * sin(a) + nq.y * cos(a));
            }
            Q[q].d = mk(nn.y, -nn.x);
            Q[q].P = scl(nn, cc);
            v2 y = select_velocity(Q, n, nobst, V, o);
            double dv = fabs(y.x - x.x) > fabs(y.y - x.y) ? fabs(y.x - x.x) : fabs(y.y - x.y);
            if (dv > worst) worst = dv;
        }
    }
    return worst;
}

/* Sensitivity of the full velocity selection (LP2, then LP3 with the first nobst lines
 * hard) to FP32-sized perturbations of the lines, one at a time (lp_sensitivity); x2
 * receives the unperturbed selection.  Returns a negative value on bad arguments. */
double oracle_lp_sensitivity(const double* lines, int n, int nobst, double V, const double* o,
                             double* x2) {
    line2 L[OR_MAXK];
    if (n < 0 || n > OR_MAXK || nobst < 0 || nobst > n) return -1.0;
    unpack(lines, n, L);
    v2 x = select_velocity(L, n, nobst, V, mk(o[0], o[1]));
    x2[0] = x.x; x2[1] = x.y;
    return lp_sensitivity(L, n, nobst, V, mk(o[0], o[1]), x);
}

typedef struct {
    int n, k, fp64, cond;
    const double *pos, *vel, *goal, *radius, *max_speed, *pref_speed, *tau;
    double nd, dt;
    float ndf;
    const float* pf;
    const bins* b;
    int nseg, kobst;          /* static obstacle segments; obstacle lines kept per agent */
    const double* seg;        /* 4 per segment: x1, y1, x2, y2 */
    const float* segf;        /* the same in FP32 (selection) */
    double tau_o;
} step_in;

static void step_agent(const step_in* S, int i, double* pos_out, double* vel_out, int32_t* nbr,
                       int32_t* obst, int32_t* status, double* margin, double* sens,
                       long long* c_scan, long long* c_lines, lpcount* c_work, long long* c_lp3) {
    cand list[OR_MAXK];
    line2 L[OR_MAXK];
    int cnt = 0, nob = 0;
    tags tg = {1e300};
    const double* pos = S->pos;
    const double* vel = S->vel;
    /* obstacle lines first: the kobst nearest reachable segments, by (d^2, index) */
    if (S->nseg > 0 && S->kobst > 0) {
        float px = S->pf[2 * i], py = S->pf[2 * i + 1];
        float vr = (float)S->max_speed[i] * (float)S->tau_o;
        float rng = vr + (float)S->radius[i];
        float rng2 = rng * rng;
        float od2[OR_MAXK];
        int oj[OR_MAXK];
        for (int j = 0; j < S->nseg; ++j) {
            float d2 = seg_dist2_f32(S->segf + 4 * j, px, py);
            if (!(d2 < rng2)) continue;
            int at = nob < S->kobst ? nob : S->kobst;
            while (at > 0 && (od2[at - 1] > d2 || (od2[at - 1] == d2 && oj[at - 1] > j))) {
                if (at < S->kobst) { od2[at] = od2[at - 1]; oj[at] = oj[at - 1]; }
                --at;
            }
            if (at < S->kobst) {
                od2[at] = d2;
                oj[at] = j;
                if (nob < S->kobst) ++nob;
            }
        }
        for (int q = 0; q < nob; ++q)
            L[q] = obstacle_line(mk(pos[2 * i], pos[2 * i + 1]), S->radius[i], S->seg + 4 * oj[q],
                                 S->tau_o, S->dt, &tg);
        if (obst) for (int q = 0; q < S->kobst; ++q) obst[q] = q < nob ? oj[q] : -1;
    }
    if (S->b) *c_scan += knn_grid_one(S->b, S->pf, pos, S->fp64, i, S->ndf, S->nd, list, &cnt, S->k);
    else { knn_brute_one(S->pf, pos, S->fp64, S->n, i, S->ndf, S->nd, list, &cnt, S->k); *c_scan += S->n - 1; }
    v2 pa = mk(pos[2 * i], pos[2 * i + 1]), va = mk(vel[2 * i], vel[2 * i + 1]);
    for (int q = 0; q < cnt; ++q) {
        int j = list[q].j;
        L[nob + q] = orca_line(pa, va, S->radius[i], mk(pos[2 * j], pos[2 * j + 1]),
                         mk(vel[2 * j], vel[2 * j + 1]), S->radius[j], S->tau[i], S->dt, i, j,
                         &tg, NULL, NULL);
    }
    *c_lines += cnt;
    v2 pv = pref_velocity(pa, mk(S->goal[2 * i], S->goal[2 * i + 1]), S->pref_speed[i], S->dt);
    v2 x;
    lpcount w = {0, 0, 0, 0, 0};
    int nl = nob + cnt;
    int bfail = lp2(L, nl, S->max_speed[i], pv, 0, &x, &tg, &w);
    int used3 = bfail < nl;
    if (used3) { lp3(L, nl, nob, bfail, S->max_speed[i], &x, &tg, &w); ++*c_lp3; }
    c_work->lp1 += w.lp1;
    c_work->bounds += w.bounds;
    c_work->checks += w.checks;
    c_work->bisectors += w.bisectors;
    c_work->problem_lines += w.problem_lines;
    if (sens) *sens = S->cond ? lp_sensitivity(L, nl, nob, S->max_speed[i], pv, x) : 0.0;
    vel_out[0] = x.x;
    vel_out[1] = x.y;
    pos_out[0] = pa.x + x.x * S->dt;
    pos_out[1] = pa.y + x.y * S->dt;
    if (nbr) for (int q = 0; q < S->k; ++q) nbr[q] = q < cnt ? list[q].j : -1;
    if (status) *status = used3;
    if (margin) *margin = tg.m;
}

static int step_all(int n, const double* pos, const double* vel, const double* goal,
                    const double* radius, const double* max_speed, const double* pref_speed,
                    const double* time_horizon, double neighbor_dist, int k, double dt,
                    int knn_mode, int fp64_knn, const float* grid_f_in, const int* grid_i_in,
                    const int32_t* subset, int n_subset, int nthreads, double* pos_out,
                    double* vel_out, int32_t* nbr, int32_t* status, double* margin,
                    long long* counters, int cond_check, double* sens, int nseg,
                    const double* seg, double tau_o, int kobst, int32_t* obst) {
    if (n < 0 || k < 1 || k > OR_MAXK || !(dt > 0.0)) return -1;
    if (nseg < 0 || kobst < 0 || k + kobst > OR_MAXK || (nseg > 0 && (!seg || !(tau_o > 0.0))))
        return -1;
    if (subset) {
        if (n_subset < 0) return -1;
        for (int q = 0; q < n_subset; ++q) if (subset[q] < 0 || subset[q] >= n) return -1;
    }
    if (counters) memset(counters, 0, 8 * sizeof(long long));
    int rows = subset ? n_subset : n;
    if (n == 0 || rows == 0) return 0;
    float* pf = (float*)malloc(sizeof(float) * 2 * (size_t)n);
    if (!pf) return -2;
    for (long long q = 0; q < 2LL * n; ++q) pf[q] = (float)pos[q];
    step_in S;
    S.n = n; S.k = k; S.fp64 = fp64_knn; S.cond = cond_check;
    S.pos = pos; S.vel = vel; S.goal = goal; S.radius = radius; S.max_speed = max_speed;
    S.pref_speed = pref_speed; S.tau = time_horizon;
    S.nd = neighbor_dist; S.dt = dt; S.ndf = (float)neighbor_dist; S.pf = pf; S.b = NULL;
    S.nseg = nseg; S.kobst = kobst; S.seg = seg; S.tau_o = tau_o; S.segf = NULL;
    float* segf = NULL;
    if (nseg > 0) {
        segf = (float*)malloc(sizeof(float) * 4 * (size_t)nseg);
        if (!segf) { free(pf); return -2; }
        for (long long q = 0; q < 4LL * nseg; ++q) segf[q] = (float)seg[q];
        S.segf = segf;
    }
    bins b;
    if (knn_mode == 1) {
        float gf[4];
        int gi[2];
        if (grid_f_in && grid_i_in) { memcpy(gf, grid_f_in, sizeof gf); memcpy(gi, grid_i_in, sizeof gi); }
        else if (oracle_grid(pf, n, S.ndf, (long long)4 * n + 1024, gf, gi) != 0) { free(pf); free(segf); return -3; }
        if (bins_build(&b, pf, n, gf, gi) != 0) { free(pf); free(segf); return -2; }
        S.b = &b;
    }
    long long c_scan = 0, c_lines = 0, c_lp3 = 0, c_lp1 = 0, c_bounds = 0, c_checks = 0, c_bis = 0,
              c_plines = 0;
#ifdef _OPENMP
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 256) num_threads(nthreads) \
    reduction(+ : c_scan, c_lines, c_lp3, c_lp1, c_bounds, c_checks, c_bis, c_plines)
#endif
    for (int q = 0; q < rows; ++q) {
        int i = subset ? subset[q] : q;
        lpcount w = {0, 0, 0, 0, 0};
        step_agent(&S, i, pos_out + 2 * (size_t)q, vel_out + 2 * (size_t)q,
                   nbr ? nbr + (size_t)q * k : NULL,
                   obst ? obst + (size_t)q * (kobst > 0 ? kobst : 1) : NULL, status ? status + q : NULL,
                   margin ? margin + q : NULL, sens ? sens + q : NULL, &c_scan, &c_lines,
                   &w, &c_lp3);
        c_lp1 += w.lp1;
        c_bounds += w.bounds;
        c_checks += w.checks;
        c_bis += w.bisectors;
        c_plines += w.problem_lines;
    }
    if (S.b) bins_free(&b);
    free(pf);
    free(segf);
    if (counters) {
        counters[0] = c_scan; counters[1] = c_lines; counters[2] = c_lp1; counters[3] = c_lp3;
        counters[4] = c_bounds; counters[5] = c_checks; counters[6] = c_bis;
        counters[7] = c_plines;
    }
    return 0;
}

int oracle_step(int n, const double* pos, const double* vel, const double* goal,
                const double* radius, const double* max_speed, const double* pref_speed,
                const double* time_horizon, double neighbor_dist, int k, double dt,
                int knn_mode, int fp64_knn, const float* grid_f_in, const int* grid_i_in,
                const int32_t* subset, int n_subset, int nthreads, double* pos_out,
                double* vel_out, int32_t* nbr, int32_t* status, double* margin,
                long long* counters, int cond_check, double* sens) {
    return step_all(n, pos, vel, goal, radius, max_speed, pref_speed, time_horizon,
                    neighbor_dist, k, dt, knn_mode, fp64_knn, grid_f_in, grid_i_in, subset,
                    n_subset, nthreads, pos_out, vel_out, nbr, status, margin, counters,
                    cond_check, sens, 0, NULL, 1.0, 0, NULL);
}

/* As oracle_step, with nseg static obstacle segments (seg: 4 doubles each, x1 y1 x2 y2),
 * obstacle time horizon tau_o and at most kobst obstacle lines per agent (k + kobst <=
 * 64); obst (kobst per row, -1 padded, may be NULL) receives the segments used. */
int oracle_step_obstacles(int n, const double* pos, const double* vel, const double* goal,
                          const double* radius, const double* max_speed, const double* pref_speed,
                          const double* time_horizon, double neighbor_dist, int k, double dt,
                          int knn_mode, int fp64_knn, const float* grid_f_in, const int* grid_i_in,
                          const int32_t* subset, int n_subset, int nthreads, double* pos_out,
                          double* vel_out, int32_t* nbr, int32_t* status, double* margin,
                          long long* counters, int cond_check, double* sens, int nseg,
                          const double* seg, double tau_o, int kobst, int32_t* obst) {
    return step_all(n, pos, vel, goal, radius, max_speed, pref_speed, time_horizon,
                    neighbor_dist, k, dt, knn_mode, fp64_knn, grid_f_in, grid_i_in, subset,
                    n_subset, nthreads, pos_out, vel_out, nbr, status, margin, counters,
                    cond_check, sens, nseg, seg, tau_o, kobst, obst);
}

/* Number of OpenMP threads the oracle would use by default (1 without OpenMP). */
/* ----------------------------------------------------------------------------------
 * Arrival (Section 4: a person who reaches the goal location is removed from the
 * simulation).  Reading: agent i has arrived when its goal lies within its own radius,
 * |goal - p| <= r, decided in FP32 with one rounding per operation:
 * dx = fl(gx - px), dy = fl(gy - py), arrived iff fl(fl(dx dx) + fl(dy dy)) <= fl(r r).
 * pos, goal: 2n floats (x, y interleaved); radius: n floats; arrived: n int32 (1 or 0).
 * Returns the number of agents that have arrived.
 * -------------------------------------------------------------------------------- */
int oracle_arrived(int n, const float* pos, const float* goal, const float* radius,
                   int32_t* arrived) {
    int count = 0;
    for (int i = 0; i < n; ++i) {
        float dx = goal[2 * i] - pos[2 * i];
        float dy = goal[2 * i + 1] - pos[2 * i + 1];
        float dx2 = dx * dx;
        float dy2 = dy * dy;
        float d2 = dx2 + dy2;
        float r2 = radius[i] * radius[i];
        arrived[i] = d2 <= r2;
        count += arrived[i];
    }
    return count;
}

/* ----------------------------------------------------------------------------------
 * Spawning without overlap (Section 4, test set-up: spawn locations are chosen so that a
 * new person overlaps nobody within a time period based on person size and speed).
 * Reading: a candidate c (position p_c, radius r_c, maximum speed V_c) enters at rest.
 * It conflicts with a present agent j (position p_j, velocity v_j, radius r_j) when the
 * two could touch within the window T moving straight at each other:
 *     |p_c - p_j| <= r_c + r_j + (V_c + |v_j|) T,
 * and with a candidate c' accepted before it (candidates are taken in index order) when
 *     |p_c - p_c'| <= r_c + r_c' + (V_c + V_c') T.
 * A candidate is accepted when it has no conflict.  Decided in FP32, one rounding per
 * operation: dx = fl(x_c - x_j), d2 = fl(fl(dx dx) + fl(dy dy)), s_j = fl(sqrt(fl(fl(vx vx)
 * + fl(vy vy)))), reach = fl(fl(r_c + r_j) + fl(fl(V_c + s_j) T)), conflict iff
 * d2 <= fl(reach reach).
 * pos, vel: 2n floats; radius: n; cand_pos: 2m; cand_radius, cand_vmax: m; accepted: m
 * int32 (1 or 0).  Returns the number accepted.  O(n m + m^2): plain loops.
 * -------------------------------------------------------------------------------- */
static int spawn_conflict(float xc, float yc, float rc, float vc, float xj, float yj, float rj,
                          float sj, float window) {
    float ex = xc - xj;
    float ey = yc - yj;
    float ex2 = ex * ex;
    float ey2 = ey * ey;
    float d2 = ex2 + ey2;
    float rr = rc + rj;
    float ss = vc + sj;
    float travel = ss * window;
    float reach = rr + travel;
    float reach2 = reach * reach;
    return d2 <= reach2;
}

int oracle_spawn(int n, const float* pos, const float* vel, const float* radius, int m,
                 const float* cand_pos, const float* cand_radius, const float* cand_vmax,
                 float window, int32_t* accepted) {
    int count = 0;
    for (int c = 0; c < m; ++c) {
        const float xc = cand_pos[2 * c], yc = cand_pos[2 * c + 1];
        int ok = 1;
        for (int j = 0; j < n && ok; ++j) {
            float vx2 = vel[2 * j] * vel[2 * j];
            float vy2 = vel[2 * j + 1] * vel[2 * j + 1];
            float v2 = vx2 + vy2;
            float sj = sqrtf(v2);
            if (spawn_conflict(xc, yc, cand_radius[c], cand_vmax[c], pos[2 * j], pos[2 * j + 1],
                               radius[j], sj, window))
                ok = 0;
        }
        for (int e = 0; e < c && ok; ++e)
            if (accepted[e] && spawn_conflict(xc, yc, cand_radius[c], cand_vmax[c], cand_pos[2 * e],
                                              cand_pos[2 * e + 1], cand_radius[e], cand_vmax[e], window))
                ok = 0;
        accepted[c] = ok;
        count += ok;
    }
    return count;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
