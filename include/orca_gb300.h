/*
 * orca_gb300.h -- C ABI of the GB300 (sm_103a) ORCA crowd-simulation step.
 *
 * One call to orca_step advances every agent by one synchronous ORCA step
 * ("Fast Simulation of Crowd Collision Avoidance", Section 3; all agents update
 * simultaneously, Section 2):
 *   1. preferred velocity towards the goal at the preferred speed (Section 3, first
 *      paragraph after Fig. 1; Section 4 test set-up);
 *   2. agents binned into a uniform grid of square cells (Fig. 2), sorted by cell;
 *   3. each agent's neighbours: the max_neighbors nearest agents whose squared distance is
 *      strictly below neighbor_dist^2 (the observation radius r_obs of Fig. 2), nearest
 *      first, equal distances broken by lower agent index;
 *   4. one ORCA half-plane per neighbour from the relative position, relative velocity,
 *      radius sum and time horizon (Fig. 1 a-c);
 *   5. the velocity closest to the preferred velocity inside the maximum-speed disc and
 *      all half-planes, or, when they have no common point, the velocity that least
 *      penetrates them (Section 3, LP paragraphs);
 *   6. velocity and position update, pos += vel * dt.
 *
 * Conventions
 *   - Every function returns an int status: ORCA_OK (0) or a negative ORCA_ERR_* code.
 *     orca_last_error() gives a message for the last failure on a context.  No C++
 *     exception crosses this ABI; the library never exits, aborts or traps the GPU.
 *   - Arrays are FP32 structure-of-arrays indexed by agent (the order of
 *     orca_set_agents).  "xy" arrays hold interleaved (x, y) pairs, 2*n floats.
 *   - `where` says whether a pointer is host memory (ORCA_HOST) or device memory on the
 *     context's GPU (ORCA_DEVICE).  Host pointers need not be pinned; with pinned memory
 *     copies overlap better.  The caller keeps ownership of every pointer it passes.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is enqueued
 *     asynchronously on it; calls that return data to the host synchronise it.  All calls
 *     on one context must be ordered on the same stream (or ordered by the caller).
 *   - Errors detected on the device (non-finite velocities, exhausted bounded waits) are
 *     latched in a device word and reported by the next synchronising call
 *     (orca_get_state / orca_sync).
 *   - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef ORCA_GB300_H
#define ORCA_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define ORCA_API __attribute__((visibility("default")))
#else
#define ORCA_API
#endif

/* status codes */
#define ORCA_OK 0
#define ORCA_ERR_ARG (-1)      /* invalid argument */
#define ORCA_ERR_NOMEM (-2)    /* workspace allocation failed or too small */
#define ORCA_ERR_CUDA (-3)     /* a CUDA runtime call failed (message has the CUDA error) */
#define ORCA_ERR_STATE (-4)    /* call not valid in the context's state (e.g. no agents) */
#define ORCA_ERR_NUMERIC (-5)  /* a non-finite velocity or position was produced */
#define ORCA_ERR_TIMEOUT (-6)  /* a bounded device-side wait gave up */
#define ORCA_ERR_CAPACITY (-7) /* more agents / scenes / cells than the context was sized for */
#define ORCA_ERR_BOUNDS (-8)   /* a device-side index check failed (library built with ORCA_CHECKS) */

/* pointer location */
#define ORCA_HOST 0
#define ORCA_DEVICE 1

/* orca_params.flags */
#define ORCA_FLAG_RECORD 1u   /* keep each step's neighbour lists and cells for readout */
#define ORCA_FLAG_NO_GRAPH 2u /* launch kernels directly instead of replaying a CUDA graph */

typedef struct orca_ctx orca_ctx;

/*
 * Scene-wide parameters, fixed for the life of a context.
 *   max_agents     capacity in agents (>= 1).
 *   max_neighbors  k, the neighbours kept per agent (1..32).
 *   max_cells      capacity of the cell table (0 -> max(4*max_agents, 65536)).  If the
 *                  crowd's bounding box would need more cells, the cell edge doubles until
 *                  it fits (the neighbour sets do not depend on the cell edge).
 *   neighbor_dist  observation radius r_obs in metres (> 0).
 *   dt             time step in seconds (> 0).
 *   cell_size      grid cell edge in metres (0 -> neighbor_dist / 4).
 *   flags          ORCA_FLAG_*.
 *   max_scenes     scenes a batch may hold (orca_set_scenes); 0 or 1 for single scenes.
 */
typedef struct orca_params {
    int32_t max_agents;
    int32_t max_neighbors;
    int32_t max_cells;
    float neighbor_dist;
    float dt;
    float cell_size;
    uint32_t flags;
    int32_t max_scenes;  /* capacity in scenes for orca_set_scenes (0 or 1: single scene) */
} orca_params;

/*
 * One scene of a batch (orca_set_scenes): `count` consecutive agents that interact only
 * with each other, with their own ORCA parameters.
 *   count          agents in the scene (>= 0).
 *   max_neighbors  k for this scene (1 .. the context's max_neighbors).
 *   neighbor_dist  r_obs (> 0).  dt: time step (> 0).  cell_size: grid edge (0 -> r_obs/4).
 */
typedef struct orca_scene {
    int32_t count;
    int32_t max_neighbors;
    float neighbor_dist;
    float dt;
    float cell_size;
    int32_t reserved;
} orca_scene;

/* Bytes of device workspace orca_create needs for these parameters (256-byte aligned). */
ORCA_API int orca_workspace_size(const orca_params* params, size_t* bytes);

/*
 * Create a context on the current CUDA device.
 *   workspace       device buffer of at least orca_workspace_size() bytes, 256-byte
 *                   aligned, owned by the caller and kept alive until orca_destroy; or
 *                   NULL, in which case the library allocates (cudaMalloc) and frees it.
 *   workspace_bytes size of `workspace` (ignored when it is NULL).
 *   out             receives the context.  On failure *out is NULL.
 */
ORCA_API int orca_create(const orca_params* params, void* workspace, size_t workspace_bytes,
                         orca_ctx** out);

/* Destroy a context (waits for its work; frees what the library allocated). */
ORCA_API int orca_destroy(orca_ctx* ctx);

/*
 * Load n agents (0 <= n <= max_agents), replacing the current crowd.
 *   pos_xy, vel_xy, goal_xy  2*n floats each (metres, metres/second, metres).
 *   radius                   n floats, agent radius (m, > 0).
 *   max_speed                n floats, radius of the velocity disc (m/s, >= 0).
 *   pref_speed               n floats, preferred walking speed (m/s, >= 0).
 *   time_horizon             n floats, tau of Fig. 1 (s, > 0).
 * Agent i of later readouts is agent i of these arrays.  Values are copied on `stream`;
 * host arrays may be reused when the call returns.
 */
ORCA_API int orca_set_agents(orca_ctx* ctx, int32_t n, const float* pos_xy,
                             const float* vel_xy, const float* goal_xy, const float* radius,
                             const float* max_speed, const float* pref_speed,
                             const float* time_horizon, int where, void* stream);

/*
 * Replace the positions and/or velocities of the current agents and keep everything else:
 * their parameters, their order in memory and each agent's search-radius prediction (its
 * last k-th neighbour distance).  For a host-driven loop that writes back a state it read
 * (or edited), so the next step keeps its full speed; orca_set_agents would reset the
 * predictions.  The neighbour search is exact whatever the predictions, so any new state is
 * valid; one far from the old state only makes the next search slower.
 *   pos_xy, vel_xy  2*n floats each in agent order (n = the current count), host or device
 *                   per `where`; either may be NULL to keep that half.
 * Pinned (page-locked) host arrays are read by a kernel directly over the CPU-GPU link;
 * other host arrays go through the context's staging buffers.  For host input the call
 * synchronises `stream` before returning.  A context without agents ignores the call.
 */
ORCA_API int orca_update_state(orca_ctx* ctx, const float* pos_xy, const float* vel_xy, int where,
                               void* stream);

/*
 * One round of a host-driven loop in a single call: write positions and/or velocities from
 * host arrays (as orca_update_state; either may be NULL to keep that half), advance nsteps
 * steps (as orca_step), and read the new state into host arrays (as orca_get_state; either
 * may be NULL).  Input and output arrays may be the same.  Everything is enqueued on
 * `stream` and the call synchronises once, at the end, reporting device-side errors as
 * orca_get_state does; host arrays may be reused when it returns.  Pinned arrays are read
 * and written by kernels over the CPU-GPU link, others through staging copies.
 *   pos_in, vel_in, pos_out, vel_out  2*n floats each, agent order, host memory.
 */
ORCA_API int orca_step_host(orca_ctx* ctx, const float* pos_in, const float* vel_in, int32_t nsteps,
                            float* pos_out, float* vel_out, void* stream);

/*
 * Load a batch of n_scenes independent scenes (1 <= n_scenes <= max_scenes) that advance
 * together: scene s owns the next scenes[s].count agents of the arrays (laid out as for
 * orca_set_agents, scene after scene), and its agents see only each other.  Each scene has
 * its own grid over its own bounding box; the cell table is shared, each scene's share
 * of max_cells being proportional to its agents (at least one cell; a scene that would
 * need more doubles its cell edge).  `scenes` is a host array.  orca_step then advances
 * every scene with one persistent launch of the per-agent kernel per step, inside the
 * captured graph.  orca_set_agents returns the context to a single scene.
 */
ORCA_API int orca_set_scenes(orca_ctx* ctx, int32_t n_scenes, const orca_scene* scenes,
                             const float* pos_xy, const float* vel_xy, const float* goal_xy,
                             const float* radius, const float* max_speed,
                             const float* pref_speed, const float* time_horizon, int where,
                             void* stream);

/*
 * Grids of the last step (needs a batch): for scene s, grid_f[4s..4s+3] = xmin, ymin, cell
 * edge, 1/edge and grid_i[3s..3s+2] = gx, gy, first global cell id.  Host pointers;
 * synchronises `stream`.  orca_get_cells reports global cell ids (first id + cy*gx + cx).
 */
ORCA_API int orca_get_scene_grids(orca_ctx* ctx, float* grid_f, int32_t* grid_i, void* stream);

/*
 * Advance nsteps (>= 0) synchronous ORCA steps on `stream`, asynchronously.
 * The first call after orca_set_agents captures one step into a CUDA graph (unless
 * ORCA_FLAG_NO_GRAPH); later calls replay it.  Capture happens on an internal stream, so
 * `stream` may be the default stream.
 */
ORCA_API int orca_step(orca_ctx* ctx, int32_t nsteps, void* stream);

/*
 * Read the current state in agent order: pos_xy and vel_xy (2*n floats each; either may be
 * NULL).  With ORCA_HOST the call synchronises `stream` and reports device-side errors;
 * pinned host arrays are written by a kernel directly over the CPU-GPU link, other host
 * arrays through staging copies.
 */
ORCA_API int orca_get_state(orca_ctx* ctx, float* pos_xy, float* vel_xy, int where,
                            void* stream);

/*
 * Read the neighbour lists used by the last step (needs ORCA_FLAG_RECORD): n*k int32
 * (k = the context's max_neighbors), row i = agent i's neighbours as agent indices,
 * nearest first, -1 padded.
 */
ORCA_API int orca_get_neighbors(orca_ctx* ctx, int32_t* nbr, int where, void* stream);

/*
 * Read the grid cell of every agent in the last step (needs ORCA_FLAG_RECORD): n uint32,
 * cell = cy * gx + cx.  grid_f (4 floats: xmin, ymin, cell edge, 1/edge) and grid_i
 * (2 int32: gx, gy) receive the grid (host pointers; either may be NULL).  Synchronises.
 */
ORCA_API int orca_get_cells(orca_ctx* ctx, uint32_t* cell, float* grid_f, int32_t* grid_i,
                            int where, void* stream);

/*
 * Counters accumulated since orca_set_agents (synchronises `stream`):
 *   counters[0] agent-steps executed, [1] agent-steps that needed the least-penetration
 *   fallback, [2] neighbour candidates examined, [3] half-planes built.
 */
ORCA_API int orca_get_counters(orca_ctx* ctx, int64_t* counters4, void* stream);

/*
 * Cost of the neighbour searches (Fig. 2: the r_obs filter, here the k nearest inside
 * r_obs) and of the least-penetration fallback, accumulated since orca_set_agents
 * (synchronises `stream`):
 *   counters[0] search passes beyond the first (the start radius held fewer than k agents
 *               inside r_obs and grew 1.5x);
 *   [1] searches that started without a radius prediction (the first step after a load:
 *       the start comes from the density of the cells around the agent);
 *   [2] grid rows scanned (a search stops at a row once its bound has tightened past it,
 *       which depends on the order of the agents inside a cell, so this count varies
 *       slightly between runs);
 *   [3] the lines of the least-penetration LP's projected problems (Section 3: each line
 *       violated by more than the penetration reached so far opens a problem over itself
 *       and the bisectors with the lines before it; a problem for line i, 0-based,
 *       counts i + 1).
 * Counted by every step.
 */
ORCA_API int orca_get_search_counters(orca_ctx* ctx, int64_t* counters4, void* stream);

/*
 * Static obstacles: n_seg line segments (0 <= n_seg <= 256; 0 clears them), seg_xyxy 4*n_seg
 * floats (x1, y1, x2, y2 per segment, host or device per `where`).  Not in the paper's
 * experiments; the ORCA obstacle rule the paper defers to (van den Berg et al.): the
 * optimisation velocity is 0 and the agent takes full responsibility, so with q the
 * segment's nearest point relative to the agent and d = |q|, the permitted velocities are
 * v.q/d <= (d - r)/time_horizon (dt in place of time_horizon when the agent overlaps the
 * segment).  Each agent keeps the max_obstacle_neighbors (1..4) nearest segments it could
 * reach within time_horizon -- FP32 squared distance, by the clamped projection, strictly
 * below fl(fl(max_speed*time_horizon) + radius)^2 -- ordered by (distance, index); their
 * half-planes come first in the LP and stay hard in the least-penetration fallback.  The
 * segments stay until replaced; they apply to single-scene steps (ORCA_ERR_STATE in a
 * batch, with operation counting, or in rollouts).  Rebuilds the step graphs.
 * A step with segments runs two more kernels: one flags the tiles of agents that could
 * reach a segment, and an obstacle instantiation of the ORCA kernel steps those tiles on a
 * second stream beside the plain launch (joined before the step ends, so a step stays
 * ordered on the caller's stream).  The first call with segments creates that stream and
 * two events; orca_destroy frees them.
 */
ORCA_API int orca_set_obstacles(orca_ctx* ctx, int32_t n_seg, const float* seg_xyxy,
                                float time_horizon, int32_t max_obstacle_neighbors, int where,
                                void* stream);

/*
 * The segments each agent used in the last step (needs ORCA_FLAG_RECORD): n*4 int32 in agent
 * order, nearest first, -1 padded.  Synchronises `stream` for host output.
 */
ORCA_API int orca_get_obstacle_neighbors(orca_ctx* ctx, int32_t* obst, int where, void* stream);

/*
 * Remove the agents that have reached their goal (Section 4: a person who reaches the
 * goal location is removed from the simulation).  An agent has arrived when its goal lies
 * within its radius on the current state, decided in FP32 with one rounding per operation:
 * dx = fl(gx - px), dy = fl(gy - py), arrived iff fl(fl(dx*dx) + fl(dy*dy)) <= fl(r*r).
 * The survivors keep their relative order and are renumbered 0..n'-1 (the next step sorts
 * them into cells again; their radius predictions are kept).  *n_remaining receives n';
 * kept_ids (n' int32, host or device memory per `where`, may be NULL) receives each new
 * index's old index.  Synchronises `stream` (the host needs n').  The next orca_step
 * re-captures its CUDA graphs for the new count.  Single-scene contexts only:
 * ORCA_ERR_STATE for a batch; ORCA_ERR_ARG for a null ctx or n_remaining.
 */
ORCA_API int orca_remove_arrived(orca_ctx* ctx, int32_t* n_remaining, int32_t* kept_ids, int where,
                                 void* stream);

/*
 * Spawning during a run (Section 4, test set-up: people are spawned at random locations
 * chosen so that they overlap nobody within a time period based on their size and speed).
 * Candidates c = 0..m-1 -- cand_pos, goal_xy (2m floats), radius, max_speed, pref_speed,
 * time_horizon (m floats), host or device memory per `where` -- enter at rest.  Candidate c
 * is refused when it could touch a present agent j within `window` seconds, both moving
 * straight at each other, |p_c - p_j| <= r_c + r_j + (V_c + |v_j|) window, or likewise a
 * candidate accepted before it (candidates are taken in index order, with that
 * candidate's maximum speed in place of |v_j|).  Decided in FP32, one rounding per
 * operation.  The accepted ones are appended with agent indices n, n+1, ... in candidate
 * order and no search-radius prediction; accepted (m int32 per `where`, may be NULL)
 * receives 1 or 0 per candidate and *n_after the new agent count.  O(n m) work (every
 * candidate against every present agent).  Synchronises `stream` (the host needs the
 * count); the next orca_step re-captures its graphs.  Errors: ORCA_ERR_ARG, ORCA_ERR_STATE
 * (a batch), ORCA_ERR_CAPACITY (n + m above max_agents), ORCA_ERR_CUDA.
 */
ORCA_API int orca_spawn_agents(orca_ctx* ctx, int32_t m, const float* cand_pos, const float* goal_xy,
                               const float* radius, const float* max_speed, const float* pref_speed,
                               const float* time_horizon, float window, int where, int32_t* accepted,
                               int32_t* n_after, void* stream);

/*
 * Operation counting (measurement; the paper has no counterpart).  With on != 0, later
 * steps launch an instantiation of the ORCA kernel that also counts the LP's algorithmic
 * operations of Section 3: LP1 calls, LP1 bounds evaluated, violation checks of the LP2
 * and LP3 scans, and LP3 bisectors formed (i per line i that LP3 solves for).  Results are
 * unchanged; the counting kernel is slower, so time nothing with it on.  Switching drops
 * the captured CUDA graphs.  Returns ORCA_OK or ORCA_ERR_ARG (null ctx).
 */
ORCA_API int orca_count_ops(orca_ctx* ctx, int32_t on);

/*
 * The four operation counts above, summed over the steps launched with counting on since
 * orca_set_agents (synchronises `stream`): counters4[0] LP1 calls, [1] LP1 bounds,
 * [2] violation checks, [3] bisectors.  Zero when counting was never on.
 */
ORCA_API int orca_get_op_counters(orca_ctx* ctx, int64_t* counters4, void* stream);

/*
 * FP64 validation rollout (validation only; the paper has no counterpart).  Runs T steps
 * of the ORCA step in FP64 from (pos0, vel0) -- neighbours decided in FP32 on the
 * FP32-rounded positions as the FP32 step decides them (k nearest by (fl32 d^2, index)
 * strictly inside r_obs), half-planes (Fig. 1), preferred velocity and the LP of Section 3
 * in double -- and, when dL_dpos is not NULL, the double instantiation of the library's
 * adjoint back through it (the same kernels the FP32 rollouts use, with the same record of
 * what fixed each selected velocity).  This separates adjoint errors from the FP32
 * trajectory's drift: the FP64 trajectory follows an FP64 reference to rounding.
 *
 * All arrays are device memory in agent order, double: pos0, vel0, goal (2n), radius,
 * max_speed, pref_speed, time_horizon (n); dL_dpos (T x n x 2, the loss gradient of
 * positions p(1..T), may be NULL); traj_pos (T x n x 2) receives p(1..T); g_pref_speed,
 * g_radius, g_time_horizon (n) and g_pos0, g_vel0 (2n) receive the gradients (each may be
 * NULL).  n <= 65,536 (the neighbour search scans all agents).  Allocates its scratch
 * with cudaMalloc and synchronises `stream` before returning.  Errors: ORCA_ERR_ARG,
 * ORCA_ERR_NOMEM, ORCA_ERR_CUDA, with a message in orca_last_error(NULL).
 */
ORCA_API int orca_validate_rollout_fp64(int32_t n, int32_t max_neighbors, float neighbor_dist, double dt,
                                        int32_t T, const double* pos0, const double* vel0,
                                        const double* goal, const double* radius,
                                        const double* max_speed, const double* pref_speed,
                                        const double* time_horizon, const double* dL_dpos,
                                        double* traj_pos, double* g_pref_speed, double* g_radius,
                                        double* g_time_horizon, double* g_pos0, double* g_vel0,
                                        void* stream);

/*
 * FP32 FMA throughput microbenchmark (measurement; the paper has no counterpart): the peak
 * against which the ORCA kernel's arithmetic roofline is quoted.  Enqueues one kernel on
 * `stream` of `blocks` CTAs of 256 threads (blocks <= 0: 8 per SM), each thread running
 * iters x 32 dependent-free FMAs; out (device, >= blocks floats) receives one value per CTA
 * that keeps the work live.  *flops receives the FP32 operations enqueued (an FMA counts
 * two); the caller times the kernel (CUDA events on `stream`).  Asynchronous.  Errors:
 * ORCA_ERR_ARG (null pointer, iters < 1), ORCA_ERR_CUDA (launch failure).
 */
ORCA_API int orca_fma_bench(int32_t blocks, int32_t iters, float* out, int64_t* flops, void* stream);

/*
 * Per-phase device timing.  With enable != 0 the step records CUDA events (event-record
 * nodes inside the captured graph) between its three phases: binning (bounding box, cell
 * keys and counts, cell table), reorder (agents into cell order) and the per-agent
 * ORCA kernel.  Toggling rebuilds the graphs on the next orca_step.
 */
ORCA_API int orca_profile(orca_ctx* ctx, int enable);

/*
 * Durations in milliseconds of the three phases of the most recent profiled step:
 * ms3[0] binning, ms3[1] reorder, ms3[2] ORCA kernel (with obstacles: the tile flags and
 * the plain and obstacle launches together).  Waits for that step to finish.
 */
ORCA_API int orca_profile_read(orca_ctx* ctx, float* ms3);

/* Number of kernels one orca_step enqueues per step: five (bounding box -- for a batch,
 * the scenes' boxes and cell ranges --, cell keys and counts, cell table, reorder, ORCA
 * kernel); static obstacles add two: the tile flags and the obstacle launch. */
ORCA_API int orca_launches_per_step(const orca_ctx* ctx, int32_t* count);

/*
 * One ORCA step without any memory allocation, for callers that cannot allocate GPU
 * memory: code inside a host framework that must route every device allocation through
 * its own pool, or call sites where cudaMalloc's implicit device synchronisation is not
 * allowed.  (The paper has no counterpart; this is a deployment convenience.)
 *
 * Inputs are device arrays in agent order, laid out as for orca_set_agents (pos_xy,
 * vel_xy, goal_xy: 2*n floats; radius, max_speed, pref_speed, time_horizon: n floats);
 * neighbor_dist, max_neighbors (1..32), dt and cell_size (0 -> neighbor_dist/4) as in
 * orca_params.  Outputs pos_out_xy, vel_out_xy: device arrays of 2*n floats receiving the
 * state after one step, in agent order; they must not overlap the inputs.  The result is
 * the same as one orca_step of a context holding these agents.
 *
 * All scratch space lives in a fixed device array inside the library, sized for at most
 * 65,536 agents and 262,144 grid cells (about 7 MiB, held on every GPU that loads the
 * library until the process exits); n above 65,536 returns ORCA_ERR_CAPACITY.  More cells
 * than that only coarsen the grid (results do not change).  Every call looks up the
 * array's device address in the current context (so a reset of the primary context is
 * safe); the first call on a device may load the library's device code, so make it
 * before any stream capture.
 * The call is asynchronous on `stream` and never synchronises, so errors that arise on
 * the GPU are not reported here: non-finite inputs give non-finite outputs, and a crowd
 * whose extent fits no grid of the scratch's cell table (which, with the cell edge
 * doubling until the grid fits, happens only for non-finite or astronomically large
 * coordinates) is stepped in a single cell -- slowly, still exactly -- without an error
 * code.  Every call shares the one array, so calls whose work overlaps
 * on the GPU (different streams, or different host threads) race and corrupt each other:
 * order them.  Errors: ORCA_ERR_ARG, ORCA_ERR_CAPACITY, ORCA_ERR_CUDA, with a message in
 * orca_last_error(NULL).
 */
ORCA_API int orca_step_static(int32_t n, const float* pos_xy, const float* vel_xy,
                              const float* goal_xy, const float* radius, const float* max_speed,
                              const float* pref_speed, const float* time_horizon,
                              float neighbor_dist, int32_t max_neighbors, float dt,
                              float cell_size, float* pos_out_xy, float* vel_out_xy,
                              void* stream);

/*
 * Change the grid cell edge (metres, > 0; 0 -> neighbor_dist / 4) used from the next
 * orca_step on.  Results do not depend on it (the neighbour search is exact for any
 * edge); speed does.  Rebuilds the step graphs.
 */
ORCA_API int orca_set_cell_size(orca_ctx* ctx, float cell_size);

/*
 * Launch shape of the per-agent ORCA kernel: threads per CTA (64, 128 or 256; default 128)
 * and the mode, lp3_lanes: 1 -- one lane per agent, which solves its LPs alone; 4 -- agent
 * split: a quad of lanes steps each agent (the neighbour search's candidates, the
 * half-planes and the least-penetration solve shared out over the four lanes; for crowds
 * too small to fill the GPU; a batch keeps one lane per agent); 32 -- work units: every
 * lane keeps its agent's LPs, but the bound evaluations of all the LP1 solves a warp needs
 * at once are dealt out over its 32 lanes (the paper's load-balanced LP, Section 3); 0 ->
 * default: 1 for max_neighbors <= 16, else 32.  Results are bitwise the same in every mode;
 * speed differs.  Until this is first called, a context steps a single scene of at most
 * 12,000 agents with k <= 16 in the agent split (64 threads) and anything else with 128
 * threads and the default mode.  Rebuilds the step graphs.
 */
ORCA_API int orca_set_launch(orca_ctx* ctx, int32_t threads_per_block, int32_t lp3_lanes);

/*
 * Differentiable rollouts (single scene).  A rollout of T steps from the loaded state
 * records the positions p(1..T); its adjoint returns the gradient of a loss L(p(1..T))
 * with respect to every agent's preferred speed, radius and time horizon (and initial
 * position and velocity).  The adjoint is hand-written: it differentiates each step
 * through the constraints that fixed the selected velocity, with neighbour sets and every
 * branch held fixed (the step is piecewise smooth).  With ckpt_every >= 1 the forward pass
 * keeps a checkpoint of the state every ckpt_every steps and the backward pass re-runs each
 * segment from its checkpoint, recording, and sweeps it in reverse (memory for ckpt_every
 * steps' records).  With ckpt_every = 0 the forward pass records every step (state,
 * neighbour lists, LP records: (20 + 4 max_neighbors) bytes per agent-step) and the
 * backward pass only sweeps them in reverse, with no recomputation.  Both modes give
 * bitwise the same trajectory and gradients.
 *
 * orca_rollout_workspace_size: device bytes for (T, ckpt_every) on this context.
 */
ORCA_API int orca_rollout_workspace_size(const orca_ctx* ctx, int32_t T, int32_t ckpt_every,
                                         size_t* bytes);

/*
 * Run T >= 1 steps from the loaded state, checkpointing every ckpt_every >= 1 steps, or
 * recording every step (ckpt_every = 0).
 *   traj_pos  device, T*n*2 floats: p(t) for t = 1..T in agent order (may be NULL).
 *   workspace device buffer of orca_rollout_workspace_size bytes, 256-byte aligned, kept by
 *             the caller until orca_rollout_backward.
 * The context's state ends at step T.
 */
ORCA_API int orca_rollout_forward(orca_ctx* ctx, int32_t T, int32_t ckpt_every, float* traj_pos,
                                  void* workspace, size_t workspace_bytes, void* stream);

/*
 * Gradients of L from dL/dp(t) (device, T*n*2 floats, t = 1..T) for the last
 * orca_rollout_forward with this workspace.  Outputs (device, n floats each; overwritten;
 * any may be NULL): g_pref_speed, g_radius, g_time_horizon; g_pos0, g_vel0 (2n floats):
 * dL/dp(0), dL/dv(0).  The context's state is left undefined (reload it).
 */
ORCA_API int orca_rollout_backward(orca_ctx* ctx, const float* dL_dpos, float* g_pref_speed,
                                   float* g_radius, float* g_time_horizon, float* g_pos0,
                                   float* g_vel0, void* workspace, size_t workspace_bytes,
                                   void* stream);

/* Synchronise `stream` and report any latched device-side error. */
ORCA_API int orca_sync(orca_ctx* ctx, void* stream);

/* Agents currently loaded (0 if none). */
ORCA_API int orca_num_agents(const orca_ctx* ctx, int32_t* n);

/* Message of the last failure on ctx ("" if none).  ctx may be NULL for the entry points
 * without a context (orca_create, orca_workspace_size, orca_step_static); that message is
 * kept per host thread, so it is the calling thread's own last failure. */
ORCA_API const char* orca_last_error(const orca_ctx* ctx);

/* Fixed text for a status code. */
ORCA_API const char* orca_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* ORCA_GB300_H */
