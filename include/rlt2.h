/*
 * rlt2.h -- C ABI of the GB300 (sm_103a) RLT2 dual-ascent library.
 *
 * Lower bounds for the Quadratic Assignment Problem by Lagrangian dual ascent
 * on the level-2 RLT formulation (Date & Nagi, arXiv:1710.03732).  Problem
 * statement: Section 1, Eq. 1.1-1.4 (flow F, distance D, fixed cost B);
 * RLT2 and its Lagrangian dual: Section 2.3, Eq. 2.6-2.16; the three-stage
 * LAP decomposition: Figure 1 and the Theta/Delta definitions after it; the
 * ascent rules: Eq. 2.20-2.23 and their combination in the proof of
 * Theorem 1; the iteration: Algorithm 1 / Algorithm 2 (S and F variants,
 * one or two phases, Section 3.4; the half-Z scheme and the Type 4 rule,
 * Sections 2.3 and 5); branch and bound: Section 4.
 *
 * General conventions
 *  - Every function returns an rlt2_status; nothing throws or aborts.
 *  - All floating point is IEEE FP64.  Matrices are row-major, n x n.
 *  - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *    global memory of the current device.  Inputs are borrowed for the
 *    duration of the call only (copied where kept); outputs are written into
 *    caller-owned buffers of the documented length.
 *  - The library owns every buffer it allocates inside a context and frees it
 *    in rlt2_destroy.  All GPU work of a context runs on the stream given at
 *    creation (a cudaStream_t passed as void*; NULL = legacy default stream).
 *  - A context is not thread-safe; distinct contexts are independent.
 *  - Sizes: 3 <= n (after removing fixed facilities) and n <= 32.
 *
 * Array layouts (residual size n, m = n-2; compressed index of j != i is
 * j' = j - (j > i), of k != i,j is k' = k - (k > i) - (k > j); same for
 * locations):
 *   tile t(i,p,j',q') = ((i*n + p)*(n-1) + j')*(n-1) + q',  T = n^2 (n-1)^2 tiles
 *   C^[t] (y costs, Section 3.3), pi_y[t]
 *   D^[t*m*m + k'*m + r'] (z costs, E = T*m*m entries)
 *   xi[t*m + k'], psi[t*m + r']              (Z-LAP duals, Eq. 2.15)
 *   gamma[(i*n+p)*(n-1) + j'], delta[(i*n+p)*(n-1) + q']  (Y-LAP duals)
 *   alpha[i], beta[p] (X-LAP duals), pi_x[i*n + p]
 */
#ifndef RLT2_H
#define RLT2_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RLT2_OK = 0,
  RLT2_EINVAL = 1,   /* bad argument: NULL, size out of range, non-finite input, bad parameters */
  RLT2_ENOMEM = 2,   /* device allocation failed or the memory budget is too small */
  RLT2_ECUDA = 3,    /* a CUDA call failed; rlt2_last_error() has the message */
  RLT2_ETIMEOUT = 4, /* a bounded device-side wait gave up */
  RLT2_EADMIT = 5    /* a node does not fit the memory budget even alone */
} rlt2_status;

/* Dual-ascent parameters.
 *  kz, ky, kx : kappa^z, kappa^y, kappa^x of Eq. 2.20, 2.22, 2.23, each in [0,1]
 *  phi_y      : varphi of Eq. 2.21 (y_ijpq <-> y_jiqp), in [0,1], phi_y + ky <= 1
 *  phi_z[5]   : phi_1..phi_5 of Eq. 2.20 (used by rules 1-3), each in [0,1],
 *               summing to 1 within 1e-12
 *  dual_mode  : 0 = the Hungarian's own duals (FP64, the CPU oracle's
 *               operation order), 1 = canonical duals (the pointwise-largest
 *               optimal row duals with u_0 = 0; unique for a given cost
 *               matrix) computed exactly in 64-bit fixed point on a per-tile
 *               grid of 2^-48 of the tile's magnitude bound, so warm and cold
 *               solves agree bit for bit, 2 = canonical duals computed in FP64
 *  warm       : 0 = cold LAPs, 1 = start every Z, Y and X LAP from its
 *               previous iteration's row duals, 2 = as 1 but the Z-LAPs start
 *               from row duals predicted by the network attached with
 *               rlt2_set_mlp (column-min repair keeps any start feasible; with
 *               canonical duals the bound does not depend on the start)
 *  min_gap    : stop once (UB - LB)/UB < min_gap (needs ub > 0 or a found UB)
 *  ub         : known upper bound on the node's QAP value (<= 0: unknown)
 *  feas_tol   : tolerance of the feasibility check after Algorithm 1
 *               (relative to max(1, |LB|)); the check stops the ascent when
 *               every y and z of the X-LAP primal has |reduced cost| <= tol
 *               (<= 0 disables it)
 *  stall_window, stall_tol : early termination of the branch-and-bound
 *               experiments (Section 5): stop once the best bound improved by
 *               less than stall_tol * |UB| over the last stall_window
 *               iterations (stall_window <= 0 disables it; at most 64)
 *  variant    : 0 = S (slow) RLT2-DA: the LAPs are solved on the full
 *               multiplier-adjusted costs b', C^, D^ (Section 3.4);
 *               1 = F (fast): the LAPs are solved on the incremental costs of
 *               the constraint set Psi_2 of Eq. 3.6 -- what remains of each
 *               reduced cost after the ascent step, (1-kz) pi_z + inflow for
 *               z, (1-ky-phi_y) pi_y(ijpq) + phi_y pi_y(jiqp) for y,
 *               (1-kx) pi_x for x -- and the bound is the previous bound
 *               plus the X-LAP value (Eq. 3.7)
 *  two_phase  : 1 = after the Z-LAPs, move every class's z slack from its
 *               members with pi_z > 0 (S_N) evenly onto its members with zero
 *               slack (S_B) and solve the Z-LAPs again (Section 3.4)
 *  phase2_tol : a z belongs to S_B when pi_z <= phase2_tol (1 + |xi| + |psi|)
 *               (its row and column duals)
 *  sa_t0, sa_cool, sa_period : annealing schedule of the Type 4 rule
 *               (Section 2.3, rule 4; Section 5): temperature sa_t0 * ub,
 *               multiplied by sa_cool every sa_period iterations; the draws
 *               are given with rlt2_set_sa (needs ub > 0)
 *  half_z     : 1 = the half-Z-LAP scheme of Section 5 (after Goncalves et
 *               al.): the z whose first facility index exceeds the second
 *               ("lower order") keep cost 0, so their Z-LAPs (i > j) are not
 *               solved.  The y move of Eq. 2.21 runs with phi_y (1/2 in the
 *               paper) on every y; each of the three upper members of a class
 *               then pools kz (2/3) of its z slack, ky (1) of its tile's y
 *               slack as left by the y move and the Type 3 part of pi_x (kx = 1),
 *               and gives half of the pool to each other upper member; a lower
 *               y (i > j) passes kx pi_x(ip)/(n-1) to its mirror on the y level.
 *               S variant, one phase, no Type 4 rule; phi_z ignored; the
 *               phi_y + ky <= 1 limit does not apply (each y's slack is
 *               first split by the y move, then pushed into z).
 *  pipeline   : 1 = run the z move of each ascent step and the Z-LAPs of
 *               the next solve as one launch, a tile's LAP starting once the
 *               move has finished every class of its facility pair (identical
 *               results; the FP64 move and the integer LAPs share the SMs);
 *               0 (default) = two launches.  On GB300 it pays for cold starts
 *               around n = 20 (13 % there) and loses elsewhere: the LAPs need
 *               the warp slots the move takes.  Not used with half_z or
 *               warm = 2, nor by rlt2_bound_nodes and the no-allocation entry
 *               point.  A pipelined wait that gives up (about a second; only a
 *               fault can cause it) stops the ascent and rlt2_iterate returns
 *               RLT2_ETIMEOUT. */
typedef struct rlt2_params {
  double kz, ky, kx, phi_y;
  double phi_z[5];
  int dual_mode;
  int warm;
  double min_gap;
  double ub;
  double feas_tol;
  int stall_window;
  double stall_tol;
  int variant;
  int two_phase;
  double phase2_tol;
  double sa_t0;
  double sa_cool;
  int sa_period;
  int half_z;
  int pipeline;
} rlt2_params;

typedef struct rlt2_ctx rlt2_ctx;

/* Default parameters: kz = kx = 1, ky = 1/2, phi_y = 1/2, phi_z = 1/5 each,
 * canonical duals, cold start, min_gap = 0, ub unknown, feas_tol = 1e-9,
 * no stall stop (stall_window = 0, stall_tol = 0.0002), S variant, one phase,
 * phase2_tol = 1e-9, sa_t0 = 0.04, sa_cool = 0.99, sa_period = 100 (Section 5),
 * z move and Z-LAPs as two launches. */
void rlt2_params_default(rlt2_params* p);

/* Create a dual-ascent context for one QAP node (Eq. 1.1; a branch-and-bound
 * node fixes some facilities, Section 4).
 *  n        : problem size, 3 <= n - (#fixed) and n <= 64 (residual <= 32)
 *  F, D     : host, n*n flow and distance matrices (finite)
 *  B        : host, n*n fixed costs, or NULL for B = 0
 *  partial  : host, n ints, partial[i] = location of facility i or -1 (free);
 *             NULL = root node.  Must be injective.
 *  p        : host parameters (NULL = defaults); copied
 *  stream   : cudaStream_t used for all work of this context
 *  out      : receives the context (NULL on failure)
 * Multipliers start at 0 (Algorithm 1 step 1), so the first iteration's bound
 * is the Gilmore-Lawler bound.  Errors: EINVAL, ENOMEM, ECUDA. */
rlt2_status rlt2_create(int n, const double* F, const double* D, const double* B, const int* partial,
                        const rlt2_params* p, void* stream, rlt2_ctx** out);

/* Child context of a branch-and-bound node (Section 4, step 3): the parent's
 * problem with facility `facility` fixed at location `location` (original
 * indices, both free in the parent), starting from the parent's multipliers --
 * its multiplier-adjusted costs of the last solve (the pending ascent step is
 * not applied): in LRLT2(v), y_{i f p l} and y_{f i l p} become x_ip and each
 * z with (f,l) in one position becomes the y of the other two, so
 *   D^_c(i,j,k|p,q,r) = D^_p(i,j,k|p,q,r),
 *   C^_c(i,j|p,q) = ((C^_p(i,j|p,q) + D^_p(i,j,f|p,q,l)) + D^_p(i,f,j|p,l,q)) + D^_p(f,i,j|l,p,q),
 *   b'_c(i|p) = (b'_p(i|p) + C^_p(i,f|p,l)) + C^_p(f,i|l,p),  const_c = const_p + b'_p(f|l);
 * the child's upper bounds use the plain QAP reduction of b.  Built on the
 * parent's stream, on the device; the parent is not changed and may be
 * destroyed afterwards.  p: the child's parameters (NULL = the parent's).
 * Errors: EINVAL (NULL, not free, residual below 3, parent or p not the S
 * variant), ENOMEM, ECUDA. */
rlt2_status rlt2_create_child(rlt2_ctx* parent, int facility, int location, const rlt2_params* p,
                              rlt2_ctx** out);

/* Run up to `iters` iterations of RLT2-DA (Algorithm 1 / 2; S or F, one or two
 * phases, as the parameters select): the ascent
 * step from the previous iteration's reduced costs (if any), then the Z, Y and
 * X LAP stages.  After return, the bound, duals, reduced costs and state all
 * belong to the same multipliers (the last solved ones).
 *  lb_hist : host, iters doubles (nullable): bound of each iteration
 *            (including the fixed facilities' constant); entries after an
 *            early stop are set to NaN
 *  done    : host (nullable): receives the number of iterations performed
 * Stops early (returns OK) once the feasibility check, min_gap or the stall
 * rule fires: iterations are enqueued in chunks of 8, 16, 32, ... and the call
 * returns after the chunk in which the device stopped.  A context's first 64
 * iterations are launched kernel by kernel, later ones as replays of captured
 * CUDA graphs of eight iterations and of one (same kernels, same results).
 * Synchronises the context's stream before returning. */
rlt2_status rlt2_iterate(rlt2_ctx* ctx, int iters, double* lb_hist, int* done);

/* Up to `iters` iterations of several contexts' ascents in lockstep: every
 * stage of an iteration is one launch over all of them (the batched node
 * kernels of rlt2_bound_nodes, Z-LAPs launched per size with the tuned shapes
 * of rlt2_node_tuning), so many small ascents, such as the children of a
 * branch-and-bound node, share the GPU instead of taking turns.  Each context
 * follows exactly the trajectory rlt2_iterate would give it and stops on its
 * own rules; the call returns once every context has stopped (checked between
 * chunks of 8, 16, 32, ... iterations) or after `iters` iterations.
 *  ctxs  : count distinct contexts, 1 <= count <= 1024, all on the current
 *          device, sharing dual_mode, warm (0 or 1) and two_phase; the
 *          half-Z scheme and Type 4 draws are not supported (EINVAL)
 *  done  : host, count ints (nullable): iterations each context ran
 * Work runs on ctxs[0]'s stream after every context's stream is synchronised;
 * the call synchronises before returning.  The contexts' augmentation and
 * relaxation counters (rlt2_stats) do not count these iterations.  Calls from
 * several host threads are serialised.  Errors: EINVAL, ECUDA. */
rlt2_status rlt2_iterate_many(rlt2_ctx* const* ctxs, int count, int iters, int* done);

/* Enqueue `iters` iterations without synchronising or reading anything back
 * (for timing and for callers that overlap work).  The bounds can be read
 * later with rlt2_bound. */
rlt2_status rlt2_iterate_async(rlt2_ctx* ctx, int iters);

/* Bounds of the last solve (host outputs, each nullable):
 *  lb      : bound of the last iteration;  best_lb : best bound so far
 *  ub      : best upper bound seen (QAP value of an X-LAP primal), or +inf
 *  perm    : n ints (full problem), location of every facility in the last
 *            X-LAP primal (fixed facilities keep their location)
 *  ub_perm : n ints, the permutation whose value is ub (same convention)
 *  iters   : iterations performed so far. Synchronises the stream. */
rlt2_status rlt2_bound(rlt2_ctx* ctx, double* lb, double* best_lb, double* ub, int* perm, int* ub_perm,
                       int* iters);

/* Duals of the last solve (Section 2.3: alpha, beta of Eq. 1.2-1.3; gamma,
 * delta of Eq. 2.2-2.3; xi, psi of Eq. 2.7-2.8).  Lengths: alpha, beta: n;
 * gamma, delta: n*n*(n-1); xi, psi: T*(n-2).  Any pointer may be NULL.
 * on_device != 0: the pointers are device memory (copied on the stream). */
rlt2_status rlt2_duals(rlt2_ctx* ctx, double* alpha, double* beta, double* gamma, double* delta, double* xi,
                       double* psi, int on_device);

/* Reduced costs of the last solve (Eq. 2.19 and the DLRLT2 constraints):
 *  pi_x: n*n, pi_y: T, pi_z: E = T*(n-2)^2; each nullable. */
rlt2_status rlt2_reduced_costs(rlt2_ctx* ctx, double* pi_x, double* pi_y, double* pi_z, int on_device);

/* Checkpoint / restore of the multiplier-adjusted costs (Section 3.3: the
 * multipliers live inside D^ and C^).  Dhat: E doubles, Chat: T doubles.
 * Import discards the pending ascent step, so the next iteration solves the
 * imported costs directly. */
rlt2_status rlt2_export_state(rlt2_ctx* ctx, double* Dhat, double* Chat, int on_device);
rlt2_status rlt2_import_state(rlt2_ctx* ctx, const double* Dhat, const double* Chat, int on_device);

/* The rest of an F-variant checkpoint: the incremental x costs bx (host, n*n)
 * and the bound the next solve adds its X-LAP value to (*lb_base).  Export
 * after an iteration returns the base of that iteration's solve, so importing
 * D^, C^, bx and lb_base and iterating repeats that solve and continues as the
 * uninterrupted run would.  S variant: bx is b' and lb_base the constant.
 * Errors: EINVAL (NULL context or, on import, NULL bx / non-finite values). */
rlt2_status rlt2_export_xstate(rlt2_ctx* ctx, double* bx, double* lb_base);
rlt2_status rlt2_import_xstate(rlt2_ctx* ctx, const double* bx, double lb_base);

/* Draws of the Type 4 rule with simulated annealing (Section 2.3, rule 4;
 * Section 5).  Draw d belongs to the ascent step after the d-th solve
 * (d = 0, 1, ...):
 *  kappa_fac : host, count*n doubles (residual n), kappa^lb_i of draw d at [d*n+i]
 *  kappa_loc : host, count*n doubles, kappa^lb_p of draw d at [d*n+p]
 *  neglog_u  : host, count doubles, -ln(u_d) of the draw's uniform u_d in (0, 1]
 * With kappa^lb = sum_i kappa_fac + sum_p kappa_loc (facilities first, in index
 * order), temperature T_d = sa_t0 * ub * sa_cool^floor(d / sa_period)
 * (one multiplication per period) and nu the bound of the d-th solve, the
 * draw is accepted when kappa^lb * nu <= neglog_u[d] * T_d (u_d <=
 * exp(-kappa^lb nu / T_d)); then every z with first facility i and first
 * location p adds kappa_fac[i] g + kappa_loc[p] g, g = nu / (n (n-1) (n-2)),
 * to the amount it gives to its symmetric partners (and, in F, takes it from
 * its own cost).  count = 0 switches the rule off.  Copied; rebuilds the CUDA
 * graph.  Errors: EINVAL (ub <= 0, sa_t0 <= 0, sa_cool not in (0, 1],
 * sa_period < 1, a kappa outside [0, 1], a sum above 1, a negative or
 * non-finite neglog_u), ENOMEM, ECUDA. */
rlt2_status rlt2_set_sa(rlt2_ctx* ctx, int count, const double* kappa_fac, const double* kappa_loc,
                        const double* neglog_u);

/* Counters since creation, out[8] = {iterations, Z augmentations, Z relaxations,
 * Y augmentations, Y relaxations, X augmentations, X relaxations, stopped}. */
rlt2_status rlt2_stats(rlt2_ctx* ctx, long long* out);

/* Sizes: *T = n^2 (n-1)^2, *E = T (n-2)^2, *n_res = residual n, *cst = constant
 * of the fixed facilities (each nullable). */
rlt2_status rlt2_sizes(rlt2_ctx* ctx, int* n_res, long long* T, long long* E, double* cst);

/* Per-kernel timing with CUDA events on the context's stream (disables CUDA
 * graph replay while on).  rlt2_kernel_times fills ms[k] (total milliseconds)
 * and count[k] (launches) for k = 0..nk-1 in the order
 * {move_y, move_z, lap_z, lap_y, lap_x, finalize, phase2_move, lap_z2}
 * (the last two are empty intervals without two_phase); synchronises. */
rlt2_status rlt2_set_timing(rlt2_ctx* ctx, int on);
rlt2_status rlt2_kernel_times(rlt2_ctx* ctx, double* ms, long long* count, int nk);

rlt2_status rlt2_destroy(rlt2_ctx* ctx);

/* Measured instruction throughputs of the current device, the denominators of
 * the hot kernels' rooflines (no counterpart in the paper: the z move is bound
 * by the FP64 pipe, the fixed-point LAPs by the integer ALU pipe, and GB300's
 * data sheet gives no per-instruction rates).  Each probe keeps 8 independent
 * accumulators per thread over a grid of resident warps; the best of three
 * timed launches (CUDA events on `stream`) after a warm-up is reported.
 *  rates        : host, 5 doubles, in G lane-operations per second:
 *                 [0] add.rn.f64, [1] fma.rn.f64, [2] add.s64, [3] add.s32,
 *                 [4] the integer-pipe binary64 addition (rlt2_fp64_add_emulated)
 *  sm_clock_ghz : host (nullable): the device's rated SM clock
 * Allocates and frees two small buffers; synchronises `stream`.  Errors:
 * EINVAL (rates NULL), ECUDA. */
rlt2_status rlt2_probe_rates(double* rates, double* sm_clock_ghz, void* stream);

/* The integer-pipe binary64 addition the z move uses for part of its exactly
 * rounded additions (no counterpart in the paper), exposed so that tests can
 * hold it to the FP64 pipe bit for bit: sum[i] = a[i] + b[i] and diff[i] =
 * a[i] - b[i], round to nearest, ties to even, computed with integer
 * operations only.  count >= 0; a, b, sum, diff: device arrays of count
 * doubles (finite inputs; an overflowing result is infinity).  Asynchronous
 * on `stream`.  Errors: EINVAL, ECUDA. */
rlt2_status rlt2_fp64_add_emulated(long long count, const double* a, const double* b, double* sum, double* diff,
                                   void* stream);

/* Bounds-checked build only (compiled with -DRLT2_BOUNDS_CHECK): the number of
 * kernel indices found outside their array since the library was loaded (each
 * is replaced by 0, never dereferenced); -1 in the normal build, -2 if a
 * counter cannot be read. */
long long rlt2_debug_bounds_violations(void);

/* Batched LAPs, one warp per LAP (the tiled-LAP idea of Section 3.2: many
 * small LAPs solved in one launch).
 *  batch, m : number of LAPs and their size, 1 <= m <= 32
 *  cost     : device, batch*m*m, LAP b at cost + b*m*m, row-major
 *  u0       : device, batch*m starting row duals, or NULL (cold start: a
 *             column reduction, preceded in dual_mode 1 by a row reduction;
 *             the canonical results do not depend on the start, n_aug does)
 *  value    : device, batch optimal values (sum of the assigned costs)
 *  u, v     : device, batch*m row / column duals (nullable)
 *  row_to_col: device, batch*m assignment (nullable)
 *  n_aug    : device, batch augmenting searches per LAP (nullable)
 *  dual_mode: 0 raw (FP64), 1 canonical (exact fixed point), 2 canonical
 *             (FP64), as in rlt2_params.  Asynchronous on `stream`; dual_mode
 *             1 takes 8 bytes of stream-ordered device memory for its work
 *             queue (cudaMallocAsync, freed on `stream` after the launch). */
rlt2_status rlt2_lap_batched(int batch, int m, const double* cost, const double* u0, double* value, double* u,
                             double* v, int* row_to_col, int* n_aug, int dual_mode, void* stream);

/* Bound a batch of branch-and-bound nodes (Section 4: a node fixes some
 * facilities; its bound is the constant of the fixed part plus the RLT2 dual
 * ascent bound of the residual QAP, see rlt2_create).  Nodes are admitted into
 * waves whose arenas fit `mem_budget`; within a wave every stage of an
 * iteration runs as one launch over all nodes (a persistent LAP kernel pulling
 * work from a device queue), and the iteration is replayed as one CUDA graph.
 *  n, F, D, B : as for rlt2_create (host)
 *  n_nodes    : number of nodes, >= 1
 *  partials   : host, n_nodes*n ints, row k = partial assignment of node k
 *               (-1 = free); every node's residual size must be in [3, 32]
 *  p          : parameters (NULL = defaults), shared by all nodes
 *  mlp        : network for warm == 2 (learned starts), else NULL
 *  iters      : iterations per node, 1..65536 (a node stops early on its own
 *               feasibility / gap / stall rule)
 *  mem_budget : device bytes the node arenas may use (0 = 80 % of free memory)
 *  lb_out     : host, n_nodes doubles: best bound of each node
 *  lb_hist    : host, n_nodes*iters doubles (nullable): bound per iteration,
 *               NaN after a node stopped
 *  iters_out  : host, n_nodes ints (nullable): iterations each node ran
 *  stats_out  : host, 5 long longs (nullable): {waves, Z augmentations,
 *               Z relaxations, lanes per Z-LAP, warps per block} where the
 *               last two are the autotuned Z-stage launch shape of the
 *               largest Z-LAP size (rlt2_node_tuning lists every size)
 *  stream     : cudaStream_t; the call synchronises it before returning
 * Errors: EINVAL (bad input), EADMIT (a node alone exceeds mem_budget),
 * ENOMEM, ECUDA.  Device memory is allocated for the call and freed on return. */
typedef struct rlt2_mlp rlt2_mlp;

/* Failure-detection check of the tensor-core inference kernel (no counterpart
 * in the paper): runs it on one tile with its MMA and commit withheld, so its
 * bounded mbarrier wait runs out (about 2^22 polls); the kernel then sets the
 * network's error flag, releases its TMEM and returns, and the device stays
 * usable.  Returns RLT2_ETIMEOUT when the timeout was detected and reported
 * (the expected outcome, error flag cleared again), RLT2_OK if the wait did
 * not run out, EINVAL for a network whose width is not 256, ECUDA otherwise. */
rlt2_status rlt2_mlp_check_wait_timeout(rlt2_mlp* mlp);

/* The same check for the training GEMM of the tall products (the persistent
 * TMA / tcgen05 kernel: a producer, an MMA issuer and four epilogue warps):
 * runs the second forward layer's product on 1,024 zero rows with no MMA
 * issued and none committed, so the producer's and the epilogue's bounded
 * waits run out; each role then stops the others, lets its started copies
 * land and releases the TMEM, and the network's error flag is set.  Returns
 * RLT2_ETIMEOUT when that was detected (flag cleared again), RLT2_OK if no
 * wait ran out, EINVAL for a width other than 256, ECUDA otherwise.  The
 * network's activation buffers are overwritten. */
rlt2_status rlt2_mlp_check_gemm_wait_timeout(rlt2_mlp* mlp);

/* Failure-detection check of the pipelined launch (rlt2_params.pipeline = 1;
 * no counterpart in the paper): enqueues one iteration whose Z-LAP warps wait
 * for facility-pair counts that the z move never reaches, with the polls
 * capped at 2^12 (a few milliseconds) instead of 2^22.  The first wait to give
 * up stops the ascent (the same path as a real timeout), the launch skips its
 * remaining LAPs and ends, and the device stays usable.  Needs a context
 * created with pipeline = 1 and warm 0 or 1 that has run at least one
 * iteration (so that a move is pending), else RLT2_EINVAL.  Returns
 * RLT2_ETIMEOUT when the timeout was detected and reported (the expected
 * outcome), RLT2_OK if no wait gave up.  Afterwards the context is stopped
 * (rlt2_iterate makes no progress and returns RLT2_ETIMEOUT) and holds the
 * state of an incomplete step: destroy it.  Synchronises the context's stream. */
rlt2_status rlt2_pipeline_check_wait_timeout(rlt2_ctx* ctx);

rlt2_status rlt2_bound_nodes(int n, const double* F, const double* D, const double* B, int n_nodes,
                             const int* partials, const rlt2_params* p, rlt2_mlp* mlp, int iters, size_t mem_budget,
                             double* lb_out, double* lb_hist, int* iters_out, long long* stats_out, void* stream);

/* The Z-stage launch shapes rlt2_bound_nodes has tuned in this process (no
 * counterpart in the paper).  Within a wave the Z-LAPs are launched per size
 * (adjacent sizes with the same shape share a launch); the shape of each size,
 * lanes per LAP (8, 16, 32) and warps per block (4, 8), is chosen the first
 * time that size occurs by timing the candidates on live iterations, and kept
 * for the life of the process.  cap: capacity of the output arrays; m, group,
 * wpb: host, cap ints (Z-LAP size, lanes per LAP, warps per block), ms: host,
 * cap doubles (nullable; the chosen shape's Z-stage time for that size when it
 * was tuned, milliseconds), sorted by size; *count: the number of sizes in the
 * table (may exceed cap).  Errors: EINVAL. */
rlt2_status rlt2_node_tuning(int cap, int* m, int* group, int* wpb, double* ms, int* count);

/* Branch and bound to optimality (Section 4) on one GPU, every node bounded by
 * RLT2-DA.  Facilities are placed in a fixed order (order_rule 1: index order;
 * 2: largest total interaction first, then largest interaction with those
 * already placed; 3: the same with smallest -- the paper's best); a node at
 * depth d fixes the first d facilities of the order and branches the next one
 * over every free location (polytomic).  Open nodes wait in a best-first heap
 * (deeper first among equal bounds); a node is fathomed when its bound reaches
 * the incumbent minus abs_tol.  Children of a parent at depth <= warm_depth
 * start from the parent's multipliers (rlt2_create_child) while at most
 * max_states parent contexts, together at most max_state_bytes of device
 * memory, are kept; other children start from zero.  Each
 * node's ascent stops at iters_node iterations (iters_root at the root), when
 * it is fathomed (min-gap against the incumbent) or by the stall rule of p.
 * Nodes with at most two free facilities are enumerated.  Every bounded node's
 * X-LAP primal is an incumbent candidate. */
typedef struct rlt2_bnb_options {
  int order_rule;       /* 1, 2 or 3; default 3 */
  int iters_root;       /* default 200 */
  int iters_node;       /* default 100 */
  int warm_depth;       /* default 64 (all); -1: every node starts from zero multipliers */
  int max_states;       /* parent contexts kept for warm starts at once; default 4096 */
  long long max_nodes;  /* stop after this many bounded nodes (0: no limit) */
  double time_limit_s;  /* stop after this many seconds (0: no limit) */
  double ub0;           /* known incumbent value (<= 0: none) */
  double abs_tol;       /* fathom when LB >= UB - abs_tol; < 0 (default): 1 - 1e-6 when F, D, B are
                           integral (the optimum is then an integer), else 1e-9 max(1, |UB|) */
  double max_state_bytes; /* device memory for kept parent contexts; 0 (default): half the free memory */
  int batch_children;   /* 1 (default): the children of a branched node are bounded together in lockstep
                           launches (rlt2_iterate_many); 0: one after the other (rlt2_iterate).  The
                           half-Z scheme and the learned start always bound one after the other */
} rlt2_bnb_options;
void rlt2_bnb_options_default(rlt2_bnb_options* o);

/* n, F, D, B as in rlt2_create (root node); p: node parameters (S variant;
 * NULL = defaults).  Outputs (host): *best = the best value found, perm (n
 * ints) its permutation, *root_lb (nullable) the root bound, stats (nullable,
 * 8) = {nodes bounded, nodes branched, completions enumerated, ascent
 * iterations, deepest level, proven optimal (0/1), warm-started children,
 * cold-started children}.  Not proven when max_nodes or time_limit_s stopped
 * the search.  Errors: EINVAL, ENOMEM, ECUDA (from the node contexts). */
rlt2_status rlt2_bnb_solve(int n, const double* F, const double* D, const double* B, const rlt2_params* p,
                           const rlt2_bnb_options* o, double* best, int* perm, double* root_lb, long long* stats,
                           void* stream);

/* Dual ascent of a small QAP that allocates no device memory.  The paper has no
 * counterpart; this entry point exists for callers that cannot call cudaMalloc:
 * code running under a framework that owns the whole device memory pool (an
 * extra cudaMalloc would fail or break its accounting), loops that must not hit
 * the allocator's implicit device synchronisation, and deployments that forbid
 * allocation after start-up.
 *  n        : problem size, 3 <= n <= 10 (root node, no fixed facilities);
 *             larger n returns RLT2_EINVAL with a message naming the limit
 *  F, D     : device, n*n flow and distance matrices (finite; not checked)
 *  B        : device, n*n fixed costs, or NULL for B = 0
 *  p        : host parameters (NULL = defaults), as for rlt2_create; the
 *             S and F variants (variant 0, 1), the two-phase Z solve and warm
 *             starts 0 and 1 run exactly as on a context.  Rejected with
 *             RLT2_EINVAL: the half-Z scheme (half_z) and the learned start
 *             (warm = 2), which need a context.  Not available on this path
 *             (a context's set-up calls): the Type 4 draws (rlt2_set_sa); the
 *             pipelined launch is ignored (pipeline = 1 runs unpipelined, with
 *             the same results)
 *  iters    : 1..65536 iterations of the dual ascent, as rlt2_iterate runs them
 *  lb_hist  : device, iters doubles: bound of each iteration (NaN after a stop)
 *  stream   : cudaStream_t the work is enqueued on; the call returns without
 *             waiting for it
 * All working memory is one fixed 8 MiB device array inside the library, held
 * by every GPU that loads the library until the process exits; nothing is
 * allocated or freed, by this call or by any library routine it uses.  The first
 * call on a device looks up the array's device address with that device
 * current; make that first call before any stream capture.  Every call reuses
 * the same array and starts by clearing what must start at zero, so calls that
 * overlap on the GPU (different streams, or different host threads on one
 * device) race and give undefined results: serialise them.  The array's
 * address is cached per device, so the library must not be used across a
 * cudaDeviceReset. */
rlt2_status rlt2_iterate_noalloc(int n, const double* F, const double* D, const double* B, const rlt2_params* p,
                                 int iters, double* lb_hist, void* stream);

/* ---- learned warm start (not in the paper) ------------------------------
 * A per-row network predicts the change of each Z-LAP row dual since the
 * previous iteration from the row's sorted, column-min-reduced, max-scaled
 * costs (FP32), the row's previous dual and m/32 (34 features); the start is
 * u0 = u_prev + scale * prediction.  34 -> hidden -> hidden -> 1, ReLU, BF16
 * weights and activations, FP32 accumulation on the tensor cores.  Predictions only seed
 * the exact Hungarian.  An rlt2_mlp is not thread-safe and must not be used by
 * two contexts whose work overlaps on the GPU. */

/* hidden: multiple of 64 in [64, 1024]; seed: deterministic initialisation. */
rlt2_status rlt2_mlp_create(int hidden, unsigned long long seed, void* stream, rlt2_mlp** out);
rlt2_status rlt2_mlp_destroy(rlt2_mlp* m);
/* Host FP32 copies: W1 34*hidden (input index first), b1 hidden, W2
 * hidden*hidden, b2 hidden, w3 hidden, b3 1.  set_weights rounds W1, W2 to
 * BF16 for the tensor cores and resets the optimiser state. */
rlt2_status rlt2_mlp_get_weights(rlt2_mlp* m, float* W1, float* b1, float* W2, float* b2, float* w3, float* b3);
rlt2_status rlt2_mlp_set_weights(rlt2_mlp* m, const float* W1, const float* b1, const float* W2, const float* b2,
                                 const float* w3, const float* b3);
/* Append training rows: ntiles m x m tiles (device), their previous row duals
 * (device, nullable) and their optimal (canonical) row duals (device); the
 * stored target is the scaled change (optimal - previous). */
rlt2_status rlt2_mlp_add_samples(rlt2_mlp* m, long long ntiles, int mz, const double* tiles, const double* prev_u,
                                 const double* target_u);
/* Number of rows; optional host copies of the BF16 feature rows (rows*64 of
 * 2-byte values, 34 used) and FP32 targets (rows). */
rlt2_status rlt2_mlp_samples(rlt2_mlp* m, long long* rows, void* X_bf16, float* targets);
rlt2_status rlt2_mlp_clear_samples(rlt2_mlp* m);
/* Loss 1/(2N) sum (out - target)^2 on the first `rows` samples (<= 262144) and
 * its gradients (host, same shapes as the weights); no update. */
rlt2_status rlt2_mlp_grad(rlt2_mlp* m, long long rows, double* loss, float* gW1, float* gb1, float* gW2,
                          float* gb2, float* gw3, float* gb3);
/* `steps` AdamW steps on minibatches of batch_rows (multiple of 64, <= 262144)
 * drawn from the samples; loss_hist (host, steps, nullable). */
rlt2_status rlt2_mlp_fit(rlt2_mlp* m, int steps, int batch_rows, double lr, double weight_decay,
                         unsigned long long seed, double* loss_hist);
/* Drop predicted changes smaller than `gate` (in units of the tile scale):
 * such rows start from their previous dual exactly (default 0). */
rlt2_status rlt2_mlp_set_gate(rlt2_mlp* m, double gate);
/* Predicted row duals u0 (device, ntiles*mz) for device tiles / previous duals. */
rlt2_status rlt2_mlp_predict(rlt2_mlp* m, long long ntiles, int mz, const double* tiles, const double* prev_u,
                             double* u0);
/* Attach a network to a context (used when its params have warm == 2). */
rlt2_status rlt2_set_mlp(rlt2_ctx* ctx, rlt2_mlp* m);

/* Human-readable name of a status, and the last error message of this thread. */
const char* rlt2_strerror(rlt2_status s);
const char* rlt2_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* RLT2_H */
