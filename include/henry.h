/*
 * henry.h -- C ABI of the GB300 (sm_103a) solver for the stochastic Henry
 * problem and its multilevel Monte Carlo (MLMC) level statistics.
 *
 * Method (arxiv 2403.17018):
 *   section 2.1, Eqs. 1-5: density-driven Darcy flow coupled to salt
 *     transport, rho(c) = rho0 + (rho1 - rho0) c, D_tensor = phi D I;
 *     boundary conditions of the Henry problem (seawater on the right,
 *     freshwater inflow on the left, no flow top and bottom);
 *   section 2.3: implicit Euler with r = T / tau steps, Newton on the
 *     coupled (p, c) system, geometric multigrid V-cycles for the linear
 *     solves, Gaussian elimination on the coarsest grid;
 *   section 3, Eqs. EgL/A, Def. of Y_l and V_l: MLMC telescoping estimator
 *     built from level pairs (g_l, g_{l-1}) that share one random input xi.
 * The discretisation is cell-centred finite volumes with harmonic face K and
 * phi, arithmetic face density, full upwinding of the advected rho and rho c.
 *
 * Conventions (all entry points):
 *   - Return HENRY_OK (0) or a negative HENRY_E_* code; no exception crosses
 *     the ABI. henry_strerror() names the code; henry_last_error() gives a
 *     message for the last failing call on this host thread.
 *   - Pointers marked "device" are CUDA device pointers owned by the caller
 *     (the Python binding passes torch tensors). "host" pointers are plain
 *     host memory. Arrays are C-contiguous FP64 unless stated otherwise.
 *   - Work is enqueued on `stream` (a cudaStream_t, NULL = legacy default
 *     stream) and is asynchronous unless the entry point says otherwise.
 *   - Per-sample failures (Newton iteration cap, non-finite values) are
 *     reported in status[] and do not fail the call.
 *   - A context is not thread-safe. Calls for different levels may run
 *     concurrently on different streams; two calls that use the same
 *     level's workspace must not overlap (fine level l and coarse level l-1
 *     of a pair have separate workspaces).
 */
#ifndef HENRY_H
#define HENRY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
#define HENRY_OK 0
#define HENRY_E_INVALID (-1)     /* bad argument (NULL, size, level, config)  */
#define HENRY_E_CUDA (-2)        /* a CUDA runtime call failed                */
#define HENRY_E_NOMEM (-3)       /* device allocation failed                  */
/* (-4 is not used: no entry point waits on the device with a time limit) */
#define HENRY_E_UNSUPPORTED (-5) /* grid cannot be coarsened to <= 32 cells  */

/* Largest batch B of one call of the entry points that launch one grid row
 * per sample (henry_solve, henry_solve_series, henry_sample_pairs,
 * henry_adjoint, henry_fields, henry_residual_jacobian[_noalloc]): larger
 * batches are rejected with HENRY_E_INVALID before any work is enqueued;
 * split them into several calls. */
#define HENRY_MAX_BATCH 65535

/* ---- per-sample status bits (status[] outputs) ------------------------- */
#define HENRY_S_OK 0
#define HENRY_S_MAXIT 1          /* some time step hit newton_maxit          */
#define HENRY_S_NONFINITE 2      /* a residual norm became NaN or Inf        */
#define HENRY_S_BADINPUT 4       /* xi was not finite                        */
#define HENRY_S_STALL 8          /* a kernel's bounded wait for its own bulk
                                    copies into shared memory gave up; the
                                    sample is dropped from later work       */

/* ---- quantities of interest (q[] outputs, HENRY_NQ per sample) --------- */
#define HENRY_NQ 22
/* 0  Q_S   = int c rho dx                    (section 4, Eq. integral_s)
 * 1  M     = int phi rho c dx                (stored salt mass, Eq. 2)
 * 2  toe   = int c (Lx - x) dx               (salt-wedge penetration)
 * 3..5     c at (1.40,0.05), (1.65,0.25), (1.90,0.50): the paper's points
 *          3, 9 and 15 of Eq. 12points shifted into y in [0,1]; bilinear
 *          interpolation of cell values clamped to the outer cell centres.
 * 6  Q_FW  = area where c <= 0.012178        (fresh water, Eq. integral_fw)
 * 7..21    Q_1..Q_15 = int c rho dx over [x_i - 0.1, x_i + 0.1] x
 *          [y_i - 0.1, y_i + 0.1] clipped to the domain (Eq. integral_box),
 *          points of Eq. 12points in the order printed there (rows y_p =
 *          -0.95, -0.75, -0.50, i.e. y = 0.05, 0.25, 0.50; x = 0.90, 1.15,
 *          1.40, 1.65, 1.90); c constant per cell. */

#define HENRY_PREC_FP64 0        /* multigrid in FP64                        */
#define HENRY_PREC_FP32_MG 1     /* FP32 V-cycles inside FP64 defect correction */

#define HENRY_LOOP_HOST 0        /* host checks convergence once per iteration */
#define HENRY_LOOP_GRAPH 1       /* one CUDA graph per time step with a device-
                                    side while loop over Newton iterations   */

typedef struct henry_config {
  /* physics (Table 1; g from Eq. 3; q0 = 6.6e-2 kg/s / rho0) */
  double rho0, rho1, mu, g, D, K0, phi0, q0;
  double Lx, Ly;       /* domain [0,Lx] x [0,Ly], y upward                  */
  double T;            /* final time [s]                                    */
  /* level hierarchy: level l has nx0*2^l x ny0*2^l cells, nt0*2^l steps    */
  int nx0, ny0, nt0, nlevels;
  int n_xi;            /* 3 or 6 random variables                           */
  /* solver */
  int precision;       /* HENRY_PREC_*                                      */
  int loop_mode;       /* HENRY_LOOP_*                                      */
  double newton_rtol;  /* stop when ||R|| <= max(rtol ||R(u^0)||, atol), u^0 */
  double newton_atol;  /*   the step's initial guess; ||.|| the RMS residual
                          scaled to units of c per step. The default atol
                          1e-11 sits just above the FP64 rounding floor of
                          the finest grids and keeps max|c - c_exact| well
                          inside 1e-9 (measured <= 5e-11)                   */
  int newton_maxit;    /* iteration cap per step -> HENRY_S_MAXIT           */
  int nu1, nu2;        /* red-black block Gauss-Seidel sweeps pre / post    */
  int vcycles;         /* V-cycles per defect-correction iteration          */
  int guess_extrapolation; /* Newton's initial guess for u^{n+1}: the
                              polynomial extrapolation in time of order q
                              through u^n, ..., u^{n-q} (q = 1: 2u^n -
                              u^{n-1}; q = 2: 3u^n - 3u^{n-1} + u^{n-2}),
                              q = min(guess_extrapolation, steps done - 1)
                              so that the initial state is never used; 0
                              starts from u^n. 0..6, default 4; c clamped
                              to [0, 1]. Changes the iterations, not the
                              converged solution; the adjoint's checkpoints
                              grow by two state components per order above
                              1 (the vertex-centred variant uses q <= 1) */
  double newton_stag_tol;  /* also converged when r <= this and the last
                              iteration reduced r by less than half (the
                              FP64 rounding floor, which grows with
                              resolution, has been reached); 0 disables */
  int mg_fusion;       /* 1: V-cycles of small levels fused into one kernel
                          (a block per sample in shared memory up to 512
                          cells, a thread-block cluster per sample up to
                          mg_cluster_cells); 0: one launch per operation */
  int mg_cluster_cells; /* largest multigrid level (cells per sample) run by
                           the cluster kernel; 0 (default) disables it */
  int mg_small_cells;   /* largest multigrid level (cells per sample, at most
                           512) run by the shared-memory kernel; default 512 */
  int jac_lag;          /* 0: Jacobian and multigrid operators rebuilt at
                           every defect-correction iteration (Newton).
                           k > 0: rebuilt at the first iteration of a step
                           and after any iteration that reduced the residual
                           by less than a factor k, reused otherwise (the
                           residual is always the current FP64 one, so the
                           converged solution satisfies the same tolerance) */
  int field_model;      /* 0 (default): the smooth fields of k_fields' 3 or 6
                           variables; 1: the paper's two-layer multiscale
                           porosity (Eq. poro_2levels), Kozeny-Carman
                           permeability K = kappa phi^3 / (1 - phi^2) with
                           kappa = K0 (1 - phi0^2) / phi0^3 (Eq.
                           e_perm_Kozeny_Carman; Table 1's kappa_KC), and the
                           recharge q0 (1 + 0.5 xi3)(1 + sin(pi t / 40)) taken
                           at the end of each step (Eq. e_recharge_of_param);
                           needs n_xi = 3 */
  int krylov_iters;     /* 0 (default): each defect-correction iteration
                           applies `vcycles` V-cycles. k > 0: it runs k
                           iterations of BiCGStab on the finest-level
                           system instead, right-preconditioned by one
                           V-cycle per application (two per iteration).
                           k = 1 is rejected: with a single BiCGStab step
                           per correction some samples of the smooth field
                           model broke down (non-finite residual) */
  double adjoint_rtol;  /* henry_adjoint: each transposed step system
                           J_n^T lam = rhs is solved until its FP64 residual
                           norm is below adjoint_rtol times its initial one,
                           or, once below 1e3 adjoint_rtol times it, an
                           iteration reduces it by less than half (the FP64
                           rounding floor). Default 1e-14 */
  int res_rows;         /* rows of cells one thread of the residual/Jacobian
                           kernel walks (its tile height per row group),
                           1..64; 0 (default): 8. A schedule knob for the
                           autotuner: it trades blocks per sample against
                           recomputed faces at tile edges */
  int discretisation;   /* HENRY_DISC_CELL (default) or HENRY_DISC_VERTEX:
                           the vertex-centred variant of section 2.3 (box
                           method with partial upwinding; see
                           henry_residual_jacobian_vc). With the vertex
                           variant henry_solve, henry_sample_pairs and
                           henry_sample_levels return nodal fields c_out,
                           p_out of shape [B][ny_l + 1][nx_l] (the unknown
                           nodes i = 0..nx_l-1; x = Lx is Dirichlet);
                           henry_adjoint, henry_solve_series, henry_fields
                           and henry_time_kernel return HENRY_E_UNSUPPORTED */
  int mg_tb_cells;      /* largest multigrid level (cells per sample) above
                           the shared-memory kernel whose V-cycle legs run
                           temporally blocked: the nu1 pre-sweeps and the
                           residual restriction in one launch, the
                           prolongation and the nu2 post-sweeps in another,
                           a tile of cells plus a halo per block (needs
                           nu1, nu2 >= 1; results bitwise those of one launch
                           per operation). 0 (default): one launch per
                           operation. A schedule knob for the autotuner */
  int jac_keep;         /* with jac_lag > 0: 1 keeps the operators across
                           time steps (rebuilt before the first iteration of a
                           solve and after any iteration that reduced the
                           residual by less than jac_lag), 0 (default)
                           rebuilds them at the first iteration of every step.
                           Changes the iterations, not the converged
                           solution; henry_adjoint's forward always rebuilds
                           per step. A schedule knob for the autotuner */
} henry_config;

#define HENRY_DISC_CELL 0        /* cell-centred, full upwind (default)      */
#define HENRY_DISC_VERTEX 1      /* vertex-centred, exponentially fitted
                                    partial upwind, the paper's Dirichlet
                                    boundaries                               */

typedef struct henry_ctx henry_ctx; /* opaque: owns device workspaces */

/* Running per-QoI statistics of one MLMC level: count, mean and sum of
 * squared deviations (M2) of g_l and of g_l - g_{l-1} (g_{-1} = 0). */
typedef struct henry_level_stats {
  int64_t n;
  double mean_f[HENRY_NQ], m2_f[HENRY_NQ];
  double mean_d[HENRY_NQ], m2_d[HENRY_NQ];
} henry_level_stats;

/* Fill *cfg with the default configuration: Table 1 physics (rho1 =
 * 1024.99, D = 18.8571e-6, K0 = 1.020408e-9, phi0 = 0.35, mu = 1e-3,
 * g = 9.8), q0 = 6.6e-5 m/s, [0,2]x[0,1], T = 43200 s, 32x16 cells and 24
 * steps on level 0, 2 levels, 3 random variables, FP64 multigrid, rtol
 * 1e-10, atol 1e-11, stagnation tolerance 1e-9, maxit 30, V(2,2), 3 V-cycles
 * per iteration, extrapolated Newton guess on, shared-memory V-cycle fusion
 * on, cluster V-cycle off (measured slower on the configured workloads). */
int henry_default_config(henry_config* cfg);

/* Validate *cfg and create a context for levels 0..cfg->nlevels-1.
 * Device workspaces are allocated lazily, per (level, role), on the first
 * call that needs them and grown when a larger batch arrives; growing
 * synchronises the device. The device current at creation is used.
 * Errors: HENRY_E_INVALID, HENRY_E_UNSUPPORTED (a level's grid does not
 * coarsen to at most 32 cells with an even nx on every multigrid level). */
int henry_create_levels(const henry_config* cfg, henry_ctx** out);

/* Free the context and its device memory (synchronises the device). */
void henry_destroy(henry_ctx* ctx);

/* Batched deterministic solves of one level (section 2.3): for each of the
 * B samples, the random fields from xi (and the optional per-cell log-K
 * perturbation), then r_l implicit Euler steps from c = 0, then the QoIs.
 *   xi      device [B][n_xi]
 *   logk    device [B][ny_l][nx_l] added to log K, or NULL
 *   q       device [B][HENRY_NQ] out
 *   c_out   device [B][ny_l][nx_l] out (c at T), or NULL
 *   p_out   device [B][ny_l][nx_l] out (p at T), or NULL
 *   status  device int [B] out (HENRY_S_* bits)
 *   iters   device int [B] out (total defect-correction iterations), or NULL
 * B may be 0 (no work). Errors: HENRY_E_INVALID, HENRY_E_CUDA, HENRY_E_NOMEM. */
int henry_solve(henry_ctx* ctx, int level, const double* xi, const double* logk, int B,
                double* q, double* c_out, double* p_out, int* status, int* iters,
                void* stream);

/* henry_solve with the QoI time series (section 4, test A3: realisations
 * and quantiles of Q_FW(t) and Q_S(t)): after steps every, 2 every, ..., of
 * the r_l steps of the level, the HENRY_NQ QoIs of every sample.
 *   q_series  device [B][r_l / every][HENRY_NQ] out (step k*every in slot k-1)
 *   q         device [B][HENRY_NQ] out (at T);  status as henry_solve
 * Errors: HENRY_E_INVALID (every < 1, NULL), HENRY_E_CUDA, HENRY_E_NOMEM. */
int henry_solve_series(henry_ctx* ctx, int level, const double* xi, const double* logk, int B,
                       int every, double* q_series, double* q, int* status, void* stream);

/* MLMC level pair (Eq. A): the same xi drives a level-l solve and a
 * level-(l-1) solve. At level 0 only the fine solve runs and q_coarse,
 * c_coarse must be NULL.
 *   q_fine, q_coarse   device [B][HENRY_NQ] out
 *   c_fine             device [B][ny_l][nx_l] out, or NULL
 *   c_coarse           device [B][ny_{l-1}][nx_{l-1}] out, or NULL
 *   status             device int [B] out, OR of both solves' bits
 * The coarse result is bitwise equal to henry_solve at level l-1 on the same
 * xi. The coarse half runs on an internal stream forked from `stream` (and
 * joined back before the call's last operation), concurrently with the fine
 * half. Errors as henry_solve. */
int henry_sample_pairs(henry_ctx* ctx, int level, const double* xi, int B,
                       double* q_fine, double* q_coarse, double* c_fine, double* c_coarse,
                       int* status, void* stream);

/* Multigrid schedule of one MLMC level (the autotuner's knobs; meanings as
 * the henry_config fields of the same names). */
typedef struct henry_schedule {
  int vcycles, nu1, nu2, mg_small_cells, jac_lag, res_rows, mg_tb_cells, jac_keep;
} henry_schedule;

/* Give MLMC level `level` its own schedule: the fine solves of level l
 * (henry_solve, the fine half of the pairs of level l) and the coarse half
 * (level l-1) of the pairs of level l use it; the context's config is kept
 * for every other field. Synchronises the device and drops that level's
 * workspaces (rebuilt on the next call). Errors: HENRY_E_INVALID (bad
 * level or out-of-range knob), HENRY_E_CUDA. */
int henry_set_schedule(henry_ctx* ctx, int level, const henry_schedule* sched);

/* One level's pairs for henry_sample_levels; arguments as henry_sample_pairs. */
typedef struct henry_level_batch {
  int level, B;
  const double* xi;   /* device [B][n_xi]                                    */
  double* q_fine;     /* device [B][HENRY_NQ] out                            */
  double* q_coarse;   /* device [B][HENRY_NQ] out; NULL at level 0           */
  double* c_fine;     /* device [B][ny_l][nx_l] out, or NULL                 */
  double* c_coarse;   /* device [B][ny_{l-1}][nx_{l-1}] out, or NULL         */
  int* status;        /* device int [B] out, OR of both solves' bits         */
} henry_level_batch;

/* The level pairs of one MLMC round, several levels at once (Eq. A, one
 * batch per level, at most one batch per level): results bitwise equal to
 * henry_sample_pairs called for each batch. With the graph loop (the
 * default) every solver involved advances together: the implicit steps of
 * one coarse (level-0) time step -- 2^l steps of each level-l solve and
 * 2^(l-1) of its coarse half, each step with its device-side Newton loop --
 * form ONE CUDA graph whose branches run concurrently, launched nt0 times
 * on `stream` (one launch per coarse step for all levels); the field
 * set-up before and the QoIs after are plain launches on `stream`. The
 * graph is kept and relaunched while the levels, batches and workspaces are
 * unchanged. With the host loop the batches run one level after another.
 * Errors: HENRY_E_INVALID (n outside 1..nlevels, a level twice, B outside
 * 0..HENRY_MAX_BATCH, NULL arrays), HENRY_E_CUDA, HENRY_E_NOMEM. */
int henry_sample_levels(henry_ctx* ctx, const henry_level_batch* batches, int n, void* stream);

/* Discrete adjoint of one QoI through the implicit Euler time stepping
 * (section 2.3), for B samples of level `level`: with R^n(u^n, u^{n-1}) = 0
 * the residual of step n and Q = Q(u^r),
 *   J_r^T lam_r = dQ/du^r,  J_n^T lam_n = -(dR^{n+1}/du^n)^T lam_{n+1},
 *   dQ/dtheta = -sum_n (dR^n/dtheta)^T lam_n,
 * for theta = xi (through the random fields of henry_fields) and the
 * per-cell log-permeability perturbation. The forward stores its state every
 * ckpt_every steps and the backward recomputes each segment from its
 * checkpoint (bitwise the forward's states); each transposed step system is
 * solved by FP64 defect correction preconditioned by the multigrid of the
 * context's precision applied to the transposed operators (relative
 * residual 1e-11).
 *   qoi_id     0 = Q_S (int c rho), 2 = toe (int c (Lx - x)); others invalid
 *   xi         device [B][n_xi];  logk device [B][ny][nx] or NULL
 *   q          device [B] out: the QoI at T
 *   dq_dxi     device [B][n_xi] out
 *   dq_dlogk   device [B][ny][nx] out, or NULL
 *   status     device int [B] out (HENRY_S_* bits of forward and adjoint)
 * Synchronises the stream once per defect-correction iteration of the
 * backward pass. Both field models: with field_model 1 the inflow
 * sensitivity of each step carries that step's recharge factor. Errors as
 * henry_solve. */
int henry_adjoint(henry_ctx* ctx, int level, const double* xi, const double* logk, int B,
                  int qoi_id, int ckpt_every, double* q, double* dq_dxi, double* dq_dlogk,
                  int* status, void* stream);

/* Merge one batch into the running statistics of a level (Def. of Y_l and
 * V_l; V_l = m2_d / (n - 1)). Samples with status != 0 are skipped.
 * Welford per thread in sample order, then a fixed pairwise Chan merge tree
 * on the device (deterministic for a given B), then a Chan merge into
 * *inout on the host. Synchronous: returns when the batch is merged.
 *   q_fine    device [B][HENRY_NQ]
 *   q_coarse  device [B][HENRY_NQ] or NULL (level 0: g_{-1} = 0)
 *   status    device int [B] or NULL (all samples valid)
 *   inout     host, running state updated in place */
int mlmc_level_stats(henry_ctx* ctx, int level, const double* q_fine, const double* q_coarse,
                     int B, const int* status, henry_level_stats* inout, void* stream);

/* Per-cell running statistics of the c field of one level (section 4, Test
 * A1): for every cell of the level-l grid, Welford over the batch in sample
 * order of g = c_l and of d = c_l - P0 c_{l-1}, P0 the piecewise-constant
 * transfer from the level-(l-1) grid. Samples with status != 0 are skipped.
 *   c_fine    device [B][ny_l][nx_l];  c_coarse device [B][ny_{l-1}][nx_{l-1}] or NULL
 *   n         device int64 [ny_l*nx_l]  running count (all cells equal)
 *   mean_f, m2_f, mean_d, m2_d  device [ny_l][nx_l], updated in place */
int mlmc_field_stats(henry_ctx* ctx, int level, const double* c_fine, const double* c_coarse,
                     int B, const int* status, int64_t* n, double* mean_f, double* m2_f,
                     double* mean_d, double* m2_d, void* stream);

/* Per-cell exceedance counts of the c field of one level (section 4: the
 * probability that the salt mass fraction at a location exceeds a threshold,
 * P(c(T, x) > threshold), estimated as count / n by the caller):
 * count[cell] += number of samples b with status[b] == 0 and
 * c[b][cell] > threshold. Integer counts, so the result does not depend on
 * how the samples are batched. Asynchronous on `stream`.
 *   c         device [B][ny_l][nx_l]
 *   status    device int [B] or NULL (all samples valid)
 *   count     device int64 [ny_l*nx_l], accumulated in place (caller zeroes it)
 * Errors: HENRY_E_INVALID (bad level, B < 0, NaN threshold, NULL), HENRY_E_CUDA. */
int mlmc_field_exceedance(henry_ctx* ctx, int level, const double* c, int B, const int* status,
                          double threshold, int64_t* count, void* stream);

/* Evaluate the FP64 finite-volume residual of one implicit Euler step and,
 * optionally, its exact Jacobian, for B states on an nx x ny grid (Eqs.
 * 1-5 integrated over each cell). Context-free; for tests and tools.
 *   phi, K          device [B][ny][nx] cell porosity and permeability
 *   qin             device [B][ny] left-side inflow velocity per row [m/s]
 *   p, c, c_old     device [B][ny][nx]
 *   R               device [B][2][ny][nx] out: R_p then R_c
 *   J               device [B][20][ny][nx] out or NULL: per cell the 2x2
 *                   blocks (row = equation p|c, column = variable p|c,
 *                   stored pp, pc, cp, cc) of d R_P / d u_Q for
 *                   Q = P, W, E, S, N (in that order); blocks of missing
 *                   neighbours are zero.
 * Errors: HENRY_E_INVALID, HENRY_E_CUDA. */
int henry_residual_jacobian(const henry_config* cfg, int nx, int ny, double tau, int B,
                            const double* phi, const double* K, const double* qin,
                            const double* p, const double* c, const double* c_old,
                            double* R, double* J, void* stream);

/* henry_residual_jacobian without any device allocation. The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory during the call -- processes whose device memory is
 * entirely owned by another allocator (a framework's caching pool or a
 * fixed memory budget, where a cudaMalloc of our own could fail or fragment
 * it), and latency-critical loops where an allocation could synchronise the
 * device or fail part-way. Arguments, layouts, outputs and errors are those
 * of henry_residual_jacobian; the caller still provides every input and
 * output buffer.
 * Scratch: 5 doubles per cell and sample in a file-scope device array of
 * 2^20 doubles (8 MiB), held by every GPU that loads the library until the
 * process exits; B * nx * ny above 209715 cells is rejected with
 * HENRY_E_INVALID (as is B > HENRY_MAX_BATCH). The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that
 * device current and caches it for the process; make that first call
 * before any stream capture. The cached address does not survive
 * cudaDeviceReset() (the module is reloaded at a new address): do not call
 * this entry point on a device after resetting it. Every call shares the array and it keeps
 * the last call's contents; each call writes every scratch element it reads
 * before reading it, so nothing needs to start at zero. Calls that overlap
 * on the GPU (on different streams, or from different host threads) race on
 * the array and must be serialised by the caller. */
int henry_residual_jacobian_noalloc(const henry_config* cfg, int nx, int ny, double tau, int B,
                                    const double* phi, const double* K, const double* qin,
                                    const double* p, const double* c, const double* c_old,
                                    double* R, double* J, void* stream);

/* The residual of one implicit Euler step of the vertex-centred variant
 * (section 2.3: vertex-centred finite volumes, partial upwinding of the
 * convective terms) and, optionally, its exact Jacobian, for B states on
 * the nodes of an nx x ny cell grid. Context-free; for tests and tools.
 * Scheme (this library's reading; the paper refers to ug4 for it): node
 * boxes clipped to the domain; the random field of `xi` (field model and
 * n_xi of cfg) evaluated at integration points -- phi at the quarter-cell
 * centres of each box for its storage, K and phi at the midpoints of the
 * two half segments of each box face for its transmissibility and
 * diffusive conductance; two-point Darcy fluxes with the mean density in
 * the gravity and diffusion terms; advected rho and rho c weighted by
 * w = (1 + alpha(Pe) sgn Q) / 2, alpha(Pe) = coth(Pe/2) - 2/Pe (exponential
 * fitting, Allen-Southwell / Il'in), Pe = |Q| / (diffusive conductance);
 * boundaries of section 2.1: x = Lx Dirichlet p = rho1 g (Ly - y), c = 1
 * (not unknowns), x = 0 inflow rho0 q_in and c = 0, its salt row being
 * (V phi0 rho0 / tau) c; top and bottom closed.
 *   xi              device [B][n_xi]
 *   p, c, c_old     device [B][ny+1][nx]: nodes i = 0..nx-1, j = 0..ny;
 *                   p is the full pressure
 *   R               device [B][2][ny+1][nx] out: R_p then R_c
 *   J               device [B][20][ny+1][nx] out or NULL: blocks P, W, E,
 *                   S, N of d R_P / d u_Q as in henry_residual_jacobian
 * nx must be even and >= 2, ny >= 1, 0 <= B <= HENRY_MAX_BATCH. Allocates
 * its scratch (stream-ordered). Errors: HENRY_E_INVALID, HENRY_E_CUDA. */
int henry_residual_jacobian_vc(const henry_config* cfg, int nx, int ny, double tau, int B,
                               const double* xi, const double* p, const double* c,
                               const double* c_old, double* R, double* J, void* stream);

/* Random fields of the level-l grid for B samples (cell centres):
 *   phi = phi0 (1 + 0.1 xi1 cos(pi x/2) sin(pi y) [+ 0.05 xi4 cos(pi x) sin(2 pi y)])
 *   K   = K0 exp(0.5 xi2 sin(pi x/2) cos(pi y) [+ 0.05 xi5 sin(pi x) cos(2 pi y)] + logk)
 *   qin = q0 (1 + 0.1 xi3 [+ 0.05 xi6 cos(pi y)])
 * (the bracketed terms when n_xi = 6). Outputs device [B][ny][nx] and
 * [B][ny]. logk may be NULL. */
int henry_fields(henry_ctx* ctx, int level, const double* xi, const double* logk, int B,
                 double* phi, double* K, double* qin, void* stream);

/* Grid of level l: *nx, *ny, *nt (steps), *n_mg (multigrid levels). */
int henry_level_info(const henry_ctx* ctx, int level, int* nx, int* ny, int* nt, int* n_mg);

/* Diagnostics: copy an internal array of the solver that serves `level`
 * (role 0: fine solves and level-l halves of pairs; role 1: the level-(l-1)
 * halves of pairs, addressed by their own level l-1) for multigrid level
 * mg_level (0 = coarsest). what: 0 J [B][24][ncell] (colour-split planes:
 * inverse diagonal block, W, E, S, N blocks row-scaled by it, diagonal
 * block),
 * 1 b, 2 x ([B][2][ncell], colour-split), 3 p, 4 c, 5 phi, 6 K ([B][ncell],
 * natural), 7..10 face constants tx, dx, ty, dy, 11..12 face fluxes of the
 * linearisation point qx (east faces; the right side in the last column),
 * qy (north faces), 13 the BiCGStab scalars of the last defect correction
 * ([B][8] FP64: rho, alpha, omega, beta, then unused; only with
 * krylov_iters > 0). Element size is 4 bytes for J, b, x with FP32
 * multigrid, else 8. Copies min(bytes, size) bytes
 * to the device or host pointer dst and synchronises the device.
 * Errors: HENRY_E_INVALID if the solver does not exist yet or an index is
 * out of range. */
int henry_debug_copy(henry_ctx* ctx, int level, int role, int mg_level, int what, void* dst,
                     int64_t bytes);

/* Kernel timing for roofline reports: replays one kernel of the solver that
 * served `level` (role as in henry_debug_copy) on its current workspace,
 * `reps` times on `stream`, after one untimed launch; the solver must have
 * run a solve before (the replay uses that solve's batch).
 * which: 0 red half-sweep of the block Gauss-Seidel smoother on the finest
 * multigrid level; 1 the FP64 residual + Jacobian kernel of the finest level;
 * 2 the residual-only evaluation of that kernel (iterations that reuse
 * their operators).
 * flush, flush_bytes: optional device buffer (NULL, 0 for none). When
 * given, every timed launch is preceded by a write of flush_bytes bytes to
 * it (larger than the L2 cache: each launch starts cold) and is timed by its
 * own pair of CUDA events, the flush excluded; without it the reps launches
 * run back to back between two events.
 * Outputs the average duration of one launch [ms], its algorithmic DRAM
 * bytes (the method's per-cell figures: smoother 26 values of the multigrid
 * type per updated cell -- operator 20, b 2, x read 2 and written 2;
 * residual + Jacobian 56 B + 20 values per cell, residual only 56 B) and
 * its FP64 + FP32
 * floating point operations (FMA = 2). Synchronises the stream. The replay
 * changes the workspace (not the caller's outputs). */
int henry_time_kernel(henry_ctx* ctx, int level, int role, int which, int reps, void* flush,
                      int64_t flush_bytes, void* stream, double* avg_ms, double* bytes,
                      double* flops);

/* Measured FP64 FMA throughput of this GPU [TFLOP/s], the denominator of
 * the FP64-pipe fraction in roofline reports (GB300 has no published
 * dense-FP64 figure to use instead): one launch of 152 x 8 blocks of 256
 * threads, each running 16 independent FMA chains of 512 * reps steps,
 * timed with CUDA events on `stream` after one warm-up launch; reps 1..1000.
 * Allocates and frees a small result buffer (stream-ordered). Synchronises
 * the stream. */
int henry_probe_fp64(int reps, void* stream, double* tflops);

/* Device kernel launches issued by this context since creation (counts
 * every launch, including those replayed inside CUDA graphs). */
int64_t henry_launch_count(const henry_ctx* ctx);

const char* henry_strerror(int code);
const char* henry_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HENRY_H */
