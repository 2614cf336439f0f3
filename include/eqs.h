/*
 * eqs.h - C ABI of the GB300 explicit Runge-Kutta-Chebyshev solver for
 * nonlinear electro-quasistatic (EQS) fields on P1 tetrahedra.
 *
 * Method (Richter, Schoeps, Clemens, "GPU Accelerated Explicit Time
 * Integration Methods for Electro-Quasistatic Fields"):
 *   Eq. 1  div(kappa(|grad phi|) grad phi) + div(eps grad dphi/dt) = 0
 *   Eq. 2  M dx/dt + K(x) x = b    (P1 finite elements)
 *   Sec. II   explicit RKC time stepping; every stage needs one solve with
 *             the constant Laplace-type matrix M (multiple right-hand sides)
 *   Sec. III  K(x)x is formed tet by tet without assembling K(x)
 *   Sec. IV   the M-solves use CG with a constant AMG preconditioner and a
 *             start vector estimated from earlier solutions
 *
 * Conventions (all entry points):
 *  - Every call returns eqs_status; EQS_OK == 0, errors are negative.  The
 *    library never throws or aborts; eqs_last_error() returns a text for the
 *    last failing call on a context.
 *  - "host" pointers are read (or written) during the call only and are
 *    never retained.  "device" pointers are CUDA global-memory pointers owned
 *    by the caller; the library never frees them.  Everything the library
 *    allocates is owned by the context and released by eqs_destroy().
 *  - Node vectors of length n_nodes are in the caller's (mesh) node order.
 *    "Free" vectors of length n_free hold the free (non-Dirichlet) nodes in
 *    ascending mesh-node order.
 *  - Device work is enqueued on the context stream (eqs_set_stream; initially
 *    the legacy default stream) and is asynchronous unless stated.
 *  - Call order: eqs_mesh_create -> eqs_set_materials -> eqs_amg_setup ->
 *    apply / solve / step; otherwise EQS_ERR_STATE.
 */
#ifndef EQS_H
#define EQS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct eqs_ctx eqs_ctx;

typedef enum {
  EQS_OK = 0,
  EQS_ERR_ARG = -1,     /* invalid argument (null pointer, size, range)      */
  EQS_ERR_MESH = -2,    /* inverted/degenerate tet, bad index, bad tag       */
  EQS_ERR_CUDA = -3,    /* a CUDA runtime call failed                        */
  EQS_ERR_NOCONV = -4,  /* CG reached max_iter before the tolerance          */
  EQS_ERR_TIMEOUT = -5, /* a bounded device wait (grid barrier) gave up       */
  EQS_ERR_NAN = -6,     /* non-finite value in an input or residual          */
  EQS_ERR_STATE = -7    /* call order violated                               */
} eqs_status;

/* Material law of Eq. 1: eps = eps0 * eps_r (eps0 = 8.8541878128e-12 F/m) and
 * kappa(E) = kappa_lo + (kappa_hi - kappa_lo) / (1 + exp(-(E - E0) / w)),
 * E = |grad phi| per tet.  kappa_hi == kappa_lo marks a constant
 * conductivity (E0 and w are then ignored). */
typedef struct {
  double eps_r, kappa_lo, kappa_hi, E0, w;
} eqs_material;

typedef enum {
  EQS_PREC_FP64 = 0,  /* every kernel in FP64                                */
  EQS_PREC_MIXED = 1  /* FP32 element kernel and AMG V-cycle (coarsest
                         level: FP32 dense inverse, or FP32 pairs with
                         eqs_opts.coarse_split 1); FP64 CG residual, dot
                         products and RKC recurrence                        */
} eqs_precision;

typedef enum {
  EQS_GUESS_PREV = 0, /* start vector = previous M-solve solution           */
  EQS_GUESS_MLP = 1,  /* learned per-node network (eqs_guess_* calls)       */
  EQS_GUESS_ZERO = 2, /* start vector = 0                                   */
  EQS_GUESS_SPE = 3,  /* subspace projection extrapolation over the last
                         spe_n solutions (Sec. IV, Eq. 4-5)                 */
  EQS_GUESS_POD = 4,  /* POD-MOR (Sec. IV, "MOR"): the first pod_k
                         solutions are the snapshots, their leading pod_m
                         POD modes span the projection of Eq. 5, computed
                         once; earlier solves start from the previous one  */
  EQS_GUESS_POD2 = 5, /* rolling POD-MOR (Sec. IV, "MOR2"): a solution whose
                         solve took more than pod_min_iters iterations
                         replaces the oldest of pod_k snapshots and the
                         basis is recomputed                                */
  EQS_GUESS_SPE_MLP = 6 /* the SPE start x0 corrected along the learned
                         network's direction by an M-norm line search (its
                         second mode, inputs: solution increments)          */
} eqs_guess_mode;

/* Options of eqs_amg_setup (fill with eqs_opts_default). */
typedef struct {
  int precision;       /* eqs_precision                                      */
  double theta;        /* strength threshold on level 0 (halved per level)   */
  int coarse_max;      /* stop coarsening at <= coarse_max rows              */
  int max_levels;      /* hierarchy depth limit                              */
  int cheb_degree;     /* Chebyshev smoother degree (1..4), pre and post     */
  double cheb_alpha;   /* smoothing interval [lambda/alpha, lambda]          */
  double rtol;         /* M-solve stopping test ||R - M z||/||R|| <= rtol    */
  int max_iter;        /* CG iteration limit per solve                       */
  int guess;           /* eqs_guess_mode                                     */
  int flexible;        /* 1: Polak-Ribiere CG                                */
  int persistent;      /* 1: each M-solve is one cooperative persistent
                          kernel (grid barriers); 0: one kernel per CG/V-cycle
                          phase inside a device-side graph loop               */
  int blocks_per_sm;   /* CTAs per SM of the persistent solve (0: 1)         */
  int spe_n;           /* solutions spanning the SPE subspace (1..6, def. 4) */
  int host_loop;       /* 1: eqs_rkc_step launches the same kernels directly
                          and drives each CG loop from the host (reads the
                          convergence flag after every iteration) instead of
                          replaying a graph; for profilers that cannot enter
                          graph loops.  Default 0.                            */
  long long barrier_polls; /* wait budget of one grid barrier of the persistent
                          solve, in polls: 0 = default (2^22, about a second),
                          < 0 = no waiting at all (every wait gives up at
                          once; for testing the EQS_ERR_TIMEOUT path)        */
  int split_m;         /* EQS_PREC_MIXED only: 1 (default) forms the CG
                          operator product M z of the FP32 preconditioned
                          residual z with M held as two FP32 parts and an
                          error-free FP32-pair row sum (accuracy a few
                          2^-48 of sum |m_ij z_j|, no FP64 multiply per
                          non-zero); 0 uses FP64 M.  Ignored in FP64 mode.  */
  int pod_k;           /* POD snapshots (1..16, default 12)                  */
  int pod_m;           /* POD modes kept (1..pod_k, default 6); fewer when
                          the snapshots have lower numerical rank           */
  int pod_min_iters;   /* EQS_GUESS_POD2: a solution becomes a snapshot when
                          its solve needed more CG iterations (default 3)   */
  int fill_lanes;      /* 1 (default): rows of AMG levels too small to fill
                          the GPU get lane groups (up to 32 lanes per row)
                          until they do; 0: lanes by row length only (for
                          contexts that run together in a batch, where each
                          instance owns a few CTAs)                         */
  int coarse_split;    /* EQS_PREC_MIXED only: 0 (default) applies the FP32
                          rounding of the coarsest level's dense inverse with
                          FP32 row sums; 1 applies it as two FP32 parts with
                          FP32-pair row sums (twice the bytes).  Ignored in
                          FP64 mode.                                        */
  int defer_sums;      /* bit 0 (EQS_PREC_MIXED, degree-1 smoother, >= 2
                          levels): the CG dot products of the fused smoothing
                          pass and of the operator pass are left as
                          per-block partial sums that every block of the
                          consuming kernel adds in the same fixed order (no
                          grid-wide ticket between the kernels); bit 1
                          (EQS_GUESS_SPE in eqs_rkc_step): the same for the
                          SPE Gram pass, whose sums one block then adds
                          before the small solve.  Cleared
                          bits form the sums in the producer's last block.
                          0..3, default 2 (bit 1 only: measured faster; the
                          CG hand-over was not).  Same results up to the
                          order of the additions.                           */
} eqs_opts;

#define EQS_MAX_STAGES 64

/* Per-step statistics (filled after a device synchronisation). */
typedef struct {
  int s;                        /* stages of the step                         */
  int total_iters;              /* CG iterations summed over the s solves     */
  int max_iters;                /* largest CG iteration count of one solve    */
  int iters[EQS_MAX_STAGES];    /* CG iterations of solve j = 0..s-1          */
  double max_relres;            /* largest final ||r||/||R|| of the s solves  */
  int status;                   /* EQS_OK or EQS_ERR_NOCONV                   */
  int64_t launches;             /* kernels the step launched (graph kernel
                                   nodes outside loops + loop-body kernel
                                   nodes x CG iterations)                    */
  int guess_kept;               /* solves that started from the learned guess
                                   (EQS_GUESS_MLP, EQS_GUESS_SPE_MLP; else 0) */
} eqs_step_stats;

/* Fill *o with the defaults (precision FP64, theta 0.08, coarse_max 500,
 * max_levels 10, degree 2, alpha 30, rtol 1e-8, max_iter 500, GUESS_PREV,
 * flexible 1, persistent 0, blocks_per_sm 1, spe_n 4, host_loop 0,
 * barrier_polls 0, split_m 1, pod_k 12, pod_m 6, pod_min_iters 3,
 * fill_lanes 1, coarse_split 0, defer_sums 2). */
void eqs_opts_default(eqs_opts* o);

/* Create a context from a tetrahedral mesh (Eq. 2 discretisation input).
 * xyz: host, n_nodes x 3 doubles, node-major (x0 y0 z0 x1 ...), metres.
 * tets: host, n_tets x 4 int32 node indices (0-based), positively oriented
 *   (det[p1-p0, p2-p0, p3-p0] > 0); an inverted or flat tet is rejected.
 * node_tag: host, n_nodes bytes: 0 free, 1 Dirichlet phi = 0,
 *   2 Dirichlet phi = g(t) (eqs_set_dirichlet).
 * Errors: EQS_ERR_ARG (null/size), EQS_ERR_MESH (index out of range,
 *   inverted or flat tet, non-finite coordinate, tag > 2, no free node).
 * Host work only; the GPU is first touched by eqs_amg_setup.
 * *out is NULL on error. */
eqs_status eqs_mesh_create(const double* xyz, int64_t n_nodes, const int32_t* tets,
                           int64_t n_tets, const uint8_t* node_tag, eqs_ctx** out);

/* Quadratic (P2) mesh (Section V's 2nd order ansatz functions): as
 * eqs_mesh_create with tets10: host, n_tets x 10 int32 node indices, the
 * four vertices (positively oriented) followed by the midpoint nodes of the
 * edges (0,1), (0,2), (0,3), (1,2), (1,3), (2,3) (straight edges).  K(x)x
 * and M use the ten quadratic shape functions with the symmetric 4-point
 * quadrature rule of degree 2 (the conductivity is evaluated at each
 * quadrature point).  The single-trajectory paths (apply, solve, step,
 * adaptive step, start vectors) accept it; the ensemble and batched serving
 * take linear tets only. */
eqs_status eqs_mesh_create_p2(const double* xyz, int64_t n_nodes, const int32_t* tets10,
                              int64_t n_tets, const uint8_t* node_tag, eqs_ctx** out);

/* Material of every tet (Eq. 1 coefficients).  tet_mat: host, n_tets bytes,
 * values < n_mat; mats: host array of n_mat (1..255) laws.
 * Errors: EQS_ERR_ARG, EQS_ERR_MESH (id out of range), EQS_ERR_STATE. */
eqs_status eqs_set_materials(eqs_ctx* ctx, const uint8_t* tet_mat, int n_mat,
                             const eqs_material* mats);

/* Drive of the tag-2 nodes: g(t) = V0 sin(2 pi freq_hz t + phase) [V]
 * (the inhomogeneous Dirichlet data that makes up b in Eq. 2). */
eqs_status eqs_set_dirichlet(eqs_ctx* ctx, double V0, double freq_hz, double phase);

/* Assemble M (Eq. 2: eps-weighted P1 Laplacian, free-free block after
 * Dirichlet elimination) and build the smoothed-aggregation AMG hierarchy
 * once on the host, then upload it (Sec. II: the preconditioner of the
 * constant M is set up once and reused for every right-hand side).
 * opts may be NULL (defaults).  Calling it again rebuilds everything. */
eqs_status eqs_amg_setup(eqs_ctx* ctx, const eqs_opts* opts);

/* y = K(x) x for all nodes, before any boundary condition (Sec. III:
 * formed tet by tet, never assembling K).  x, y: device, n_nodes doubles,
 * mesh order; y is overwritten.  Uses the precision chosen at setup. */
eqs_status eqs_apply_K(eqs_ctx* ctx, const double* x, double* y);

/* y = K(x) x as eqs_apply_K computes it (the same element kernel; results
 * differ only by the order of the atomic additions), for callers that must
 * not allocate device memory during the call: code running where cudaMalloc
 * is not allowed or not wanted, e.g. under a fixed device-memory budget that
 * was claimed up front, or on a real-time or callback path where an
 * allocation could block or fail.  The paper has no counterpart; this is a
 * library convenience.  The call allocates nothing: its scratch (the
 * potential and the result staged in the library's internal node order) is
 * a static 12 MiB device array inside the library, which every GPU that
 * loads the library holds until the process exits.  Limit: n_nodes <=
 * 524288, else EQS_ERR_ARG.  The first call on a device looks up the
 * array's address and keeps it for the rest of the process; make that first
 * call before any stream capture.  A device reset (cudaDeviceReset) may move
 * the array, so after one this entry point must not be used again in that
 * process.  All calls share the one array, so calls whose work overlaps on
 * the GPU (other streams, other threads, several contexts on one device)
 * race; serialise them.  x, y: device, n_nodes doubles, mesh order; the
 * context's device must be current.  Asynchronous on the context stream. */
eqs_status eqs_apply_K_static(eqs_ctx* ctx, const double* x, double* y);

/* Solve M_ff z = rhs for nrhs right-hand sides (Sec. IV) by AMG-PCG.
 * rhs: device, n_free x nrhs doubles, column-major (column k at
 *   rhs + k*n_free).  z: device, same shape; on entry the start vectors,
 *   on exit the solutions.  rtol <= 0 uses the setup value.
 * iters_out: host, nrhs ints or NULL.  Synchronises the stream.
 * Returns EQS_ERR_NOCONV if any column hit max_iter (z then holds the last
 * iterate). */
eqs_status eqs_solve_M(eqs_ctx* ctx, const double* rhs, double* z, int nrhs, double rtol,
                       int* iters_out);

/* Apply the AMG V-cycle once: z = B r (device, n_free doubles each). */
eqs_status eqs_vcycle(eqs_ctx* ctx, const double* r, double* z);

/* y = M_ff x (device, n_free doubles each). */
eqs_status eqs_spmv_M(eqs_ctx* ctx, const double* x, double* y);

/* y = M_ff x for an FP32 x (device, n_free floats) through the split-M
 * product of the mixed CG operator (see eqs_opts.split_m); y: device,
 * n_free doubles.  EQS_ERR_STATE unless the context was set up in
 * EQS_PREC_MIXED with split_m 1. */
eqs_status eqs_spmv_M32(eqs_ctx* ctx, const float* x, double* y);

/* One RKC step of s stages (Sec. II; scheme of its ref. [9], damping 2/13)
 * from time t to t + dt.  x: device, n_nodes doubles, mesh order: on entry
 * x(t) (Dirichlet entries are ignored and replaced by g(t)), on exit
 * x(t + dt) with Dirichlet entries g(t + dt).  2 <= s <= EQS_MAX_STAGES.
 * The whole step runs as one CUDA graph (cached per s) whose CG loops are
 * device-side while-loops.  stats: host or NULL; when non-NULL the call
 * synchronises and returns EQS_ERR_NOCONV if a solve did not converge. */
eqs_status eqs_rkc_step(eqs_ctx* ctx, double* x, double t, double dt, int s,
                        eqs_step_stats* stats);

/* ---- Adaptive stepping (the paper runs RKC with a local time-integration
 * error below 1e-2; ref. [9] controls it).  One accepted step from t: the
 * number of stages is the smallest s <= s_max with beta_s >= h rho (rho the
 * a-priori stiffness bound of eqs_rkc_dt_bound; h is cut when s_max does
 * not suffice), the step runs as eqs_rkc_step, then F(t + h, x_new) is
 * evaluated and the local error estimate
 *   Est = (12 (x_n - x_n+1) + 6 h (F_n + F_n+1)) / 15
 * is measured in the weighted RMS norm with weights atol + rtol
 * max(|x_n|, |x_n+1|) over the free nodes.  err <= 1 accepts; otherwise x
 * is restored and the step retried with h 0.8 err^(-1/3) (factor kept in
 * [0.1, 10]).  x: device, n_nodes doubles, mesh order, in x(t), out
 * x(t + h_used).  Synchronises.  EQS_ERR_NOCONV after 50 rejected tries (x
 * restored), or when a stage solve did not converge. */
typedef struct {
  double h_used;     /* accepted step                                        */
  double h_next;     /* proposed next step (h_used 0.8 err^(-1/3), clipped)  */
  double err;        /* error norm of the accepted step (<= 1)                */
  int s;             /* stages of the accepted step                          */
  int tries;         /* 1 + rejected tries                                   */
  int total_iters;   /* CG iterations of all tries and error evaluations     */
} eqs_adapt_stats;

eqs_status eqs_rkc_adaptive_step(eqs_ctx* ctx, double* x, double t, double h_try, double atol,
                                 double rtol, int s_max, eqs_adapt_stats* out);

/* Statistics of the last eqs_rkc_step on ctx (synchronises the stream). */
eqs_status eqs_get_step_stats(eqs_ctx* ctx, eqs_step_stats* stats);

/* Largest stable step for s stages: beta_s / rho with the a-priori bound
 * rho = max over materials and E of max(kappa, d(kappa E)/dE) / eps of the
 * spectral radius of M^-1 dK/dx; returns a negative value on error. */
double eqs_rkc_dt_bound(const eqs_ctx* ctx, int s);

/* Use this CUDA stream (cudaStream_t passed as void*) for all later work;
 * NULL selects the legacy default stream (the initial setting). */
eqs_status eqs_set_stream(eqs_ctx* ctx, void* cuda_stream);

/* Sizes: any pointer may be NULL. */
eqs_status eqs_get_sizes(const eqs_ctx* ctx, int64_t* n_nodes, int64_t* n_free,
                         int64_t* n_tets);

/* AMG hierarchy description: *n_levels, and per level (host arrays of at
 * least 16 entries, may be NULL) its rows and non-zeros. */
eqs_status eqs_amg_info(const eqs_ctx* ctx, int* n_levels, int64_t* rows, int64_t* nnz);

/* Aggregate index of every row of AMG level `level` (host, rows[level]
 * int32 entries), for checking the setup. */
eqs_status eqs_amg_aggregates(const eqs_ctx* ctx, int level, int32_t* agg_out);

/* ---- Learned start vector (Sec. IV estimates start vectors from earlier
 * solutions; the per-node network is an addition without counterpart in the
 * paper).  Inputs at a free node: its last four M-solve solutions h1..h4
 * and their means over the free mesh neighbours, divided by the RMS s_h of
 * h1; network 8 -> 32 -> 32 -> 1 with exact-erf GELU, BF16 weights, FP32
 * accumulation; start vector z0 = h1 + s_h * output.  In EQS_GUESS_MLP mode
 * each solve starts from z0 unless ||R - M h1|| < ||R - M z0||.  Its second
 * mode (EQS_GUESS_SPE_MLP, eqs_guess_eval_spe) corrects the SPE start x0
 * along the network's direction instead. */

/* Select the start vector of the stage solves (an eqs_guess_mode value). */
eqs_status eqs_set_guess(eqs_ctx* ctx, int mode);

/* Set / read the 1377 FP32 master parameters, packed as W1 (32x8 row-major),
 * b1 (32), W2 (32x32), b2 (32), w3 (32), b3 (host arrays).  Setting resets
 * the Adam state. */
eqs_status eqs_guess_set_params(eqs_ctx* ctx, const float* theta, int n);
eqs_status eqs_guess_get_params(eqs_ctx* ctx, float* theta, int n);

/* Record the next `capacity` stage solutions of eqs_rkc_step (device, FP32)
 * as training data, with steps in an SPE mode also each solution's distance
 * z - x0 from its SPE start; 0 stops recording and frees the record.
 * Restarts the solution history. */
eqs_status eqs_guess_record(eqs_ctx* ctx, int64_t capacity);

/* Train on the recorded solutions: `iters` Adam steps (learning rate lr) on
 * mini-batches of `batch` (solve, node) samples drawn on the device from the
 * splitmix64 stream `seed`; target (z - h1)/s_h, MSE loss.  loss_first /
 * loss_last (host, nullable) receive the first and last mini-batch losses. */
eqs_status eqs_guess_train(eqs_ctx* ctx, int iters, int batch, float lr, uint64_t seed,
                           float* loss_first, float* loss_last);

/* Gradient of the mini-batch MSE loss for given normalised inputs X (host,
 * B x 8) and targets T (host, B) with the current BF16 weights: grad (host,
 * 1377), loss (host, nullable).  For checking the training kernel. */
eqs_status eqs_guess_grad(eqs_ctx* ctx, const float* X, const float* T, int B, float* grad,
                          float* loss);

/* n_batches Adam steps (Kingma & Ba; FP32 master weights, BF16 copies for
 * the forward and backward passes) on given mini-batches: X (host,
 * n_batches x B x 8 normalised inputs), T (host, n_batches x B targets),
 * with the training and update kernels of eqs_guess_train.  The Adam step
 * counter continues from earlier training (eqs_guess_set_params resets it).
 * losses (host, n_batches floats, nullable): the loss of each mini-batch
 * before its update.  For checking the training loop against a reference. */
eqs_status eqs_guess_train_batches(eqs_ctx* ctx, const float* X, const float* T, int B, int n_batches,
                                   float lr, float* losses);

/* The start of the network's SPE-correction mode (EQS_GUESS_SPE_MLP): the
 * network, fed the increments x0 - h1, h1 - h2, h2 - h3, h3 - h4 at the node
 * and their 1-ring means divided by s = RMS(x0 - h1), gives a direction
 * d = s * output; the start is z0 = x0 + alpha d with the step that
 * minimises the M-norm error along d, alpha = d.(R - M x0) / d.(M d)
 * (0 when d.Md = 0), so z0 is never further from the solution in the
 * M-norm than x0.  x0 (device, n_free doubles: the SPE start), H (device,
 * 4 x n_free doubles: h1 first), R (device, n_free: the right-hand side),
 * z0 (device, n_free doubles).  In EQS_GUESS_SPE_MLP mode eqs_guess_train
 * trains this mode on steps recorded with EQS_GUESS_SPE or
 * EQS_GUESS_SPE_MLP (target (z - x0)/RMS(z - x0); EQS_ERR_STATE
 * otherwise).  Synchronises. */
eqs_status eqs_guess_eval_spe(eqs_ctx* ctx, const double* x0, const double* H, const double* R, double* z0);

/* z0 of the network for the history H (device, 4 x n_free doubles: h1 first)
 * into z0 (device, n_free doubles); synchronises. */
eqs_status eqs_guess_eval(eqs_ctx* ctx, const double* H, double* z0);

/* ---- Ensemble: EQS_ENS_W trajectories on one mesh that differ only in the
 * amplitude of their drive (column c is driven by v0_scale[c] g(t)).  Every
 * stage solves the EQS_ENS_W right-hand sides together: Sec. IV's multiple
 * right-hand-side problem with the constant M, here as a blocked CG in
 * which each matrix entry of M, of the AMG operators and of the transfer
 * matrices is read once for all columns (sparse matrix times a block of
 * vectors), while every column keeps its own CG coefficients and stopping
 * test (||R_c - M z_c|| <= rtol ||R_c||; a converged column is frozen).
 * Needs a context set up in EQS_PREC_MIXED with split_m 1; starts every
 * solve from the column's previous solution.  Device memory for the
 * ensemble is allocated by the first ensemble call. */
#define EQS_ENS_W 4

typedef struct {
  int s;
  int total_iters[EQS_ENS_W];  /* CG iterations of each column, summed over the s solves */
  int passes;                  /* CG loop passes summed over the solves (per solve:
                                  the largest column count)                     */
  int max_iters;               /* largest pass count of one solve                */
  double max_relres;           /* largest final ||r||/||R|| of all columns       */
  int status;                  /* EQS_OK, EQS_ERR_NOCONV or EQS_ERR_NAN          */
  int64_t launches;            /* kernels of the step (graph kernel nodes outside
                                  loops + loop-body kernel nodes x passes)      */
} eqs_ens_stats;

/* One RKC step of s stages (as eqs_rkc_step) for the EQS_ENS_W trajectories.
 * x: device, EQS_ENS_W x n_nodes doubles, column-major (trajectory c at
 *   x + c n_nodes), mesh order; in x(t), out x(t + dt), Dirichlet entries
 *   replaced by v0_scale[c] g(t).
 * v0_scale: host, EQS_ENS_W finite doubles.
 * The step is one CUDA graph per s (x reaches it through a per-call
 * parameter block, so any buffer reuses it); stats: host or NULL (then the
 * call is asynchronous).  EQS_ERR_STATE if the context is not mixed /
 * split. */
eqs_status eqs_ens_rkc_step(eqs_ctx* ctx, double* x, const double* v0_scale, double t, double dt,
                            int s, eqs_ens_stats* stats);

/* Y = K(X) X for the EQS_ENS_W columns at once with the ensemble's element
 * kernel (Sec. III: formed tet by tet, never assembling K; the four columns
 * share each tet's geometry), before any boundary condition.  X, Y: device,
 * EQS_ENS_W x n_nodes doubles, column-major (column c at X + c n_nodes), mesh
 * order; Y is overwritten.  FP32 arithmetic as in the mixed step: X is
 * carried as FP32 (hi, lo) pairs, Y is the FP32 result widened.  Needs a
 * context set up in EQS_PREC_MIXED on linear (4-node) tets, else
 * EQS_ERR_STATE.  Device memory for the staged columns is allocated by the
 * first call.  Asynchronous on the context stream. */
eqs_status eqs_ens_apply_K(eqs_ctx* ctx, const double* X, double* Y);

/* Statistics of the last ensemble step (synchronises). */
eqs_status eqs_ens_get_step_stats(eqs_ctx* ctx, eqs_ens_stats* stats);

/* Solve M_ff z_c = rhs_c for the EQS_ENS_W columns together with the blocked
 * CG of the ensemble at the setup's rtol.  rhs, z: device, n_free x
 * EQS_ENS_W doubles, column-major; z holds the start vectors on entry and
 * the solutions on exit.  iters_out: host, EQS_ENS_W ints or NULL.
 * Synchronises; EQS_ERR_NOCONV if a column hit max_iter. */
eqs_status eqs_ens_solve_M(eqs_ctx* ctx, const double* rhs, double* z, int* iters_out);

/* SPE start vectors of the four columns (Sec. IV, Eq. 4-5) from a given
 * history, as the ensemble step forms them: X (device, 6 x 4 x n_free
 * doubles; solution k of column c at X + (4 k + c) n_free, k = 0 the most
 * recent), b (device, 4 x n_free: the right-hand sides).  x0 (device,
 * 4 x n_free) receives the start vectors, r0 (device, 4 x n_free) the start
 * residuals b - W y as the CG starts from them (W = M X from the Gram pass,
 * no further product with M).  Synchronises.  For checking the pass. */
eqs_status eqs_ens_spe_eval(eqs_ctx* ctx, const double* X, const double* b, double* x0, double* r0);

/* The CG kernels of the mixed path widen FP32 values to FP64 with integer
 * operations (GB300 executes the hardware conversion on its slow FP64 pipe).
 * This call applies that widening to n values on the current device (f
 * device float input, f_wide device double output) so it can be checked
 * against the exact conversion.  Synchronises the device.  No counterpart
 * in the paper. */
eqs_status eqs_convert_check(const float* f, int n, double* f_wide);

/* ---- One kernel of the step, launched alone (measurement).
 * Enqueues ONE launch of the named kernel of the last step
 * (eqs_rkc_step, or eqs_ens_rkc_step for the EQS_KERNEL_ENS_* ids) on the
 * context stream, with the arguments that step's last stage solve used, so
 * that a caller can time the kernel with events on that stream:
 *   SPE_GRAM: the SPE Gram pass of Sec. IV, Eq. 4-5 (the product W = M x
 *             of the newest solution, the new Gram column and the
 *             projections of the right-hand side; the small solve that
 *             follows it in a step is not launched); ENS_SPE_GRAM is two
 *             launches, the product alone and then the dot products with
 *             the four small solves in the last block;
 *   ELEM:     the element kernel of Sec. III on the last stage state, its
 *             K(x)x scattered into a private buffer of the context
 *             (allocated on the first such call);
 *   PCG_PQ:   the CG operator pass q = M z + beta q of Sec. IV (for the
 *             ensemble with all four columns active: their convergence
 *             flags are cleared first, one small memset on the stream).
 * The Gram pass recomputes the last solve's column (same values); the CG
 * pass overwrites CG vectors that the next solve re-initialises.  So a
 * later step is unaffected, but the call must not overlap a step.
 * EQS_ERR_STATE when no such step has run (or SPE is not in use for the
 * Gram ids), EQS_ERR_ARG for an unknown id.  Asynchronous. */
enum {
  EQS_KERNEL_SPE_GRAM = 0, EQS_KERNEL_ELEM = 1, EQS_KERNEL_PCG_PQ = 2,
  EQS_KERNEL_ENS_SPE_GRAM = 16, EQS_KERNEL_ENS_ELEM = 17, EQS_KERNEL_ENS_PCG_PQ = 18
};
eqs_status eqs_launch_kernel(eqs_ctx* ctx, int kernel);

/* ---- Batched serving: many independent instances advance together.
 * Every RKC stage of all instances is one cooperative launch in which each
 * instance owns a group of CTAs proportional to its free rows (at least
 * rows_per_block rows per CTA; scaled up until all CTAs are co-resident) and
 * runs its recurrence, element kernel, right-hand side and whole CG solve
 * with its own bounded group barrier (EQS_ERR_TIMEOUT when a wait gives up).
 * The step is one CUDA graph per s.  Contexts must be set up in
 * EQS_PREC_MIXED with equal rtol on one device; while a batch uses them they
 * must not run other work concurrently.  The batch keeps the context
 * pointers (the caller keeps the contexts alive) and owns the rest. */
typedef struct eqs_batch eqs_batch;

typedef struct {
  int n_inst, s;
  int64_t total_iters;   /* CG iterations summed over instances and stages  */
  int max_iters;         /* largest iteration count of one solve            */
  double max_relres;     /* largest final ||r||/||R||                        */
  int status;            /* EQS_OK, EQS_ERR_NOCONV or EQS_ERR_TIMEOUT        */
  int64_t launches;      /* kernels of the step graph                        */
} eqs_batch_stats;

eqs_status eqs_batch_create(eqs_ctx* const* ctxs, int n, int rows_per_block, eqs_batch** out);

/* When every context selects EQS_GUESS_SPE, each batched solve starts from
 * the SPE vector of its instance (Sec. IV, Eq. 4-5, six solutions; the
 * Gram pass and the small solve run inside the instance's CTA group, on
 * the context's solution ring, so a context must not step on its own
 * between batched steps); otherwise from the previous solution.
 *
 * Wait budget of every group barrier of the batched launches, in polls
 * (0: the default, 2^22); a wait that runs out sets the instance's error
 * flag, every CTA of the group returns, and the step reports
 * EQS_ERR_TIMEOUT (x of that step is then undefined).  Takes effect from
 * the next step. */
eqs_status eqs_batch_set_barrier_polls(eqs_batch* b, long long polls);

/* One RKC step of s stages for every instance: x is a host array of n
 * device pointers (instance k: n_nodes of ctx k doubles, mesh order, in x(t),
 * out x(t + dt)); drive, materials and tolerances come from each context.
 * stats: host or NULL (then the call is asynchronous). */
eqs_status eqs_batch_rkc_step(eqs_batch* b, double* const* x, double t, double dt, int s,
                              eqs_batch_stats* stats);

/* Statistics of the last batched step (synchronises); inst_iters: host array
 * of n totals per instance, or NULL. */
eqs_status eqs_batch_get_stats(eqs_batch* b, eqs_batch_stats* stats, int64_t* inst_iters);

/* CTAs of the batched stage launch and the rows per CTA finally used. */
eqs_status eqs_batch_info(const eqs_batch* b, int* total_blocks, int* rows_per_block);

eqs_status eqs_batch_destroy(eqs_batch* b);
const char* eqs_batch_last_error(const eqs_batch* b);

/* SPE start vector x0 = V (V^T M V)^-1 V^T b (Sec. IV, Eq. 4-5) for a given
 * history X (device, n x n_free doubles, most recent first), right-hand side
 * b and result x0 (device, n_free doubles).  The history is pushed oldest
 * first through the same kernels the step uses (M x of each pushed solution,
 * incremental Gram matrix), then x0 is formed.  n must equal the setup's
 * spe_n.  Overwrites the context's SPE history and right-hand side buffer;
 * synchronises.  For checking the projection. */
eqs_status eqs_spe_eval(eqs_ctx* ctx, const double* X, const double* b, int n, double* x0);

/* POD-MOR start vector (Sec. IV) for K given snapshots X (device, K x
 * n_free doubles, oldest first, K <= pod_k): the basis of the leading
 * pod_m POD modes is built by the kernels of the step (Gram matrices,
 * Jacobi eigendecomposition, reduced system) and x0 = V (V^T M V)^-1 V^T b
 * is written (b, x0: device, n_free doubles).  Replaces the context's
 * snapshot set by X (eqs_pod_info then describes this basis); synchronises.
 * For checking the projection. */
eqs_status eqs_pod_eval(eqs_ctx* ctx, const double* X, int K, const double* b, double* x0);

/* POD state of the context (synchronises): snapshots stored, modes kept,
 * bases computed, snapshots added, and (host, 16 doubles, nullable) the
 * eigenvalues of X^T X of the last basis, descending. */
eqs_status eqs_pod_info(eqs_ctx* ctx, int* count, int* modes, int* rebuilds, int* adds, double* lam);

/* Release everything owned by ctx (NULL is accepted). */
eqs_status eqs_destroy(eqs_ctx* ctx);

/* Text of the last error on ctx (or of the last failed eqs_mesh_create when
 * ctx is NULL). Never NULL. */
const char* eqs_last_error(const eqs_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* EQS_H */
