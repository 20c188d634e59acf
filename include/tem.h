/* tem.h -- C ABI of the GB300 shifted-system TEM library (libtem.so).
 *
 * The library evaluates, on one GPU, the hot path of a Gauss-Newton step of
 * 3-D transient EM inversion with a rational approximation of the matrix
 * exponential (Borner, Guttel, Gunther, "Scalable Parallel 3-D TEM Inversion
 * via Rational Approximation of the Matrix Exponential"):
 *
 *   u(t_j) ~ 2 Re sum_i alpha_i^[j] (K - xi_i M)^-1 f            (Section 2.3)
 *   d_j    = Q u(t_j)                                            (Section 3)
 *   J_j v  = 2 Re sum_i alpha_i^[j] xi_i Q A_i^-1 [(dM/dm) g_i v]  (Section 3.1)
 *   J^T w  = sum_j J_j^T w_j                                     (Section 3.1)
 *   LSQR on [W_d J; sqrt(lambda) L^1/2]                          (Section 3.3, eq. lsqr)
 *
 * with K the Whitney-edge curl-curl matrix (1/mu0), M(sigma) the
 * conductivity mass matrix, A_i = K - xi_i M complex symmetric, g_i = A_i^-1 f,
 * m = ln(sigma) on the parameter cells, dM/dm_e = sigma_e M1_e.
 *
 * Conventions
 *  - Every call returns an int status: TEM_OK (0) or a negative TEM_ERR_*.
 *    tem_last_error() returns a message owned by the context (valid until the
 *    next call on that context).
 *  - "host" arrays are read during the call only.  "dev" arrays are
 *    caller-owned device pointers on the context's GPU, contiguous, valid for
 *    the duration of the call; the library never frees them.
 *  - The library owns every factor, symbolic table and work buffer; all are
 *    released by tem_destroy().
 *  - Device work is issued on the stream given to tem_create(); calls return
 *    after the stream is synchronised (status words are read back), unless
 *    the context is asynchronous (tem_set_async): then calls return once
 *    their work is issued and tem_status reports the device status.
 *  - Calls out of order (e.g. tem_jvp before tem_forward) return
 *    TEM_ERR_STATE.  Sizes that do not match the context return TEM_ERR_ARG.
 *  - Data vectors are laid out d[x][r][j] (transmitter, receiver, time),
 *    row-major, FP64.  Model vectors are FP64 over the parameter cells in
 *    tetrahedron order.
 */
#ifndef TEM_H
#define TEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TEM_OK 0
#define TEM_ERR_ARG (-1)     /* bad argument or size */
#define TEM_ERR_OOM (-2)     /* device memory exhausted */
#define TEM_ERR_PIVOT (-3)   /* a pivot of some A_i underflowed (singular shift) */
#define TEM_ERR_TIMEOUT (-4) /* a bounded device wait expired */
#define TEM_ERR_CUDA (-5)    /* CUDA runtime error */
#define TEM_ERR_STATE (-6)   /* call out of order */
#define TEM_ERR_MESH (-7)    /* degenerate mesh / source / receiver */

/* Arithmetic of the factors and solves. */
#define TEM_FP64 0         /* complex double throughout */
#define TEM_FP32_REFINED 1 /* complex float factors and solves, FP64 iterative
                              refinement (residual K - xi M in FP64) */

typedef struct tem_ctx tem_ctx;

typedef struct tem_stats {
  int64_t n_dof;         /* N: interior edges (unknowns) */
  int64_t n_tet;         /* tetrahedra */
  int64_t n_param;       /* P: parameter cells */
  int64_t n_faces_reg;   /* rows of the regulariser root W */
  int64_t n_fronts;      /* supernodes of the assembly tree */
  int64_t n_levels;      /* height of the assembly tree + 1 */
  int64_t nnz_a;         /* nonzeros of A (full symmetric pattern) */
  int64_t nnz_l;         /* stored factor entries per pole (incl. diagonal) */
  double flops_factor;   /* complex MACs of one pole's factorisation */
  int64_t max_front;     /* largest front order */
  int64_t bytes_device;  /* device bytes held by the context */
  int32_t m;             /* pole pairs */
  int32_t n_times;       /* K */
  int32_t n_tx, n_rx;
  int32_t precision;
  int32_t refine_steps;  /* refinement corrections per forward and J v solve (FP32 mode) */
  int32_t last_pivot_front; /* front of the last pivot failure, -1 if none */
  double min_pivot_abs;  /* smallest |d_kk| seen in the last factorisation */
  int64_t nnz_l11;       /* factor entries in the pivot blocks (sum k(k+1)/2) */
  int64_t n_solve_launch;/* kernel launches of one solve (forward + backward sweep) */
  int64_t pole_solves;   /* poles x (forward + backward sweep) issued so far */
  int64_t solve_calls;   /* multi-pole solves issued so far (each with its refinement) */
  int32_t tc_ctas_per_sm; /* resident CTAs per SM of the tensor-core product kernel (0 before its first launch) */
  int32_t refine_steps_adjoint; /* refinement corrections per adjoint (J^T w) solve (FP32 mode) */
  int64_t tc_prod_launches;   /* FP32 solve products run on the tensor cores, library-wide since load */
  int64_t simt_prod_launches; /* FP32 solve products run on the FP32 pipes, library-wide since load */
  int64_t n_nodes;       /* FP32 mode: interior vertices (gradient-space unknowns) */
  int64_t nnz_l_nodal;   /* FP32 mode: stored factor entries of the nodal Laplacian */
  int32_t nodal;         /* FP32 mode: 1 = gradient-space correction on */
  int32_t reserved0;
  int64_t tc_update_launches; /* FP32 factor trailing updates run on the tensor cores, library-wide since load */
} tem_stats;

/* Create a context on the current CUDA device.  precision: TEM_FP64 or
 * TEM_FP32_REFINED.  stream: a cudaStream_t (NULL = legacy default stream). */
int tem_create(tem_ctx **ctx, int precision, void *stream);

/* Release everything the context owns.  ctx may be NULL. */
int tem_destroy(tem_ctx *ctx);

/* Message of the last failure on ctx (or on context creation if ctx NULL). */
const char *tem_last_error(tem_ctx *ctx);

/* Mesh, conductivity and parameterisation (Section 2.2, Section 3).
 *   xyz      host [n_vert][3]  vertex coordinates (m)
 *   tets     host [n_tet][4]   vertex ids of each tetrahedron (any order)
 *   sigma    host [n_tet]      conductivity (S/m) of every cell; the values
 *                              of parameter cells are overwritten by
 *                              exp(log_sigma) in tem_factor
 *   is_param host [n_tet]      1 = inverted cell (model parameter), else 0
 * Builds edges, removes edges on the outer boundary (PEC, Section 2.1), the element
 * matrices, the nested-dissection ordering, the assembly tree and the
 * regulariser root W = M_div^-1/2 D^T over the parameter cells (Section 3.2), and
 * uploads the index tables.  leaf_max: largest leaf of the dissection
 * (0 = default).  May be called once per context. */
int tem_mesh(tem_ctx *ctx, int64_t n_vert, const double *xyz, int64_t n_tet,
             const int32_t *tets, const double *sigma, const uint8_t *is_param,
             int32_t leaf_max);

/* Poles and residues of the rational approximant (Section 2.3).
 *   xi    host [m][2]        (re, im) of xi_i; each stands for the pair
 *                            {xi_i, conj xi_i}; system A_i = K - xi_i M
 *   alpha host [m][n_times][2] (re, im) of alpha_i^[j]
 * Re xi_i must be < 0 (keeps A_i's real part positive definite). */
int tem_poles(tem_ctx *ctx, int32_t m, const double *xi, int32_t n_times,
              const double *alpha);

/* New observation times for the poles of tem_poles (Section 2.3: the poles
 * are shared by every time and only the residues alpha_i^[j] depend on t_j,
 * so new times need no new factorisation).  The residues are fitted on the
 * device in FP64 by penalised linear least squares, per time t_j:
 *   min over alpha_.^[j] of  sum_z ( exp(-t_j z) - 2 Re sum_i alpha_i^[j] / (z - xi_i) )^2
 *                            + mu^2 sum_i |alpha_i^[j]|^2 / |xi_i|^2
 * over the sample set z in {0} and n_z log-spaced points in [z_min, z_max]
 * (the spectrum of M^-1 K lies on z >= 0), by Householder QR of the
 * (n_z + 1 + 2m) x 2m matrix once and one reduction and back-substitution per
 * time.  The penalty bounds each partial fraction (max over z >= 0 of
 * |alpha_i / (z - xi_i)| = |alpha_i| / |xi_i|).  Defaults of the stored tables:
 * n_z = 2200, z_min = 1e-2, z_max = 1e9, mu = 1e-4.
 *   t         host [n_times], every t_j > 0 (1 <= n_times <= 2^20)
 *   alpha_out host [m][n_times][2] (re, im) of the fitted alpha_i^[j], or NULL
 * The data, J v and J^T w shapes become [n_tx][n_rx][n_times].  The factors stay
 * valid; the forward solutions too, but the next tem_jvp / tem_jtvp / tem_lsqr
 * needs a tem_forward first (TEM_ERR_STATE until then).  Synchronises and
 * reallocates the buffers sized by the data: not in asynchronous mode
 * (TEM_ERR_STATE) and not inside a stream capture, and a CUDA graph captured
 * before the call still refers to the old buffers, so it must not be replayed
 * after it.  TEM_ERR_ARG for bad
 * arguments, a fit larger than (n_z + 1 + 2m) n_times = 2^31, or a rank-deficient
 * fit (mu = 0 with too few samples). */
int tem_times(tem_ctx *ctx, int32_t n_times, const double *t, int32_t n_z, double z_min,
              double z_max, double mu, double *alpha_out);

/* Poles of the rational approximant fitted on the device (Section 2.3; the
 * paper fits them with RKFIT).  Variable projection: for given poles the
 * residues of every time are the penalised least-squares fit of tem_times
 * (same sample set, same penalty), and the poles minimise the sum over the
 * times of the squared residuals,
 *   f(xi) = sum_j || (I - Q Q^T) [exp(-t_j z); 0] ||^2   (Q from the QR of the basis),
 * by Levenberg-Marquardt steps on p = (log(-Re xi_i), log(Im xi_i)) (which
 * keeps Re xi < 0 < Im xi) with Kaufman's Jacobian -(I - Q Q^T)(dB/dp) c_j,
 * formed and reduced to the normal equations on the device (FP64); the host
 * solves the 2m x 2m step, and at most a factor e^2 per step in any part of
 * a pole.  Stops after max_iter steps, when no step decreases f, or when the
 * relative decrease is below 1e-12.
 *   t      host [n_times] fitting times (> 0; 1 <= n_times <= 4096), 1 <= m <= 32
 *   xi     host [m][2] starting poles in (Re < 0 < Im), fitted poles out
 *   obj    host [3] out: f at the start, f at the end, steps taken
 *   stream cudaStream_t (NULL: the default stream) of the current device
 * Needs no context (errors: tem_last_error(NULL)); allocates and frees its
 * own work arrays and synchronises.  TEM_ERR_ARG for bad arguments, a fit
 * larger than (n_z + 1 + 2m) 2m n_times = 2^31, or starting poles that leave
 * the fit rank deficient. */
int tem_fit_poles(int32_t m, int32_t n_times, const double *t, int32_t n_z, double z_min, double z_max,
                  double mu, int32_t max_iter, double *xi, double *obj, void *stream);

/* Transmitters and receivers (Section 2.1 source, Section 4.2 observation).
 *   loop_ptr  host [n_tx+1]  offsets into loop_verts
 *   loop_verts host          closed polylines of vertex ids; consecutive ids
 *                            (and last->first) must share a mesh edge; I = 1 A
 *   rx        host [n_rx][3] receiver positions on a horizontal mesh surface;
 *                            Q = -(curl e)_z by Stokes on the surface
 *                            triangles whose closure holds the receiver
 *                            (area-weighted when it lies on an edge/vertex). */
int tem_sources(tem_ctx *ctx, int32_t n_tx, const int64_t *loop_ptr,
                const int32_t *loop_verts, int32_t n_rx, const double *rx);

/* Factor every shifted matrix A_i = K - xi_i M(sigma) (Algorithm 1), with
 * sigma = exp(log_sigma) on the parameter cells.
 *   log_sigma dev [P] FP64.
 * Returns TEM_ERR_PIVOT if a pivot underflows. */
int tem_factor(tem_ctx *ctx, const double *log_sigma);

/* Forward responses: g_i = A_i^-1 f_x for all poles and transmitters
 * (kept for the Jacobian products), then d[x][r][j] = 2 Re sum_i
 * alpha_i^[j] (Q g_i,x)_r.   d dev [n_tx][n_rx][n_times] FP64. */
int tem_forward(tem_ctx *ctx, double *d);

/* J v.   v dev [P] FP64,  jv dev [n_tx][n_rx][n_times] FP64. */
int tem_jvp(tem_ctx *ctx, const double *v, double *jv);

/* J^T w.  w dev [n_tx][n_rx][n_times] FP64,  jtw dev [P] FP64. */
int tem_jtvp(tem_ctx *ctx, const double *w, double *jtw);

/* One Gauss-Newton LSQR solve (Section 3.3, eq. lsqr): n_iter iterations of
 * Paige-Saunders LSQR, no stopping test, on
 *   min || [W_d J; sqrt(lambda) W] dm + [W_d (d - d_obs); sqrt(lambda) W (m - m_ref)] ||
 * at the model of the last tem_factor and the data of the last tem_forward.
 *   d_obs dev [n_tx][n_rx][n_times], wd dev [same] (diagonal of W_d),
 *   m_ref dev [P], dm dev [P] (output).  Each iteration is one J v and one
 *   J^T w ("pair"); all scalars stay on the device in FP64. */
int tem_lsqr(tem_ctx *ctx, const double *d_obs, const double *wd,
             const double *m_ref, double lambda, int32_t n_iter, double *dm);

/* tem_lsqr for callers that cannot allocate device memory while an
 * inversion runs: programs whose device memory belongs to their own
 * allocator (a framework's caching pool), or that must not risk a cudaMalloc
 * failing, or cudaMalloc/cudaFree synchronising the device, between
 * Gauss-Newton steps.  Same arguments, results and errors as tem_lsqr, but
 * the LSQR work vectors and scalars live in one file-scope device array of
 * 4 Mi doubles (32 MiB) that every GPU loading the library holds until the
 * process exits; a problem needing more (3 nd + 2 n_faces + 3 P doubles,
 * nd = n_tx n_rx n_times) returns TEM_ERR_ARG and nothing runs.  The call
 * allocates nothing itself; the factors and solve buffers it uses come from
 * tem_factor.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress, with the context's device current), so make
 * that first call before any stream capture.  All calls on a device share the
 * array and it keeps the last call's contents: calls that overlap on the GPU
 * (other streams, other contexts on the same device) race.  This entry point
 * has no counterpart in the paper. */
int tem_lsqr_noalloc(tem_ctx *ctx, const double *d_obs, const double *wd,
                     const double *m_ref, double lambda, int32_t n_iter, double *dm);

/* Gauss-Newton bookkeeping at the model of the last tem_factor and the data of
 * the last tem_forward (Section 3, phi; Section 3.3, line search), on the
 * device: the objective phi = 1/2 ||W_d (d - d_obs)||^2 + lambda R(m) with
 * R = 1/2 ||W (m - m_ref)||^2 (W^T W = L), and optionally its gradient
 *   grad = J^T W_d^2 (d - d_obs) + lambda L (m - m_ref)     (one J^T w)
 * and the directional derivative grad . dm.
 *   d_obs, wd dev [n_tx][n_rx][n_times]; m_ref dev [P]; grad dev [P] or NULL;
 *   dm dev [P] or NULL (needs grad); out host [5]: phi, 1/2 ||W_d r||^2, R,
 *   chi^2 = ||W_d r||^2 / (n_tx n_rx n_times), grad . dm (0 without dm).
 * Synchronises (the scalars are returned): TEM_ERR_STATE in asynchronous
 * mode. */
int tem_gn_eval(tem_ctx *ctx, const double *d_obs, const double *wd, const double *m_ref,
                double lambda, const double *dm, double *grad, double *out);

/* out = m + eta dm over the parameter cells (the Gauss-Newton trial model,
 * Section 3.3).  m, dm, out dev [P]; out may alias m. */
int tem_model_step(tem_ctx *ctx, const double *m, const double *dm, double eta, double *out);

/* Supernode amalgamation of the assembly tree (Algorithm 1, factorise; no
 * paper counterpart in its details): a child separator of at most
 * max_pivots unknowns is merged into its parent front (its pivots first) and
 * its children become the parent's, while the parent keeps at most four
 * children.  The plane separators between two leaf boxes of the dissection
 * are small (21 unknowns on the 46^3 box); merged, they cost some explicit
 * zeros in the parent's dense front instead of a tree level of fronts that
 * fill a fraction of the device tiles.  Default 32; 0 switches it off.  Call
 * before tem_mesh, which builds the tree (TEM_ERR_STATE after it);
 * max_pivots in 0..4096 (TEM_ERR_ARG otherwise). */
int tem_set_amalgamation(tem_ctx *ctx, int32_t max_pivots);

/* TEM_FP32_REFINED mode: refinement corrections per forward and J v solve
 * (default 3) and the conductivity floor of the factored matrices (default
 * 1e-6).
 *
 * The complex-float factor is of P_i = K - xi_i M(s_i) with the cell
 * conductivity raised to s_i,t = max(sigma_t, floor_tau / (|xi_i| mu0 h_t^2)),
 * h_t^2 = vol_t^(2/3); every correction solves with P_i, the residual
 * b - (K - xi_i M(sigma)) x is formed with the true matrix in double-float
 * pairs (compensated products on the FP32 pipes).  Without
 * the floor the gradient fields of resistive cells (air, 1e-8 S/m) have pivots
 * below float resolution and the refinement diverges.  P_i^-1 A_i is then
 * ~sigma / s on the gradients of the floored cells: the gradient-space
 * correction (tem_set_nodal) removes those error components every step,
 * which lets the floor go down to 1e-6, where the remaining modes contract
 * by ~1e-3 per step.  The FP64 mode factors A_i itself.  With tol > 0 a pole stops refining once its last correction,
 * over the unknowns every output reads (edges of parameter cells), is below
 * tol times the solution there; the remaining sweeps run over the poles still
 * refining (one host read per step).  steps in 0..40 (the maximum),
 * floor_tau in [0, 1], tol in [0, 1] (0: always steps corrections). */
int tem_set_refine(tem_ctx *ctx, int32_t steps, double floor_tau, double tol);

/* TEM_FP32_REFINED mode: refinement corrections per adjoint solve, the
 * solves of tem_jtvp (and of tem_lsqr's J^T w), default 1.  Their output is
 * the cell sums over parameter cells (formed in double-float pairs), which
 * converge in fewer corrections than the receivers' fields of tem_forward
 * and tem_jvp.  steps in 0..40; TEM_ERR_ARG otherwise. */
int tem_set_refine_adjoint(tem_ctx *ctx, int32_t steps);

/* TEM_FP32_REFINED mode: run the update-row products of the solves on the
 * tensor cores (tcgen05, TF32 split into hi + lo parts, three MMAs per
 * product, FP32 accumulation; default 1) or on the FP32 pipes (0).  A
 * tensor-core completion wait that gives up makes the call return
 * TEM_ERR_TIMEOUT.  No effect in TEM_FP64 mode. */
int tem_set_tensor_cores(tem_ctx *ctx, int enable);

/* Asynchronous mode (default 0): tem_factor, tem_forward, tem_jvp, tem_jtvp,
 * tem_lsqr and tem_lsqr_noalloc return as soon as their work is issued on the
 * context's stream, without synchronising or reading the device status, so
 * that a caller can overlap them with its own work or capture them into a
 * CUDA graph (stream capture on the context's stream) and replay it.
 * Arguments are checked as usual; device-side failures (a pivot underflow, an
 * expired tensor-core wait) are reported by the next tem_status.  Calls that
 * allocate on first use (tem_factor's first call allocates the numeric
 * storage, tem_lsqr's first call its work vectors) must have run once before
 * a capture.  A refinement tolerance (tem_set_refine tol > 0) needs host
 * reads and is refused (TEM_ERR_ARG) in this mode.  Switching it off
 * synchronises the stream. */
int tem_set_async(tem_ctx *ctx, int enable);

/* Synchronise the context's stream and report the device status words of the
 * work issued so far: TEM_ERR_TIMEOUT (cleared once reported), TEM_ERR_PIVOT
 * (the last tem_factor failed; solves need a new tem_factor), else TEM_OK. */
int tem_status(tem_ctx *ctx);

/* A batch of independent surveys (uneven meshes, each its own context):
 * for every context i, in order, the operations of `ops` on its own stream:
 *   TEM_BATCH_FACTOR  tem_factor(ctx[i], log_sigma[i])
 *   TEM_BATCH_FORWARD tem_forward(ctx[i], d[i])
 *   TEM_BATCH_JTVP    tem_jtvp(ctx[i], w[i], jtw[i])
 * issued asynchronously, with no synchronisation between contexts, so that
 * contexts on different streams run concurrently on the GPU.  Arrays are per
 * context and follow the single calls' layouts (NULL where an operation is
 * not requested).  Contexts in asynchronous mode stay unsynchronised (read
 * their status with tem_status; the whole call can then be captured into one
 * CUDA graph, whose branches are the contexts' streams); for the others the
 * call synchronises each and returns the first failing status.  Each context
 * must have run the requested calls once before a capture (allocation). */
#define TEM_BATCH_FACTOR 1
#define TEM_BATCH_FORWARD 2
#define TEM_BATCH_JTVP 4
int tem_batch(tem_ctx **ctx, int32_t n, int32_t ops, const double *const *log_sigma, double *const *d,
              const double *const *w, double *const *jtw);

/* TEM_FP32_REFINED mode: the trailing updates of the dense fronts (Algorithm 1,
 * factorise) on the tensor cores (default 1) or on the FP32 pipes (0).  On the
 * tensor cores the pivots of a front go in blocks of 128: each 32-wide panel
 * updates the rest of its block, and the block then updates the whole
 * trailing part at once, F22 -= L21 D L21^T of rank 128, as tcgen05 TF32
 * MMAs (hi / lo split, three MMAs per product, FP32 accumulation in TMEM)
 * fed by TMA.  Takes effect at the next tem_factor (solves before it return
 * TEM_ERR_STATE).  No effect in TEM_FP64 mode. */
int tem_set_tc_fronts(tem_ctx *ctx, int enable);

/* Limits of the bounded waits inside the tensor-core solve kernel (library
 * wide; defaults 2^26 polls and 1 s).  A wait that runs out makes the kernel
 * stop issuing work, drain its loads and MMAs in flight (with the default
 * limits) and return; the call then fails with TEM_ERR_TIMEOUT, whose flag is
 * cleared once reported.  For tests of that status: tiny limits make the
 * waits run out on purpose.  max_polls >= 1, 0 < max_seconds <= 60. */
int tem_set_wait_limit(tem_ctx *ctx, uint32_t max_polls, double max_seconds);

/* TEM_FP32_REFINED mode: the gradient-space correction of every refinement
 * step (default 1).  The floored factor P_i leaves the gradient fields of the
 * floored cells almost uncorrected (P_i^-1 A_i ~ sigma / s ~ 0 there), so each
 * step also solves the residual equation on the discrete gradients G psi of
 * the interior vertices.  With K G = 0 (Section 2.2, curl grad = 0),
 * G^T A_i G = -xi_i G^T M(sigma) G: one real sigma-weighted nodal Laplacian
 * L = G^T M G for every pole, factored with A_i in tem_factor, and per step
 * psi = L^-1 G^T r, x += -G psi / xi_i, r -= M G psi, before the correction
 * with P_i.  Switching it on after tem_factor without it requires a new
 * tem_factor (TEM_ERR_STATE until then).  No effect in TEM_FP64 mode. */
int tem_set_nodal(tem_ctx *ctx, int enable);

/* Time one class of kernels with CUDA events on the context's stream:
 * 0 trailing update, 1 panel, 2 forward pivot-block step, 3 backward
 * pivot-block step, 4 backward update-row product (L21^T), 5 extend-add,
 * 6 forward update-row product (L21), 7 forward super-block product,
 * 8 backward super-block product, 9 pivot-block inversion, 10 refinement
 * residual, 11 refinement vector kernels (split, scaling, accumulation, join),
 * 12 Jacobian kernels (J v right-hand sides, J^T w right-hand sides, residue
 * sums, cell sums), 13 gradient-space correction (G^T r, nodal sweeps,
 * M G psi; its sweeps count in no other class), and its parts: 14 G^T r and
 * scaling, 15 nodal sweeps, 16 M G psi and x update; 17 tensor-core trailing
 * updates of the factorisation (panel copies and rank-128 updates); -1
 * switches timing off (the default).
 * class + 64 (h + 1) times only the launches of assembly-tree level h.
 * Timing adds an event pair around each launch of that class. */
int tem_set_profiling(tem_ctx *ctx, int kernel_class);

/* Accumulated device time (ms) and launch count of the timed class since the
 * last tem_set_profiling. */
int tem_kernel_time(tem_ctx *ctx, double *total_ms, int64_t *launches);

/* Kernel launches issued by the library since it was loaded (all contexts). */
int64_t tem_launch_count(void);

/* Sizes and counters. */
int tem_info(tem_ctx *ctx, tem_stats *out);

/* Host copy of the assembled matrices in the library's DoF numbering, for
 * inspection and tests: K (and M at the last factor) in CSR, FP64.
 * Pass NULL pointers to query nnz first (returned in *nnz). */
int tem_export_pattern(tem_ctx *ctx, int64_t *nnz, int64_t *row_ptr,
                       int32_t *col, double *k_val, double *m_val);

/* Host copy of the forward solutions g_i = A_i^-1 f_x of the last tem_forward
 * (Algorithm 1, solve), for inspection and tests: g host [m][N][n_tx][2]
 * (re, im) FP64, unknowns in the library's numbering (tem_export_dofs).
 * TEM_ERR_STATE before tem_forward. */
int tem_export_forward(tem_ctx *ctx, double *g);

/* Permutation: perm[new] = interior-edge index in the library's own edge
 * numbering, and the edge's two vertex ids (lower first), host arrays of
 * length N and [N][2]. */
int tem_export_dofs(tem_ctx *ctx, int64_t *edge_verts);

/* Assembly-tree levels of the edge system (for per-level measurements with
 * tem_set_profiling): out host [n_levels][4], per level h (0 = leaves) the
 * number of fronts, the pivot-block entries sum k (k + 1) / 2, the
 * update-row entries sum k b and the largest k.  After tem_mesh. */
int tem_level_info(tem_ctx *ctx, int64_t *out);

#ifdef __cplusplus
}
#endif
#endif /* TEM_H */
