/*
 * rcg.h -- C ABI of librcg: inner-outer recycled Krylov solves for the
 * symmetric diffusion operator of diffuse optical tomography and the
 * one-sided reduced model built from them (O'Connell, Kilmer, de Sturler,
 * Gugercin, "Computing Reduced Order Models via Inner-Outer Krylov Recycling
 * in Diffuse Optical Tomography", arXiv 1602.00138).
 *
 * Problem (Sec. 2.1, eqs. ModelPDE1-4; Sec. 3): on the unit square (2D) or
 * cube (3D) with N unknown nodes per axis, h = 1/(N+1), the zero-frequency
 * diffusion operator with homogeneous Dirichlet lateral faces and Robin
 * faces at z = 0 and z = 1 is discretised by centred differences, and the
 * Robin boundary unknowns are eliminated (Sec. 3, Schur complement
 * A~ = F - D2 G^-1 D1).  A~(p) = A~_* + diag(h^2 mu(p)) is SPD (eq. sum).
 * Node index: i + Nx*(j + Ny*k), x fastest; (Nx,Ny,Nz) = (N,1,N) in 2D
 * (axes x and z) and (N,N,N) in 3D.  Interior rows are scaled by h^2:
 *   (A~ x)_p = sum_f w_f (x_p - x_q) + h^2 mu_p x_p,
 *   w_f = (D_p + D_q)/2 between unknowns; w_f = D_p towards a lateral ghost
 *   (x_q = 0); on a Robin face the eliminated boundary unknown leaves
 *   D_p / (1 + alpha_p) on the diagonal, alpha_p = 2 A D_p / h.
 * Effective sources / receivers (Sec. 3.1): a source of weight s at face
 * point (i,j) of z = 0 is b~ = s D_p / (1 + alpha_p) e_p, a detector of
 * weight c at face point (i,j) of z = 1 is c~ = c alpha_p / (1 + alpha_p) e_p,
 * p the unknown next to the face point.  Right-hand sides are ordered
 * [B~ (sources), C~ (detectors)] (Sec. 3.3 eq. solves).
 *
 * Method (Algorithm 2, Sec. 4.3): a seed U_0 (k_u smallest eigenvectors of
 * A~_0) and X_0 = A~_0^-1 [B~, C~] give V = basis([U_0, X_0]) and per-RHS
 * recycle spaces U_j = [U_0, X_0(:,j)].  For every sample point and RHS the
 * Galerkin guess from range(V) is checked; if its relative residual exceeds
 * tol_j the correction equation A~ g = r (eq. resi) is solved by CG deflated
 * with U_j and the new direction is appended to V and to U_j.
 *
 * Conventions for every call:
 *   - return value: RCG_OK (0) or a negative RCG_ERR_* code; the context
 *     keeps the last error message (rcg_last_error).  No C++ exception
 *     crosses this boundary.
 *   - host pointers ("host") are read during the call and never retained;
 *     the caller keeps ownership.  Device pointers ("device") must be
 *     cudaMalloc'ed memory of the device current at rcg_create.
 *   - matrices are column-major; an n-vector per column.
 *   - all device work is issued on the stream given to rcg_create; a call
 *     returns after that stream has finished the call's work unless stated.
 *   - one context per host thread; contexts are independent.
 */
#ifndef RCG_H
#define RCG_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define RCG_OK                 0
#define RCG_ERR_INVALID       -1   /* bad argument or call order            */
#define RCG_ERR_CUDA          -2   /* a CUDA runtime call failed            */
#define RCG_ERR_OOM           -3   /* device allocation failed or over cap  */
#define RCG_ERR_NOT_SPD       -4   /* a small FP64 Cholesky found d <= 0    */
#define RCG_ERR_NOT_CONVERGED -5   /* some RHS hit maxit or the refinement-
                                      restart cap; stats still filled        */
#define RCG_ERR_BREAKDOWN     -6   /* p^T A p <= 0 or non-finite in CG      */
#define RCG_ERR_TIMEOUT       -7   /* a bounded device wait ran out         */
#define RCG_ERR_RANK_CAP      -8   /* basis V would exceed r_max            */

/* ---- option values --------------------------------------------------- */
#define RCG_FP64        0   /* every vector and product in float64             */
#define RCG_MIXED       1   /* float32 vectors / stencil / basis products, float64
                               refinement residuals, Galerkin matrices and
                               rank decisions                                  */
#define RCG_MAX_PRIVATE 8   /* private columns of a recycle space U_j       */
/* check of Algorithm 2: the Galerkin guess x0 = V (V^T A~ V)^-1 V^T b (this
 * library's default) or the paper's minimum-residual guess x0 = U K^T b with
 * A~ V = K R, U = V R^-1 (Sec. 4.2.1, eq. initialz); both with an explicitly
 * recomputed float64 residual */
#define RCG_GALERKIN    0
#define RCG_MR          1
/* inner solver of the correction equation (eq. resi): CG deflated by U_j
 * (Saad et al. 2000) or the paper's recycled MINRES with K_j = A~ U_j
 * (Sec. 4.1, eqs. eq01 and SmallMin) */
#define RCG_CG          0
#define RCG_MINRES      1
/* recycling: the paper's inner-outer method (global V and per-RHS U_j) or
 * per-RHS recycle spaces only, the comparison method of Sec. 6.3 / Table 2
 * (no V check: each system from the minimum-residual guess in range(U_j),
 * new directions into U_j only) */
#define RCG_INNER_OUTER 0
#define RCG_PER_RHS     1
/* diffusion coefficient: fixed (Sec. 2.1: D known, set by rcg_set_diffusion)
 * or tracking the absorption at every sample and parameter point,
 * D = 1 / (3 (mu + mu_s')) (the diffusion approximation's coefficient; an
 * extension).  Tracking makes A~ change off the diagonal (every face weight
 * and the Robin term D/(1 + alpha) of the Schur complement, Sec. 3), moves
 * the effective source / detector weights of Sec. 3.1 with the sample, and
 * gives the Jacobian of eq. newjac the stencil term and the weights'
 * derivatives.  With tracking, the D of rcg_set_diffusion is only the
 * reference for the solver's right-hand sides: the systems are solved with
 * those weights and the solutions scaled to the sample's own (relative
 * tolerances and Algorithm 2's decisions do not change under that scaling);
 * rcg_solution_get, rcg_full_eval and the reduced model use the sample's
 * weights.  Runs the scalar CG path (the float4 stencils share one D). */
#define RCG_LEARN_DEFLATE 0
#define RCG_LEARN_START   1
#define RCG_D_FIXED       0
#define RCG_D_TRACKS_MU   1
#define RCG_SEQUENTIAL  0   /* the paper's order: V grows between RHS          */
#define RCG_WAVE        1   /* all RHS of `wave_samples` samples at once with V
                               frozen; ordered append afterwards               */

typedef struct rcg_ctx rcg_ctx;

typedef struct {
    int    dim;        /* 2 or 3                                             */
    int    N;          /* unknown nodes per axis (>= 2)                      */
    double robin_A;    /* reflection constant A of eq. ModelPDE2 (> 0)       */
} rcg_grid;

typedef struct {
    int    precision;     /* RCG_FP64 | RCG_MIXED                           */
    int    order;         /* RCG_SEQUENTIAL | RCG_WAVE                      */
    int    wave_samples;  /* samples per wave in RCG_WAVE (0 = all given)   */
    double tau_rank;      /* append iff ||new part|| / ||x|| > tau_rank     */
    int    k_u;           /* seed eigenvectors (Sec. 4.2.2: 10)             */
    int    k_cap;         /* max columns of a recycle space U_j = [U_0,
                             private columns]; the private part holds at
                             most RCG_MAX_PRIVATE columns, so values above
                             k_u + RCG_MAX_PRIVATE act as that bound; when
                             full, the oldest private column goes first     */
    int    r_max;         /* max columns of V (device memory is sized by it)*/
    int    max_samples;   /* sample slots (0..max_samples-1)                */
    int    maxit;         /* CG iterations per RHS before NOT_CONVERGED     */
    double inner_eta;     /* RCG_MIXED: float32 CG cycle stops at
                             eta * ||r_restart|| before an FP64 refinement  */
    int    check_refine;  /* extra Galerkin refinement steps of the check   */
    int    keep_solutions;/* keep every delivered x (for rcg_solution_get)  */
    int    seed_degree;   /* Chebyshev filter degree of the eigen seed      */
    long long spin_budget;/* polls of a tensor-core kernel's main-loop waits
                             for its MMAs (0 = 2^22; negative = none, so
                             every such wait runs out: exercises the error
                             path); on running out the call returns
                             RCG_ERR_TIMEOUT after the kernel has waited
                             (full bound) for its last MMAs               */
    int    learned;       /* RCG_MIXED: add the learned network's column to
                             the private U_j of every CG solve (needs
                             weights: rcg_learn_set_weights or _train)      */
    int    wave_rhs;      /* RCG_WAVE: right-hand sides per wave (0 = all):
                             a wave takes `wave_samples` samples x wave_rhs
                             consecutive RHS, so V grows between the RHS
                             blocks of a sample as in the paper's order      */
    int    check;         /* RCG_GALERKIN (default) | RCG_MR                */
    int    inner;         /* RCG_CG (default) | RCG_MINRES                  */
    int    recycle;       /* RCG_INNER_OUTER (default) | RCG_PER_RHS        */
    int    d_model;       /* RCG_D_FIXED (default) | RCG_D_TRACKS_MU        */
    double mu_s_prime;    /* reduced scattering mu_s' of RCG_D_TRACKS_MU
                             (> 0; default 1)                                */
    int    learned_mode;  /* with `learned`: RCG_LEARN_DEFLATE (default) keeps
                             the network's column in U_j for every CG
                             iteration of the solve (augmented CG);
                             RCG_LEARN_START uses it in the first Galerkin
                             projection x0 += W (W^T A~ W)^-1 W^T r only and
                             then iterates deflated by U_j alone (no
                             per-iteration cost)                             */
} rcg_options;

typedef struct {
    int    sample, rhs;   /* sample slot and RHS index                      */
    int    iters;         /* CG iterations (0: V sufficed)                  */
    int    restarts;      /* refinement restarts                            */
    int    appended;      /* 1 if a column was appended to V                */
    int    status;        /* RCG_OK / RCG_ERR_NOT_CONVERGED / _BREAKDOWN    */
    double relres0;       /* relres of the Galerkin guess from V            */
    double relres;        /* final relres, float64 residual recomputed      */
    double ratio;         /* ||new part|| / ||x|| at the append decision    */
    int    augmented;     /* 1 if the learned column joined U_j of this solve */
} rcg_stat;

/* Fill *o with defaults: FP64, sequential, tau_rank 1e-12, k_u 10,
 * k_cap 256, r_max 2048, max_samples 32, maxit 20000, inner_eta 1e-4,
 * check_refine 0, keep_solutions 0, seed_degree 0 (automatic), learned 0,
 * wave_rhs 0, check RCG_GALERKIN, inner RCG_CG, recycle RCG_INNER_OUTER,
 * d_model RCG_D_FIXED, mu_s_prime 1, learned_mode RCG_LEARN_DEFLATE. */
void rcg_options_default(rcg_options *o);

/* Create a context on the current CUDA device.  `cuda_stream` is a
 * cudaStream_t (NULL = legacy default stream).  Device memory for the grid,
 * the basis (r_max columns) and the coefficient fields is allocated here;
 * per-wave workspaces grow on demand.  Returns RCG_ERR_OOM if it fails. */
int  rcg_create(rcg_ctx **out, const rcg_grid *g, const rcg_options *o, void *cuda_stream);
void rcg_destroy(rcg_ctx *c);
const char *rcg_last_error(const rcg_ctx *c);
const char *rcg_strerror(int code);

/* Diffusion coefficient D at the n unknowns (host, float64, > 0, finite).
 * Fixed across samples (Sec. 2.1: D known). Must precede rcg_set_sample. */
int rcg_set_diffusion(rcg_ctx *c, const double *D);

/* Sources on the z = 0 face and detectors on the z = 1 face (Sec. 2.1):
 * face points as (i, j) pairs, 1-based (j = 1 in 2D), and weights
 * (NULL = 1).  Defines nrhs = nsrc + ndet effective right-hand sides. */
int rcg_set_sources_detectors(rcg_ctx *c, int nsrc, const int *src_ij, const double *src_w,
                              int ndet, const int *det_ij, const double *det_w);

/* Per-RHS tolerance (host, nrhs values in (0, 1)); default 1e-8. */
int rcg_set_tolerances(rcg_ctx *c, const double *tol);

/* Absorption mu at the n unknowns for sample slot s (host / device float64,
 * >= 0).  A~_s = A~_* + diag(h^2 mu_s) (eq. sum).  Setting the slot that
 * rcg_seed used as s0 discards the seed (rcg_seed must run again). */
int rcg_set_sample(rcg_ctx *c, int s, const double *mu);
int rcg_set_sample_device(rcg_ctx *c, int s, const double *mu_dev);

/* Apply A~_s to ncols device vectors: y_j = A~_s x_j (n per column, leading
 * dimension n).  prec RCG_FP64 takes double*, RCG_MIXED float* (the float32
 * operator of the inner iterations).  Parity / benchmarking entry. */
int rcg_apply(rcg_ctx *c, int s, int prec, const void *x_dev, void *y_dev, int ncols);

/* The same operator application as rcg_apply, for callers that cannot
 * allocate device memory during the call: for example a caller whose device
 * memory is owned by another allocator (a framework's caching pool) or that
 * cannot afford cudaMalloc / cudaFree (cudaFree waits for the whole device)
 * on a repeated call.  rcg_apply allocates its per-column tables on each
 * call; this entry point calls no cudaMalloc, cudaFree or allocating library
 * routine and keeps the tables in one static device array of the library,
 * sized for RCG_NOALLOC_MAX_COLS columns (24 KiB), which every GPU that
 * loads the library holds until the process exits.  The paper has no
 * counterpart; it is a property of this library's interface.
 *   - ncols > RCG_NOALLOC_MAX_COLS returns RCG_ERR_INVALID (message in
 *     rcg_last_error); x_dev / y_dev as in rcg_apply (caller-owned).
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) once for that device; make that first call
 *     before any stream capture begins.
 *   - All calls share the array and it keeps the last call's tables: calls
 *     that overlap on the GPU (other streams or host threads) race on it.
 *   - Returns after the context's stream has finished the application. */
#define RCG_NOALLOC_MAX_COLS 1024
int rcg_apply_noalloc(rcg_ctx *c, int s, int prec, const void *x_dev, void *y_dev, int ncols);

/* The float32 operator of the inner CG iteration (the stencil of eq. sum,
 * A~_s = A~_* + diag(h^2 mu_s), applied to every Lanczos / CG vector, Sec.
 * 5.3): y_j = A~_s x_j for ncols device columns of n floats (leading
 * dimension n, 16-byte aligned; needs N % 4 == 0), and dots[j] += x_j^T y_j
 * (device, ncols doubles, may be NULL).  variant: -1 the autotuned choice
 * (the one the solver uses for this grid and column count), or one of the
 * RCG_STENCIL_VARIANTS kernels named by rcg_stencil_variant_name (0: rows,
 * 1: plane ring, 2..13: z-marching tiles, 14..15: z-marching tiles with
 * registers for three CTAs per SM, 16..18: planes of 64 x 16 or 64 x 8
 * tiles copied by TMA into a shared-memory ring, Nx % 64 == 0).
 * RCG_ERR_INVALID if the variant does not support the grid;
 * RCG_ERR_TIMEOUT if a TMA copy's wait ran out.  Parity / timing entry;
 * returns after the context's stream has finished. */
#define RCG_STENCIL_VARIANTS 19
int rcg_apply_f32(rcg_ctx *c, int s, int variant, const float *x_dev, float *y_dev, int ncols, double *dots_dev);
/* Name of stencil variant v (NULL if out of range); 1 if the variant runs on
 * the grid of c, else 0. */
const char *rcg_stencil_variant_name(int v);
int rcg_stencil_variant_ok(const rcg_ctx *c, int v);
/* The autotuner's record (one line per tuned grid and lane-count class: the
 * time of every candidate and the choice) into buf (len bytes, NUL-
 * terminated); returns the full length. */
int rcg_tuning_report(char *buf, int len);

/* The basis product of the orthogonalisation in the append (Sec. 5.3
 * incremental QR: V^T W, W^T W, V^T Q, Q^T Q), exposed for testing and
 * timing: C = A^T diag(w) B (w == NULL: C = A^T B; w != NULL is the weighted
 * Gram V^T Delta V of the check and the reduced model, eq. newreduced, with
 * w = h^2 (mu - mu_*) of finite support) with A (n x ka) and B (n x kb)
 * float32, column-major with
 * leading dimensions lda, ldb, and C (ka x kb, leading dimension ldc)
 * float64, all three in device memory and owned by the caller.
 *   - engine 0: CUDA-core kernel (float32 products, float64 partial sums);
 *     engine 1: tensor cores (tcgen05 kind::tf32, three MMAs per product,
 *     float64 sum of the split-K slices), which needs A and B 16-byte
 *     aligned and lda, ldb multiples of 4 (else RCG_ERR_INVALID); with w it
 *     visits only the 32-row blocks where w does not vanish.  w (float64,
 *     n, device, 16-byte aligned) scales the rows of A in float32.
 *   - n == 0 gives C = 0 (A and B may then be NULL).
 *   - symmetric != 0: A == B, ka == kb, lda == ldb (engine 1 computes the
 *     upper tiles and mirrors them).
 *   - Runs on `stream` (a cudaStream_t, NULL = default stream) and returns
 *     after it has finished.  The split-K scratch is one library buffer per
 *     GPU, grown on demand and kept until exit; calls from several host
 *     threads take turns.
 *   - RCG_ERR_INVALID for bad sizes or pointers, RCG_ERR_CUDA for a CUDA
 *     error, RCG_ERR_TIMEOUT if a tensor-core wait ran out (C undefined). */
int rcg_gemm_tn_f32(const float *A, long long lda, int ka, const float *B, long long ldb, int kb, long long n,
                    const double *w, double *C, int ldc, int engine, int symmetric, void *stream);

/* Seed step of Algorithm 2 at sample s0: U_0 = U0 (host n x k_u, column-
 * major) or, if U0 == NULL, the k_u smallest eigenvectors of A~_{s0} by a
 * Chebyshev-filtered subspace iteration on the device; X_0 by deflated CG
 * with U_0; V = basis([U_0, X_0]); U_j = [U_0, X_0(:,j)].  A~_{s0} becomes
 * A~_* of the cached Galerkin matrix V^T A~_* V.  stats (host, nrhs) may be
 * NULL.  Resets any previous basis. */
int rcg_seed(rcg_ctx *c, int s0, const double *U0, rcg_stat *stats);

/* Return to the state right after rcg_seed (V, U_j, caches) without
 * recomputing it: O(1). */
int rcg_reset_to_seed(rcg_ctx *c);

/* The seed step's result of context src (Algorithm 2's first three lines:
 * U_0, X_0, V = basis([U_0, X_0]), U_j = [U_0, X_0(:, j)], C_* = V^T A~_* V)
 * copied into c, which then behaves as if rcg_seed had run on it (the paper
 * computes the seed once, offline, and reuses it, Sec. 5.3).  Both contexts
 * on the same device, with the same grid, D, sources / detectors and the
 * seed sample's mu in the same slot (checked; RCG_ERR_INVALID otherwise).
 * Precision: equal, or a float32 seed into a float64 context (the float32
 * values are exact in float64; V^T X_0 is recomputed in float64); a float64
 * seed into a float32 context is refused.  src is not changed. */
int rcg_seed_copy(rcg_ctx *c, const rcg_ctx *src);

/* Algorithm 2 outer loop over samples s_first .. s_first+s_count-1 (each
 * set by rcg_set_sample), in the order of options.order.  stats (host,
 * s_count*nrhs, [sample][rhs]) may be NULL.  Returns RCG_ERR_NOT_CONVERGED
 * if any RHS hit maxit (stats still filled), RCG_ERR_RANK_CAP if V is full. */
int rcg_solve_all(rcg_ctx *c, int s_first, int s_count, rcg_stat *stats);

/* Current number of columns of V and a copy of V (host, n x r float64). */
int rcg_basis_rank(const rcg_ctx *c, int *r);
int rcg_basis_get(rcg_ctx *c, double *V);

/* Algorithm 1 (Sec. 4.2.2, "Generate Symmetric Global Basis via Truncated
 * SVD"), steps 2-3, on the delivered solutions kept so far (needs
 * options.keep_solutions): S = [X_s1, X_s2, ...], the kept samples in
 * ascending order, each X_s = the n x nrhs solutions of sample s; V becomes
 * the first r left singular vectors of S with
 * r = min(r_max, #{i : sigma_i > tau sigma_1}) (r_max <= 0: options.r_max).
 * The singular values come from the float64 Gram S^T S (parallel Jacobi), so
 * values below ~1e-7 sigma_1 are not resolved.  Afterwards C_* is rebuilt for
 * the new V, the leading min(k_u, r) columns of V serve as the shared
 * deflation space, the private recycle lists restart empty, and
 * rcg_reset_to_seed returns to the compressed basis.  sigma (host, may be
 * NULL): the first min(sigma_len, m) singular values, descending; nsnap (may
 * be NULL): m, the number of columns of S.  RCG_ERR_INVALID before rcg_seed,
 * without kept solutions, for tau < 0, for m > RCG_COMPRESS_MAX_COLS, or if
 * no singular value exceeds tau sigma_1 (V is unchanged then). */
#define RCG_COMPRESS_MAX_COLS 4096
int rcg_basis_compress(rcg_ctx *c, int r_max, double tau, double *sigma, int sigma_len, int *nsnap);

/* Delivered solutions of sample s (host, n x nrhs float64) from the last
 * rcg_solve_all (or rcg_seed for s0); needs options.keep_solutions. */
int rcg_solution_get(rcg_ctx *c, int s, double *X);

/* Reduced model at absorption mu (host, n): Psi_r = C~_r^T A~_r^-1 B~_r with
 * A~_r = V^T A~(mu) V, B~_r = V^T B~, C~_r = V^T C~ (eq. newreduced) into
 * Psi (host, ndet x nsrc column-major: Psi[d + ndet*s]); if dmu != NULL
 * (host, n x nparam) also J[d + ndet*(s + nsrc*k)] =
 * -Z_r^T V^T diag(h^2 dmu_k) V X_r (eq. newjac). */
int rcg_rom_eval(rcg_ctx *c, const double *mu, int nparam, const double *dmu,
                 double *Psi, double *J);

/* The full-order transfer function and Jacobian of sample s from its
 * delivered solutions (needs options.keep_solutions): Psi = C~^T X (Sec. 3.1)
 * with X the source columns, and, if dmu != NULL (host, n x nparam),
 * J[d + ndet*(s' + nsrc*k)] = -Z^T diag(h^2 dmu_k) X (eq. newjac) with Z the
 * detector columns; same layouts as rcg_rom_eval.  For comparing the reduced
 * model against the full one (the interpolation property of Sec. 3.4). */
int rcg_full_eval(rcg_ctx *c, int s, int nparam, const double *dmu, double *Psi, double *J);

/* The basis update of the append (Sec. 5.3: W - V (V^T W), Q = W R^-1,
 * V <- Q R2^-1), exposed for testing and timing: Out = alpha V C + beta Out
 * with V (n x k, ld ldv) float32, C (k x m, ld ldc) float64 and Out (n x m,
 * ld ldo) float32, all in device memory and owned by the caller.  engine 0:
 * CUDA cores (float32); engine 1: tensor cores (3xTF32; V 16-byte aligned
 * with ldv a multiple of 4, else RCG_ERR_INVALID).  Runs on `stream` and
 * returns after it has finished; RCG_ERR_TIMEOUT if a tensor-core wait ran
 * out (Out undefined). */
int rcg_gemm_nn_f32(const float *V, long long ldv, int k, const double *C, int ldc, int m, long long n, float *Out,
                    long long ldo, double alpha, double beta, int engine, void *stream);

/* Save the recycling state (V, C_* = V^T A~_* V and the mu_* it belongs to,
 * X_0 and V^T X_0, the private recycle lists, the state right after the seed,
 * the learned network's weights if any) to a file, and load it into a
 * context created with the same grid, precision, D and sources/detectors
 * (checked: RCG_ERR_INVALID otherwise).  The paper reuses the basis across
 * optimisation steps (Sec. 4.2.2); this lets a later process continue from
 * it.  The seed sample slot is set to the saved mu_*; rcg_reset_to_seed
 * returns to the saved seed state. */
int rcg_save(rcg_ctx *c, const char *path);
int rcg_load(rcg_ctx *c, const char *path);

/* Device-resident variant of rcg_rom_eval: mu_dev (n), dmu_dev (n x nparam),
 * Psi_dev, J_dev device float64. */
int rcg_rom_eval_device(rcg_ctx *c, const double *mu_dev, int nparam, const double *dmu_dev,
                        double *Psi_dev, double *J_dev);

/* The reduced model at nq parameter points in one call (Sec. 4.2.2: the
 * optimisation evaluates Psi_r and its Jacobian at many p through the same
 * V).  Device float64 arrays: mu_dev nq x n (point q at mu_dev + q n),
 * dmu_dev nq x nparam x n (d mu / d p_k of point q at dmu_dev + (q nparam + k) n)
 * or NULL, Psi_dev nq x ndet x nsrc (point q as in rcg_rom_eval at
 * Psi_dev + q ndet nsrc), J_dev nq x nparam x ndet x nsrc or NULL (needs
 * dmu_dev).  Each point's values equal rcg_rom_eval's at that point up to
 * rounding.  The points are processed in chunks of
 * rcg_rom_eval_batch_chunk() points, so the workspace stays within
 * RCG_ROM_BATCH_WORKSPACE bytes (one point at a time if a single point needs
 * more).  The caller owns every array; the call returns after the results
 * are written.  RCG_ERR_INVALID for nq < 0, missing arrays or an empty basis,
 * RCG_ERR_NOT_SPD if a reduced matrix is not positive definite. */
int rcg_rom_eval_batch(rcg_ctx *c, int nq, const double *mu_dev, int nparam, const double *dmu_dev,
                       double *Psi_dev, double *J_dev);

/* Points per chunk of rcg_rom_eval_batch for n unknowns, a basis of r
 * columns, nsrc sources, ndet detectors and nparam parameters (0: no
 * Jacobian): the largest count, at least 1 and at most 256, whose workspace
 * (per point the reduced matrix, its weights, block lists and solves; per
 * point and parameter a Gram, its block list and its tensor-core partial
 * sums) fits in RCG_ROM_BATCH_WORKSPACE bytes.  Host arithmetic only:
 * allocates nothing, needs no context; -1 for negative sizes. */
#define RCG_ROM_BATCH_WORKSPACE (4LL << 30)
int rcg_rom_eval_batch_chunk(long long n, int r, int nsrc, int ndet, int nparam);

/* Elapsed device milliseconds of the named phase in the last call that ran
 * it ("check", "cg", "append", "seed_eig", "seed_x0", "rom", "rom_batch",
 * "compress");
 * -1 if none. */
double rcg_phase_ms(const rcg_ctx *c, const char *phase);

/* Number of kernel launches issued by this context since creation. */
long long rcg_launch_count(const rcg_ctx *c);

/* Device-side profile of the kernels of one inner CG iteration (kernel
 * 0: stencil q = A~ p with the fused p^T q; 1: update of x, r with the fused
 * r^T r and private (A~ U_j)^T r; 2: the shared (A~ U_0)^T r dots; 3: the
 * per-lane scalars (decision, beta, mu); 4: direction p = r + beta p - U_j mu;
 * the float64 path has no separate kernels 2 and 3).
 * rcg_profile_enable(c, 1) resets and starts it (CUDA events around every
 * launch on the context's stream, plus device work counters); 0 stops it.
 * rcg_profile_get fills: launches, total device ms, lane_units (sum over
 * launches of the active right-hand-side lanes: stencil columns for 0,
 * update lanes for 1, direction lanes for 2-4) and defl_cols (sum over those
 * lanes of their recycle-space columns). */
typedef struct {
    long long launches;
    double    ms;
    double    lane_units;
    double    defl_cols;
} rcg_kprof;
int rcg_profile_enable(rcg_ctx *c, int on);
int rcg_profile_get(rcg_ctx *c, int kernel, rcg_kprof *out);

/* ---------------------------------------------------------------- learned
 * Learned augmentation of the private recycle spaces (not in the paper; the
 * learned step of this library's mixed-precision contender).  For a
 * right-hand side whose Galerkin check fails, a 3D CNN on a coarse grid
 * (block means over f^3 fine nodes, f = 4, 2 or 1) maps the features
 * [coarse(r0) / max|coarse(r0)|, coarse(mu) / mean(mu) - 1] (bfloat16) of its
 * check residual r0 and the sample's mu to the shape of the correction
 * A~^-1 r0; the trilinear upsampling x_hat joins that solve's private U_j
 * (never V) iff its Galerkin pivot sqrt(s/d) > tau_rank, where d = x_hat^T
 * A~ x_hat and s = d - c^T (U_j^T A~ U_j)^-1 c, c = U_j^T A~ x_hat.  Network:
 * a 3-level U-Net on the coarse grid (levels halved by 2x2x2 block means,
 * dims ceil(G/2); nearest-cell doubling on the way up), ten 3x3x3
 * zero-padded convolutions with bias, (Cin, Cout) = (2,16) (16,16) | (16,32)
 * (32,32) | (32,64) | (96,32) (32,32) | (48,16) (16,16) (16,1), where layers
 * 5 and 7 read [up(deeper level), skip of their level]; ReLU after every
 * layer but the last.  rcg_learn_nparams() = 243,473 parameters laid out per
 * layer as W [Cout][Cin][27] (offset (dz+1)*9+(dy+1)*3+(dx+1)) then
 * b [Cout].  The convolutions run on the tensor cores with bfloat16 weights
 * and activations (every ReLU and halving output rounded to bfloat16) and
 * float32 accumulation; training keeps float32 master weights (Adam, mean
 * squared error against coarse(x - x0) / max|coarse(x - x0)| of recorded
 * solves) and forms the gradient from bfloat16 operands.  All arrays below
 * are host memory owned by the caller; coarse arrays are
 * [batch][channel][Gz][Gy][Gx], x fastest. */
int rcg_learn_nparams(void);
/* dims[0..3] = Gx, Gy, Gz, f of the context's grid. */
int rcg_learn_geometry(rcg_ctx *c, int *dims);
int rcg_learn_set_weights(rcg_ctx *c, const float *theta, int nparam);
int rcg_learn_get_weights(rcg_ctx *c, float *theta, int nparam);
/* on != 0: every later rcg_solve_all records one (features, target) pair per
 * CG solve (held in device memory); *npairs = pairs recorded so far. */
int rcg_learn_record(rcg_ctx *c, int on);
int rcg_learn_pairs(rcg_ctx *c, int *npairs);
/* Adam (beta 0.9 / 0.999) over the recorded pairs: `epochs` passes in
 * shuffled batches of `batch` (shuffles seeded by `seed`); *loss (may be NULL)
 * = mean loss of the last epoch.  RCG_ERR_INVALID if nothing was recorded. */
int rcg_learn_train(rcg_ctx *c, int epochs, int batch, double lr, unsigned long long seed, double *loss);
/* The network (inference: bfloat16 weights and activations) on B inputs
 * in[B][2][V] -> out[B][V]. */
int rcg_learn_forward(rcg_ctx *c, const float *in, int B, float *out);
/* Loss and its gradient grad[nparam] with respect to the master weights for
 * one batch in[B][2][V], targets tg[B][V] (the training pass: bfloat16
 * operands, so both approximate those of the exact network to bfloat16
 * precision). */
int rcg_learn_gradient(rcg_ctx *c, const float *in, const float *tg, int B, float *grad, double *loss);
/* Features feat[2][V] (may be NULL) and x_hat[n] (may be NULL) of one
 * residual r0[n] (float32) at sample slot s, with the bfloat16 weights. */
int rcg_learn_predict(rcg_ctx *c, int s, const float *r0, float *feat, float *xhat);

#ifdef __cplusplus
}
#endif
#endif /* RCG_H */
