/*
 * hypersara.h - C ABI of the GB300 HyperSARA primal-dual hot path.
 *
 * Operations follow Abdulaziz, Dabbech & Wiaux, "Wideband super-resolution
 * imaging in radio interferometry via low rankness and joint average sparsity
 * models (HyperSARA)":
 *   - measurement operator Phi_l = Theta_l G_l F Z and its adjoint
 *     (Sec. 2.1, Eq. "inverse"; adjoint in Sec. 3.2 after Eq. "min-problem-d");
 *   - SARA dictionary Psi^dagger / Psi: Dirac + Daubechies 1-8 (Sec. 2.3);
 *   - proximity operators (Sec. 3.3, Eqs. "proj-plus", "prox-L*", "prox-L21")
 *     and their Moreau duals (Eq. "md");
 *   - one iteration of the preconditioned primal-dual algorithm (Algorithm 2:
 *     steps 2-23, data blocks, fixed or adaptive l2 bounds), its variants
 *     (Sec. 4.2) and the re-weighting outer loop (Algorithm 1).
 *
 * Conventions shared by every entry point
 *   Precision   a plan is FP32 (HS_F32: real = float, complex = float2 {re, im})
 *               or FP64 (HS_F64: real = double, complex = double2). Every
 *               real/complex buffer passed to that plan uses its precision.
 *               l2-ball norms, epsilon, singular values, weights of the nuclear
 *               norm and the Gram eigendecomposition are always FP64.
 *   Layout      image cube X: L x ny x nx reals, channel-major, row-major images;
 *               pixel (iy, ix) has centred coordinates (ix - nx/2, iy - ny/2).
 *               coefficient cube A: 9 x L x ny x nx reals; basis 0 is Dirac,
 *               basis p (1..8) the Mallat-layout periodic DWT with db_p; the
 *               whole frame is scaled by 1/3 so that Psi Psi^dagger = I.
 *               visibilities: sum_l M_l complex values, channel-concatenated in
 *               the order the plan was created with (the "caller order").
 *   Memory      pointers named "device" are CUDA device pointers the caller owns;
 *               the library never frees them and keeps no reference after the
 *               call returns, except where a create function says so. Plans and
 *               states own only what they derive (sorted coordinates, gridding lists,
 *               tables, scratch), allocated at creation: the compute entry points
 *               allocate nothing.
 *   Streams     `stream` is a cudaStream_t (NULL = legacy default stream). Compute
 *               entry points are asynchronous on it unless stated otherwise.
 *               One plan or state must not be used from two streams at once
 *               (they share scratch).
 *   Errors      every function returns an hs_status; argument errors are detected
 *               on the host before any launch and leave outputs untouched.
 *               hs_last_error() returns a thread-local message for the last failure.
 */
#ifndef HYPERSARA_H
#define HYPERSARA_H

#include <stdint.h>

#if defined(__GNUC__)
#define HS_API __attribute__((visibility("default")))
#else
#define HS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HS_OK = 0,
    HS_ERR_ARG = -1,      /* invalid argument (null pointer, size, mode) */
    HS_ERR_CUDA = -2,     /* a CUDA runtime call failed */
    HS_ERR_NOMEM = -3,    /* device or host allocation failed at creation */
    HS_ERR_TIMEOUT = -4,  /* a bounded device-side wait gave up */
    HS_ERR_STATE = -5     /* object used in the wrong state */
} hs_status;

typedef enum { HS_F32 = 0, HS_F64 = 1 } hs_prec;

/* plan flags */
/* Gridding adds one window per warp at a time into per-warp tiles with
 * Kahan-compensated sums (FP32 plans). Without it grids of at least 64 x 64
 * cells use the register sweep (uncompensated, faster) and smaller grids add 4
 * non-overlapping windows per warp pass into per-warp tiles. Every form sums in
 * a fixed order, so all are bitwise reproducible. */
#define HS_PLAN_COMPENSATED 1u
/* FP32 plans: form the nuclear prox's L x L Gram matrix with register-blocked
 * FMA on the CUDA cores instead of the tensor cores (tcgen05 BF16 products of
 * exact digit splits). Without it the autotuner picks the faster form (the
 * tensor cores when timing is off); the CUDA-core form is also used when a
 * buffer is not 16-byte aligned. */
#define HS_PLAN_GRAM_FMA 2u
/* Keep the default parameters instead of timing candidates at creation. By
 * default a plan times, on itself, the sweep-gridding row cut and list cap
 * ((32, 512), (64, 1024), (128, 2048)), F^H over all channels at once against
 * L2-sized channel chunks and, for FP32 plans, the tensor-core against the
 * CUDA-core Gram matrix, and keeps the fastest (choices cached per
 * process by grid, L, visibilities, precision and flags; hs_plan_info reports
 * them and the candidate times). */
#define HS_PLAN_NO_TUNE 4u
/* Apply F^H in L2-sized channel chunks (the row pass of each chunk, on a stream
 * of the plan, overlapping the next chunk's column pass) without timing it
 * against the single pass over all channels. Same arithmetic either way. */
#define HS_PLAN_FFT_CHUNKED 8u

typedef struct hs_plan* hs_plan_t;
typedef struct hs_pd_state* hs_pd_state_t;

/* Library version and build information (static string). */
HS_API const char* hs_version(void);

/* Thread-local description of the last error ("" if none). */
HS_API const char* hs_last_error(void);

/*
 * hs_plan_create - measurement setup for one wideband problem (Sec. 2.1).
 *   nx, ny        image size; powers of two in [16, 2048], divisible by 2^wavelet_levels.
 *   L             number of channels, 1..1024 (the nuclear-norm prox needs L <= 64).
 *   vis_offsets   HOST array of L+1 int64: visibilities of channel l are
 *                 [vis_offsets[l], vis_offsets[l+1]); vis_offsets[0] = 0,
 *                 nondecreasing; empty channels are allowed; total < 2^31.
 *   uv            DEVICE array (total x 2) of the plan's real type: (u, v) in
 *                 radians, u pairs with the x axis; values must lie in [-pi, pi).
 *                 Read once during the call (copied to the host and sorted).
 *   weights       DEVICE array (total) of the plan's real type: diagonal natural
 *                 weights Theta (Sec. 2.1), or NULL for Theta = I. Copied.
 *   precond       DEVICE array (total) of the plan's real type: diagonal
 *                 preconditioner U > 0 (Sec. 3.3), or NULL for U = I. Copied.
 *                 Used by hs_op_norm2 and the primal-dual states.
 *   oversample    grid oversampling o; must be 2.
 *   J             interpolation kernel support; must be 8.
 *   kb_beta       Kaiser-Bessel shape; <= 0 selects pi sqrt((J/o)^2 (o-1/2)^2 - 0.8).
 *   wavelet_levels  DWT levels of the SARA bases, 1..8.
 *   prec          HS_F32 or HS_F64.
 *   flags         bitwise OR of HS_PLAN_* flags.
 *   stream        stream used for the set-up copies; the call synchronises it.
 * On success *out owns device memory until hs_plan_destroy. Errors: HS_ERR_ARG
 * (sizes, uv outside [-pi, pi) or non-finite, bad offsets), HS_ERR_NOMEM, HS_ERR_CUDA.
 */
HS_API hs_status hs_plan_create(hs_plan_t* out, int nx, int ny, int L, const int64_t* vis_offsets,
                         const void* uv, const void* weights, const void* precond,
                         int oversample, int J, double kb_beta, int wavelet_levels,
                         hs_prec prec, unsigned flags, void* stream);

/*
 * hs_plan_create_blocks - hs_plan_create with intra-channel data blocks
 * (Sec. 2.1, masks M_l^b): block_offsets, HOST nblocks + 1 int64, splits the
 * visibility vector (caller order) into contiguous blocks; it runs from 0 to
 * the total, is nondecreasing and contains every channel boundary of
 * vis_offsets (so nblocks >= L). PD states on the plan then keep one l2 bound,
 * one ball projection and one residual per block (eps and rho of nblocks
 * values). hs_plan_create is this call with one block per channel.
 */
HS_API hs_status hs_plan_create_blocks(hs_plan_t* out, int nx, int ny, int L, const int64_t* vis_offsets,
                                int nblocks, const int64_t* block_offsets, const void* uv, const void* weights,
                                const void* precond, int oversample, int J, double kb_beta,
                                int wavelet_levels, hs_prec prec, unsigned flags, void* stream);

/* Frees everything the plan owns. The caller must make sure no work using the
 * plan is still running. NULL is accepted. */
HS_API hs_status hs_plan_destroy(hs_plan_t plan);

/* Sizes derived by a plan (all host values). */
typedef struct {
    int nx, ny, L, Kx, Ky, levels, prec, flags;
    int64_t total_vis;
    int64_t grid_tile_entries;    /* gridding list slots: visibility-tile pairs plus group padding */
    int tile_x, tile_y;           /* gridding tile size in grid cells */
    int kb_terms;                 /* coefficients per kernel polynomial piece */
    double kb_beta;
    double kb_fit_max_err;        /* max |poly - phi| / phi(0) of the kernel fit */
    int64_t device_bytes;         /* device memory held by the plan */
    int nblocks;                  /* data blocks (L unless created with hs_plan_create_blocks) */
    int gram_tc;                  /* FP32 Gram matrix on the tensor cores (1) or CUDA cores (0) */
    int sweep_hmax, sweep_cap;    /* sweep gridding: rows per work item, window cap per list */
    int tuned;                    /* 0 defaults, 1 timed at creation, 2 from the process cache */
    double tune_ms;               /* host time spent choosing */
    double tune_grid_ms[3];       /* gridding launch per candidate (32, 64, 128 rows); 0 if not timed */
    double tune_gram_ms[2];       /* Gram matrix: tensor cores, CUDA cores; 0 if not timed */
    int fft_adj_chunk;            /* channels per F^H chunk (0: all at once) */
    double tune_fft_ms[2];        /* F^H: all channels, L2-sized chunks; 0 if not timed */
} hs_plan_info_t;

HS_API hs_status hs_plan_info(hs_plan_t plan, hs_plan_info_t* info);

/*
 * hs_set_device_limit - cap the device memory the library's plans and PD
 * states may hold in this process, in bytes (0: no cap, the default). An
 * allocation that would pass it fails with HS_ERR_NOMEM before cudaMalloc is
 * called, and the plan or state being created is released. Existing
 * allocations are not affected. hs_device_bytes reports what is held now.
 */
HS_API hs_status hs_set_device_limit(int64_t bytes);
HS_API hs_status hs_device_bytes(int64_t* out);

/*
 * hs_plan_check - synchronise the stream and report whether a kernel of this
 * plan (or of a PD state on it) failed on the device since the last check
 * (the flag is then cleared): HS_ERR_TIMEOUT if a bounded device-side wait
 * expired, HS_ERR_ARG if an input was outside a kernel's range, HS_OK
 * otherwise. The tensor-core Gram kernel of the nuclear prox (hs_gram) is the
 * one that waits on the device (for its own tensor-core operations, 1 s
 * bound) and the one with a range (|z| < 2^60); after such a failure its
 * output is invalid. hs_pd_get performs the same check when it synchronises.
 */
HS_API hs_status hs_plan_check(hs_plan_t plan, void* stream);

/*
 * hs_phi_fwd - Y = Phi(X): Y_l = Theta_l G_l F Z x_l for every channel
 * (Sec. 2.1, Eq. "inverse"). X: DEVICE L x ny x nx reals. Y: DEVICE total
 * complex values, caller order. F is the unnormalised DFT with a negative
 * exponent; G_l interpolates the spectrum with the separable Kaiser-Bessel
 * kernel over 8 x 8 cells at t = u K / (2 pi).
 */
HS_API hs_status hs_phi_fwd(hs_plan_t plan, const void* X, void* Y, void* stream);

/*
 * hs_phi_adj - X = Phi^dagger(Y): x_l = Re(Z^T F^H G_l^H Theta_l y_l)
 * (adjoint stated after Eq. "min-problem-d"; Re because x_l is real, Sec. 2.1).
 * Y: DEVICE total complex (caller order). X: DEVICE L x ny x nx reals.
 */
HS_API hs_status hs_phi_adj(hs_plan_t plan, const void* Y, void* X, void* stream);

/*
 * hs_psi_fwd - A = Psi^dagger X (analysis, Sec. 2.3): for every channel,
 * A[0] = x / 3 and A[p] = W_p x / 3 (p = 1..8), W_p the periodic orthonormal
 * 2-D DWT with db_p, Mallat layout. X: DEVICE L x ny x nx; A: DEVICE 9 x L x ny x nx.
 */
HS_API hs_status hs_psi_fwd(hs_plan_t plan, const void* X, void* A, void* stream);

/*
 * hs_psi_adj - X = Psi A = (A[0] + sum_p W_p^T A[p]) / 3 (synthesis, the
 * adjoint and, for this frame, the left inverse of hs_psi_fwd).
 */
HS_API hs_status hs_psi_adj(hs_plan_t plan, const void* A, void* X, void* stream);

/*
 * hs_prox_l21 - row-wise soft threshold over channels (Eq. "prox-L21").
 * Row n = (basis b, pixel) collects A[b][0..L-1][pixel]. With
 * lambda_n = thr * w_rows[n] (w_rows: DEVICE 9 x ny x nx reals, or NULL for 1):
 *   dual = 0:  out_n = max(||a_n|| - lambda_n, 0) a_n / ||a_n||   (0 for a zero row)
 *   dual = 1:  out_n = a_n - prox(a_n) = a_n min(1, lambda_n / ||a_n||)   (Eq. "md")
 * A and out: DEVICE 9 x L x ny x nx; out may equal A. thr >= 0.
 */
HS_API hs_status hs_prox_l21(hs_plan_t plan, const void* A, const void* w_rows, double thr,
                      int dual, void* out, void* stream);

/*
 * hs_l21_grad - gradient of the weighted l2,1 norm sum_n w_n ||a_n||_2 (Sec.
 * 2.3): out_n = w_n a_n / ||a_n|| for every row n (across channels), 0 for a
 * zero row (the minimum-norm subgradient there). A, w_rows and out as in
 * hs_prox_l21; out may equal A. Used by the backward pass of the l2,1 term of
 * differentiable objectives.
 */
HS_API hs_status hs_l21_grad(hs_plan_t plan, const void* A, const void* w_rows, void* out, void* stream);

/*
 * hs_prox_nuclear - singular value soft threshold of the N x L matrix whose
 * column l is channel l (Eq. "prox-L*"), through the L x L Gram matrix
 * Z^T Z (FP64 accumulation) and its FP64 Jacobi eigendecomposition:
 *   dual = 0:  out = U diag(max(s - thr w, 0)) V^T
 *   dual = 1:  out = X - prox(X) = U diag(min(s, thr w)) V^T
 * w_sv: DEVICE L doubles (weight of the j-th largest singular value) or NULL
 * for 1. sv_out: DEVICE L doubles receiving the singular values of X in
 * descending order, or NULL. Requires L <= 64. out may equal X.
 * FP64 plans diagonalise the Gram matrix with an FP64 Jacobi method. FP32 plans
 * use an FP32 Jacobi method for the whole spectrum and refine in FP64 the
 * eigenpairs with sigma_j > thr w_j (the only ones whose factor differs from 1
 * in the dual form or from 0 in the prox form); singular values below the
 * threshold are then resolved to ~1e-7 sigma_max^2 / sigma_j.
 */
HS_API hs_status hs_prox_nuclear(hs_plan_t plan, const void* X, const double* w_sv, double thr,
                          int dual, void* out, double* sv_out, void* stream);

/*
 * hs_gram - the L x L Gram matrix S = Z^T Z of the N x L matrix Z whose column
 * l is channel l of X (+ Xadd when not NULL): the dense contraction inside
 * the nuclear prox (Eq. "prox-L*", Algorithm 2 step 5). S_out: DEVICE L x L
 * doubles, row-major (symmetric). Requires L <= 64.
 * FP32 plans use the tensor cores (tcgen05, BF16 operands) on exact integer
 * digits of z: per 64-pixel chunk and channel, z is quantised to 24 bits
 * relative to the chunk's largest magnitude, split into three base-256 digits,
 * and every digit product and tensor-core partial sum is an exact integer;
 * chunk partials are combined with compensated FP32 sums and FP64 across
 * CTAs, so |S - S_exact|_ij <~ 1e-7 sqrt(S_ii S_jj). Inputs need |z| < 2^60
 * (else HS_ERR_ARG from hs_plan_check). The CUDA-core form (HS_PLAN_GRAM_FMA,
 * and buffers not 16-byte aligned) sums runs of 32 pixels in FP32 with two-sum
 * compensation. FP64 plans sum in FP64. form: 0 the plan's choice (autotuner),
 * 1 tensor cores, 2 CUDA cores (FP32 plans; FP64 plans ignore it).
 */
HS_API hs_status hs_gram(hs_plan_t plan, const void* X, const void* Xadd, int form, double* S_out, void* stream);

/*
 * hs_proj_l2ball - per-channel projection onto B(y_l, eps_l) =
 * {z : ||z - y_l||_2 <= eps_l} (Sec. 3.2, functions g_l):
 *   dual = 0:  out_l = P_B(z_l) = y_l + (z_l - y_l) min(1, eps_l / ||z_l - y_l||)
 *   dual = 1:  out_l = z_l - P_B(z_l)
 * Z, Yd, out: DEVICE total complex (caller order); eps: DEVICE L doubles >= 0.
 * The norms are accumulated in FP64. rho_out: DEVICE L doubles receiving
 * ||z_l - y_l||, or NULL. out may equal Z.
 */
HS_API hs_status hs_proj_l2ball(hs_plan_t plan, const void* Z, const void* Yd, const double* eps,
                         int dual, void* out, double* rho_out, void* stream);

/*
 * hs_proj_l2ball_static - the projection of hs_proj_l2ball without a plan and
 * without any device allocation (the paper has no counterpart: it exists for
 * callers that hold only device pointers and must not allocate). Its scratch
 * is a fixed device array of HS_L2BALL_STATIC_DOUBLES doubles inside the
 * library (partial sums and per-channel scales); nothing in it needs to start
 * at zero.
 *   L:           channels, 1 <= L <= HS_L2BALL_STATIC_MAX_L (else HS_ERR_ARG,
 *                detected on the host before any launch);
 *   vis_offsets: DEVICE L + 1 int64, channel l owns [vis_offsets[l], vis_offsets[l+1]);
 *   Z, Yd, out:  DEVICE complex of `prec`, indexed by those offsets; out may equal Z;
 *   eps, rho_out, dual: as in hs_proj_l2ball (rho_out may be NULL).
 * The first call on a device (that device current) looks up the scratch
 * address with cudaGetSymbolAddress, which may load the library's device
 * code, and caches it; make that call before any stream capture. The scratch
 * is shared by every call on the device: calls whose executions overlap (two
 * streams or host threads) race and give wrong results.
 */
#define HS_L2BALL_STATIC_DOUBLES 65536
#define HS_L2BALL_STATIC_MAX_L 16384
HS_API hs_status hs_proj_l2ball_static(int L, const int64_t* vis_offsets, const void* Z, const void* Yd,
                                const double* eps, hs_prec prec, int dual, void* out, double* rho_out,
                                void* stream);

/*
 * hs_norm_l21 - sum_n w_n ||a_n||_2 over the rows of a coefficient cube
 * (the weighted l2,1 norm of Sec. 2.3). w_rows as in hs_prox_l21. The result is
 * written to *out_host after the stream has been synchronised.
 */
HS_API hs_status hs_norm_l21(hs_plan_t plan, const void* A, const void* w_rows, double* out_host,
                      void* stream);

/*
 * hs_estimate_mu - the regularisation parameter mu = ||X_d||_* / ||Psi^dagger X_d||_{2,1}
 * of the dirty cube X_d,l = eta_l Phi_l^dagger y_l (Sec. 2.3), with the PSF
 * normalisation eta_l = 1 / max(Phi_l^dagger Phi_l delta), delta the unit image
 * at the phase centre (Sec. 4.3). Y: DEVICE total complex (caller order);
 * A_work: DEVICE 9 x L x ny x nx reals of scratch (the caller's); eta_out:
 * DEVICE L doubles or NULL; Xd_out: DEVICE L x ny x nx reals or NULL (the
 * dirty cube). The nuclear norm comes from the Gram route of hs_prox_nuclear
 * (L <= 64). Synchronises the stream; *mu_host is valid on return.
 */
HS_API hs_status hs_estimate_mu(hs_plan_t plan, const void* Y, void* A_work, double* eta_out, void* Xd_out,
                                double* mu_host, void* stream);

/*
 * hs_op_norm2 - max_l ||U_l^{1/2} Phi_l||_S^2 by power iteration on
 * Phi_l^dagger U_l Phi_l, all channels at once (step sizes, Sec. 3.4).
 * Start vector drawn from `seed`; stops when every channel's estimate changes
 * by less than tol (relative) or after `iters` iterations. Synchronous:
 * *out_host is valid on return. Uses plan scratch.
 */
HS_API hs_status hs_op_norm2(hs_plan_t plan, int iters, double tol, uint64_t seed, double* out_host,
                      void* stream);

/* Parameters of Algorithm 2 (Sec. 3.4); see hs_pd_state_create. */
typedef struct {
    double tau;         /* primal step, 0 < tau; convergence needs tau (k1 + k2 + k3 ||U^1/2 Phi||^2) < 1 */
    double kappa1;      /* weight of the nuclear dual, default 1 */
    double kappa2;      /* weight of the sparsity dual, 1 / ||Psi^dagger||^2 = 1 */
    double kappa3;      /* weight of the data duals, 1 / ||U^1/2 Phi||^2 */
    double mu;          /* regularisation parameter of the l2,1 term (Sec. 2.3) */
    double psi_norm2;   /* ||Psi^dagger||_S^2 = 1 for the normalised frame */
    int use_nuclear;    /* 0 drops the low-rankness prior (LR / JAS variants) */
    int use_l21;        /* 0 drops the joint-sparsity prior */
    const double* w_nuc;   /* DEVICE L doubles (nuclear weights) or NULL = 1; referenced, not copied */
    const void* w_l21;     /* DEVICE 9 x ny x nx reals (row weights) or NULL = 1; referenced
                              (sparsity = 1: 9 x L x ny x nx per-coefficient weights) */
    int sparsity;          /* 0: l2,1 rows across channels (HyperSARA, JAS); 1: l1 per
                              coefficient (SARA, Sec. 4.2: the channels decouple) */
} hs_pd_params;

/*
 * hs_pd_state_create - primal-dual state for Algorithm 2 with one block per
 * channel and fixed l2 bounds. Y: DEVICE total complex data y_l (caller order,
 * copied). eps: DEVICE nblocks doubles, one l2 bound per data block (nblocks =
 * L unless the plan has blocks; copied). All primal and dual variables start
 * at zero. The state keeps references to params->w_nuc / w_l21, which must stay
 * valid while it is used. Errors: HS_ERR_ARG, HS_ERR_NOMEM, HS_ERR_CUDA.
 */
HS_API hs_status hs_pd_state_create(hs_plan_t plan, const void* Y, const double* eps,
                             const hs_pd_params* params, hs_pd_state_t* out, void* stream);

HS_API hs_status hs_pd_state_destroy(hs_pd_state_t state);

/*
 * hs_pd_set_data - replace the data y_l (DEVICE total complex, caller order) and
 * the bounds eps (DEVICE nblocks doubles) of a state, keeping its primal and dual
 * variables (warm start on new data of the same coverage). Asynchronous.
 */
HS_API hs_status hs_pd_set_data(hs_pd_state_t state, const void* Y, const double* eps, void* stream);

/* One iteration of Algorithm 2 (steps 2-12 and 20-23), asynchronous on stream. */
HS_API hs_status hs_pd_step(hs_pd_state_t state, void* stream);

/*
 * hs_pd_solve - `iters` iterations. graph = 1 captures one iteration as a CUDA
 * graph on first use and replays it; graph = 0 launches kernels directly.
 * Asynchronous on stream.
 */
HS_API hs_status hs_pd_solve(hs_pd_state_t state, int iters, int graph, void* stream);

/*
 * hs_pd_get - copy the current primal estimate X (DEVICE L x ny x nx, may be
 * NULL) and the last iteration's diagnostics: *beta_host = ||X - X_prev|| / ||X||
 * (Algorithm 2 step 23) and rho_host[b] = ||U^{-1/2} vbar_b - y_b|| per data
 * block (HOST nblocks doubles, may be NULL). Synchronises the stream when beta_host or rho_host is
 * given, and then returns HS_ERR_TIMEOUT if a bounded device-side wait of the
 * plan's kernels expired (see hs_plan_check).
 */
HS_API hs_status hs_pd_get(hs_pd_state_t state, void* X, double* beta_host, double* rho_host,
                    void* stream);

/*
 * hs_pd_set_data_host - hs_pd_set_data from HOST buffers: y_l (HOST total
 * complex of the plan's precision, caller order; pinned memory makes the copy
 * asynchronous) and eps (HOST nblocks doubles) are copied to the device on the
 * stream, then y is permuted into the state's order. The first call allocates
 * a device staging buffer of the visibilities' size (kept by the state);
 * later calls allocate nothing. The host buffers must stay valid until the
 * stream reaches the copies.
 */
HS_API hs_status hs_pd_set_data_host(hs_pd_state_t state, const void* Y_host, const double* eps_host, void* stream);

/*
 * hs_pd_get_host - hs_pd_get into HOST memory: X_host (L x ny x nx reals of
 * the plan's precision), *beta_host and rho_host (nblocks doubles) may be
 * NULL except X_host. Synchronises the stream; returns HS_ERR_TIMEOUT or
 * HS_ERR_ARG as hs_plan_check does when a kernel failed on the device.
 */
HS_API hs_status hs_pd_get_host(hs_pd_state_t state, void* X_host, double* beta_host, double* rho_host,
                                void* stream);

/* Number of kernel nodes in the state's captured iteration graph (0 before the
 * first hs_pd_solve with graph = 1): the kernel launches of one iteration. */
HS_API hs_status hs_pd_graph_kernels(hs_pd_state_t state, int* out);

/*
 * hs_pd_nuclear_info - diagnostics of the last nuclear-norm step (Algorithm 2
 * step 5) of a state: sv_host (HOST L doubles, may be NULL) receives the
 * singular values of P + X~, *active_host (may be NULL) the number of them above
 * the threshold. Synchronises the stream.
 */
HS_API hs_status hs_pd_nuclear_info(hs_pd_state_t state, double* sv_host, int* active_host,
                                    void* stream);

/*
 * hs_pd_reweight - weight update of the re-weighting outer loop (Sec. 3.5,
 * Algorithm 1) from the state's current primal X:
 *   w_l21[n] = gamma_l21 / (gamma_l21 + ||(Psi^dagger X)_n||_2)   (Eq. "weights-l21"),
 *     n a row (basis, pixel) of the coefficient cube, norm across channels;
 *     DEVICE 9 x ny x nx reals of the plan's precision, or NULL;
 *   w_nuc[j] = gamma_nuc / (gamma_nuc + sigma_j(X))              (Eq. "weights-n"),
 *     sigma_j the singular values of the N x L matrix X, descending;
 *     DEVICE L doubles, or NULL (needs L <= 64);
 *   sv_out: DEVICE L doubles receiving sigma_j, or NULL.
 * Pass the buffers the state was created with as params->w_l21 / w_nuc to make
 * the next iterations use the new weights (the state reads them in place).
 * gamma_* must be finite and > 0 for the outputs requested. Asynchronous on
 * `stream`; it uses the state's and plan's scratch, so it must not overlap an
 * iteration of the same state. FP32 plans refine every eigenpair with a
 * positive eigenvalue in FP64.
 */
HS_API hs_status hs_pd_reweight(hs_pd_state_t st, double gamma_l21, double gamma_nuc, void* w_l21,
                         double* w_nuc, double* sv_out, void* stream);

/* Number of iterations performed by a state. */
HS_API hs_status hs_pd_iterations(hs_pd_state_t state, int64_t* out);

/*
 * Adaptive l2 bounds (Algorithm 2 steps 13-19, Sec. 3.6). Each iteration t
 * (counted from 1) computes rho_b = ||y_b - Phibar_b X~|| per data block at the
 * extrapolated image it uses; if beta of the previous iteration < lambda1,
 * t - vartheta_b > min_gap and |rho_b - eps_b| / eps_b > lambda2, the bound
 * becomes lambda3 rho_b + (1 - lambda3) eps_b (used from the next iteration)
 * and vartheta_b = t. The first iteration never adjusts (beta undefined).
 * hs_pd_set_adaptive(st, NULL) or enable = 0 switches it off; changing it
 * re-captures the iteration graph at the next hs_pd_solve. The paper's values:
 * lambda1 = 5e-4, lambda2 = 0.01, lambda3 = 0.618, min_gap = 100.
 */
typedef struct {
    int enable;
    double lambda1, lambda2, lambda3;
    int64_t min_gap;   /* vartheta_bar */
} hs_adapt_params;

HS_API hs_status hs_pd_set_adaptive(hs_pd_state_t st, const hs_adapt_params* params);

/* Current bounds eps_b, last residuals rho_b = ||y_b - Phibar_b X~|| (adaptive
 * runs) and vartheta_b per data block, copied to HOST arrays of nblocks
 * entries (each may be NULL); synchronises the stream. */
HS_API hs_status hs_pd_bounds(hs_pd_state_t st, double* eps_host, double* resid_host, int64_t* theta_host,
                       void* stream);

/* Stages of the measurement path that hs_time_stage can launch alone. */
typedef enum {
    HS_STAGE_FFT_FWD = 0,   /* X (L x ny x nx) -> plan grid: Z, then F (row and column passes) */
    HS_STAGE_DEGRID = 1,    /* plan grid -> Y (caller order): G Theta */
    HS_STAGE_GRID = 2,      /* Y (caller order) -> plan grid: G^H Theta^H */
    HS_STAGE_FFT_ADJ = 3,   /* plan grid -> X: F^H, then Z^T */
    HS_STAGE_PSI_FWD = 4,   /* X -> A: Psi^dagger */
    HS_STAGE_PSI_ADJ = 5    /* A -> X: Psi */
} hs_stage;

/*
 * hs_time_stage - profiling aid: launches one stage `reps` times on `stream`
 * and returns in *avg_ms the mean duration per launch, measured with CUDA
 * events recorded on that stream (synchronises it). `in` / `out` are the
 * stage's DEVICE input and output as listed in hs_stage (unused ones may be
 * NULL); stages that read or write "plan grid" use the plan's scratch grid.
 */
HS_API hs_status hs_time_stage(hs_plan_t plan, int stage, const void* in, void* out, int reps,
                               float* avg_ms, void* stream);

/*
 * Host-only helpers (no GPU needed). Used by the plan; exported so that the
 * derived tables can be inspected.
 * hs_daubechies_lowpass: db_p low-pass filter, p = 1..8, by spectral
 *   factorisation (Daubechies, Ten Lectures 6.1), minimum phase, sum = sqrt 2;
 *   writes 2p doubles to out.
 * hs_kb_poly_fit: piecewise polynomial fit of the Kaiser-Bessel kernel used by
 *   the gridding kernels; returns the maximum error relative to phi(0) for
 *   the given number of coefficients per unit interval.
 * hs_kb_poly_coefs: the fit itself: J x terms doubles, piece p (x in
 *   [p - J/2, p - J/2 + 1), x = p - J/2 + (s + 1) / 2) as monomial coefficients
 *   of s in increasing degree. The kernel is even, so piece J - 1 - p at s is
 *   piece p at -s; the gridding kernels evaluate the two together.
 */
HS_API hs_status hs_daubechies_lowpass(int p, double* out);
HS_API hs_status hs_kb_poly_fit(int J, double beta, int terms, double* max_rel_err);
HS_API hs_status hs_kb_poly_coefs(int J, double beta, int terms, double* coef_out);

/*
 * hs_sweep_lists (host only): the gridding work lists a plan builds for the
 * register-sweep kernel on grids of at least 64 x 64 cells (G_l^H of step 12,
 * Sec. 2.1), for inspection. Input: L channels of windows given by their start
 * cells k0x[r], k0y[r] (0 <= k0 < K: the cell of t = u K / (2 pi), minus 3,
 * wrapped), channel-concatenated with offsets[L + 1] (offsets[0] = 0). Output:
 * work items, 6 ints each (channel, 32-column strip, first output row, end
 * row, entry range e0, e1), heaviest first; entries: window positions r in
 * groups of 4 (-1 = padding) whose windows start in the same 8-row band of the
 * item (relative rows -7 .. end - first - 1) and cover disjoint columns of the
 * strip, groups in band order. Two-call form: with items or ent NULL only
 * *n_items and *n_ent are written; otherwise they give the capacities (in
 * items and entries) and receive the counts. Caller-owned host buffers.
 * Rows of an item are cut after hmax rows, or earlier once its list would pass
 * cap windows (hmax, cap <= 0: the defaults 64 and 1024; the autotuner of
 * hs_plan_create chooses among (32, 512), (64, 1024) and (128, 2048)).
 * Errors: HS_ERR_ARG for grids narrower than 64 or not a multiple of 32
 * (columns) or 8 (rows), bad offsets, start cells outside the grid, or short
 * buffers.
 */
HS_API hs_status hs_sweep_lists(int Kx, int Ky, int L, const int64_t* offsets, const int* k0x, const int* k0y,
                                int hmax, int cap, int* items, int64_t* n_items, int* ent, int64_t* n_ent);

#ifdef __cplusplus
}
#endif

#endif /* HYPERSARA_H */
