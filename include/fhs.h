/*
 * libfhs: Faceted HyperSARA primal-dual forward-backward (PDFB) imaging on one
 * GPU (sm_103a).  C ABI: plain host/device pointers, sizes and a CUDA stream
 * passed as `void *` (a cudaStream_t; NULL = legacy default stream).
 *
 * The library solves, for C channel-interleaved spectral sub-cubes
 * (channel l belongs to sub-cube l % C), the problem of Eq. 3 of Thouvenin et
 * al., "Parallel faceted imaging in radio interferometry via proximal
 * splitting (Faceted HyperSARA): II", Sec. 2.2:
 *
 *   minimise_{X >= 0}  sum_{l,b} iota_{B(y_{l,b}, eps_{l,b})}(Phi_{l,b} x_l)
 *                      + mu_bar sum_q ||S_q X_c||_{*,w} + mu ||Psi^dagger X_c||_{2,1,w}
 *
 * with Phi_l = Theta_l G_l F Z the NUFFT measurement operator of Eq. 1
 * (Sec. 2.1), the l2-ball data constraints of Eq. 2, the faceted low-rankness
 * prior and the exactly faceted SARA average-joint-sparsity prior of
 * Sec. 2.2.2, and log-sum reweighting around PDFB (Sec. 2.2.3).
 *
 * Conventions shared by every entry point:
 *  - images are float32, layout [L][ny][nx] (row-major, channel-major planes);
 *    pixel (i1, i2) has coordinates n = (i1 - ny/2, i2 - nx/2);
 *  - visibilities are complex float32 stored as interleaved (re, im) pairs,
 *    concatenated by channel in the caller's order (vis_offsets);
 *  - every pointer named *_dev is device memory owned by the caller; every
 *    other pointer is host memory owned by the caller; the library keeps no
 *    caller pointer after a call returns;
 *  - device work is enqueued on `stream` and is asynchronous unless the call
 *    returns a host scalar (documented per call);
 *  - every call returns an fhs_status and never aborts; on FHS_ERR_ARG the
 *    problem is left unchanged; fhs_last_error() describes the last failure
 *    of the calling thread.
 */
#ifndef FHS_H
#define FHS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fhs_problem fhs_problem;

typedef enum {
    FHS_OK = 0,
    FHS_ERR_ARG = 1,      /* invalid argument or size; nothing was changed      */
    FHS_ERR_OOM = 2,      /* device allocation failed                           */
    FHS_ERR_CUDA = 3,     /* a CUDA / cuFFT call failed                         */
    FHS_ERR_TIMEOUT = 4,  /* a bounded device wait gave up                      */
    FHS_ERR_STATE = 5     /* call not valid in the problem's current state      */
} fhs_status;

/* Problem parameters.  Mirrors the user parameters and default internal
 * parameters of the paper's imaging pipeline (Sec. 4.2). */
typedef struct fhs_params {
    int32_t ny, nx;          /* image sides in pixels; both even, >= 16            */
    int32_t n_channels;      /* L                                                  */
    int32_t n_subcubes;      /* C; L % C == 0 (channel l -> sub-cube l % C, Eq. 3) */
    int32_t n_blocks;        /* B data blocks per channel (Sec. 2.1)               */
    int32_t qy, qx;          /* spatial facets of the low-rankness prior (Q=qy*qx) */
    double  facet_overlap;   /* facet extension on the low side, fraction of tile  */
    int32_t kb_taps;         /* J: Kaiser-Bessel taps per dimension (7)            */
    int32_t wavelet_levels;  /* SARA decomposition depth (4); bases Dirac+db1..db8 */
    double  w_max;           /* w-projection planes span [-w_max, w_max]; 0 = off  */
    int32_t n_wplanes;       /* planes per sign (>= 2 when w_max > 0)              */
    double  pixel_size;      /* radians per pixel (w-term chirp, Sec. 3.2)         */
    double  mu;              /* l21 (joint sparsity) regularisation; 0 switches the
                                prior off; < 0 selects 1 / sum_c ||Psi^dagger X_c||_{2,1}
                                of the dirty cube X (see fhs_residual)              */
    double  mu_bar;          /* nuclear (low-rankness) regularisation; 0 switches it
                                off; < 0 selects 1 / sum_{c,q} ||S_q X_c||_* of the
                                dirty cube X                                        */
    double  upsilon;         /* log-sum reweighting constant, l21 (> 0)            */
    double  upsilon_bar;     /* log-sum reweighting constant, nuclear (> 0)        */
    double  tau;             /* primal step; <= 0 selects 0.99/3                   */
    double  sigma0;          /* nuclear dual step; <= 0 selects 1/max facet cover  */
    double  sigma1;          /* l21 dual step; <= 0 selects 1 (||Psi|| = 1)        */
    double  sigma2;          /* data dual step; <= 0 selects 1/max_l ||Phi_l||^2   */
    int32_t power_iters;     /* Lanczos steps for ||Phi_l||^2 (default 100)        */
    double  power_tol;       /* relative change of the estimate that stops them    */
    int32_t gram_precision;  /* facet Gram of the nuclear dual step, fhs_gram_precision */
    int32_t data_reduction;  /* 1: visibility-gridding data reduction (Sec. 3.4), see below */
} fhs_params;

/* Data reduction (data_reduction = 1, Sec. 3.4, Eqs. 4-5).  Each channel's
 * visibilities are gridded, y'_l = Lambda_l (Theta_l G_l)^H y_l, and the data
 * term becomes one l2 ball per channel (all blocks aggregated) around y'_l for
 * Phi'_l = Lambda_l H_l F Z, H_l = (Theta_l G_l)^H (Theta_l G_l), Lambda_l =
 * diag(H_l)^(-1/2) on the M'_l grid cells some visibility reaches (0 elsewhere).
 * H_l is applied as a pass over G (it is not stored), so an iteration makes two
 * passes over G instead of one.  With data reduction:
 *  - eps (fhs_create_problem) is [L]: eps'_l; NULL selects
 *    eps'_l = sqrt(M'_l + 2 sqrt(M'_l)) (Eq. 2's bound for M'_l unit-variance
 *    values: E||Gamma n||^2 = M'_l for whitened noise n);
 *  - sigma2 <= 0 selects 1 / max_l ||Phi'_l||^2, the PSF normalisation and the
 *    dirty image of the mu / mu_bar defaults use Phi'_l, and fhs_residual
 *    returns eta'_l Re Phi'^H_l (y'_l - Phi'_l x_l);
 *  - the data dual (FHS_STATE_DUAL_DATA) is [L][2N_y][2N_x] complex on the
 *    oversampled grid (zero off the gridded cells);
 *  - fhs_measure and fhs_adjoint still apply Phi_l and Phi_l^H of the
 *    visibilities. */

/* Arithmetic of the facet Gram G_q = Z_q^T Z_q in the nuclear dual step
 * (Sec. 2.2.2).  FP32: FP32 products on the CUDA cores, FP64 sums across
 * threads.  TF32 / BF16: inputs rounded to TF32 or BF16, products summed in
 * FP32 on the tensor cores, FP64 across CTAs.  FP64: FP64 products and sums
 * on the CUDA cores (the mode that agrees with an FP64 SVD of Z_q also for
 * the small singular values).  The reweighting Gram is FP64 in every mode;
 * the eigendecomposition is FP64 in every mode. */
typedef enum { FHS_GRAM_FP32 = 0, FHS_GRAM_TF32 = 1, FHS_GRAM_BF16 = 2, FHS_GRAM_FP64 = 3 } fhs_gram_precision;

/* Fill *p with the defaults (J = 7, 4 levels, 64 w-planes, computed steps). */
void fhs_default_params(fhs_params *p);

/*
 * Build a problem on the current CUDA device.
 *  omega        host, [M_tot][2] float64: spatial frequency of each visibility
 *               in radians per pixel, (along y, along x), each in [-pi, pi).
 *  w            host, [M_tot] float64 w coordinate in wavelengths, or NULL (0).
 *  y            host, [M_tot][2] float64 raw (not whitened) visibilities.
 *  sigma        host, [L] float64 noise standard deviation per channel
 *               (Theta_l = 1/sigma_l, natural weighting, Eq. 1).
 *  vis_offsets  host, [L+1] int64: channel l owns visibilities
 *               [vis_offsets[l], vis_offsets[l+1]); vis_offsets[0] = 0.
 *  block_offsets host, [L][B+1] int64, relative to the channel start,
 *               non-decreasing from 0 to M_l: block b of channel l (Sec. 2.1).
 *  eps          host, [L][B] float64 l2-ball radii, or NULL for Eq. 2 with
 *               unit-variance whitened noise: eps_{l,b}^2 = (M_l + 2 sqrt(M_l)) M_{l,b}/M_l.
 * Copies everything it needs; builds G on the device (one row per visibility:
 * a (J+2h) x (J+2h) box of KB samples convolved with the w-kernel of its
 * plane); computes ||Phi_l||^2 (Lanczos, largest eigenvalue of
 * Re(Phi_l^H Phi_l)) when sigma2 <= 0; sets
 * X = 0, all duals to 0 and all weights to 1 (Sec. 5.2: zero initialisation).
 * Synchronises `stream` before returning.
 */
fhs_status fhs_create_problem(const fhs_params *params, const double *omega, const double *w,
                              const double *y, const double *sigma, const int64_t *vis_offsets,
                              const int64_t *block_offsets, const double *eps, void *stream,
                              fhs_problem **out);

/*
 * fhs_create_problem with direction-dependent effects folded into G
 * (Sec. 3.1: each row of G is its interpolation kernel convolved with the
 * Fourier kernel of the DDEs of its antenna pair).
 *  dde  host, [M_tot][5][5] complex as interleaved float64 (re, im), in the
 *       order of omega: the DDE kernel of each visibility on the oversampled
 *       grid, tap [j1][j2] at grid offset (j1 - 2, j2 - 2) along (y, x).
 * Every row's box grows to T + 4 taps per axis (its corner moves by -2) and
 * the row is stored as the sum of 5 separable terms, which represents the
 * 2-D convolution exactly; the factors take 5x the storage of a row without
 * DDEs.  Boxes must stay within 16 taps: with J = 7 the w-kernels may add at
 * most 2 taps per side, otherwise FHS_ERR_ARG.  dde NULL: FHS_ERR_ARG.
 * fhs_estimate_bytes does not count the DDE factors.
 */
fhs_status fhs_create_problem_dde(const fhs_params *params, const double *omega, const double *w,
                                  const double *y, const double *sigma, const int64_t *vis_offsets,
                                  const int64_t *block_offsets, const double *eps, const double *dde,
                                  void *stream, fhs_problem **out);

/* Release every device and host resource of the problem (NULL is a no-op). */
void fhs_destroy_problem(fhs_problem *prob);

typedef struct fhs_info {
    int64_t n_vis;           /* M_tot                                              */
    int64_t nnz;             /* entries of G (sum over rows of T^2)                */
    int64_t n_coef;          /* SARA coefficients per channel (Dirac + db1..db8)   */
    int64_t nuclear_size;    /* floats in the nuclear dual (all sub-cubes, facets) */
    int64_t device_bytes;    /* device memory held by the problem                  */
    int32_t n_facets;        /* Q                                                  */
    int32_t iteration;       /* PDFB iterations done                               */
    double  tau, sigma0, sigma1, sigma2;
    double  phi_norm2_max;   /* max_l ||Phi_l||^2 (0 if sigma2 was given)          */
    int64_t n_gfac;          /* stored G values: each row is the outer product of
                                two 1-D factors of T taps, kept as 2T values     */
    int32_t bin_dense_min;   /* binning of the pass over G (fhs_autotune_bins)     */
    int32_t bin_split;
    double  mu, mu_bar;      /* regularisation in use (the defaults once computed) */
    int64_t n_red;           /* gridded data points sum_l M'_l (0 without data reduction) */
} fhs_info;

fhs_status fhs_get_info(const fhs_problem *prob, fhs_info *info);

/* vis_dev[M_tot] (complex) = Phi_l x_l per channel (whitened, Eq. 1).
 * x_dev: [L][ny][nx] float32.  Asynchronous. */
fhs_status fhs_measure(fhs_problem *prob, const float *x_dev, float *vis_dev, void *stream);

/* Residual cube of Sec. 5.3: r_dev[L][ny][nx] = eta_l Re(Phi_l^H (y_l - Phi_l x_l))
 * with the whitened data y_l of the problem and eta_l = 1 / (Phi_l^H Phi_l delta)(centre)
 * (the point-spread function normalised to peak 1 at the phase centre; computed at
 * set-up, 0 for a channel without visibilities).  x_dev: [L][ny][nx] float32, or NULL
 * for x = 0, which gives the dirty image.  Asynchronous; uses the problem's
 * scratch (not the PDFB state). */
fhs_status fhs_residual(fhs_problem *prob, const float *x_dev, float *r_dev, void *stream);

/* Noise levels and l2 bounds from a model cube x0_dev ([L][ny][nx] float32,
 * device), as the paper sets them from the model image of a calibration step
 * (Sec. 3.3 (i), Sec. 5): with the whitened residual visibilities
 * r_{l,b} = Theta_l (y_{l,b} - Phi_{l,b} x0_l),
 *   sigma_out[l*B + b] = sigma_l * (sample standard deviation of r_{l,b},
 *                        complex, mean removed, M_{l,b} - 1 degrees of freedom)
 *   eps_out[l*B + b]   = ||r_{l,b}||_2.
 * With data reduction both are [L]: eps_out[l] = ||y'_l - Phi'_l x0_l||_2 (Sec.
 * 5.2, with the model visibilities Phi_l x0_l) and sigma_out[l] = eps_out[l] /
 * sqrt(M'_l).  sigma_out / eps_out (host) may be NULL.  apply != 0 makes
 * eps_out the problem's l2 bounds for the following iterations.  Synchronises
 * `stream`; FHS_ERR_TIMEOUT if a bounded device wait gave up before (see
 * fhs_device_status). */
fhs_status fhs_noise_from_model(fhs_problem *prob, const float *x0_dev, int32_t apply, double *sigma_out,
                                double *eps_out, void *stream);

/* Schedule of the adaptive noise estimation (fhs_adaptive_noise). */
typedef struct fhs_adaptive_params {
    int32_t max_iter;      /* PDFB iterations of the phase at most (>= 0)                       */
    int32_t check_every;   /* PDFB iterations between checks (>= 1)                             */
    double  settle_tol;    /* a check acts only when the relative change ||x+ - x|| / ||x+|| of
                              the last iteration is below settle_tol (> 0; INFINITY: always)    */
} fhs_adaptive_params;

typedef struct fhs_adaptive_result {
    int32_t iterations;    /* PDFB iterations run                                             */
    int32_t n_checks;      /* checks that acted                                               */
    int32_t n_updates;     /* checks that re-estimated the bounds                             */
    int32_t satisfied;     /* 1 when the last check found every l2 bound satisfied            */
} fhs_adaptive_result;

/* Adaptive estimation of the effective noise level during the first PDFB
 * iterations (Sec. 3.3 (ii)).  The paper gives the outline: image priors
 * inactive at first, noise estimates and l2 bounds updated while the
 * iteration runs, and fixed once the bounds hold.  The schedule here is a
 * reading of it built from the paper's own estimator and bound:
 *  - mu = mu_bar = 0 for the phase (SARA and nuclear steps skipped), the
 *    bounds the problem holds at the start;
 *  - every check_every iterations, if the last relative change is below
 *    settle_tol, a check takes the Sec. 3.3 (i) estimates of the current
 *    iterate (residual norms rho and noise levels, as fhs_noise_from_model);
 *    if rho <= eps for every block (every channel with data reduction) the
 *    bounds hold: the phase ends with them fixed.  Otherwise every bound is
 *    re-estimated as eps = s * eps0, with eps0 the bound of unit whitened
 *    noise (the default of fhs_create_problem: Eq. 2 with
 *    eps0^2 = (M_l + 2 sqrt(M_l)) M_{l,b} / M_l; with data reduction
 *    M'_l + 2 sqrt(M'_l)) and s the estimated whitened noise level
 *    (sigma_hat_{l,b} / sigma_l; with data reduction sigma_hat'_l);
 *  - the phase ends after max_iter iterations otherwise; mu and mu_bar are
 *    then restored (the iteration count goes on from the phase).
 * The phase starts the run: a problem that has iterated already gives
 * FHS_ERR_STATE.  sigma_out / eps_out (host, [L*B], or [L] with data
 * reduction; may be NULL) receive the noise levels of the final iterate's
 * residual and the bounds in force; res_out (may be NULL) the counts.
 * Synchronises `stream`. */
fhs_status fhs_adaptive_noise(fhs_problem *prob, const fhs_adaptive_params *params, double *sigma_out,
                              double *eps_out, fhs_adaptive_result *res_out, void *stream);

/* x_dev[L][ny][nx] = Re(Phi_l^H v_l), the adjoint of fhs_measure for real
 * images.  vis_dev: [M_tot] complex in the caller's order.  Asynchronous.
 * The gridding accumulates each tile of the oversampled grid in 32-bit fixed
 * point (the quantum is 2^-21 of a bound on the tile's largest contribution),
 * so the result agrees with exact arithmetic to a few 1e-6 relative; a tile
 * with a non-finite visibility accumulates in FP32 instead.  The PDFB
 * iteration's adjoint uses the same gridding. */
fhs_status fhs_adjoint(fhs_problem *prob, const float *vis_dev, float *x_dev, void *stream);

/* coef_dev[L][n_coef] = Psi^dagger x_l (Sec. 2.2.2): (1/3)[x; W_db1 x; ...; W_db8 x].
 * Per basis, levels 1..J in order, each level the (y-filter, x-filter) =
 * (lo,hi), (hi,lo), (hi,hi) subbands row-major, then the last (lo,lo) band.
 * Level sizes n_{j+1} = floor((n_j + 2p - 1)/2) (decimated full convolution,
 * zero extension).  Equal to the faceted transform on any tiling.  Async. */
fhs_status fhs_sara_analysis(fhs_problem *prob, const float *x_dev, float *coef_dev, void *stream);

/* Same coefficients as fhs_sara_analysis for n_images images of ny x nx
 * pixels ([n_images][ny][nx] in, [n_images][n_coef] out, layout as above),
 * without a problem handle and without allocating device memory.  The paper
 * has no counterpart: this entry point serves callers that cannot allocate
 * device memory, such as code whose device memory is fully reserved by
 * another allocator (a framework's caching allocator or a fixed pool) and
 * latency-critical loops that must not pay for cudaMalloc and the device
 * synchronisation it can imply.  Its scratch is a 16 MiB static device array
 * (2^22 floats) that every GPU loading the library holds until exit; images
 * needing more scratch than that (about 1.4e6 pixels at 4 levels) are rejected
 * with FHS_ERR_ARG.  The first call on a device looks up the array's address
 * on that device (it must be the current device); make that first call before
 * any stream capture.  The address is cached per device for the life of the
 * process: after cudaDeviceReset the module is loaded afresh and the cached
 * address may no longer be valid, so do not call this entry point after a
 * device reset.  Every call shares the one array, so calls that overlap
 * on the GPU (other streams, other threads) race: order them.  The scratch
 * needs no clearing (every value read was written earlier in the same call).
 * Asynchronous on `stream`. */
fhs_status fhs_sara_analysis_noalloc(int32_t ny, int32_t nx, int32_t n_images, int32_t levels,
                                     const float *x_dev, float *coef_dev, void *stream);

/* x_dev[L][ny][nx] = Psi c_l, the adjoint of fhs_sara_analysis.  Async. */
fhs_status fhs_sara_synthesis(fhs_problem *prob, const float *coef_dev, float *x_dev, void *stream);

/* Run n_iter PDFB iterations (Sec. 2.2.3):
 *   x+ = max(0, x - tau (sum_q S_q^T P_q + Psi W + Re Phi^H v)),  xbar = 2 x+ - x,
 *   P_q <- Z - SVT(Z, mu_bar w_q), Z = P_q + sigma0 S_q xbar    (per sub-cube, facet)
 *   W   <- Z min(1, mu w_r / ||Z_r||), Z = W + sigma1 Psi^dagger xbar (rows over channels)
 *   v_b <- (Z - sigma2 y_b)(1 - min(1, sigma2 eps_b / ||Z - sigma2 y_b||)), Z = v_b + sigma2 Phi_b xbar.
 * rel_change_out (host, may be NULL): ||x+ - x|| / ||x+|| of the last
 * iteration; when non-NULL the call synchronises `stream` and returns
 * FHS_ERR_TIMEOUT if a bounded device wait gave up (see fhs_device_status). */
fhs_status fhs_pdfb_step(fhs_problem *prob, int32_t n_iter, double *rel_change_out, void *stream);

/* n_iter PDFB iterations of each of n_prob problems, problem k on
 * streams[k] (streams may be NULL: legacy default stream).  Iterations are
 * submitted round-robin, one per problem at a time, so independent problems
 * (spectral sub-cubes or separate requests, Eq. 3) overlap on the device.
 * rel_change_out (host, [n_prob], may be NULL) as in fhs_pdfb_step; when
 * non-NULL the call synchronises every stream.                           */
fhs_status fhs_pdfb_step_batch(fhs_problem **probs, int32_t n_prob, int32_t n_iter, void **streams,
                               double *rel_change_out);

/* Replay one PDFB iteration as a CUDA graph (captured on first use for each
 * stream; on by default; never on the legacy default stream or while
 * tracing).  on = 0 launches kernel by kernel. */
fhs_status fhs_use_graphs(fhs_problem *prob, int32_t on);

/* Device bytes a problem with these parameters and n_vis visibilities with
 * coordinates w (host [n_vis], or NULL for no w-term) will hold after
 * fhs_create_problem (resident_out) and at most during it (peak_out), for
 * admission by HBM footprint.  Host only; either output may be NULL.     */
fhs_status fhs_estimate_bytes(const fhs_params *params, const double *w, int64_t n_vis, int64_t *resident_out,
                              int64_t *peak_out);

/* The admission query of the serving path under the name of the boundary
 * table: identical to fhs_estimate_bytes (same arguments, same results). */
fhs_status fhs_workspace_bytes(const fhs_params *params, const double *w, int64_t n_vis, int64_t *resident_out,
                               int64_t *peak_out);

/* Log-sum reweighting (Sec. 2.2.3): w_r = upsilon/(upsilon + ||(Psi^dagger X)_r||),
 * w_{q,i} = upsilon_bar/(upsilon_bar + sigma_i(S_q X)); duals are kept. Async. */
fhs_status fhs_reweight(fhs_problem *prob, void *stream);

/* The reweighting scheme of Sec. 2.2.3: log-sum priors handled by an outer
 * reweighting loop around PDFB.  n_reweight+1 inner runs of at most
 * max_iter/(n_reweight+1) iterations each (remainder in the last), an inner
 * run stopping early once ||x+ - x||/||x+|| < rel_tol (tested every
 * `check_every` iterations; <= 0 means 10), fhs_reweight between runs.
 * iters_out (host, may be NULL) receives the iterations done.  Synchronises;
 * returns FHS_ERR_TIMEOUT if a bounded device wait gave up during the run
 * (the image is then not to be trusted). */
fhs_status fhs_solve(fhs_problem *prob, int32_t max_iter, double rel_tol, int32_t n_reweight,
                     int32_t check_every, int32_t *iters_out, void *stream);

/* Image and state transfer (checkpoint / resume).  Device buffers, async. */
typedef enum {
    FHS_STATE_IMAGE = 0,       /* X, [L][ny][nx] float32                                 */
    FHS_STATE_DUAL_DATA = 1,   /* v, [M_tot] complex (float32 pairs), caller's order     */
    FHS_STATE_DUAL_SARA = 2,   /* W, [L][n_coef] float32, layout of fhs_sara_analysis    */
    FHS_STATE_DUAL_NUCLEAR = 3,/* P, per sub-cube c, per facet q (row-major facets),
                                  [L_c][wy_q][wx_q] float32, concatenated                */
    FHS_STATE_WEIGHTS_SARA = 4,/* w_r, [C][n_coef] float32                               */
    FHS_STATE_WEIGHTS_NUC = 5  /* w_{q,i}, [C][Q][L_c] float32                           */
} fhs_state_part;

/* Number of float32 values of one part.  Setting a dual recomputes the
 * adjoint term it feeds into the next primal step, so get_state of every part
 * followed by set_state of every part resumes the iteration exactly. */
fhs_status fhs_state_size(const fhs_problem *prob, int32_t part, int64_t *n_floats);
fhs_status fhs_get_state(fhs_problem *prob, int32_t part, float *dst_dev, void *stream);
/* The current image X (the iterate x of Eq. 3's PDFB, [L][ny][nx] float32)
 * into x_dev; the same as fhs_get_state(prob, FHS_STATE_IMAGE, ...).  Async. */
fhs_status fhs_get_image(fhs_problem *prob, float *x_dev, void *stream);
fhs_status fhs_set_state(fhs_problem *prob, int32_t part, const float *src_dev, void *stream);

/* Pick the tile binning of the pass over G by measurement (a layout choice of
 * this library; no passage of the paper defines it).  Times the
 * normal-mode pass G^H G on a random image under the binning in use and
 * under candidate binnings (dense-bin minimum 16/32/48/96 rows, bins of at
 * most 192/288/384 rows cut into equal parts), and keeps a candidate only if
 * it is at least 3 % faster.  The PDFB state is unchanged; the result of every
 * operator is the same up to the summation order of the adjoint.  Returns the
 * binning kept (either out pointer may be NULL).  Allocates the candidate
 * bins on `stream`; synchronises it.  A captured iteration graph is dropped
 * and recaptured by the next step. */
fhs_status fhs_autotune_bins(fhs_problem *prob, void *stream, int32_t *dense_min_out, int32_t *split_out);

/* ||Phi_l||^2 for every channel: the largest Ritz value after n_iter Lanczos
 * steps on Re(Phi_l^H Phi_l) from a fixed start (rises monotonically to the
 * largest eigenvalue); returns into the host array norms[L].  Uses the
 * iteration's scratch (the PDFB state is kept).  Synchronises.            */
fhs_status fhs_operator_norms(fhs_problem *prob, int32_t n_iter, double *norms, void *stream);

/* Tracing: per-phase device time of the PDFB iteration, measured with CUDA
 * events recorded on the caller's stream around each phase while enabled.
 * Phases, in iteration order: */
typedef enum {
    FHS_PHASE_PRIMAL = 0,        /* primal step + adjoint gathers + zero-pad     */
    FHS_PHASE_FFT_FWD = 1,       /* F (cuFFT)                                    */
    FHS_PHASE_DEGRID_GRID = 2,   /* dual pass over G: Phi xbar, data-dual update,
                                    block norms (data reduction: H Xhat)        */
    FHS_PHASE_L2BALL = 3,        /* block l2-ball factors, clearing of the grids */
    FHS_PHASE_FFT_INV = 4,       /* F^H (cuFFT)                                  */
    FHS_PHASE_SARA = 5,          /* Psi^dagger, weighted l21 dual, Psi           */
    FHS_PHASE_NUCLEAR = 6,       /* facet Grams, FP64 eig, SVT dual              */
    FHS_PHASE_SCATTER = 7,       /* scatter pass over G: G^H of the data dual
                                    (data reduction: H Lambda v)                */
    FHS_N_PHASES = 8
} fhs_phase;

/* on != 0 starts recording (and clears the totals); 0 stops. */
fhs_status fhs_profile_enable(fhs_problem *prob, int32_t on);
/* Synchronises the recorded events and returns, per phase, the summed
 * milliseconds (ms_out[FHS_N_PHASES]) and the number of timed iterations
 * (*iters_out).  Either pointer may be NULL.                             */
fhs_status fhs_profile_read(fhs_problem *prob, double *ms_out, int64_t *iters_out);
/* Number of libfhs kernels launched since the problem was created (cuFFT's
 * own kernels are not counted). */
fhs_status fhs_kernel_launches(const fhs_problem *prob, int64_t *count_out);

/* Device-side status of the problem's kernels: FHS_ERR_TIMEOUT if a bounded
 * wait inside a kernel gave up since the flag was last read, FHS_OK
 * otherwise; the flag is cleared.  The bounded waits are the tensor-core
 * Gram's stage mbarriers (code 1: the kernel skips its remaining stages and
 * still releases its tensor memory) and the pass over G's wait for the TMA
 * copy of its window (code 2: it waits once more, bounded, so that no copy
 * into its shared memory is in flight when it goes on).  fhs_solve,
 * fhs_pdfb_step with rel_change_out, fhs_noise_from_model and the server's
 * per-request checks read the same flag and fail with FHS_ERR_TIMEOUT (the
 * server marks the request FHS_REQ_FAILED).  Synchronises the stream. */
fhs_status fhs_device_status(fhs_problem *prob, void *stream);

/* Test aid for the failure path (the paper has no counterpart): launches one
 * CTA whose thread waits, with the same bounded wait as the pass over G's
 * window copy, on an mbarrier that nothing arrives at.  After max_polls polls
 * (1 .. 2^24; each poll may suspend the thread for a hardware-defined
 * interval, well below a millisecond) the wait gives up, records code 2 in
 * the problem's device flag and the kernel returns.  The next synchronising
 * call then reports FHS_ERR_TIMEOUT, as after a real timeout; nothing else of
 * the problem changes.  Asynchronous. */
fhs_status fhs_debug_unsatisfied_wait(fhs_problem *prob, int32_t max_polls, void *stream);

/* ------------------------------------------------------------------------
 * Serving: imaging requests solved concurrently on one GPU.  Requests are
 * independent problems (like the spectral sub-cubes of Eq. 3); a server
 * admits queued requests first-fit while their estimated peak device
 * footprint (fhs_estimate_bytes) fits its budget and fewer than max_active
 * run, builds each on a stream of its own, keeps all admitted problems
 * stepping (CUDA-graph replays of check_every iterations, relative change
 * read back asynchronously), reweights between stages as fhs_solve does, and
 * retires a request at its tolerance or iteration budget, copying the image
 * to host memory and freeing its device memory (stream-ordered), which
 * admits further requests.  Native threads: three for admission and set-up,
 * one for stepping.
 * ------------------------------------------------------------------------ */
typedef struct fhs_server fhs_server;

typedef enum { FHS_REQ_QUEUED = 0, FHS_REQ_RUNNING = 1, FHS_REQ_DONE = 2, FHS_REQ_FAILED = 3 } fhs_request_state;

typedef struct fhs_request {       /* arrays as in fhs_create_problem; copied by fhs_server_submit */
    fhs_params params;
    const double *omega, *w, *y, *sigma;
    const int64_t *vis_offsets, *block_offsets;
    const double *eps;
    int32_t max_iter;              /* iteration budget over all reweighting stages          */
    int32_t n_reweight;            /* reweightings (stages = n_reweight + 1)                  */
    double rel_tol;                /* a stage ends once ||x+ - x|| / ||x+|| < rel_tol         */
    int32_t check_every;           /* iterations between checks (<= 0: the server's default) */
} fhs_request;

typedef struct fhs_request_result {
    int32_t state;                 /* fhs_request_state                                       */
    int32_t status;                /* fhs_status of a failure                                 */
    int32_t iterations;            /* PDFB iterations done                                    */
    double rel_change;             /* last relative change read                               */
    double t_submit, t_start, t_done;   /* seconds since the server started                  */
    int64_t device_bytes;          /* bytes the problem held                                  */
} fhs_request_result;

/* Start a server on the current device with a device-memory budget (bytes). */
fhs_status fhs_server_create(int64_t hbm_budget_bytes, int32_t max_active, int32_t check_every,
                             fhs_server **out);
/* Queue a request (returns at once; FHS_ERR_OOM if it can never fit). */
fhs_status fhs_server_submit(fhs_server *server, const fhs_request *req, int64_t *id_out);
/* Non-blocking state of a request. */
fhs_status fhs_server_query(fhs_server *server, int64_t id, fhs_request_result *res_out);
/* Wait (timeout_s < 0: forever) for a request; image_out (host [L][ny][nx],
 * may be NULL) receives the image.  Returns the request's status. */
fhs_status fhs_server_wait(fhs_server *server, int64_t id, double timeout_s, float *image_out,
                           fhs_request_result *res_out);
/* Requests running or being set up, queued, and device bytes admitted. */
fhs_status fhs_server_stats(fhs_server *server, int64_t *active, int64_t *queued, int64_t *bytes_in_use);
/* Drop queued requests (their state becomes FAILED with FHS_ERR_STATE), let
 * admitted ones run to the end, stop the threads and free the server.  Call
 * it when no other thread is inside a call on this server: a caller that
 * needs a request's result waits for it first. */
void fhs_server_destroy(fhs_server *server);

/* Host utility: the library's own db_p low-pass filter (2p taps, minimum
 * phase, sum sqrt(2)), computed by spectral factorisation (Daubechies 1988). */
fhs_status fhs_daubechies_filter(int32_t p, double *h_out);

/* Text of the last error on the calling thread ("" if none). */
const char *fhs_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FHS_H */
