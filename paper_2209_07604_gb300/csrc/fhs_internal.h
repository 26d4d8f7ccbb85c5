// Internal definitions of libfhs: problem state, device layouts and kernel
// launchers.  Not part of the public ABI (see include/fhs.h).
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>

#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "fhs.h"

namespace fhs {

constexpr int kMaxLevels = 6;      // SARA depth supported
constexpr int kNumDb = 8;          // db1..db8
constexpr int kMaxF = 16;          // taps of db8
constexpr int kMaxLc = 32;         // channels per sub-cube supported
constexpr int kMaxWHalf = 4;       // largest w-kernel half-width h
constexpr int kTile = 32;
constexpr int kDdeTaps = 5;        // DDE kernels: kDdeTaps x kDdeTaps grid taps, centred
#ifndef FHS_BIN_MAX
#define FHS_BIN_MAX 384
#endif
// Rows per bin of the data kernel: at most kBinSplitMax (its shared-memory
// staging capacity); tile runs shorter than kBinDenseMin go to sparse bins.
constexpr long long kBinSplitMax = FHS_BIN_MAX, kBinDenseMin = 48;
// Pieces (runs of one data block each) a bin may hold: the blocks of a channel
// share tile bins while B <= kBinMaxPieces (otherwise every bin holds rows of
// one block, as one piece).
constexpr long long kBinMaxPieces = 16;          // grid tile (cells) used to sort visibilities
constexpr float kSaraScale = 1.0f / 3.0f;   // 1/sqrt(9 bases)

// ---------------------------------------------------------------------------
// host math (host_math.cpp)
// ---------------------------------------------------------------------------
double bessel_i0(double x);
double kb_beta(int J, double os);
double kb_hat(double nu, int J, double beta);
std::vector<double> daubechies(int p);
double chirp_phase(double n_abs, int N, int K);
void wkernel(double wp, int N, int K, double pixel_size, int h, std::complex<double> *out);

// ---------------------------------------------------------------------------
// SARA layout (constant memory in k_sara.cu)
// ---------------------------------------------------------------------------
struct SaraConst {
    int levels;
    int F[kNumDb + 1];                       // taps per basis (index 1..8)
    float h[kNumDb + 1][kMaxF];              // low-pass
    float g[kNumDb + 1][kMaxF];              // high-pass g[k] = (-1)^k h[F-1-k]
    int ny[kNumDb + 1][kMaxLevels + 1];      // level sizes (j = 0..levels)
    int nx[kNumDb + 1][kMaxLevels + 1];
    long long off_det[kNumDb + 1][kMaxLevels + 1];  // coefficient offset of level j details
    long long off_ll[kNumDb + 1];            // coefficient offset of the last LL band
    long long off_tmp[kNumDb + 1][kMaxLevels + 1];  // temp offset of approximation a_j
    long long n_coef;                        // coefficients per channel
    long long n_tmp;                         // temp floats per channel
    int img_ny, img_nx;
};

SaraConst sara_layout(int ny, int nx, int levels);

// ---------------------------------------------------------------------------
// Problem state
// ---------------------------------------------------------------------------
struct Facet {
    int y0, y1, x0, x1;
};

}  // namespace fhs

struct fhs_problem {
    fhs_params prm;
    int L = 0, C = 0, Lc = 0, B = 0, ny = 0, nx = 0, K1 = 0, K2 = 0, J = 7;
    int rank = 1;                             // separable terms per row of G (kDdeTaps with DDE kernels)
    bool narrow_rows = false;                 // at most 1 row in 10 has more than 8 taps (gathers at 5 CTAs/SM)
    long long N = 0, K = 0;                   // pixels and grid cells per channel
    long long Mtot = 0, nnz = 0, n_fac = 0;   // nnz: entries of G (sum T^2); n_fac: stored factors (sum 2T)
    std::vector<long long> vis_off;           // [L+1]
    std::vector<double> sigma_l;              // [L] whitening of each channel (Theta_l = 1 / sigma_l)
    std::vector<long long> seg_off;           // [L*B+1] sorted-order offsets of (l,b) segments
    int n_seg = 0;

    // data term (sorted visibility order)
    int2 *meta = nullptr;                     // {c1 | c2 << 16, T}
    long long *fptr = nullptr;                // [Mtot+1] offsets of the row factors
    float2 *gfac = nullptr;                   // [n_fac] per row: g1 / sigma (T values), g2 (T values)
    float *gmax = nullptr;                    // [Mtot] max |g1| max |g2| per single-term row
    float2 *y = nullptr;                      // whitened data
    float2 *dvis = nullptr;                   // data dual storage d (v = scale_b d)
    long long *perm = nullptr;                // sorted -> caller index
    float2 *vis_tmp = nullptr;                // [Mtot] scratch for measure/adjoint
    int *vis_chan = nullptr;                  // [n_seg] channel of each segment
    long long *d_seg_off = nullptr;           // [n_seg+1]
    double *blk_norm2 = nullptr;              // [n_seg]
    double *eps = nullptr;                    // [n_seg]
    float *blk_scale = nullptr;               // [n_seg]  (1 - m_b)
    int n_bin = 0, ntx = 0;                   // tile bins of the single-pass data kernel
    int bin_dense_min = 0, bin_split = 0;     // binning in use (defaults or fhs_autotune_bins)
    // a bin is a list of pieces: runs of sorted rows of one data block each (the rows of all
    // blocks of a channel whose boxes start in one grid tile, or a run of sparse rows of one block)
    int bin_slots = 1;                        // piece slots per bin (unused ones have length 0)
    long long *bin_fbase = nullptr;           // [n_bin] factor offset (fptr) of each bin's first row
    int *bin_chan = nullptr;                  // [n_bin] channel
    int *bin_tile = nullptr;                  // [n_bin] tile key, -1 = sparse (global path)
    long long *piece_start = nullptr;         // [n_bin][bin_slots] first row (sorted order)
    int *piece_len = nullptr;                 // [n_bin][bin_slots] rows
    int *piece_blk = nullptr;                 // [n_bin][bin_slots] block b of the channel
    int n_chunk = 0;
    long long *chunk_start = nullptr;         // [n_chunk+1]
    int *chunk_seg = nullptr;                 // [n_chunk]
    float *s1 = nullptr, *s2 = nullptr;       // Z scaling per axis
    // F on real images: R2C of the zero-padded image into a half grid (columns 0..K2/2 of each
    // row, row stride HS), which the passes over G read with X(k) = conj X(-k) for the other
    // columns; F^H through C2R from a half grid holding the Hermitian part of the adjoint (the
    // scatter folds it there)
    int HS = 0;                               // half-grid row stride: K2/2 + 1
    long long KH = 0;                         // half-grid cells per channel, K1 * HS
    cufftHandle plan_r2c = 0, plan_c2r = 0;
    bool plan_ok = false;
    void *fft_ws = nullptr;                   // work area shared by both plans
    size_t fft_ws_bytes = 0;
    float *grid_in = nullptr;                 // [L][K] real zero-padded input (zeros persist)
    float2 *grid_work = nullptr;              // [L][KH] forward spectrum / folded data adjoint
    float2 *grid_scr = nullptr;               // [L][KH] scratch output grids
    float2 *grid_aux = nullptr;               // [L][KH] scratch for measure/adjoint
    float *adj_real = nullptr;                // [L][K] F^H of the data adjoint grid (iteration state)
    float *real_scr = nullptr;                // [L][K] F^H output of the other calls

    // data reduction (Sec. 3.4): grids [L][K], zero off the gridded cells
    bool dr = false;
    float *dr_lam = nullptr;                  // Lambda_l
    float2 *dr_y = nullptr;                   // y'_l
    float2 *dr_v = nullptr;                   // reduced data dual
    float2 *dr_u = nullptr;                   // H Xhat (zero between uses)
    float2 *dr_w = nullptr;                   // Lambda v, input of the adjoint pass
    double *dr_norm2 = nullptr;               // [L]
    double *dr_eps = nullptr;                 // [L] eps'_l
    float *dr_scale = nullptr;                // [L]
    std::vector<long long> dr_m;              // M'_l

    // image domain
    float *X = nullptr, *Xbar = nullptr, *A_sara = nullptr;

    // SARA
    fhs::SaraConst sara{};
    float *W = nullptr;                       // [L][n_coef]
    float *coef_tmp = nullptr;                // [L][n_coef] analysis output
    float *sara_tmp = nullptr;                // [L][n_tmp] approximations
    float *w21 = nullptr;                     // [C][n_coef]

    // nuclear
    std::vector<fhs::Facet> facets;           // Q facets (row-major)
    int Q = 0;
    int4 *d_facets = nullptr;                 // [Q]
    long long *nuc_off = nullptr;             // [C*Q] float offset of P_{c,q}
    std::vector<long long> h_nuc_off;
    long long nuc_size = 0;
    float *P = nullptr;
    double *gram = nullptr;                   // [C*Q][Lc*Lc]
    float *mix = nullptr;                     // [C*Q][Lc*Lc]
    float *wnuc = nullptr;                    // [C*Q][Lc]
    double *eigv = nullptr;                   // [C*Q][n*n] eigenvectors of the last dual-step Gram (n = Lc rounded up to even)
    short *cov_row_first = nullptr, *cov_row_cnt = nullptr;   // [ny]
    short *cov_col_first = nullptr, *cov_col_cnt = nullptr;   // [nx]
    int max_cover = 1;

    // reductions
    double *red = nullptr;                    // [2]: ||x+ - x||^2, ||x+||^2

    cudaStream_t home = nullptr;              // stream of creation: stream-ordered allocations live on it
    double tau = 0, sigma0 = 0, sigma1 = 0, sigma2 = 0, phi_norm2_max = 0;
    int iteration = 0;
    long long n_launch = 0;                   // libfhs kernels launched
    double *pnorms = nullptr;                 // [2L] power-iteration reductions
    int *dev_err = nullptr;                   // [1] set by a kernel whose bounded wait gave up
    float *eta = nullptr;                     // [L] PSF-peak normalisation 1 / (Phi_l^H Phi_l delta)(centre)

    // the SARA and nuclear dual steps run on their own streams, forked after
    // the primal step and joined before the iteration ends
    cudaStream_t s_sara = nullptr, s_nuc = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_sara = nullptr, ev_nuc = nullptr;

    // CUDA graph of one iteration, replayed by fhs_pdfb_step on the stream it was captured on
    bool use_graphs = true;
    cudaGraphExec_t gexec = nullptr;
    cudaStream_t gstream = nullptr;
    long long g_launches = 0;                 // libfhs kernels in one captured iteration

    // tracing: event pairs per phase per iteration, recycled from a pool
    bool prof_on = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_used;
    double prof_ms[FHS_N_PHASES] = {0};
    long long prof_iters = 0;
    size_t bytes = 0;
    std::vector<void *> allocs;
};

namespace fhs {

// Sets the text returned by fhs_last_error() on the calling thread.
void set_last_error(const std::string &msg);

// Releases a problem whose work has all been issued on `s`: waits for s only
// (no device-wide synchronisation), frees its stream-ordered memory.
void destroy_on_stream(fhs_problem *p, cudaStream_t s);

// kernel launchers --------------------------------------------------------
// k_nufft.cu
// dde: NULL, or [Mtot][kDdeTaps^2] DDE kernels in sorted order; ext = kDdeTaps - 1 with DDEs, else 0.
cudaError_t launch_build_g(fhs_problem *p, const double2 *kap, const short *plane, const double2 *wk_table,
                           const double2 *dde, int ext, const double *inv_sigma_seg, cudaStream_t s);
cudaError_t launch_zpad(fhs_problem *p, const float *x, float *grid, cudaStream_t s);
// Set-up: the sorted rows' grid coordinates (kap), w-planes and whitened data (p->y) from the
// caller's omega, y and planes through p->perm; vis_off [L+1] and sigma [L] on the device.
cudaError_t launch_gather_rows(fhs_problem *p, const double2 *omega, const double2 *ycall, const short *cplane,
                               const long long *vis_off, const double *sigma, double2 *kap, short *plane,
                               cudaStream_t s);
// Z and Z^T of channel l alone (x and grid point at the channel-0 images and grids)
cudaError_t launch_zpad_channel(fhs_problem *p, const float *x, float *grid, int l, cudaStream_t s);
cudaError_t launch_crop_channel(fhs_problem *p, const float *grid, float *x, int l, cudaStream_t s);
cudaError_t launch_degrid(fhs_problem *p, const float2 *grid, float2 *vis_sorted, cudaStream_t s);
// test aid: a bounded wait on an mbarrier nothing arrives at, which records a timeout in p->dev_err
cudaError_t launch_unsatisfied_wait(fhs_problem *p, int max_polls, cudaStream_t s);
// fixed: dense bins accumulate their window in 32-bit fixed point (see k_binned.cu); false keeps
// FP32 atomics (the gridding of the data reduction, whose faint cells are weighted up by Lambda).
// fold: the output is a half grid that receives the Hermitian part (g(k) + conj g(-k)) / 2 of the
// adjoint, the input of the C2R transform; without fold a full grid receives g (outputs that stay
// in the frequency domain).  Gathering passes read half grids (forward spectra) unless stated.
cudaError_t launch_grid(fhs_problem *p, const float2 *vis_sorted, float2 *grid, cudaStream_t s, bool fixed, bool fold);
cudaError_t launch_crop(fhs_problem *p, const float *grid, float *x, cudaStream_t s);
cudaError_t launch_data_dual(fhs_problem *p, cudaStream_t s);      // dual pre-update + block norms
cudaError_t launch_data_scatter(fhs_problem *p, cudaStream_t s);   // grid_work += G^H (s_b d), folded
// fixed, fold: as for launch_grid; the passes of the data reduction use fixed = false.  in_half:
// the input is a half grid (a forward spectrum), else a full grid.
cudaError_t launch_normal(fhs_problem *p, const float2 *grid, bool in_half, float2 *grid_out, cudaStream_t s,
                          bool fixed, bool fold, int bin0 = 0, int nbin = -1);   // bins [bin0, bin0 + nbin)
// One Lanczos step after y = A v: y <- w, vprev <- v_{j+1}; alpha_j[l] and
// nb2_j[L + l] (= beta_{j+1}^2) accumulate, nb2_j[l] = beta_j^2 is read.
// chans (device, nch entries): the channels to step; nullptr: all L
cudaError_t launch_lanczos_step(fhs_problem *p, float *y, float *vprev, const float *v, double *alpha_j,
                                double *nb2_j, cudaStream_t s, const int *chans = nullptr, int nch = 0);
cudaError_t launch_block_finalize(fhs_problem *p, cudaStream_t s);
cudaError_t launch_permute_to_caller(fhs_problem *p, const float2 *sorted, float2 *caller, const float *scale_seg,
                                     cudaStream_t s);
cudaError_t launch_permute_from_caller(fhs_problem *p, const float2 *caller, float2 *sorted, cudaStream_t s);
cudaError_t launch_power_dots(fhs_problem *p, const float *x, const float *y, double *out, cudaStream_t s);
cudaError_t launch_power_scale(fhs_problem *p, const float *y, float *x, const double *norms, cudaStream_t s);
// k_sara.cu
cudaError_t launch_sara_analysis(fhs_problem *p, const float *x, float *coef, cudaStream_t s);
cudaError_t launch_sara_synthesis(fhs_problem *p, const float *coef, float *x, cudaStream_t s);
cudaError_t launch_l21_dual(fhs_problem *p, cudaStream_t s);
cudaError_t launch_l21_reweight(fhs_problem *p, cudaStream_t s);
// k_nuclear.cu
cudaError_t launch_nuclear_gram(fhs_problem *p, const float *img, bool with_dual, bool fp64, cudaStream_t s);
cudaError_t launch_nuclear_eig(fhs_problem *p, bool reweight, cudaStream_t s);
// Singular values (descending, FP64) of every facet whose Gram is in p->gram: svals[C*Q][Lc].
cudaError_t launch_nuclear_svals(fhs_problem *p, double *svals, cudaStream_t s);
cudaError_t launch_l21_norm(fhs_problem *p, const float *A, double *out, cudaStream_t s);
cudaError_t launch_vis_residual(fhs_problem *p, const float2 *phi, float2 *r, cudaStream_t s);
cudaError_t launch_chan_scale(fhs_problem *p, float *x, const float *f, cudaStream_t s);
// data reduction (k_reduce.cu)
cudaError_t launch_dr_diag(fhs_problem *p, double *diag, cudaStream_t s);
cudaError_t launch_dr_setup(fhs_problem *p, const double *diag, float2 *ghy, unsigned long long *cnt, cudaStream_t s);
cudaError_t launch_dr_dual(fhs_problem *p, cudaStream_t s);
cudaError_t launch_dr_finalize(fhs_problem *p, cudaStream_t s);
cudaError_t launch_dr_weight(fhs_problem *p, cudaStream_t s);      // dr_w = Lambda dr_v
cudaError_t launch_dr_resid_norm(fhs_problem *p, double *out, cudaStream_t s);   // out[l] += ||y' - Lambda dr_u||^2
cudaError_t launch_seg_stats(fhs_problem *p, const float2 *phi, double *stats, cudaStream_t s);
cudaError_t launch_dr_combine(fhs_problem *p, float2 *u, float a, float b, float2 *w, cudaStream_t s);
cudaError_t launch_nuclear_apply(fhs_problem *p, cudaStream_t s);
// Tensor-core Gram of the dual step (precision FHS_GRAM_TF32 or FHS_GRAM_BF16).
cudaError_t launch_nuclear_gram_tc(fhs_problem *p, int precision, cudaStream_t s);
// k_pdfb.cu
cudaError_t launch_primal(fhs_problem *p, cudaStream_t s);

}  // namespace fhs
