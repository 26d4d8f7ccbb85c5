// C-ABI of libfhs: problem set-up (visibility sorting, w-kernels, G build,
// SARA layout, facets, step sizes), the PDFB iteration driver, reweighting,
// state transfer.  Every device computation is one of the kernels in k_*.cu
// or a cuFFT transform; the host only orders launches.
#include "fhs_internal.h"

#include <algorithm>
#include <chrono>
#include <climits>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

using namespace fhs;

namespace {

thread_local std::string g_err;

// fn(begin, end) over [0, n) split into contiguous ranges on up to 32 host
// threads (set-up of 10^7 visibilities is otherwise host bound).  A range whose
// thread cannot be started runs on the calling thread.
template <typename F>
void parallel_for(long long n, F fn, long long min_chunk = 1 << 16) {
    const long long hc = std::max(1u, std::thread::hardware_concurrency());
    const long long nt = std::max(1LL, std::min({hc, 32LL, (n + min_chunk - 1) / std::max(1LL, min_chunk)}));
    if (nt <= 1) {
        fn(0LL, n);
        return;
    }
    const long long step = (n + nt - 1) / nt;
    std::vector<std::thread> th;
    for (long long t = 1; t < nt; ++t) {
        const long long a = std::min(n, t * step), b = std::min(n, (t + 1) * step);
        try {
            th.emplace_back(fn, a, b);
        } catch (...) {
            fn(a, b);
        }
    }
    fn(0LL, std::min(n, step));
    for (auto &x : th) x.join();
}

fhs_status fail(fhs_status st, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CU(call)                                                                                   \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(e_ == cudaErrorMemoryAllocation ? FHS_ERR_OOM : FHS_ERR_CUDA, "%s: %s (%s:%d)", #call, \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                               \
    } while (0)

#define CUFFT(call)                                                                                \
    do {                                                                                           \
        cufftResult r_ = (call);                                                                   \
        if (r_ != CUFFT_SUCCESS) return fail(FHS_ERR_CUDA, "%s: cufft error %d", #call, int(r_));  \
    } while (0)

#define TRY(call)                                                                                  \
    do {                                                                                           \
        fhs_status s_ = (call);                                                                    \
        if (s_ != FHS_OK) return s_;                                                               \
    } while (0)

// Stream-ordered device allocation on the problem's home stream (released
// with cudaFreeAsync, so retiring a problem never synchronises the device).
template <typename T>
fhs_status dev_alloc(fhs_problem *p, T **ptr, size_t count, bool zero = true) {
    *ptr = nullptr;
    if (count == 0) count = 1;
    void *q = nullptr;
    const size_t bytes = count * sizeof(T);
    cudaError_t e = cudaMallocAsync(&q, bytes, p->home);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(FHS_ERR_OOM, "cudaMallocAsync of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    p->allocs.push_back(q);
    p->bytes += bytes;
    if (zero) {
        e = cudaMemsetAsync(q, 0, bytes, p->home);
        if (e != cudaSuccess) return fail(FHS_ERR_CUDA, "cudaMemsetAsync failed: %s", cudaGetErrorString(e));
    }
    *ptr = static_cast<T *>(q);
    return FHS_OK;
}

void dev_free(fhs_problem *p, void *q) {
    auto it = std::find(p->allocs.begin(), p->allocs.end(), q);
    if (it != p->allocs.end()) {
        cudaFreeAsync(q, p->home);
        p->allocs.erase(it);
    }
}

template <typename T>
fhs_status upload(T *dst, const T *src, size_t count, cudaStream_t s) {
    if (count == 0) return FHS_OK;
    CU(cudaMemcpyAsync(dst, src, count * sizeof(T), cudaMemcpyHostToDevice, s));
    return FHS_OK;
}

void free_all(fhs_problem *p) {
    if (p->s_sara) cudaStreamSynchronize(p->s_sara);
    if (p->s_nuc) cudaStreamSynchronize(p->s_nuc);
    for (void *q : p->allocs) cudaFreeAsync(q, p->home);
    p->allocs.clear();
    cudaStreamSynchronize(p->home);
    if (p->plan_ok) {
        cufftDestroy(p->plan_r2c);
        cufftDestroy(p->plan_c2r);
    }
    p->plan_ok = false;
    for (cudaStream_t *t : {&p->s_sara, &p->s_nuc})
        if (*t) { cudaStreamDestroy(*t); *t = nullptr; }
    for (cudaEvent_t *e : {&p->ev_fork, &p->ev_sara, &p->ev_nuc})
        if (*e) { cudaEventDestroy(*e); *e = nullptr; }
}

inline cudaStream_t S(void *s) { return static_cast<cudaStream_t>(s); }

// Tile bins of the single-pass data kernel (k_binned.cu): inside each
// (channel, block) segment, a run of rows whose box corners share one grid tile
// becomes shared-memory bins when it holds at least dense_min rows, cut into
// parts of at most `split` rows (equal parts when `even`, else full parts and
// a remainder); shorter runs are packed in order into sparse bins of at most
// sparse_max rows, which take the global-memory path.
// Tile bins of the pass over G.  A channel's rows are sorted, inside each
// data block's segment, by the grid tile of their box corner.  For every tile,
// the runs of all B blocks together form dense bins when they hold at least
// dense_min rows: the runs are the bin's pieces (one block each, in block
// order), cut into parts of at most `split` rows (`even`: parts of about equal
// size).  The rows of tiles below dense_min are sparse: consecutive ones of a
// block form sparse bins (tile -1) of one piece of at most sparse_max rows.
// With B > kBinMaxPieces every block is binned on its own (tile bins of one
// piece).
struct BinList {
    std::vector<int> pptr, chan, tile, plen, pblk;
    std::vector<long long> pstart, fbase;
    void clear() {
        pptr.assign(1, 0);
        fbase.clear();
        chan.clear();
        tile.clear();
        plen.clear();
        pblk.clear();
        pstart.clear();
    }
    void piece(long long start, long long len, int blk) {
        pstart.push_back(start);
        plen.push_back(int(len));
        pblk.push_back(blk);
    }
    void close(int l, int k) {
        fbase.push_back(pstart[pptr.back()]);    // the bin's first row (its factor offset is filled in later)
        chan.push_back(l);
        tile.push_back(k);
        pptr.push_back(int(pstart.size()));
    }
    int n_bin() const { return int(chan.size()); }
};

void make_bins(const int2 *meta, const long long *fptr, const std::vector<long long> &seg_off, int L, int B, int ntx,
               long long dense_min, long long split, bool even, long long sparse_max, BinList &out) {
    out.clear();
    auto key = [&](long long i) {
        return (meta[i].x & 0xffff) / kTile * ntx + (int)((unsigned)meta[i].x >> 16) / kTile;
    };
    // blocks share bins while a bin's factor offsets stay 32-bit (rows of one channel span less
    // than 2^31 factor values)
    bool merge = B <= kBinMaxPieces;
    for (int l = 0; l < L && merge; ++l)
        merge = fptr[seg_off[(l + 1) * B]] - fptr[seg_off[l * B]] < INT_MAX;
    const int G = merge ? B : 1;                     // blocks binned together
    struct Run { long long a, e; };
    for (int l = 0; l < L; ++l) {
        for (int b0 = 0; b0 < B; b0 += G) {
            std::vector<long long> pos(G), end(G), sp_a(G, -1), sp_e(G, -1);
            for (int g = 0; g < G; ++g) {
                pos[g] = seg_off[l * B + b0 + g];
                end[g] = seg_off[l * B + b0 + g + 1];
            }
            auto flush_sparse = [&](int g) {
                for (long long q = sp_a[g]; q < sp_e[g]; q += sparse_max) {
                    out.piece(q, std::min(sparse_max, sp_e[g] - q), b0 + g);
                    out.close(l, -1);
                }
                sp_a[g] = sp_e[g] = -1;
            };
            std::vector<Run> runs(G);
            for (;;) {
                // the smallest tile key among the blocks' next runs
                int k = INT_MAX;
                for (int g = 0; g < G; ++g)
                    if (pos[g] < end[g]) k = std::min(k, key(pos[g]));
                if (k == INT_MAX) break;
                long long n = 0;
                for (int g = 0; g < G; ++g) {
                    runs[g] = {pos[g], pos[g]};
                    if (pos[g] < end[g] && key(pos[g]) == k) {
                        long long e = pos[g] + 1;
                        while (e < end[g] && key(e) == k) ++e;
                        runs[g].e = e;
                        n += e - pos[g];
                        pos[g] = e;
                    }
                }
                if (n >= dense_min) {
                    const long long parts = (n + split - 1) / split;
                    const long long cap = even ? (n + parts - 1) / parts : split;
                    // a block's pending sparse rows end where its run of this tile starts
                    for (int g = 0; g < G; ++g)
                        if (runs[g].e > runs[g].a && sp_a[g] >= 0) flush_sparse(g);
                    long long room = cap;
                    bool open = false;
                    for (int g = 0; g < G; ++g) {
                        long long a = runs[g].a;
                        while (a < runs[g].e) {
                            const long long take = std::min(room, runs[g].e - a);
                            out.piece(a, take, b0 + g);
                            open = true;
                            a += take;
                            room -= take;
                            if (room == 0) {
                                out.close(l, k);
                                open = false;
                                room = cap;
                            }
                        }
                    }
                    if (open) out.close(l, k);
                } else {
                    for (int g = 0; g < G; ++g) {
                        if (runs[g].e == runs[g].a) continue;
                        if (sp_e[g] != runs[g].a && sp_a[g] >= 0) flush_sparse(g);
                        if (sp_a[g] < 0) sp_a[g] = runs[g].a;
                        sp_e[g] = runs[g].e;
                    }
                }
            }
            for (int g = 0; g < G; ++g)
                if (sp_a[g] >= 0) flush_sparse(g);
        }
    }
    for (long long &f : out.fbase) f = fptr[f];
}

// A bin list on the device (the arrays the pass over G reads) and its bytes.
struct DevBins {
    int *chan = nullptr, *tile = nullptr, *plen = nullptr, *pblk = nullptr;
    long long *pstart = nullptr, *fbase = nullptr;
    int n_bin = 0, slots = 1, dense_min = 0, split = 0;
    size_t bytes = 0;
};

// A bin list in the device layout: every bin has `slots` piece slots (the
// most pieces any bin holds), unused ones of length 0, so that a CTA loads its
// bin's pieces in the same round trip as the bin's channel and tile.
struct SlotBins {
    int slots = 1;
    std::vector<long long> pstart;
    std::vector<int> plen, pblk;
};

SlotBins to_slots(const BinList &b) {
    SlotBins o;
    for (int k = 0; k < b.n_bin(); ++k) o.slots = std::max(o.slots, b.pptr[k + 1] - b.pptr[k]);
    const size_t n = size_t(b.n_bin()) * o.slots;
    o.pstart.assign(n, 0);
    o.plen.assign(n, 0);
    o.pblk.assign(n, 0);
    for (int k = 0; k < b.n_bin(); ++k)
        for (int q = b.pptr[k]; q < b.pptr[k + 1]; ++q) {
            const size_t d = size_t(k) * o.slots + (q - b.pptr[k]);
            o.pstart[d] = b.pstart[q];
            o.plen[d] = b.plen[q];
            o.pblk[d] = b.pblk[q];
        }
    return o;
}

DevBins current_bins(const fhs_problem *p) {
    DevBins d;
    d.slots = p->bin_slots;
    d.fbase = p->bin_fbase;
    d.chan = p->bin_chan;
    d.tile = p->bin_tile;
    d.pstart = p->piece_start;
    d.plen = p->piece_len;
    d.pblk = p->piece_blk;
    d.n_bin = p->n_bin;

    d.dense_min = p->bin_dense_min;
    d.split = p->bin_split;
    const size_t np = size_t(p->n_bin) * p->bin_slots;
    d.bytes = sizeof(int) * (2 * size_t(p->n_bin) + 2 * np) + sizeof(long long) * (np + p->n_bin);
    return d;
}

void use_bins(fhs_problem *p, const DevBins &d) {
    p->bin_slots = d.slots;
    p->bin_fbase = d.fbase;
    p->bin_chan = d.chan;
    p->bin_tile = d.tile;
    p->piece_start = d.pstart;
    p->piece_len = d.plen;
    p->piece_blk = d.pblk;
    p->n_bin = d.n_bin;

    p->bin_dense_min = d.dense_min;
    p->bin_split = d.split;
}

// The device-side error flag, already copied to the host as h after a
// synchronisation of s: FHS_OK when clear; otherwise FHS_ERR_TIMEOUT, with the
// flag cleared on s so that the next check starts afresh.  Codes: 1 the
// tensor-core Gram's mbarrier wait, 2 the pass over G's window wait.
fhs_status take_device_error(fhs_problem *p, int h, cudaStream_t s) {
    if (h == 0) return FHS_OK;
    CU(cudaMemsetAsync(p->dev_err, 0, sizeof(int), s));
    return fail(FHS_ERR_TIMEOUT, "a bounded wait in a device kernel gave up (code %d: %s)", h,
                h == 1 ? "tensor-core Gram stage barrier" : "window copy of the pass over G");
}

// Copies the device-side error flag to the host, synchronises s and returns
// take_device_error's verdict.
fhs_status device_error(fhs_problem *p, cudaStream_t s) {
    int h = 0;
    CU(cudaMemcpyAsync(&h, p->dev_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    return take_device_error(p, h, s);
}

fhs_status check_params(const fhs_params *q) {
    if (!q) return fail(FHS_ERR_ARG, "params is NULL");
    if (q->ny < 16 || q->nx < 16 || (q->ny & 1) || (q->nx & 1))
        return fail(FHS_ERR_ARG, "image sides must be even and >= 16 (got %d x %d)", q->ny, q->nx);
    if (2LL * q->ny >= 65536 || 2LL * q->nx >= 65536) return fail(FHS_ERR_ARG, "image side too large");
    if (q->n_channels < 1 || q->n_subcubes < 1 || q->n_channels % q->n_subcubes)
        return fail(FHS_ERR_ARG, "n_channels must be a positive multiple of n_subcubes");
    if (q->n_channels / q->n_subcubes > kMaxLc)
        return fail(FHS_ERR_ARG, "at most %d channels per sub-cube are supported", kMaxLc);
    if (q->n_blocks < 1) return fail(FHS_ERR_ARG, "n_blocks must be >= 1");
    if (q->qy < 1 || q->qx < 1 || q->qy > q->ny || q->qx > q->nx) return fail(FHS_ERR_ARG, "bad facet grid");
    if (!(q->facet_overlap >= 0.0 && q->facet_overlap < 1.0)) return fail(FHS_ERR_ARG, "facet_overlap must be in [0, 1)");
    if (q->kb_taps < 2 || q->kb_taps > 8) return fail(FHS_ERR_ARG, "kb_taps must be in [2, 8]");
    if (q->wavelet_levels < 1 || q->wavelet_levels > kMaxLevels) return fail(FHS_ERR_ARG, "wavelet_levels must be in [1, 6]");
    if (q->w_max < 0.0) return fail(FHS_ERR_ARG, "w_max must be >= 0");
    if (q->w_max > 0.0 && (q->n_wplanes < 2 || q->n_wplanes > 4096)) return fail(FHS_ERR_ARG, "n_wplanes must be in [2, 4096]");
    if (q->w_max > 0.0 && !(q->pixel_size > 0.0)) return fail(FHS_ERR_ARG, "pixel_size must be > 0 with w-terms");
    if (!std::isfinite(q->mu) || !std::isfinite(q->mu_bar))
        return fail(FHS_ERR_ARG, "mu and mu_bar must be finite (>= 0, or < 0 for the dirty-image default)");
    if (!(q->upsilon > 0.0) || !(q->upsilon_bar > 0.0)) return fail(FHS_ERR_ARG, "upsilon and upsilon_bar must be > 0");
    if (q->gram_precision < FHS_GRAM_FP32 || q->gram_precision > FHS_GRAM_FP64)
        return fail(FHS_ERR_ARG, "gram_precision must be one of FHS_GRAM_FP32, _TF32, _BF16, _FP64");
    if (q->data_reduction != 0 && q->data_reduction != 1) return fail(FHS_ERR_ARG, "data_reduction must be 0 or 1");
    return FHS_OK;
}

// F of a real zero-padded grid: R2C into the half grid `out` (columns 0..K2/2, row stride HS);
// the passes over G read the other columns as X(k) = conj X(-k).
fhs_status fft_forward(fhs_problem *p, const float *in, float2 *out, cudaStream_t s) {
    CUFFT(cufftSetStream(p->plan_r2c, s));
    CUFFT(cufftExecR2C(p->plan_r2c, const_cast<cufftReal *>(in), reinterpret_cast<cufftComplex *>(out)));
    return FHS_OK;
}

// Re F^H g from the half grid `in` holding the Hermitian part of g (the folded adjoint): C2R into
// the real grid `out`.  The transform overwrites `in`.
fhs_status fft_inverse(fhs_problem *p, float2 *in, float *out, cudaStream_t s) {
    CUFFT(cufftSetStream(p->plan_c2r, s));
    CUFFT(cufftExecC2R(p->plan_c2r, reinterpret_cast<cufftComplex *>(in), reinterpret_cast<cufftReal *>(out)));
    return FHS_OK;
}

// Zeroes L half grids (the target of a folded scatter).
fhs_status zero_half(fhs_problem *p, float2 *grid, cudaStream_t s) {
    CU(cudaMemsetAsync(grid, 0, sizeof(float2) * p->KH * p->L, s));
    return FHS_OK;
}

// Re F^H G^H of sorted visibilities `vis` into the real grid `out` (grid: scratch).
fhs_status adjoint_to_real(fhs_problem *p, const float2 *vis, float2 *grid, float *out, cudaStream_t s) {
    TRY(zero_half(p, grid, s));
    CU(launch_grid(p, vis, grid, s, true, true));
    TRY(fft_inverse(p, grid, out, s));
    return FHS_OK;
}

fhs_status forward_from_image(fhs_problem *p, const float *x, float2 *vis_sorted, cudaStream_t s) {
    CU(launch_zpad(p, x, p->grid_in, s));
    TRY(fft_forward(p, p->grid_in, p->grid_aux, s));
    CU(launch_degrid(p, p->grid_aux, vis_sorted, s));
    return FHS_OK;
}

fhs_status adjoint_to_image(fhs_problem *p, const float2 *vis_sorted, float *x, cudaStream_t s) {
    TRY(adjoint_to_real(p, vis_sorted, p->grid_aux, p->real_scr, s));
    CU(launch_crop(p, p->real_scr, x, s));
    return FHS_OK;
}

// y = Re(Phi^H Phi) v for every channel: one pass over G in the normal mode
// (gather and scatter of each row together) between the two FFTs.  grid_in
// keeps its zero padding (Z writes the image cells only) and grid_work and
// adj_real (Phi^H of the data dual) are iteration state, so the adjoint grids
// go to grid_scr and real_scr.
//
// With data reduction, y = Re(Phi'^H Phi') v = Re Z^T F^H H Lambda^2 H F Z v:
// two passes over G with the Lambda^2 weighting between them (dr_u and dr_w
// are zero / free between iterations).
fhs_status apply_normal(fhs_problem *p, const float *v, float *y, cudaStream_t s) {
    float2 *scratch = p->grid_scr;
    CU(launch_zpad(p, v, p->grid_in, s));
    TRY(fft_forward(p, p->grid_in, p->grid_aux, s));
    TRY(zero_half(p, scratch, s));
    if (p->dr) {
        CU(launch_normal(p, p->grid_aux, true, p->dr_u, s, false, false));
        CU(launch_dr_combine(p, p->dr_u, 0.f, 1.f, p->dr_w, s));
        CU(launch_normal(p, p->dr_w, false, scratch, s, false, true));
    } else {
        CU(launch_normal(p, p->grid_aux, true, scratch, s, true, true));
    }
    TRY(fft_inverse(p, scratch, p->real_scr, s));
    CU(launch_crop(p, p->real_scr, y, s));
    return FHS_OK;
}

// x = Re Phi^H y (the dirty image before the PSF normalisation); with data
// reduction Re Phi'^H y' = Re Z^T F^H H Lambda y'.
fhs_status dirty_image(fhs_problem *p, float *x, cudaStream_t s) {
    if (!p->dr) return adjoint_to_image(p, p->y, x, s);
    CU(launch_dr_combine(p, nullptr, 1.f, 0.f, p->dr_w, s));
    TRY(zero_half(p, p->grid_aux, s));
    CU(launch_normal(p, p->dr_w, false, p->grid_aux, s, false, true));
    TRY(fft_inverse(p, p->grid_aux, p->real_scr, s));
    CU(launch_crop(p, p->real_scr, x, s));
    return FHS_OK;
}

// Largest eigenvalue of the symmetric tridiagonal matrix with diagonal a[0..m)
// and squared off-diagonal b2[0..m-1), by bisection on the Sturm count (the
// number of negative pivots of T - x I is the number of eigenvalues below x).
double tridiag_max_eig(const double *a, const double *b2, int m) {
    if (m <= 0) return 0.0;
    double lo = a[0], hi = a[0];
    for (int i = 0; i < m; ++i) {
        const double r = (i > 0 ? std::sqrt(b2[i - 1]) : 0.0) + (i + 1 < m ? std::sqrt(b2[i]) : 0.0);
        lo = std::min(lo, a[i] - r);
        hi = std::max(hi, a[i] + r);
    }
    const double scale = std::max(std::fabs(lo), std::fabs(hi));
    if (!(scale > 0.0)) return 0.0;
    auto below = [&](double x) {
        int c = 0;
        double q = 1.0;
        for (int i = 0; i < m; ++i) {
            q = (a[i] - x) - (i > 0 ? b2[i - 1] / q : 0.0);
            if (q == 0.0) q = -1e-300 * scale;
            if (q < 0.0) ++c;
        }
        return c;
    };
    for (int it = 0; it < 200 && hi - lo > 1e-15 * scale; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (below(mid) == m) hi = mid; else lo = mid;
    }
    return hi;
}

// ||Phi_l||^2 = lambda_max(Re(Phi_l^H Phi_l)) for every channel by the Lanczos
// recurrence from a fixed random start (the largest Ritz value rises
// monotonically to lambda_max, far faster than the power method when the top of
// the spectrum is clustered).  Work vectors: Xbar (v_{j-1}), A_sara (v_j) and the
// first L*N entries of coef_tmp (w); all three are zero again on return.
// PSF-peak normalisation (Sec. 5.3): eta_l = 1 / (Re Phi_l^H Phi_l delta)(centre), delta the unit
// image at the phase centre; 0 for a channel without visibilities.  Scratch: coef_tmp, Xbar
// (zero again on return).
fhs_status psf_factors(fhs_problem *p, cudaStream_t s) {
    const long long LN = (long long)p->L * p->N;
    const long long centre = (long long)(p->ny / 2) * p->nx + p->nx / 2;
    std::vector<float> delta(LN, 0.f);
    for (int l = 0; l < p->L; ++l) delta[(size_t)l * p->N + centre] = 1.f;
    TRY(upload(p->coef_tmp, delta.data(), LN, s));
    TRY(apply_normal(p, p->coef_tmp, p->Xbar, s));
    std::vector<float> peak(p->L), eta(p->L);
    for (int l = 0; l < p->L; ++l)
        CU(cudaMemcpyAsync(&peak[l], p->Xbar + (long long)l * p->N + centre, sizeof(float), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    for (int l = 0; l < p->L; ++l) eta[l] = peak[l] > 0.f ? 1.f / peak[l] : 0.f;
    TRY(upload(p->eta, eta.data(), p->L, s));
    CU(cudaMemsetAsync(p->Xbar, 0, sizeof(float) * LN, s));
    CU(cudaMemsetAsync(p->coef_tmp, 0, sizeof(float) * LN, s));
    return FHS_OK;
}

// Dirty-image defaults of the regularisation (the paper defers its heuristics to Part I; this
// is the reading used): with X = eta_l Phi_l^H y_l, mu_bar = 1 / sum_{c,q} ||S_q X_c||_* and
// mu = 1 / sum_c ||Psi^dagger X_c||_{2,1}.  Each is computed only when its parameter is
// negative.  Scratch: A_sara, coef_tmp, the Grams (zero again on return).
fhs_status default_regularisation(fhs_problem *p, cudaStream_t s) {
    const bool want_mu = p->prm.mu < 0.0, want_mu_bar = p->prm.mu_bar < 0.0;
    if (!want_mu && !want_mu_bar) return FHS_OK;
    const long long LN = (long long)p->L * p->N;
    float *X = p->A_sara;
    TRY(dirty_image(p, X, s));
    CU(launch_chan_scale(p, X, p->eta, s));
    double *tmp = nullptr;
    const size_t n_tmp = (size_t)p->C * p->Q * p->Lc + p->C;
    CU(cudaMallocAsync(reinterpret_cast<void **>(&tmp), sizeof(double) * n_tmp, s));
    fhs_status rs = FHS_OK;
    auto run = [&]() -> fhs_status {
        CU(cudaMemsetAsync(tmp, 0, sizeof(double) * n_tmp, s));
        double *svals = tmp, *l21 = tmp + (size_t)p->C * p->Q * p->Lc;
        if (want_mu_bar) {
            CU(launch_nuclear_gram(p, X, false, true, s));
            CU(launch_nuclear_svals(p, svals, s));
        }
        if (want_mu) {
            CU(launch_sara_analysis(p, X, p->coef_tmp, s));
            CU(launch_l21_norm(p, p->coef_tmp, l21, s));
        }
        std::vector<double> h(n_tmp);
        CU(cudaMemcpyAsync(h.data(), tmp, sizeof(double) * n_tmp, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        double nuc = 0.0, l = 0.0;
        for (size_t i = 0; i < (size_t)p->C * p->Q * p->Lc; ++i) nuc += h[i];
        for (int c = 0; c < p->C; ++c) l += h[(size_t)p->C * p->Q * p->Lc + c];
        if (want_mu_bar) {
            if (!(nuc > 0.0)) return fail(FHS_ERR_ARG, "mu_bar default: the dirty image is zero");
            p->prm.mu_bar = 1.0 / nuc;
        }
        if (want_mu) {
            if (!(l > 0.0)) return fail(FHS_ERR_ARG, "mu default: the dirty image is zero");
            p->prm.mu = 1.0 / l;
        }
        return FHS_OK;
    };
    rs = run();
    cudaFreeAsync(tmp, s);
    CU(cudaMemsetAsync(X, 0, sizeof(float) * LN, s));
    CU(cudaMemsetAsync(p->coef_tmp, 0, sizeof(float) * (size_t)p->sara.n_coef * p->L, s));
    return rs;
}

// y = Re(Phi_l^H Phi_l) v for the channels `chans` alone (other channels of y are left as they
// are): per channel Z, R2C by the batch-1 plan f1, the normal-mode pass over the channel's bins
// [bfirst[l], bfirst[l] + bcount[l]), C2R by i1, Z^T.
fhs_status apply_normal_channels(fhs_problem *p, const float *v, float *y, const std::vector<int> &chans,
                                 const std::vector<int> &bfirst, const std::vector<int> &bcount, cufftHandle f1,
                                 cufftHandle i1, cudaStream_t s) {
    CUFFT(cufftSetStream(f1, s));
    CUFFT(cufftSetStream(i1, s));
    for (const int l : chans) {
        CU(launch_zpad_channel(p, v, p->grid_in, l, s));
        CUFFT(cufftExecR2C(f1, p->grid_in + (long long)l * p->K,
                           reinterpret_cast<cufftComplex *>(p->grid_aux + (long long)l * p->KH)));
        CU(cudaMemsetAsync(p->grid_scr + (long long)l * p->KH, 0, sizeof(float2) * p->KH, s));
        CU(launch_normal(p, p->grid_aux, true, p->grid_scr, s, true, true, bfirst[l], bcount[l]));
        CUFFT(cufftExecC2R(i1, reinterpret_cast<cufftComplex *>(p->grid_scr + (long long)l * p->KH),
                           p->real_scr + (long long)l * p->K));
        CU(launch_crop_channel(p, p->real_scr, y, l, s));
    }
    return FHS_OK;
}

// Batch-1 R2C / C2R plans on the problem's work area (for apply_normal_channels); false if they
// cannot be made or need more work area than the batched plans have.
bool channel_plans(fhs_problem *p, cufftHandle *f1, cufftHandle *i1) {
    int n[2] = {p->K1, p->K2}, emb[2] = {p->K1, p->K2}, hemb[2] = {p->K1, p->HS};
    size_t wf = 0, wi = 0;
    *f1 = *i1 = 0;
    if (cufftCreate(f1) != CUFFT_SUCCESS) return false;
    if (cufftCreate(i1) != CUFFT_SUCCESS) {
        cufftDestroy(*f1);
        return false;
    }
    const bool ok = cufftSetAutoAllocation(*f1, 0) == CUFFT_SUCCESS && cufftSetAutoAllocation(*i1, 0) == CUFFT_SUCCESS &&
                    cufftMakePlanMany(*f1, 2, n, emb, 1, int(p->K), hemb, 1, int(p->KH), CUFFT_R2C, 1, &wf) ==
                        CUFFT_SUCCESS &&
                    cufftMakePlanMany(*i1, 2, n, hemb, 1, int(p->KH), emb, 1, int(p->K), CUFFT_C2R, 1, &wi) ==
                        CUFFT_SUCCESS &&
                    std::max(wf, wi) <= p->fft_ws_bytes && cufftSetWorkArea(*f1, p->fft_ws) == CUFFT_SUCCESS &&
                    cufftSetWorkArea(*i1, p->fft_ws) == CUFFT_SUCCESS;
    if (!ok) {
        cufftDestroy(*f1);
        cufftDestroy(*i1);
        *f1 = *i1 = 0;
    }
    return ok;
}

// ||Phi_l||^2 for every channel by Lanczos (see above).  Only the largest value sets the data
// step, so once every estimate changes by less than kNarrowTol over 5 steps, the steps go on
// only for the channels within kNarrowMargin of the largest estimate (Ritz values rise
// monotonically to lambda_max, and these have all but stopped rising); the others keep their
// last estimate.
constexpr double kNarrowTol = 1e-2, kNarrowMargin = 0.1, kNarrowStop = 1e-3;

fhs_status norm_estimate(fhs_problem *p, int n_iter, double tol, std::vector<double> &lam, cudaStream_t s,
                         int *steps_taken = nullptr) {
    const long long LN = (long long)p->L * p->N;
    const int L = p->L;
    std::vector<float> x0(LN);
    unsigned long long st = 0x9E3779B97F4A7C15ull;
    for (long long i = 0; i < LN; ++i) {
        st = st * 6364136223846793005ull + 1442695040888963407ull;
        x0[i] = float(double(st >> 11) * (1.0 / 9007199254740992.0) - 0.5);
    }
    double *norms = p->pnorms;
    float *vprev = p->Xbar, *v = p->A_sara, *y = p->coef_tmp;
    const bool trace = std::getenv("FHS_TRACE_SETUP") != nullptr;
    double *coef = nullptr;                     // alpha[n_iter][L] then nb2[n_iter + 1][L]
    const size_t n_coef = (size_t)(2 * n_iter + 1) * L;
    CU(cudaMallocAsync(reinterpret_cast<void **>(&coef), sizeof(double) * n_coef, s));
    int *d_chans = nullptr;                     // the narrowed channels, for the vector steps
    if (cudaMallocAsync(reinterpret_cast<void **>(&d_chans), sizeof(int) * L, s) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeAsync(coef, s);
        return fail(FHS_ERR_OOM, "device allocation of the Lanczos channel list failed");
    }
    fhs_status rs = FHS_OK;
    std::vector<int> chans, bfirst, bcount;
    // the channels' bin ranges (bins are ordered by channel), for the narrowed steps
    cufftHandle f1 = 0, i1 = 0;
    bool can_narrow = !p->dr && L > 1 && p->n_bin > 0;
    if (can_narrow) {
        std::vector<int> bc(p->n_bin);
        if (cudaMemcpyAsync(bc.data(), p->bin_chan, sizeof(int) * p->n_bin, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            can_narrow = false;
        }
        bfirst.assign(L, 0);
        bcount.assign(L, 0);
        for (int b = 0; can_narrow && b < p->n_bin; ++b) {
            if (b > 0 && bc[b] < bc[b - 1]) can_narrow = false;
            else if (bcount[bc[b]]++ == 0) bfirst[bc[b]] = b;
        }
    }
    auto run = [&]() -> fhs_status {
        double *alpha = coef, *nb2 = coef + (size_t)n_iter * L;
        CU(cudaMemsetAsync(coef, 0, sizeof(double) * n_coef, s));
        CU(cudaMemsetAsync(vprev, 0, sizeof(float) * LN, s));
        TRY(upload(v, x0.data(), LN, s));
        CU(cudaMemsetAsync(norms, 0, sizeof(double) * 2 * L, s));
        CU(launch_power_dots(p, v, v, norms, s));
        CU(launch_power_scale(p, v, v, norms, s));
        lam.assign(L, 0.0);
        std::vector<double> ha, hb, prev(L, -1.0), al, bl;
        bool narrow = false;
        for (int j = 0; j < n_iter; ++j) {
            if (narrow) TRY(apply_normal_channels(p, v, y, chans, bfirst, bcount, f1, i1, s));
            else TRY(apply_normal(p, v, y, s));
            CU(launch_lanczos_step(p, y, vprev, v, alpha + (size_t)j * L, nb2 + (size_t)j * L, s,
                                   narrow ? d_chans : nullptr, int(chans.size())));
            std::swap(vprev, v);
            if (steps_taken) *steps_taken = j + 1;
            const bool last = j + 1 == n_iter;
            if (!last && !(tol > 0.0 && (j + 1) % 5 == 0)) continue;
            const int m = j + 1;
            ha.resize((size_t)m * L);
            hb.resize((size_t)m * L);
            CU(cudaMemcpyAsync(ha.data(), alpha, sizeof(double) * m * L, cudaMemcpyDeviceToHost, s));
            CU(cudaMemcpyAsync(hb.data(), nb2 + L, sizeof(double) * m * L, cudaMemcpyDeviceToHost, s));
            CU(cudaStreamSynchronize(s));
            double worst = 0.0;
            int open = 0;
            al.resize(m);
            bl.resize(m);
            for (int l = 0; l < L; ++l) {
                if (narrow && !std::binary_search(chans.begin(), chans.end(), l)) continue;
                for (int i = 0; i < m; ++i) {
                    al[i] = ha[(size_t)i * L + l];
                    bl[i] = hb[(size_t)i * L + l];
                }
                lam[l] = tridiag_max_eig(al.data(), bl.data(), m);
                const double ch = std::fabs(lam[l] - prev[l]) / std::max(std::fabs(lam[l]), 1e-300);
                worst = std::max(worst, ch);
                open += ch >= tol;
                prev[l] = lam[l];
            }
            if (trace)
                std::fprintf(stderr, "fhs set-up: Lanczos step %3d: largest relative change %.3e, %d of %d channels above %.0e\n",
                             m, worst, open, narrow ? int(chans.size()) : L, tol);
            // narrowed, the largest estimate alone would decide the stop, and a change below tol
            // over 5 steps can leave it short of its limit by far more than tol (all channels at
            // once kept it iterating while the slowest converged): the narrowed channels run on
            // until they are stationary to rounding, or to the step limit
            if (tol > 0.0 && worst < (narrow ? kNarrowStop * tol : tol)) break;
            if (!narrow && tol > 0.0 && worst < kNarrowTol && can_narrow) {
                const double top = *std::max_element(lam.begin(), lam.end());
                chans.clear();
                for (int l = 0; l < L; ++l)
                    if (lam[l] >= (1.0 - kNarrowMargin) * top) chans.push_back(l);
                if (2 * chans.size() <= size_t(L) && channel_plans(p, &f1, &i1)) {
                    CU(cudaMemcpyAsync(d_chans, chans.data(), sizeof(int) * chans.size(), cudaMemcpyHostToDevice,
                                       s));
                    CU(cudaStreamSynchronize(s));    // chans is host memory of this frame
                    narrow = true;
                    if (trace)
                        std::fprintf(stderr, "fhs set-up: Lanczos from step %d on %d of %d channels\n", m,
                                     int(chans.size()), L);
                }
            }
        }
        return FHS_OK;
    };
    rs = run();
    if (f1) cufftDestroy(f1);
    if (i1) cufftDestroy(i1);
    cudaFreeAsync(coef, s);
    cudaFreeAsync(d_chans, s);
    if (rs != FHS_OK) return rs;
    CU(cudaMemsetAsync(p->Xbar, 0, sizeof(float) * LN, s));
    CU(cudaMemsetAsync(p->A_sara, 0, sizeof(float) * LN, s));
    CU(cudaMemsetAsync(p->coef_tmp, 0, sizeof(float) * LN, s));
    return FHS_OK;
}

// Side T = J + 2h of the G box of a visibility with coordinate w (w-plane rule).
int row_side(double wv, const fhs_params &q) {
    if (!(q.w_max > 0.0)) return q.kb_taps;
    const int P1 = q.n_wplanes - 1;
    const double dw = q.w_max / P1;
    long long pa = (long long)std::floor(std::fabs(wv) / dw + 0.5);
    if (pa > P1) pa = P1;
    return q.kb_taps + 2 * int((8 * pa + P1) / (2 * P1));
}

// Facets of the low-rankness prior: tiles at floor(i n / Q), extended on the
// low side by ceil(overlap * tile) and clipped at 0, row-major.
std::vector<Facet> facet_list(const fhs_params &q) {
    auto axis = [&](int n, int Qd) {
        std::vector<std::pair<int, int>> r;
        for (int i = 0; i < Qd; ++i) {
            const int b0 = int((long long)i * n / Qd), b1 = int((long long)(i + 1) * n / Qd);
            const int ext = int(std::ceil(q.facet_overlap * double(b1 - b0)));
            r.push_back({std::max(0, b0 - ext), b1});
        }
        return r;
    };
    std::vector<Facet> f;
    for (auto &a : axis(q.ny, q.qy))
        for (auto &b : axis(q.nx, q.qx)) f.push_back({a.first, a.second, b.first, b.second});
    return f;
}

bool sara_active(const fhs_problem *p) { return p->prm.mu > 0.0; }
bool nuc_active(const fhs_problem *p) { return p->prm.mu_bar > 0.0; }

// Records an event pair around one phase of the iteration while tracing is on.
struct Phase {
    fhs_problem *p;
    cudaStream_t s;
    int id;
    cudaEvent_t a = nullptr, b = nullptr;
    Phase(fhs_problem *p_, cudaStream_t s_, int id_) : p(p_), s(s_), id(id_) {
        if (!p->prof_on) return;
        a = take();
        b = take();
        if (a) cudaEventRecord(a, s);
    }
    cudaEvent_t take() {
        if (!p->ev_pool.empty()) {
            cudaEvent_t e = p->ev_pool.back();
            p->ev_pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
        return e;
    }
    ~Phase() {
        if (!p->prof_on || !a || !b) return;
        cudaEventRecord(b, s);
        p->ev_used.push_back({id, {a, b}});
    }
};

fhs_status one_iteration(fhs_problem *p, cudaStream_t s) {
    CU(cudaMemsetAsync(p->red, 0, 2 * sizeof(double), s));
    {
        Phase ph(p, s, FHS_PHASE_PRIMAL);
        CU(launch_primal(p, s));
    }
    // the prior branches only read xbar and fork off after the dual pass over G
    // (they then overlap the l2-ball factors, the scatter pass and F^H; beside
    // the first pass they take the shared memory it needs and cost more than
    // they save); tracing keeps one stream so that its per-phase event pairs
    // time one phase at a time
    const bool fork = !p->prof_on && p->s_sara && p->s_nuc && (sara_active(p) || nuc_active(p));
    // data fidelity: F, dual pass over G, l2-ball factors, scatter pass, F^H
    {
        Phase ph(p, s, FHS_PHASE_FFT_FWD);
        TRY(fft_forward(p, p->grid_in, p->grid_work, s));
    }
    {
        Phase ph(p, s, FHS_PHASE_DEGRID_GRID);
        if (p->dr) CU(launch_normal(p, p->grid_work, true, p->dr_u, s, false, false));     // H Xhat
        else CU(launch_data_dual(p, s));                               // d, block norms
    }
    if (fork) {
        CU(cudaEventRecord(p->ev_fork, s));
        CU(cudaStreamWaitEvent(p->s_sara, p->ev_fork, 0));
        CU(cudaStreamWaitEvent(p->s_nuc, p->ev_fork, 0));
    }
    if (p->dr) {
        // reduced l2 balls, then the adjoint pass H Lambda v into grid_work
        {
            Phase ph(p, s, FHS_PHASE_L2BALL);
            CU(launch_dr_dual(p, s));
            CU(launch_dr_finalize(p, s));
            TRY(zero_half(p, p->grid_work, s));
        }
        Phase ph(p, s, FHS_PHASE_SCATTER);
        CU(launch_normal(p, p->dr_w, false, p->grid_work, s, false, true));
    } else {
        // l2-ball factors, then G^H (s_b d) straight into the channel grids
        {
            Phase ph(p, s, FHS_PHASE_L2BALL);
            CU(launch_block_finalize(p, s));
            TRY(zero_half(p, p->grid_work, s));
        }
        Phase ph(p, s, FHS_PHASE_SCATTER);
        CU(launch_data_scatter(p, s));
    }
    {
        Phase ph(p, s, FHS_PHASE_FFT_INV);
        TRY(fft_inverse(p, p->grid_work, p->adj_real, s));
    }
    // average joint sparsity
    if (sara_active(p)) {
        cudaStream_t ss = fork ? p->s_sara : s;
        Phase ph(p, s, FHS_PHASE_SARA);
        CU(launch_sara_analysis(p, p->Xbar, p->coef_tmp, ss));
        CU(launch_l21_dual(p, ss));
        CU(launch_sara_synthesis(p, p->W, p->A_sara, ss));
        if (fork) CU(cudaEventRecord(p->ev_sara, ss));
    }
    // faceted low-rankness
    if (nuc_active(p)) {
        cudaStream_t sn = fork ? p->s_nuc : s;
        Phase ph(p, s, FHS_PHASE_NUCLEAR);
        const int gp = p->prm.gram_precision;
        if (gp == FHS_GRAM_TF32 || gp == FHS_GRAM_BF16) CU(launch_nuclear_gram_tc(p, gp, sn));
        else CU(launch_nuclear_gram(p, p->Xbar, true, gp == FHS_GRAM_FP64, sn));
        CU(launch_nuclear_eig(p, false, sn));
        CU(launch_nuclear_apply(p, sn));
        if (fork) CU(cudaEventRecord(p->ev_nuc, sn));
    }
    if (fork) {                                  // join
        if (sara_active(p)) CU(cudaStreamWaitEvent(s, p->ev_sara, 0));
        if (nuc_active(p)) CU(cudaStreamWaitEvent(s, p->ev_nuc, 0));
    }
    if (p->prof_on) p->prof_iters++;
    p->iteration++;
    return FHS_OK;
}

// n iterations on stream s: replays a CUDA graph of one iteration (captured
// once per stream) when graphs are enabled, the stream is not the legacy
// default stream and tracing is off; otherwise launches kernel by kernel.
// A capture that fails (a library call that cannot be captured) turns graphs
// off for the problem and falls back to plain launches.
fhs_status run_iterations(fhs_problem *p, int n, cudaStream_t s) {
    const bool can = p->use_graphs && !p->prof_on && s != nullptr && n > 0;
    if (can && (!p->gexec || p->gstream != s)) {
        if (p->gexec) {
            cudaGraphExecDestroy(p->gexec);
            p->gexec = nullptr;
        }
        const long long l0 = p->n_launch;
        const int it0 = p->iteration;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        fhs_status st = FHS_ERR_CUDA;
        if (e == cudaSuccess) {
            st = one_iteration(p, s);
            e = cudaStreamEndCapture(s, &g);
        }
        p->iteration = it0;
        const long long per = p->n_launch - l0;
        p->n_launch = l0;
        if (st == FHS_OK && e == cudaSuccess && g) e = cudaGraphInstantiate(&p->gexec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (st != FHS_OK || e != cudaSuccess || !p->gexec) {
            cudaGetLastError();
            p->gexec = nullptr;
            p->use_graphs = false;
        } else {
            p->gstream = s;
            p->g_launches = per;
        }
    }
    if (can && p->gexec) {
        for (int it = 0; it < n; ++it) {
            CU(cudaGraphLaunch(p->gexec, s));
            p->iteration++;
            p->n_launch += p->g_launches;
        }
        return FHS_OK;
    }
    for (int it = 0; it < n; ++it) TRY(one_iteration(p, s));
    return FHS_OK;
}

// Work area of the R2C and C2R plans (one shared area: the larger of the two).
size_t cufft_workspace(int K1, int K2, int L) {
    const int hs = K2 / 2 + 1;
    int n[2] = {K1, K2}, emb[2] = {K1, K2}, hemb[2] = {K1, hs};
    size_t wf = 0, wi = 0;
    if (cufftEstimateMany(2, n, emb, 1, K1 * K2, hemb, 1, K1 * hs, CUFFT_R2C, L, &wf) != CUFFT_SUCCESS) wf = 0;
    if (cufftEstimateMany(2, n, hemb, 1, K1 * hs, emb, 1, K1 * K2, CUFFT_C2R, L, &wi) != CUFFT_SUCCESS) wi = 0;
    return std::max(wf, wi);
}

}  // namespace

void fhs::set_last_error(const std::string &msg) { g_err = msg; }

void fhs::destroy_on_stream(fhs_problem *p, cudaStream_t s) {
    if (!p) return;
    cudaStreamSynchronize(s);
    for (auto &u : p->ev_used) { cudaEventDestroy(u.second.first); cudaEventDestroy(u.second.second); }
    for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    p->home = s;
    free_all(p);
    delete p;
}

extern "C" {

const char *fhs_last_error(void) { return g_err.c_str(); }

void fhs_default_params(fhs_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->ny = p->nx = 256;
    p->n_channels = 1;
    p->n_subcubes = 1;
    p->n_blocks = 1;
    p->qy = p->qx = 1;
    p->facet_overlap = 0.0;
    p->kb_taps = 7;
    p->wavelet_levels = 4;
    p->w_max = 0.0;
    p->n_wplanes = 64;
    p->pixel_size = 0.0;
    p->mu = 0.0;
    p->mu_bar = 0.0;
    p->upsilon = 1e-3;
    p->upsilon_bar = 1e-3;
    p->tau = p->sigma0 = p->sigma1 = p->sigma2 = 0.0;
    p->power_iters = 100;
    p->power_tol = 1e-7;
    p->gram_precision = FHS_GRAM_FP32;
    p->data_reduction = 0;
}

fhs_status fhs_daubechies_filter(int32_t p, double *h_out) {
    if (p < 1 || p > kNumDb || !h_out) return fail(FHS_ERR_ARG, "p must be in [1, 8] and h_out non-NULL");
    const std::vector<double> h = daubechies(p);
    std::copy(h.begin(), h.end(), h_out);
    return FHS_OK;
}

// Wall time of the stages of the problem set-up, printed to stderr when the
// environment variable FHS_TRACE_SETUP is set (each mark waits for the stream,
// so that device work is charged to its own stage).
struct SetupTrace {
    bool on = std::getenv("FHS_TRACE_SETUP") != nullptr;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now(), t = t0;
    void mark(const char *stage, cudaStream_t s) {
        if (!on) return;
        cudaStreamSynchronize(s);
        const auto n = std::chrono::steady_clock::now();
        std::fprintf(stderr, "fhs set-up: %-34s %8.3f s (total %8.3f s)\n", stage,
                     std::chrono::duration<double>(n - t).count(), std::chrono::duration<double>(n - t0).count());
        t = n;
    }
};

// Problem set-up shared by fhs_create_problem and fhs_create_problem_dde (dde: NULL, or
// [M_tot][5][5] complex DDE kernels in the caller's visibility order).
static fhs_status create_impl(const fhs_params *params, const double *omega, const double *w, const double *y,
                              const double *sigma, const int64_t *vis_offsets, const int64_t *block_offsets,
                              const double *eps_in, const double *dde, void *stream, fhs_problem **out) {
    g_err.clear();
    if (!out) return fail(FHS_ERR_ARG, "out is NULL");
    *out = nullptr;
    TRY(check_params(params));
    SetupTrace trace;
    if (!omega || !y || !sigma || !vis_offsets || !block_offsets) return fail(FHS_ERR_ARG, "NULL input array");
    const fhs_params &q = *params;
    const int L = q.n_channels, B = q.n_blocks, J = q.kb_taps;
    if (vis_offsets[0] != 0) return fail(FHS_ERR_ARG, "vis_offsets[0] must be 0");
    for (int l = 0; l < L; ++l) {
        if (vis_offsets[l + 1] < vis_offsets[l]) return fail(FHS_ERR_ARG, "vis_offsets must be non-decreasing");
        if (!(sigma[l] > 0.0)) return fail(FHS_ERR_ARG, "sigma[%d] must be > 0", l);
        const int64_t Ml = vis_offsets[l + 1] - vis_offsets[l];
        const int64_t *bo = block_offsets + (int64_t)l * (B + 1);
        if (bo[0] != 0 || bo[B] != Ml) return fail(FHS_ERR_ARG, "block_offsets of channel %d must run from 0 to M_l", l);
        for (int b = 0; b < B; ++b)
            if (bo[b + 1] < bo[b]) return fail(FHS_ERR_ARG, "block_offsets must be non-decreasing");
    }
    const long long Mtot = vis_offsets[L];
    {
        // first invalid visibility (parallel scan), then the message for it
        std::atomic<long long> first_bad{Mtot};
        parallel_for(Mtot, [&](long long i0, long long i1) {
            for (long long i = i0; i < i1 && i < first_bad.load(std::memory_order_relaxed); ++i) {
                const double a = omega[2 * i], b = omega[2 * i + 1];
                if (!(a >= -M_PI && a < M_PI && b >= -M_PI && b < M_PI) || !std::isfinite(y[2 * i]) ||
                    !std::isfinite(y[2 * i + 1]) || (w && !std::isfinite(w[i]))) {
                    long long cur = first_bad.load();
                    while (i < cur && !first_bad.compare_exchange_weak(cur, i)) {}
                    break;
                }
            }
        });
        const long long i = first_bad.load();
        if (i < Mtot) {
            const double a = omega[2 * i], b = omega[2 * i + 1];
            if (!(a >= -M_PI && a < M_PI && b >= -M_PI && b < M_PI))
                return fail(FHS_ERR_ARG, "omega[%lld] outside [-pi, pi)", i);
            if (!std::isfinite(y[2 * i]) || !std::isfinite(y[2 * i + 1])) return fail(FHS_ERR_ARG, "y[%lld] not finite", i);
            return fail(FHS_ERR_ARG, "w[%lld] not finite", i);
        }
    }
    cudaStream_t s = S(stream);
    trace.mark("input checks", s);

    fhs_problem *p = new (std::nothrow) fhs_problem();
    if (!p) return fail(FHS_ERR_OOM, "host allocation failed");
    auto guard = [&](fhs_status st) {
        if (st != FHS_OK) {
            cudaStreamSynchronize(s);
            free_all(p);
            delete p;
        }
        return st;
    };
    p->prm = q;
    p->home = s;
    p->dr = q.data_reduction != 0;
    p->L = L; p->C = q.n_subcubes; p->Lc = L / q.n_subcubes; p->B = B; p->J = J;
    p->ny = q.ny; p->nx = q.nx; p->K1 = 2 * q.ny; p->K2 = 2 * q.nx;
    p->N = (long long)q.ny * q.nx;
    p->K = (long long)p->K1 * p->K2;
    p->HS = p->K2 / 2 + 1;
    p->KH = (long long)p->K1 * p->HS;
    p->Mtot = Mtot;
    p->vis_off.assign(vis_offsets, vis_offsets + L + 1);
    p->sigma_l.assign(sigma, sigma + L);
    p->n_seg = L * B;
    p->seg_off.resize(p->n_seg + 1);
    for (int l = 0; l < L; ++l)
        for (int b = 0; b < B; ++b) p->seg_off[l * B + b] = vis_offsets[l] + block_offsets[(int64_t)l * (B + 1) + b];
    p->seg_off[p->n_seg] = Mtot;

    // ---- per-visibility geometry, w-plane, tile key; counting sort per segment
    const int K1 = p->K1, K2 = p->K2;
    const int P1 = q.w_max > 0.0 ? q.n_wplanes - 1 : 0;
    const double dw = q.w_max > 0.0 ? q.w_max / P1 : 0.0;
    const int ntx = (K2 + kTile - 1) / kTile, nty = (K1 + kTile - 1) / kTile;
    // per visibility (caller's order) its row meta (corner c1 | c2 << 16, side T) and w-plane:
    // the sorted rows are gathered from these two and from omega and y
    std::vector<int> key(Mtot);
    std::vector<int2> cmeta(Mtot);
    std::vector<short> cplane(Mtot);
    const int n_planes = 2 * P1 + 1;
    std::vector<std::atomic<unsigned char>> used(n_planes);
    for (auto &u : used) u.store(0, std::memory_order_relaxed);
    // with DDE kernels every box grows by kDdeTaps - 1 (half on each side) and a row is the
    // sum of kDdeTaps separable terms (see build_g_kernel)
    const int ext = dde ? kDdeTaps - 1 : 0, hx = ext / 2;
    p->rank = dde ? kDdeTaps : 1;
    std::atomic<int> box_too_big{0};
    std::atomic<long long> wide_rows{0};
    parallel_for(Mtot, [&](long long i0, long long i1) {
    std::vector<unsigned char> seen(n_planes, 0);
    long long nwide = 0;
    for (long long i = i0; i < i1; ++i) {
        const double k1 = omega[2 * i] * K1 / (2.0 * M_PI);
        const double k2 = omega[2 * i + 1] * K2 / (2.0 * M_PI);
        const long long p01 = (long long)std::floor(k1 - J / 2.0) + 1;
        const long long p02 = (long long)std::floor(k2 - J / 2.0) + 1;
        int pv = 0, h = 0;
        if (P1 > 0) {
            const double wv = w ? w[i] : 0.0;
            long long pa = (long long)std::floor(std::fabs(wv) / dw + 0.5);
            if (pa > P1) pa = P1;
            pv = int(wv < 0 ? -pa : pa);
            h = (8 * std::abs(pv) + P1) / (2 * P1);
        }
        const int T = J + 2 * h + ext;
        if (T > 16) box_too_big.store(1, std::memory_order_relaxed);
        nwide += T > 8;
        long long c1 = (p01 - h - hx) % K1; if (c1 < 0) c1 += K1;
        long long c2 = (p02 - h - hx) % K2; if (c2 < 0) c2 += K2;
        cmeta[i] = make_int2(int(c1) | (int(c2) << 16), T);
        cplane[i] = short(pv + P1);
        seen[pv + P1] = 1;
        key[i] = (int(c1 / kTile) * ntx + int(c2 / kTile)) * 17 + T;   // tile, then box side
    }
    for (int k = 0; k < n_planes; ++k)
        if (seen[k]) used[k].store(1, std::memory_order_relaxed);
    wide_rows.fetch_add(nwide, std::memory_order_relaxed);
    });
    p->narrow_rows = p->rank == 1 && 10 * wide_rows.load() <= Mtot;
    if (box_too_big.load()) {
        delete p;
        return fail(FHS_ERR_ARG, "DDE kernels widen the G boxes past 16 taps: with DDEs the w-kernels may "
                                 "add at most %d taps per side (w_max too large for this pixel size)", (16 - J - ext) / 2);
    }
    trace.mark("host geometry (boxes, planes, keys)", s);
    const int nkeys = nty * ntx * 17;
    std::vector<long long> perm(Mtot);
    // sort by tile key, then (inside each (tile, T) run) by box corner, row-major within the
    // tile, so that the rows one warp gathers at once read nearby window cells: two stable
    // counting sorts per segment (corner position first, then tile key), segments in parallel
    parallel_for(p->n_seg, [&](long long s0, long long s1) {
        std::vector<long long> cnt(nkeys + 1), cpos(kTile * kTile + 1), tmp;
        for (long long sg = s0; sg < s1; ++sg) {
            const long long a = p->seg_off[sg], b = p->seg_off[sg + 1];
            auto pos = [&](long long i) {
                const int cc = cmeta[i].x;
                return ((cc & 0xffff) % kTile) * kTile + int((unsigned)cc >> 16) % kTile;
            };
            tmp.resize(size_t(b - a));
            std::fill(cpos.begin(), cpos.end(), 0);
            for (long long i = a; i < b; ++i) cpos[pos(i) + 1]++;
            for (int k = 0; k < kTile * kTile; ++k) cpos[k + 1] += cpos[k];
            for (long long i = a; i < b; ++i) tmp[cpos[pos(i)]++] = i;
            std::fill(cnt.begin(), cnt.end(), 0);
            for (long long i = a; i < b; ++i) cnt[key[i] + 1]++;
            for (int k = 0; k < nkeys; ++k) cnt[k + 1] += cnt[k];
            for (const long long i : tmp) perm[a + cnt[key[i]]++] = i;
        }
    }, 1);
    trace.mark("host sort by tile", s);
    // the sorted rows' meta and factor counts here (the bins need them on the host); their grid
    // coordinates, w-planes and whitened data are gathered on the device (launch_gather_rows)
    std::vector<int2> meta(Mtot);
    std::vector<long long> fptr(Mtot + 1);
    fptr[0] = 0;
    parallel_for(Mtot, [&](long long v0, long long v1) {
        for (long long v = v0; v < v1; ++v) {
            const int2 m = cmeta[perm[v]];
            meta[v] = m;
            fptr[v + 1] = 2LL * p->rank * m.y;
        }
    });
    trace.mark("host rows (meta, offsets)", s);
    {
        // fptr[v + 1] holds row v's factor count: prefix sums (and nnz) over fixed blocks of rows,
        // block totals first, then each block from its offset
        const long long nblk = 64, bl = (Mtot + nblk - 1) / nblk;
        std::vector<long long> bsum(nblk + 1, 0), bnnz(nblk, 0);
        parallel_for(nblk, [&](long long b0, long long b1) {
            for (long long b = b0; b < b1; ++b) {
                long long t = 0, z = 0;
                for (long long v = b * bl; v < std::min(Mtot, (b + 1) * bl); ++v) {
                    t += fptr[v + 1];
                    z += (long long)meta[v].y * meta[v].y;
                }
                bsum[b + 1] = t;
                bnnz[b] = z;
            }
        }, 1);
        p->nnz = 0;
        for (long long b = 0; b < nblk; ++b) {
            bsum[b + 1] += bsum[b];
            p->nnz += bnnz[b];
        }
        parallel_for(nblk, [&](long long b0, long long b1) {
            for (long long b = b0; b < b1; ++b) {
                long long run = bsum[b];
                for (long long v = b * bl; v < std::min(Mtot, (b + 1) * bl); ++v) {
                    run += fptr[v + 1];
                    fptr[v + 1] = run;
                }
            }
        }, 1);
    }
    std::vector<double2> dde_sorted;
    if (dde) {
        dde_sorted.resize((size_t)Mtot * kDdeTaps * kDdeTaps);
        parallel_for(Mtot, [&](long long v0, long long v1) {
            for (long long v = v0; v < v1; ++v) {
                const long long i = perm[v];
                for (int j = 0; j < kDdeTaps * kDdeTaps; ++j)
                    dde_sorted[(size_t)v * kDdeTaps * kDdeTaps + j] =
                        make_double2(dde[2 * (i * kDdeTaps * kDdeTaps + j)], dde[2 * (i * kDdeTaps * kDdeTaps + j) + 1]);
            }
        });
    }
    p->n_fac = fptr[Mtot];
    { std::vector<int> t; t.swap(key); }

    trace.mark("host row offsets (prefix sums)", s);
    // ---- w-kernel table: planes -P1..P1, per axis up to 2*kMaxWHalf+1 taps (those in use)
    { std::vector<int2> t; t.swap(cmeta); }
    std::vector<double2> wk((size_t)n_planes * 2 * (2 * kMaxWHalf + 1), make_double2(0.0, 0.0));
    for (int pi = 0; pi < n_planes; ++pi) {
        if (!used[pi].load(std::memory_order_relaxed)) continue;
        const int pv = pi - P1;
        const int h = P1 > 0 ? (8 * std::abs(pv) + P1) / (2 * P1) : 0;
        const double wp = pv * dw;
        std::complex<double> ck[2 * kMaxWHalf + 1];
        for (int dim = 0; dim < 2; ++dim) {
            wkernel(wp, dim ? q.nx : q.ny, dim ? K2 : K1, q.pixel_size, h, ck);
            for (int jj = 0; jj < 2 * h + 1; ++jj)
                wk[((size_t)pi * 2 + dim) * (2 * kMaxWHalf + 1) + jj] = make_double2(ck[jj].real(), ck[jj].imag());
        }
    }

    // ---- chunks of at most CH visibilities inside one segment
    long long CH = (Mtot + 152 * 8 - 1) / (152 * 8);
    CH = std::max(32LL, std::min(1024LL, CH));
    std::vector<long long> cstart;
    std::vector<int> cseg;
    for (int sg = 0; sg < p->n_seg; ++sg)
        for (long long a = p->seg_off[sg]; a < p->seg_off[sg + 1]; a += CH) {
            cstart.push_back(a);
            cseg.push_back(sg);
        }
    p->n_chunk = int(cseg.size());
    cstart.push_back(Mtot);

    // ---- tile bins for the single-pass data kernel (make_bins); fhs_autotune_bins
    // may replace them with a measured choice
    BinList bins;
    p->ntx = ntx;
    make_bins(meta.data(), fptr.data(), p->seg_off, L, B, ntx, kBinDenseMin, kBinSplitMax, false, kBinSplitMax, bins);
    p->bin_dense_min = int(kBinDenseMin);
    p->bin_split = int(kBinSplitMax);
    p->n_bin = bins.n_bin();
    const SlotBins sb = to_slots(bins);
    p->bin_slots = sb.slots;
    const size_t n_slot = sb.pstart.size();

    trace.mark("host w-kernels, chunks, bins", s);
    std::vector<double> eps(p->n_seg), inv_sig(p->n_seg);
    for (int l = 0; l < L; ++l) {
        const double Ml = double(vis_offsets[l + 1] - vis_offsets[l]);
        for (int b = 0; b < B; ++b) {
            const double Mb = double(block_offsets[(int64_t)l * (B + 1) + b + 1] - block_offsets[(int64_t)l * (B + 1) + b]);
            eps[l * B + b] = (eps_in && !q.data_reduction) ? eps_in[l * B + b]
                                    : (Ml > 0 ? std::sqrt((Ml + 2.0 * std::sqrt(Ml)) * Mb / Ml) : 0.0);
            inv_sig[l * B + b] = 1.0 / sigma[l];
        }
    }

    // ---- device state: data term
    fhs_status st;
    double2 *d_kap = nullptr, *d_wk = nullptr;
    short *d_plane = nullptr;
    double *d_isg = nullptr;
    if ((st = guard(dev_alloc(p, &p->meta, Mtot, false))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &p->fptr, Mtot + 1, false))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &p->gfac, p->n_fac, false))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &p->gmax, Mtot, false))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &p->y, Mtot, false))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &p->dvis, Mtot))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &p->vis_tmp, Mtot))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &p->perm, Mtot, false))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &p->d_seg_off, p->n_seg + 1, false))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &p->blk_norm2, p->n_seg))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &p->eps, p->n_seg, false))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &p->blk_scale, p->n_seg, false))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &p->bin_fbase, p->n_bin, false))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &p->bin_chan, p->n_bin, false))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &p->bin_tile, p->n_bin, false))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &p->piece_start, n_slot, false))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &p->piece_len, n_slot, false))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &p->piece_blk, n_slot, false))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &p->chunk_start, p->n_chunk + 1, false))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &p->chunk_seg, p->n_chunk, false))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &d_kap, Mtot, false))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &d_plane, Mtot, false))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &d_wk, wk.size(), false))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &d_isg, p->n_seg, false))) != FHS_OK) return st;
    double2 *d_dde = nullptr;
    if (dde) {
        if ((st = guard(dev_alloc(p, &d_dde, dde_sorted.size(), false))) != FHS_OK) return st;
        if ((st = guard(upload(d_dde, dde_sorted.data(), dde_sorted.size(), s))) != FHS_OK) return st;
    }
    std::vector<float> ones(p->n_seg, 1.0f);
    if ((st = guard(upload(p->meta, meta.data(), Mtot, s))) != FHS_OK) return st;
    if ((st = guard(upload(p->fptr, fptr.data(), Mtot + 1, s))) != FHS_OK) return st;

    if ((st = guard(upload(p->perm, perm.data(), Mtot, s))) != FHS_OK) return st;
    if ((st = guard(upload(p->d_seg_off, p->seg_off.data(), p->n_seg + 1, s))) != FHS_OK) return st;
    if ((st = guard(upload(p->eps, eps.data(), p->n_seg, s))) != FHS_OK) return st;
    if ((st = guard(upload(p->blk_scale, ones.data(), p->n_seg, s))) != FHS_OK) return st;
    if ((st = guard(upload(p->bin_fbase, bins.fbase.data(), bins.fbase.size(), s))) != FHS_OK) return st;
    if ((st = guard(upload(p->bin_chan, bins.chan.data(), bins.chan.size(), s))) != FHS_OK) return st;
    if ((st = guard(upload(p->bin_tile, bins.tile.data(), bins.tile.size(), s))) != FHS_OK) return st;
    if ((st = guard(upload(p->piece_start, sb.pstart.data(), n_slot, s))) != FHS_OK) return st;
    if ((st = guard(upload(p->piece_len, sb.plen.data(), n_slot, s))) != FHS_OK) return st;
    if ((st = guard(upload(p->piece_blk, sb.pblk.data(), n_slot, s))) != FHS_OK) return st;
    if ((st = guard(upload(p->chunk_start, cstart.data(), cstart.size(), s))) != FHS_OK) return st;
    if ((st = guard(upload(p->chunk_seg, cseg.data(), cseg.size(), s))) != FHS_OK) return st;
    {
        // the caller's omega, y and w-planes in its order, gathered into the sorted order on the device
        double2 *d_om = nullptr, *d_yc = nullptr;
        short *d_pc = nullptr;
        long long *d_vo = nullptr;
        double *d_sg = nullptr;
        if ((st = guard(dev_alloc(p, &d_om, Mtot, false))) != FHS_OK) return st;
        if ((st = guard(dev_alloc(p, &d_yc, Mtot, false))) != FHS_OK) return st;
        if ((st = guard(dev_alloc(p, &d_pc, Mtot, false))) != FHS_OK) return st;
        if ((st = guard(dev_alloc(p, &d_vo, L + 1, false))) != FHS_OK) return st;
        if ((st = guard(dev_alloc(p, &d_sg, L, false))) != FHS_OK) return st;
        std::vector<long long> vo(vis_offsets, vis_offsets + L + 1);
        if ((st = guard(upload(d_om, reinterpret_cast<const double2 *>(omega), Mtot, s))) != FHS_OK) return st;
        if ((st = guard(upload(d_yc, reinterpret_cast<const double2 *>(y), Mtot, s))) != FHS_OK) return st;
        if ((st = guard(upload(d_pc, cplane.data(), Mtot, s))) != FHS_OK) return st;
        if ((st = guard(upload(d_vo, vo.data(), L + 1, s))) != FHS_OK) return st;
        if ((st = guard(upload(d_sg, sigma, L, s))) != FHS_OK) return st;
        cudaError_t e = launch_gather_rows(p, d_om, d_yc, d_pc, d_vo, d_sg, d_kap, d_plane, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return guard(fail(FHS_ERR_CUDA, "row gather failed: %s", cudaGetErrorString(e)));
        for (void *t : {(void *)d_om, (void *)d_yc, (void *)d_pc, (void *)d_vo, (void *)d_sg}) dev_free(p, t);
        p->bytes -= (sizeof(double2) * 2 + sizeof(short)) * Mtot + sizeof(long long) * (L + 1) + sizeof(double) * L;
        { std::vector<short> t; t.swap(cplane); }
    }
    if ((st = guard(upload(d_wk, wk.data(), wk.size(), s))) != FHS_OK) return st;
    if ((st = guard(upload(d_isg, inv_sig.data(), p->n_seg, s))) != FHS_OK) return st;
    trace.mark("device allocation and upload", s);
    {
        cudaError_t e = launch_build_g(p, d_kap, d_plane, d_wk, d_dde, ext, d_isg, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return guard(fail(FHS_ERR_CUDA, "G build failed: %s", cudaGetErrorString(e)));
        if (d_dde) {
            dev_free(p, d_dde);
            p->bytes -= sizeof(double2) * dde_sorted.size();
            std::vector<double2>().swap(dde_sorted);
        }
    }

    // scaling of Z
    {
        const double beta = kb_beta(J, 2.0);
        std::vector<float> s1(q.ny), s2(q.nx);
        for (int i = 0; i < q.ny; ++i) s1[i] = float(1.0 / kb_hat(double(i - q.ny / 2) / K1, J, beta));
        for (int i = 0; i < q.nx; ++i) s2[i] = float(1.0 / kb_hat(double(i - q.nx / 2) / K2, J, beta));
        if ((st = guard(dev_alloc(p, &p->s1, q.ny, false))) != FHS_OK) return st;
        if ((st = guard(dev_alloc(p, &p->s2, q.nx, false))) != FHS_OK) return st;
        if ((st = guard(upload(p->s1, s1.data(), q.ny, s))) != FHS_OK) return st;
        if ((st = guard(upload(p->s2, s2.data(), q.nx, s))) != FHS_OK) return st;
    }
    {
        // R2C: real [L][K1][K2] -> half grids [L][K1][HS]; C2R the reverse.  One work area serves
        // both (they never run at the same time on a problem's streams).
        int n[2] = {K1, K2}, emb[2] = {K1, K2}, hemb[2] = {K1, p->HS};
        size_t ws_f = 0, ws_i = 0;
        if (cufftCreate(&p->plan_r2c) != CUFFT_SUCCESS) return guard(fail(FHS_ERR_CUDA, "cufftCreate failed"));
        if (cufftCreate(&p->plan_c2r) != CUFFT_SUCCESS) {
            cufftDestroy(p->plan_r2c);
            return guard(fail(FHS_ERR_CUDA, "cufftCreate failed"));
        }
        p->plan_ok = true;
        if (cufftSetAutoAllocation(p->plan_r2c, 0) != CUFFT_SUCCESS ||
            cufftSetAutoAllocation(p->plan_c2r, 0) != CUFFT_SUCCESS ||
            cufftMakePlanMany(p->plan_r2c, 2, n, emb, 1, int(p->K), hemb, 1, int(p->KH), CUFFT_R2C, L, &ws_f) !=
                CUFFT_SUCCESS ||
            cufftMakePlanMany(p->plan_c2r, 2, n, hemb, 1, int(p->KH), emb, 1, int(p->K), CUFFT_C2R, L, &ws_i) !=
                CUFFT_SUCCESS)
            return guard(fail(FHS_ERR_CUDA, "cuFFT plan set-up failed"));
        const size_t ws = std::max<size_t>(std::max(ws_f, ws_i), 1);
        char *w = nullptr;
        if ((st = guard(dev_alloc(p, &w, ws, false))) != FHS_OK) return st;
        p->fft_ws = w;
        p->fft_ws_bytes = ws;
        if (cufftSetWorkArea(p->plan_r2c, p->fft_ws) != CUFFT_SUCCESS ||
            cufftSetWorkArea(p->plan_c2r, p->fft_ws) != CUFFT_SUCCESS)
            return guard(fail(FHS_ERR_CUDA, "cufftSetWorkArea failed"));
    }
    if ((st = guard(dev_alloc(p, &p->grid_in, p->K * L))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &p->grid_work, p->KH * L))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &p->grid_aux, p->KH * L))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &p->grid_scr, p->KH * L))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &p->adj_real, p->K * L))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &p->real_scr, p->K * L, false))) != FHS_OK) return st;
    if (p->dr) {
        // gridding (Sec. 3.4): diag(H_l) by one pass over the rows, Lambda_l, y'_l, M'_l
        const size_t LK = (size_t)p->K * L;
        if ((st = guard(dev_alloc(p, &p->dr_lam, LK, false))) != FHS_OK) return st;
        if ((st = guard(dev_alloc(p, &p->dr_y, LK, false))) != FHS_OK) return st;
        if ((st = guard(dev_alloc(p, &p->dr_v, LK))) != FHS_OK) return st;
        if ((st = guard(dev_alloc(p, &p->dr_u, LK))) != FHS_OK) return st;
        if ((st = guard(dev_alloc(p, &p->dr_w, LK))) != FHS_OK) return st;
        if ((st = guard(dev_alloc(p, &p->dr_norm2, L))) != FHS_OK) return st;
        if ((st = guard(dev_alloc(p, &p->dr_eps, L, false))) != FHS_OK) return st;
        if ((st = guard(dev_alloc(p, &p->dr_scale, L))) != FHS_OK) return st;
        double *diag = nullptr;
        unsigned long long *cnt = nullptr;
        if ((st = guard(dev_alloc(p, &diag, LK))) != FHS_OK) return st;
        if ((st = guard(dev_alloc(p, &cnt, L))) != FHS_OK) return st;
        std::vector<unsigned long long> hc(L);
        cudaError_t e = launch_dr_diag(p, diag, s);
        if (e == cudaSuccess) e = launch_grid(p, p->y, p->dr_u, s, false, false);
        if (e == cudaSuccess) e = launch_dr_setup(p, diag, p->dr_u, cnt, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hc.data(), cnt, sizeof(unsigned long long) * L, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return guard(fail(FHS_ERR_CUDA, "data reduction set-up failed: %s", cudaGetErrorString(e)));
        dev_free(p, diag);
        dev_free(p, cnt);
        p->bytes -= sizeof(double) * LK + sizeof(unsigned long long) * L;
        p->dr_m.assign(hc.begin(), hc.end());
        std::vector<double> de(L);
        for (int l = 0; l < L; ++l) {
            const double m = double(p->dr_m[l]);
            de[l] = eps_in ? eps_in[l] : (m > 0 ? std::sqrt(m + 2.0 * std::sqrt(m)) : 0.0);
        }
        if ((st = guard(upload(p->dr_eps, de.data(), L, s))) != FHS_OK) return st;
    }

    // ---- image domain
    if ((st = guard(dev_alloc(p, &p->X, p->N * L))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &p->Xbar, p->N * L))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &p->A_sara, p->N * L))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &p->red, 2))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &p->pnorms, 2 * L))) != FHS_OK) return st;
    if ((st = guard(dev_alloc(p, &p->dev_err, 1))) != FHS_OK) return st;

    // ---- SARA layout
    {
        p->sara = sara_layout(q.ny, q.nx, q.wavelet_levels);
        const SaraConst &c = p->sara;
        if ((st = guard(dev_alloc(p, &p->W, c.n_coef * L))) != FHS_OK) return st;
        if ((st = guard(dev_alloc(p, &p->coef_tmp, c.n_coef * L))) != FHS_OK) return st;
        if ((st = guard(dev_alloc(p, &p->sara_tmp, c.n_tmp * L))) != FHS_OK) return st;
        if ((st = guard(dev_alloc(p, &p->w21, c.n_coef * p->C, false))) != FHS_OK) return st;
        std::vector<float> w1(c.n_coef * p->C, 1.0f);
        if ((st = guard(upload(p->w21, w1.data(), w1.size(), s))) != FHS_OK) return st;
    }

    // ---- nuclear facets: tiles at floor(i n / Q), low side extended by ceil(overlap * tile)
    {
        auto axis = [&](int n, int Qd) {
            std::vector<std::pair<int, int>> r;
            for (int i = 0; i < Qd; ++i) {
                const int b0 = int((long long)i * n / Qd), b1 = int((long long)(i + 1) * n / Qd);
                const int ext = int(std::ceil(q.facet_overlap * double(b1 - b0)));
                r.push_back({std::max(0, b0 - ext), b1});
            }
            return r;
        };
        const auto ay = axis(q.ny, q.qy), ax = axis(q.nx, q.qx);
        p->Q = q.qy * q.qx;
        p->facets = facet_list(q);
        std::vector<int4> fz;
        for (const Facet &f : p->facets) fz.push_back(make_int4(f.y0, f.y1, f.x0, f.x1));
        auto cover = [&](const std::vector<std::pair<int, int>> &ff, int n, std::vector<short> &first,
                         std::vector<short> &cnt) {
            first.assign(n, 0);
            cnt.assign(n, 0);
            for (int i = 0; i < n; ++i) {
                int f0 = -1, c0 = 0;
                for (int k = 0; k < (int)ff.size(); ++k)
                    if (ff[k].first <= i && i < ff[k].second) {
                        if (f0 < 0) f0 = k;
                        ++c0;
                    }
                first[i] = short(f0);
                cnt[i] = short(c0);
            }
        };
        std::vector<short> rf, rc, cf, cc;
        cover(ay, q.ny, rf, rc);
        cover(ax, q.nx, cf, cc);
        int mr = 0, mc = 0;
        for (short v : rc) mr = std::max(mr, int(v));
        for (short v : cc) mc = std::max(mc, int(v));
        p->max_cover = mr * mc;
        p->h_nuc_off.resize((size_t)p->C * p->Q);
        long long off = 0;
        for (int c = 0; c < p->C; ++c)
            for (int k = 0; k < p->Q; ++k) {
                p->h_nuc_off[(size_t)c * p->Q + k] = off;
                const Facet &f = p->facets[k];
                off += (long long)p->Lc * (f.y1 - f.y0) * (f.x1 - f.x0);
            }
        p->nuc_size = off;
        if ((st = guard(dev_alloc(p, &p->d_facets, p->Q, false))) != FHS_OK) return st;
        if ((st = guard(dev_alloc(p, &p->nuc_off, p->C * p->Q, false))) != FHS_OK) return st;
        if ((st = guard(dev_alloc(p, &p->P, off))) != FHS_OK) return st;
        if ((st = guard(dev_alloc(p, &p->gram, (size_t)p->C * p->Q * p->Lc * p->Lc))) != FHS_OK) return st;
        if ((st = guard(dev_alloc(p, &p->mix, (size_t)p->C * p->Q * p->Lc * p->Lc))) != FHS_OK) return st;
        if ((st = guard(dev_alloc(p, &p->wnuc, (size_t)p->C * p->Q * p->Lc, false))) != FHS_OK) return st;
        {
            const int ne = p->Lc + (p->Lc & 1);
            std::vector<double> eye((size_t)p->C * p->Q * ne * ne, 0.0);
            for (size_t m = 0; m < (size_t)p->C * p->Q; ++m)
                for (int i = 0; i < ne; ++i) eye[m * ne * ne + (size_t)i * ne + i] = 1.0;
            if ((st = guard(dev_alloc(p, &p->eigv, eye.size(), false))) != FHS_OK) return st;
            if ((st = guard(upload(p->eigv, eye.data(), eye.size(), s))) != FHS_OK) return st;
        }
        if ((st = guard(dev_alloc(p, &p->cov_row_first, q.ny, false))) != FHS_OK) return st;
        if ((st = guard(dev_alloc(p, &p->cov_row_cnt, q.ny, false))) != FHS_OK) return st;
        if ((st = guard(dev_alloc(p, &p->cov_col_first, q.nx, false))) != FHS_OK) return st;
        if ((st = guard(dev_alloc(p, &p->cov_col_cnt, q.nx, false))) != FHS_OK) return st;
        std::vector<float> w1((size_t)p->C * p->Q * p->Lc, 1.0f);
        if ((st = guard(upload(p->wnuc, w1.data(), w1.size(), s))) != FHS_OK) return st;
        if ((st = guard(upload(p->d_facets, fz.data(), fz.size(), s))) != FHS_OK) return st;
        if ((st = guard(upload(p->nuc_off, p->h_nuc_off.data(), p->h_nuc_off.size(), s))) != FHS_OK) return st;
        if ((st = guard(upload(p->cov_row_first, rf.data(), rf.size(), s))) != FHS_OK) return st;
        if ((st = guard(upload(p->cov_row_cnt, rc.data(), rc.size(), s))) != FHS_OK) return st;
        if ((st = guard(upload(p->cov_col_first, cf.data(), cf.size(), s))) != FHS_OK) return st;
        if ((st = guard(upload(p->cov_col_cnt, cc.data(), cc.size(), s))) != FHS_OK) return st;
    }

    if (cudaStreamCreateWithFlags(&p->s_sara, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p->s_nuc, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_sara, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_nuc, cudaEventDisableTiming) != cudaSuccess)
        return guard(fail(FHS_ERR_CUDA, "stream/event creation failed"));

    trace.mark("G build and the other device state", s);
    // ---- step sizes (Condat-Vu: tau * sum_i sigma_i ||L_i||^2 < 1)
    p->tau = q.tau > 0 ? q.tau : 0.99 / 3.0;
    p->sigma1 = q.sigma1 > 0 ? q.sigma1 : 1.0;
    p->sigma0 = q.sigma0 > 0 ? q.sigma0 : 1.0 / double(p->max_cover);
    if (q.sigma2 > 0) {
        p->sigma2 = q.sigma2;
    } else {
        std::vector<double> lam;
        const int n_it = q.power_iters > 0 ? q.power_iters : 100;
        const double tol = q.power_tol > 0 ? q.power_tol : 1e-7;
        int steps = 0;
        if ((st = guard(norm_estimate(p, n_it, tol, lam, s, &steps))) != FHS_OK) return st;
        char what[64];
        std::snprintf(what, sizeof what, "operator norms (%d Lanczos steps)", steps);
        trace.mark(what, s);
        p->phi_norm2_max = *std::max_element(lam.begin(), lam.end());
        if (!(p->phi_norm2_max > 0)) return guard(fail(FHS_ERR_ARG, "operator norm is zero (no visibilities?)"));
        p->sigma2 = 1.0 / p->phi_norm2_max;
    }
    if ((st = guard(dev_alloc(p, &p->eta, L, false))) != FHS_OK) return st;
    if ((st = guard(psf_factors(p, s))) != FHS_OK) return st;
    if ((st = guard(default_regularisation(p, s))) != FHS_OK) return st;
    trace.mark("PSF peaks, default regularisation", s);
    {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return guard(fail(FHS_ERR_CUDA, "set-up failed: %s", cudaGetErrorString(e)));
    }
    // set-up temporaries are no longer needed
    for (void *t : {(void *)d_kap, (void *)d_plane, (void *)d_wk, (void *)d_isg}) dev_free(p, t);
    p->bytes -= sizeof(double2) * Mtot + sizeof(short) * Mtot + sizeof(double2) * wk.size() + sizeof(double) * p->n_seg;
    *out = p;
    return FHS_OK;
}

fhs_status fhs_create_problem(const fhs_params *params, const double *omega, const double *w, const double *y,
                              const double *sigma, const int64_t *vis_offsets, const int64_t *block_offsets,
                              const double *eps_in, void *stream, fhs_problem **out) {
    return create_impl(params, omega, w, y, sigma, vis_offsets, block_offsets, eps_in, nullptr, stream, out);
}

fhs_status fhs_create_problem_dde(const fhs_params *params, const double *omega, const double *w, const double *y,
                                  const double *sigma, const int64_t *vis_offsets, const int64_t *block_offsets,
                                  const double *eps_in, const double *dde, void *stream, fhs_problem **out) {
    if (!dde) return fail(FHS_ERR_ARG, "dde is NULL (use fhs_create_problem without DDE kernels)");
    return create_impl(params, omega, w, y, sigma, vis_offsets, block_offsets, eps_in, dde, stream, out);
}

void fhs_destroy_problem(fhs_problem *p) {
    if (!p) return;
    cudaDeviceSynchronize();
    for (auto &u : p->ev_used) { cudaEventDestroy(u.second.first); cudaEventDestroy(u.second.second); }
    for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
    if (p->gexec) cudaGraphExecDestroy(p->gexec);
    p->home = nullptr;          // the creation stream may be gone; the device is idle
    free_all(p);
    delete p;
}

fhs_status fhs_use_graphs(fhs_problem *p, int32_t on) {
    if (!p) return fail(FHS_ERR_ARG, "NULL problem");
    p->use_graphs = on != 0;
    if (!p->use_graphs && p->gexec) {
        cudaGraphExecDestroy(p->gexec);
        p->gexec = nullptr;
    }
    return FHS_OK;
}

fhs_status fhs_pdfb_step_batch(fhs_problem **probs, int32_t n_prob, int32_t n_iter, void **streams,
                               double *rel_change_out) {
    if (!probs || n_prob < 0 || n_iter < 0) return fail(FHS_ERR_ARG, "bad argument");
    for (int k = 0; k < n_prob; ++k)
        if (!probs[k]) return fail(FHS_ERR_ARG, "probs[%d] is NULL", k);
    // one iteration of every problem in turn, so that their work overlaps on the device
    for (int it = 0; it < n_iter; ++it)
        for (int k = 0; k < n_prob; ++k) TRY(run_iterations(probs[k], 1, streams ? S(streams[k]) : nullptr));
    if (rel_change_out) {
        std::vector<double> h(2 * (size_t)n_prob, 0.0);
        for (int k = 0; k < n_prob; ++k)
            CU(cudaMemcpyAsync(h.data() + 2 * k, probs[k]->red, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                               streams ? S(streams[k]) : nullptr));
        for (int k = 0; k < n_prob; ++k) CU(cudaStreamSynchronize(streams ? S(streams[k]) : nullptr));
        for (int k = 0; k < n_prob; ++k)
            rel_change_out[k] = h[2 * k + 1] > 0 ? std::sqrt(h[2 * k] / h[2 * k + 1]) : INFINITY;
    }
    return FHS_OK;
}

fhs_status fhs_estimate_bytes(const fhs_params *params, const double *w, int64_t n_vis, int64_t *resident_out,
                              int64_t *peak_out) {
    TRY(check_params(params));
    if (n_vis < 0) return fail(FHS_ERR_ARG, "n_vis must be >= 0");
    const fhs_params &q = *params;
    const long long L = q.n_channels, B = q.n_blocks, C = q.n_subcubes, Lc = L / C;
    const long long N = (long long)q.ny * q.nx, K = 4 * N, M = n_vis;
    long long n_fac = 0;
    for (long long i = 0; i < M; ++i) n_fac += 2LL * row_side(w ? w[i] : 0.0, q);
    const long long nseg = L * B, nchunk = M / 32 + nseg + 1, nbin = M / 32 + 2 * nseg + 1;
    const SaraConst c = sara_layout(q.ny, q.nx, q.wavelet_levels);
    long long nuc = 0;
    const std::vector<Facet> fac = facet_list(q);
    for (const Facet &f : fac) nuc += Lc * (long long)(f.y1 - f.y0) * (f.x1 - f.x0);
    nuc *= C;
    const long long Q = (long long)fac.size();
    long long r = 0;
    r += 8 * M + 8 * (M + 1) + 8 * n_fac + 8 * M * 4 + 4 * M;        // meta, factor offsets, G factors, y, d, scratch,
                                                                     // perm, row bounds
    r += 8 * (nseg + 1) + 8 * nseg + 8 * nseg + 4 * nseg;            // segments, norms, eps, scales
    // bins (first piece, channel, tile) and their pieces (start, length, block): a piece is a run of one
    // block inside one tile, or a sparse run, so there are at most bins + (segments x tiles) of them
    const long long ntiles = (long long)((2 * q.ny + kTile - 1) / kTile) * ((2 * q.nx + kTile - 1) / kTile);
    (void)ntiles;
    const long long npiece = nbin * std::min<long long>(B <= kBinMaxPieces ? B : 1, kBinMaxPieces);
    r += 16 * nbin + 16 * npiece + 8 * (nchunk + 1) + 4 * nchunk;
    r += 4 * (q.ny + q.nx);                                          // Z scaling
    const long long KH = (long long)(2 * q.ny) * (q.nx + 1);         // half-grid cells: K1 x HS
    r += 8 * KH * L * 3 + 4 * K * L * 3;                             // half grids, real grids
    r += 4 * N * L * 3 + 16 + 16 * L + 4 * L;                        // images, reductions, PSF factors
    r += 4 * c.n_coef * L * 2 + 4 * c.n_tmp * L + 4 * c.n_coef * C;  // SARA
    const long long ne = Lc + (Lc & 1);
    r += 16 * Q + 8 * C * Q + 4 * nuc + 12 * C * Q * Lc * Lc + 4 * C * Q * Lc + 4 * (q.ny + q.nx);
    r += 8 * C * Q * ne * ne;                                        // eigenvector warm starts
    r += (long long)cufft_workspace(2 * q.ny, 2 * q.nx, int(L));
    if (q.data_reduction) r += 36 * K * L + 20 * L;                  // Lambda, y', v', u, w; norms, eps', scales
    const long long n_planes = q.w_max > 0.0 ? 2LL * (q.n_wplanes - 1) + 1 : 1;
    // set-up temporaries: grid coordinates and w-planes (sorted), and the caller's omega, y and planes
    // while they are gathered
    const long long peak = r + (q.data_reduction ? 8 * K * L : 0) + (16 + 2 + 16 + 16 + 2) * M +
                           16 * n_planes * 2 * (2 * kMaxWHalf + 1) + 8 * nseg;
    if (resident_out) *resident_out = r;
    if (peak_out) *peak_out = peak;
    return FHS_OK;
}

fhs_status fhs_workspace_bytes(const fhs_params *params, const double *w, int64_t n_vis, int64_t *resident_out,
                               int64_t *peak_out) {
    return fhs_estimate_bytes(params, w, n_vis, resident_out, peak_out);
}

fhs_status fhs_get_image(fhs_problem *p, float *x_dev, void *stream) {
    return fhs_get_state(p, FHS_STATE_IMAGE, x_dev, stream);
}

fhs_status fhs_profile_enable(fhs_problem *p, int32_t on) {
    if (!p) return fail(FHS_ERR_ARG, "NULL problem");
    if (on) {
        for (auto &u : p->ev_used) { p->ev_pool.push_back(u.second.first); p->ev_pool.push_back(u.second.second); }
        p->ev_used.clear();
        for (double &v : p->prof_ms) v = 0.0;
        p->prof_iters = 0;
    }
    p->prof_on = on != 0;
    return FHS_OK;
}

fhs_status fhs_profile_read(fhs_problem *p, double *ms_out, int64_t *iters_out) {
    if (!p) return fail(FHS_ERR_ARG, "NULL problem");
    for (auto &u : p->ev_used) {
        CU(cudaEventSynchronize(u.second.second));
        float ms = 0.f;
        CU(cudaEventElapsedTime(&ms, u.second.first, u.second.second));
        p->prof_ms[u.first] += ms;
        p->ev_pool.push_back(u.second.first);
        p->ev_pool.push_back(u.second.second);
    }
    p->ev_used.clear();
    if (ms_out)
        for (int i = 0; i < FHS_N_PHASES; ++i) ms_out[i] = p->prof_ms[i];
    if (iters_out) *iters_out = p->prof_iters;
    return FHS_OK;
}

fhs_status fhs_kernel_launches(const fhs_problem *p, int64_t *count_out) {
    if (!p || !count_out) return fail(FHS_ERR_ARG, "NULL argument");
    *count_out = p->n_launch;
    return FHS_OK;
}

fhs_status fhs_device_status(fhs_problem *p, void *stream) {
    if (!p) return fail(FHS_ERR_ARG, "NULL problem");
    cudaStream_t s = S(stream);
    int h = 0;
    CU(cudaMemcpyAsync(&h, p->dev_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    return take_device_error(p, h, s);
}

fhs_status fhs_debug_unsatisfied_wait(fhs_problem *p, int32_t max_polls, void *stream) {
    if (!p) return fail(FHS_ERR_ARG, "NULL problem");
    if (max_polls < 1 || max_polls > (1 << 24)) return fail(FHS_ERR_ARG, "max_polls must be in [1, 2^24]");
    CU(launch_unsatisfied_wait(p, max_polls, S(stream)));
    return FHS_OK;
}

fhs_status fhs_get_info(const fhs_problem *p, fhs_info *info) {
    if (!p || !info) return fail(FHS_ERR_ARG, "NULL argument");
    info->n_vis = p->Mtot;
    info->nnz = p->nnz;
    info->n_coef = p->sara.n_coef;
    info->nuclear_size = p->nuc_size;
    info->device_bytes = (int64_t)p->bytes;
    info->n_facets = p->Q;
    info->iteration = p->iteration;
    info->tau = p->tau;
    info->sigma0 = p->sigma0;
    info->sigma1 = p->sigma1;
    info->sigma2 = p->sigma2;
    info->phi_norm2_max = p->phi_norm2_max;
    info->n_gfac = p->n_fac;
    info->bin_dense_min = p->bin_dense_min;
    info->bin_split = p->bin_split;
    info->mu = p->prm.mu;
    info->mu_bar = p->prm.mu_bar;
    long long nr = 0;
    for (long long m : p->dr_m) nr += m;
    info->n_red = nr;
    return FHS_OK;
}

fhs_status fhs_measure(fhs_problem *p, const float *x_dev, float *vis_dev, void *stream) {
    if (!p || !x_dev || !vis_dev) return fail(FHS_ERR_ARG, "NULL argument");
    cudaStream_t s = S(stream);
    TRY(forward_from_image(p, x_dev, p->vis_tmp, s));
    CU(launch_permute_to_caller(p, p->vis_tmp, reinterpret_cast<float2 *>(vis_dev), nullptr, s));
    return FHS_OK;
}

fhs_status fhs_adjoint(fhs_problem *p, const float *vis_dev, float *x_dev, void *stream) {
    if (!p || !x_dev || !vis_dev) return fail(FHS_ERR_ARG, "NULL argument");
    cudaStream_t s = S(stream);
    CU(launch_permute_from_caller(p, reinterpret_cast<const float2 *>(vis_dev), p->vis_tmp, s));
    TRY(adjoint_to_image(p, p->vis_tmp, x_dev, s));
    return FHS_OK;
}

fhs_status fhs_residual(fhs_problem *p, const float *x_dev, float *r_dev, void *stream) {
    if (!p || !r_dev) return fail(FHS_ERR_ARG, "NULL argument");
    cudaStream_t s = S(stream);
    if (p->dr) {
        // eta' Re Phi'^H (y' - Phi' x) = eta' Re Z^T F^H H Lambda (y' - Lambda H F Z x)
        float2 *u = nullptr;
        if (x_dev) {
            CU(launch_zpad(p, x_dev, p->grid_in, s));
            TRY(fft_forward(p, p->grid_in, p->grid_aux, s));
            CU(launch_normal(p, p->grid_aux, true, p->dr_u, s, false, false));
            u = p->dr_u;
        }
        CU(launch_dr_combine(p, u, 1.f, -1.f, p->dr_w, s));
        TRY(zero_half(p, p->grid_aux, s));
        CU(launch_normal(p, p->dr_w, false, p->grid_aux, s, false, true));
        TRY(fft_inverse(p, p->grid_aux, p->real_scr, s));
        CU(launch_crop(p, p->real_scr, r_dev, s));
        CU(launch_chan_scale(p, r_dev, p->eta, s));
        return FHS_OK;
    }
    if (x_dev) {
        TRY(forward_from_image(p, x_dev, p->vis_tmp, s));
        CU(launch_vis_residual(p, p->vis_tmp, p->vis_tmp, s));
    } else {
        CU(cudaMemcpyAsync(p->vis_tmp, p->y, sizeof(float2) * p->Mtot, cudaMemcpyDeviceToDevice, s));
    }
    TRY(adjoint_to_image(p, p->vis_tmp, r_dev, s));
    CU(launch_chan_scale(p, r_dev, p->eta, s));
    return FHS_OK;
}

fhs_status fhs_noise_from_model(fhs_problem *p, const float *x0_dev, int32_t apply, double *sigma_out,
                                double *eps_out, void *stream) {
    if (!p || !x0_dev) return fail(FHS_ERR_ARG, "NULL argument");
    cudaStream_t s = S(stream);
    const int n = p->dr ? p->L : p->n_seg;
    const size_t n_st = p->dr ? (size_t)p->L : 3 * (size_t)p->n_seg;
    double *st = nullptr;
    CU(cudaMallocAsync(reinterpret_cast<void **>(&st), sizeof(double) * n_st, s));
    std::vector<double> h(n_st), sig(n), eps(n);
    auto run = [&]() -> fhs_status {
        CU(cudaMemsetAsync(st, 0, sizeof(double) * n_st, s));
        if (p->dr) {
            CU(launch_zpad(p, x0_dev, p->grid_in, s));
            TRY(fft_forward(p, p->grid_in, p->grid_aux, s));
            CU(launch_normal(p, p->grid_aux, true, p->dr_u, s, false, false));
            CU(launch_dr_resid_norm(p, st, s));
        } else {
            TRY(forward_from_image(p, x0_dev, p->vis_tmp, s));
            CU(launch_seg_stats(p, p->vis_tmp, st, s));
        }
        CU(cudaMemcpyAsync(h.data(), st, sizeof(double) * n_st, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        return FHS_OK;
    };
    const fhs_status rs = run();
    cudaFreeAsync(st, s);
    if (rs != FHS_OK) return rs;
    TRY(device_error(p, s));
    for (int i = 0; i < n; ++i) {
        if (p->dr) {
            eps[i] = std::sqrt(h[i]);
            sig[i] = p->dr_m[i] > 0 ? eps[i] / std::sqrt(double(p->dr_m[i])) : 0.0;
        } else {
            const double m = double(p->seg_off[i + 1] - p->seg_off[i]);
            const double sr = h[3 * i], si = h[3 * i + 1], s2 = h[3 * i + 2];
            eps[i] = std::sqrt(s2);
            const double var = m > 1 ? (s2 - (sr * sr + si * si) / m) / (m - 1) : 0.0;
            sig[i] = p->sigma_l[i / p->B] * std::sqrt(std::max(var, 0.0));
        }
    }
    if (sigma_out) std::copy(sig.begin(), sig.end(), sigma_out);
    if (eps_out) std::copy(eps.begin(), eps.end(), eps_out);
    if (apply) {
        CU(cudaMemcpyAsync(p->dr ? p->dr_eps : p->eps, eps.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
        CU(cudaStreamSynchronize(s));
    }
    return FHS_OK;
}

// Adaptive noise estimation (Sec. 3.3 (ii)): PDFB iterations with the priors
// inactive, the l2 bounds re-estimated from the current iterate's residual
// (the Sec. 3.3 (i) estimator) until they hold.
fhs_status fhs_adaptive_noise(fhs_problem *p, const fhs_adaptive_params *ap, double *sigma_out, double *eps_out,
                              fhs_adaptive_result *res_out, void *stream) {
    if (!p || !ap) return fail(FHS_ERR_ARG, "NULL argument");
    if (ap->max_iter < 0 || ap->check_every < 1)
        return fail(FHS_ERR_ARG, "max_iter must be >= 0 and check_every >= 1");
    if (!(ap->settle_tol > 0.0)) return fail(FHS_ERR_ARG, "settle_tol must be > 0 (INFINITY: every check acts)");
    if (p->iteration != 0)
        return fail(FHS_ERR_STATE, "the adaptive phase starts the run: the problem has iterated already");
    cudaStream_t s = S(stream);
    const int n = p->dr ? p->L : p->n_seg;
    double *eps_dev = p->dr ? p->dr_eps : p->eps;
    // eps0: the bounds of unit-variance whitened noise (the default rule of the set-up)
    std::vector<double> eps0(n), cur(n), sig(n), rho(n), scale(n);
    for (int i = 0; i < n; ++i) {
        if (p->dr) {
            const double m = double(p->dr_m[i]);
            eps0[i] = m > 0 ? std::sqrt(m + 2.0 * std::sqrt(m)) : 0.0;
            scale[i] = 1.0;
        } else {
            const int l = i / p->B;
            const double Ml = double(p->seg_off[(l + 1) * p->B] - p->seg_off[l * p->B]);
            const double Mb = double(p->seg_off[i + 1] - p->seg_off[i]);
            eps0[i] = Ml > 0 ? std::sqrt((Ml + 2.0 * std::sqrt(Ml)) * Mb / Ml) : 0.0;
            scale[i] = 1.0 / p->sigma_l[l];
        }
    }
    CU(cudaMemcpyAsync(cur.data(), eps_dev, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    // the captured iteration holds the regularisation: capture it again on each side of the phase
    auto drop_graph = [&]() {
        if (p->gexec) {
            cudaGraphExecDestroy(p->gexec);
            p->gexec = nullptr;
        }
    };
    const double mu = p->prm.mu, mu_bar = p->prm.mu_bar;
    drop_graph();
    p->prm.mu = 0.0;
    p->prm.mu_bar = 0.0;
    int it = 0, n_chk = 0, n_up = 0, sat = 0;
    fhs_status st = FHS_OK;
    while (it < ap->max_iter) {
        const int k = std::min(ap->check_every, ap->max_iter - it);
        double rel = INFINITY;
        if ((st = fhs_pdfb_step(p, k, &rel, stream)) != FHS_OK) break;
        it += k;
        if (!(rel < ap->settle_tol)) continue;
        if ((st = fhs_noise_from_model(p, p->X, 0, sig.data(), rho.data(), stream)) != FHS_OK) break;
        ++n_chk;
        bool hold = true;
        for (int i = 0; i < n; ++i) hold = hold && rho[i] <= cur[i];
        if (hold) {
            sat = 1;
            break;
        }
        for (int i = 0; i < n; ++i) cur[i] = sig[i] * scale[i] * eps0[i];
        if (cudaMemcpyAsync(eps_dev, cur.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            st = fail(FHS_ERR_CUDA, "%s", cudaGetErrorString(cudaGetLastError()));
            break;
        }
        ++n_up;
    }
    cudaStreamSynchronize(s);
    drop_graph();
    p->prm.mu = mu;
    p->prm.mu_bar = mu_bar;
    if (st != FHS_OK) return st;
    if (sigma_out) TRY(fhs_noise_from_model(p, p->X, 0, sigma_out, nullptr, stream));
    if (eps_out) std::copy(cur.begin(), cur.end(), eps_out);
    if (res_out) {
        res_out->iterations = it;
        res_out->n_checks = n_chk;
        res_out->n_updates = n_up;
        res_out->satisfied = sat;
    }
    return FHS_OK;
}

fhs_status fhs_sara_analysis(fhs_problem *p, const float *x_dev, float *coef_dev, void *stream) {
    if (!p || !x_dev || !coef_dev) return fail(FHS_ERR_ARG, "NULL argument");
    CU(launch_sara_analysis(p, x_dev, coef_dev, S(stream)));
    return FHS_OK;
}

fhs_status fhs_sara_synthesis(fhs_problem *p, const float *coef_dev, float *x_dev, void *stream) {
    if (!p || !x_dev || !coef_dev) return fail(FHS_ERR_ARG, "NULL argument");
    CU(launch_sara_synthesis(p, coef_dev, x_dev, S(stream)));
    return FHS_OK;
}

fhs_status fhs_pdfb_step(fhs_problem *p, int32_t n_iter, double *rel_change_out, void *stream) {
    if (!p) return fail(FHS_ERR_ARG, "NULL problem");
    if (n_iter < 0) return fail(FHS_ERR_ARG, "n_iter must be >= 0");
    cudaStream_t s = S(stream);
    TRY(run_iterations(p, n_iter, s));
    if (rel_change_out) {
        // the relative change and the device error flag in one synchronisation: an iteration
        // whose bounded wait gave up must not be reported as a good one
        double h[2] = {0, 0};
        int herr = 0;
        CU(cudaMemcpyAsync(h, p->red, sizeof h, cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(&herr, p->dev_err, sizeof herr, cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
        TRY(take_device_error(p, herr, s));
        *rel_change_out = h[1] > 0 ? std::sqrt(h[0] / h[1]) : INFINITY;
    }
    return FHS_OK;
}

fhs_status fhs_reweight(fhs_problem *p, void *stream) {
    if (!p) return fail(FHS_ERR_ARG, "NULL problem");
    cudaStream_t s = S(stream);
    CU(launch_sara_analysis(p, p->X, p->coef_tmp, s));
    CU(launch_l21_reweight(p, s));
    CU(launch_nuclear_gram(p, p->X, false, true, s));
    CU(launch_nuclear_eig(p, true, s));
    return FHS_OK;
}

fhs_status fhs_solve(fhs_problem *p, int32_t max_iter, double rel_tol, int32_t n_reweight, int32_t check_every,
                     int32_t *iters_out, void *stream) {
    if (!p) return fail(FHS_ERR_ARG, "NULL problem");
    if (max_iter < 0 || n_reweight < 0) return fail(FHS_ERR_ARG, "max_iter and n_reweight must be >= 0");
    if (check_every <= 0) check_every = 10;
    const int per = max_iter / (n_reweight + 1);
    int done = 0;
    for (int r = 0; r <= n_reweight; ++r) {
        const int k = (r < n_reweight) ? per : max_iter - per * n_reweight;
        int it = 0;
        while (it < k) {
            const int n = std::min(check_every, k - it);
            double rel = 0;
            TRY(fhs_pdfb_step(p, n, &rel, stream));
            it += n;
            if (rel < rel_tol) break;
        }
        done += it;
        if (r < n_reweight) TRY(fhs_reweight(p, stream));
    }
    if (iters_out) *iters_out = done;
    return device_error(p, S(stream));     // synchronises; FHS_ERR_TIMEOUT if a device wait gave up
}

fhs_status fhs_state_size(const fhs_problem *p, int32_t part, int64_t *n) {
    if (!p || !n) return fail(FHS_ERR_ARG, "NULL argument");
    switch (part) {
        case FHS_STATE_IMAGE: *n = p->N * p->L; break;
        case FHS_STATE_DUAL_DATA: *n = p->dr ? 2 * p->K * p->L : 2 * p->Mtot; break;
        case FHS_STATE_DUAL_SARA: *n = p->sara.n_coef * p->L; break;
        case FHS_STATE_DUAL_NUCLEAR: *n = p->nuc_size; break;
        case FHS_STATE_WEIGHTS_SARA: *n = p->sara.n_coef * p->C; break;
        case FHS_STATE_WEIGHTS_NUC: *n = (int64_t)p->C * p->Q * p->Lc; break;
        default: return fail(FHS_ERR_ARG, "unknown state part %d", part);
    }
    return FHS_OK;
}

fhs_status fhs_get_state(fhs_problem *p, int32_t part, float *dst, void *stream) {
    int64_t n = 0;
    TRY(fhs_state_size(p, part, &n));
    if (!dst) return fail(FHS_ERR_ARG, "NULL destination");
    cudaStream_t s = S(stream);
    const size_t b = sizeof(float) * n;
    switch (part) {
        case FHS_STATE_IMAGE: CU(cudaMemcpyAsync(dst, p->X, b, cudaMemcpyDeviceToDevice, s)); break;
        case FHS_STATE_DUAL_DATA:
            if (p->dr) CU(cudaMemcpyAsync(dst, p->dr_v, b, cudaMemcpyDeviceToDevice, s));
            else CU(launch_permute_to_caller(p, p->dvis, reinterpret_cast<float2 *>(dst), p->blk_scale, s));
            break;
        case FHS_STATE_DUAL_SARA: CU(cudaMemcpyAsync(dst, p->W, b, cudaMemcpyDeviceToDevice, s)); break;
        case FHS_STATE_DUAL_NUCLEAR: CU(cudaMemcpyAsync(dst, p->P, b, cudaMemcpyDeviceToDevice, s)); break;
        case FHS_STATE_WEIGHTS_SARA: CU(cudaMemcpyAsync(dst, p->w21, b, cudaMemcpyDeviceToDevice, s)); break;
        case FHS_STATE_WEIGHTS_NUC: CU(cudaMemcpyAsync(dst, p->wnuc, b, cudaMemcpyDeviceToDevice, s)); break;
    }
    return FHS_OK;
}

fhs_status fhs_set_state(fhs_problem *p, int32_t part, const float *src, void *stream) {
    int64_t n = 0;
    TRY(fhs_state_size(p, part, &n));
    if (!src) return fail(FHS_ERR_ARG, "NULL source");
    cudaStream_t s = S(stream);
    const size_t b = sizeof(float) * n;
    switch (part) {
        case FHS_STATE_IMAGE: CU(cudaMemcpyAsync(p->X, src, b, cudaMemcpyDeviceToDevice, s)); break;
        case FHS_STATE_DUAL_DATA: {
            if (p->dr) {
                // the reduced dual and its adjoint grid F^H H Lambda v (what the next primal step reads)
                CU(cudaMemcpyAsync(p->dr_v, src, b, cudaMemcpyDeviceToDevice, s));
                CU(launch_dr_weight(p, s));
                TRY(zero_half(p, p->grid_work, s));
                CU(launch_normal(p, p->dr_w, false, p->grid_work, s, false, true));
                TRY(fft_inverse(p, p->grid_work, p->adj_real, s));
                CU(cudaStreamSynchronize(s));
                break;
            }
            CU(launch_permute_from_caller(p, reinterpret_cast<const float2 *>(src), p->dvis, s));
            std::vector<float> ones(p->n_seg, 1.0f);
            CU(cudaMemcpyAsync(p->blk_scale, ones.data(), sizeof(float) * p->n_seg, cudaMemcpyHostToDevice, s));
            TRY(adjoint_to_real(p, p->dvis, p->grid_work, p->adj_real, s));
            CU(cudaStreamSynchronize(s));
            break;
        }
        case FHS_STATE_DUAL_SARA:
            if (!sara_active(p))
                return fail(FHS_ERR_STATE, "SARA dual set while mu = 0: it would not enter the iteration");
            CU(cudaMemcpyAsync(p->W, src, b, cudaMemcpyDeviceToDevice, s));
            CU(launch_sara_synthesis(p, p->W, p->A_sara, s));
            break;
        case FHS_STATE_DUAL_NUCLEAR:
            if (!nuc_active(p))
                return fail(FHS_ERR_STATE, "nuclear dual set while mu_bar = 0: it would not enter the iteration");
            CU(cudaMemcpyAsync(p->P, src, b, cudaMemcpyDeviceToDevice, s));
            break;
        case FHS_STATE_WEIGHTS_SARA: CU(cudaMemcpyAsync(p->w21, src, b, cudaMemcpyDeviceToDevice, s)); break;
        case FHS_STATE_WEIGHTS_NUC: CU(cudaMemcpyAsync(p->wnuc, src, b, cudaMemcpyDeviceToDevice, s)); break;
    }
    return FHS_OK;
}

fhs_status fhs_autotune_bins(fhs_problem *p, void *stream, int32_t *dense_min_out, int32_t *split_out) {
    if (!p) return fail(FHS_ERR_ARG, "NULL problem");
    cudaStream_t s = S(stream);
    if (p->Mtot == 0 || p->n_bin == 0) {
        if (dense_min_out) *dense_min_out = p->bin_dense_min;
        if (split_out) *split_out = p->bin_split;
        return FHS_OK;
    }
    CU(cudaStreamSynchronize(s));
    std::vector<int2> meta(p->Mtot);
    std::vector<long long> fptr(p->Mtot + 1);
    CU(cudaMemcpyAsync(meta.data(), p->meta, sizeof(int2) * p->Mtot, cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(fptr.data(), p->fptr, sizeof(long long) * (p->Mtot + 1), cudaMemcpyDeviceToHost, s));
    // a forward grid of a random image (scratch: coef_tmp, grid_in, grid_aux); the
    // normal-mode pass accumulates into the first L block grids, zero again after
    const long long LN = (long long)p->L * p->N;
    std::vector<float> x0(LN);
    unsigned long long st = 0x2545F4914F6CDD1Dull;
    for (long long i = 0; i < LN; ++i) {
        st = st * 6364136223846793005ull + 1442695040888963407ull;
        x0[i] = float(double(st >> 11) * (1.0 / 9007199254740992.0) - 0.5);
    }
    TRY(upload(p->coef_tmp, x0.data(), LN, s));
    CU(launch_zpad(p, p->coef_tmp, p->grid_in, s));
    TRY(fft_forward(p, p->grid_in, p->grid_aux, s));

    const DevBins cur = current_bins(p);
    cudaStream_t home = p->home;
    p->home = s;                                       // candidate arrays live on this call's stream
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    fhs_status rs = FHS_OK;
    auto release = [&](const DevBins &b) {
        dev_free(p, b.fbase);
        dev_free(p, b.chan);
        dev_free(p, b.tile);
        dev_free(p, b.pstart);
        dev_free(p, b.plen);
        dev_free(p, b.pblk);
        p->bytes -= b.bytes;
    };
    auto time_bins = [&](const DevBins &b, float &ms) -> fhs_status {
        use_bins(p, b);
        CU(launch_normal(p, p->grid_aux, true, p->grid_scr, s, !p->dr, true));    // warm-up
        CU(cudaEventRecord(e0, s));
        for (int r = 0; r < 3; ++r) CU(launch_normal(p, p->grid_aux, true, p->grid_scr, s, !p->dr, true));
        CU(cudaEventRecord(e1, s));
        CU(cudaEventSynchronize(e1));
        CU(cudaEventElapsedTime(&ms, e0, e1));
        return FHS_OK;
    };
    DevBins best = cur;
    float best_ms = 0.f;
    auto run = [&]() -> fhs_status {
        CU(cudaEventCreate(&e0));
        CU(cudaEventCreate(&e1));
        TRY(time_bins(cur, best_ms));
        const long long dmins[] = {16, 32, 48, 96};
        const long long splits[] = {192, 288, kBinSplitMax};
        BinList bl;
        for (long long dm : dmins)
            for (long long sp : splits) {
                if (sp > kBinSplitMax) continue;
                make_bins(meta.data(), fptr.data(), p->seg_off, p->L, p->B, p->ntx, dm, sp, true, kBinSplitMax, bl);
                DevBins c;
                c.n_bin = bl.n_bin();
                const SlotBins sl = to_slots(bl);
                c.slots = sl.slots;
                c.dense_min = int(dm);
                c.split = int(sp);
                TRY(dev_alloc(p, &c.fbase, bl.fbase.size(), false));
                TRY(dev_alloc(p, &c.chan, bl.chan.size(), false));
                TRY(dev_alloc(p, &c.tile, bl.tile.size(), false));
                TRY(dev_alloc(p, &c.pstart, sl.pstart.size(), false));
                TRY(dev_alloc(p, &c.plen, sl.plen.size(), false));
                TRY(dev_alloc(p, &c.pblk, sl.pblk.size(), false));
                c.bytes = sizeof(int) * (bl.chan.size() + bl.tile.size() + sl.plen.size() + sl.pblk.size()) +
                          sizeof(long long) * (sl.pstart.size() + bl.fbase.size());
                TRY(upload(c.fbase, bl.fbase.data(), bl.fbase.size(), s));
                TRY(upload(c.chan, bl.chan.data(), bl.chan.size(), s));
                TRY(upload(c.tile, bl.tile.data(), bl.tile.size(), s));
                TRY(upload(c.pstart, sl.pstart.data(), sl.pstart.size(), s));
                TRY(upload(c.plen, sl.plen.data(), sl.plen.size(), s));
                TRY(upload(c.pblk, sl.pblk.data(), sl.pblk.size(), s));
                float ms = 0.f;
                TRY(time_bins(c, ms));
                DevBins loser = c;
                if (ms < 0.97f * best_ms) {            // keep a candidate only for a clear gain
                    loser = best;
                    best = c;
                    best_ms = ms;
                }
                if (loser.chan != cur.chan) release(loser);
            }
        return FHS_OK;
    };
    rs = run();
    if (rs != FHS_OK && best.chan != cur.chan) {        // a failed search keeps the original bins
        release(best);
        best = cur;
    }
    use_bins(p, best);
    if (best.chan != cur.chan) release(cur);
    p->home = home;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (p->gexec) {                                    // the captured iteration holds the old bins
        cudaGraphExecDestroy(p->gexec);
        p->gexec = nullptr;
    }
    TRY(zero_half(p, p->grid_scr, s));
    CU(cudaMemsetAsync(p->coef_tmp, 0, sizeof(float) * LN, s));
    CU(cudaStreamSynchronize(s));
    if (rs != FHS_OK) return rs;
    if (dense_min_out) *dense_min_out = p->bin_dense_min;
    if (split_out) *split_out = p->bin_split;
    return FHS_OK;
}

fhs_status fhs_operator_norms(fhs_problem *p, int32_t n_iter, double *norms, void *stream) {
    if (!p || !norms || n_iter < 1) return fail(FHS_ERR_ARG, "bad argument");
    cudaStream_t s = S(stream);
    // the work images are part of the iteration state: keep them
    const long long LN = p->N * p->L;
    float *save = nullptr;
    cudaStream_t home = p->home;
    p->home = s;                // the work buffer lives on this call's stream
    fhs_status ast = dev_alloc(p, &save, 2 * LN, false);
    p->home = home;
    TRY(ast);
    CU(cudaMemcpyAsync(save, p->Xbar, sizeof(float) * LN, cudaMemcpyDeviceToDevice, s));
    CU(cudaMemcpyAsync(save + LN, p->A_sara, sizeof(float) * LN, cudaMemcpyDeviceToDevice, s));
    std::vector<double> lam;
    fhs_status st = norm_estimate(p, n_iter, 0.0, lam, s);
    CU(cudaMemcpyAsync(p->Xbar, save, sizeof(float) * LN, cudaMemcpyDeviceToDevice, s));
    CU(cudaMemcpyAsync(p->A_sara, save + LN, sizeof(float) * LN, cudaMemcpyDeviceToDevice, s));
    CU(cudaStreamSynchronize(s));
    p->home = s;
    dev_free(p, save);
    p->home = home;
    p->bytes -= sizeof(float) * 2 * LN;
    if (st != FHS_OK) return st;
    std::copy(lam.begin(), lam.end(), norms);
    return FHS_OK;
}

}  // extern "C"
