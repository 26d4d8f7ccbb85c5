// Visibility-gridding data reduction (Sec. 3.4, Eqs. 4-5) on sm_103a.
//
// Per channel l, with the whitened rows of G (Theta_l G_l, 1/sigma_l folded
// into the first factor):
//   H_l      = (Theta_l G_l)^H (Theta_l G_l),  applied without being stored:
//              one normal-mode pass over G (gather then scatter of every row)
//   Lambda_l = 1 / sqrt(H_l[k][k]) on the grid cells some row reaches, else 0
//   y'_l     = Lambda_l (Theta_l G_l)^H y_l          (Eq. 4)
//   Phi'_l   = Lambda_l H_l F Z                       (Eq. 5)
// All blocks of a channel are gridded together: one l2 ball per channel.
// The reduced data, the reduced dual and Lambda live on the oversampled grid
// ([L][K], zero off the M'_l gridded points), so the dual update is a
// coalesced elementwise pass between the two passes over G.
#include "fhs_internal.h"

namespace fhs {

namespace {

constexpr int kWarps = 8;

// two complex cells as one float4, two Lambda values as one float2
inline float4 *f4(float2 *p) { return reinterpret_cast<float4 *>(p); }
inline const float2 *f2(const float *p) { return reinterpret_cast<const float2 *>(p); }

__device__ __forceinline__ int chan_of(const long long *seg_off, int n_seg, int B, long long v) {
    int lo = 0, hi = n_seg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (seg_off[mid] <= v) lo = mid; else hi = mid - 1;
    }
    return lo / B;
}

// diag[l][k] += |G_m[k]|^2 over the rows m of channel l: one warp per row,
// lanes over the T x T box; an entry is sum_r A_r[a] B_r[b] (R separable
// terms, R = 1 without DDE kernels), squared in FP64.
__global__ void __launch_bounds__(256) dr_diag_kernel(const int2 *__restrict__ meta, const long long *__restrict__ fptr,
                                                      const float2 *__restrict__ gfac,
                                                      const long long *__restrict__ seg_off, int n_seg, int B, int R,
                                                      long long Mtot, int K1, int K2, long long K,
                                                      double *__restrict__ diag) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (long long v = (long long)blockIdx.x * kWarps + warp; v < Mtot; v += (long long)gridDim.x * kWarps) {
        const int2 m = meta[v];
        const int T = m.y;
        const int c1 = m.x & 0xffff, c2 = (int)((unsigned)m.x >> 16);
        const float2 *f = gfac + fptr[v];
        double *dl = diag + (long long)chan_of(seg_off, n_seg, B, v) * K;
        for (int e = lane; e < T * T; e += 32) {
            const int a = e / T, b = e - a * T;
            double re = 0.0, im = 0.0;
            for (int r = 0; r < R; ++r) {
                const float2 x = f[r * 2 * T + a], y = f[r * 2 * T + T + b];
                re += double(x.x) * y.x - double(x.y) * y.y;
                im += double(x.x) * y.y + double(x.y) * y.x;
            }
            int k1 = c1 + a, k2 = c2 + b;
            k1 -= (k1 >= K1) ? K1 : 0;
            k2 -= (k2 >= K2) ? K2 : 0;
            atomicAdd(dl + (long long)k1 * K2 + k2, re * re + im * im);
        }
    }
}

// Lambda = 1/sqrt(diag) where diag > 0; y' = Lambda (G^H y) (ghy is zeroed
// after it is read); cnt[l] = M'_l.  blockIdx.y is the channel.
__global__ void dr_setup_kernel(const double *__restrict__ diag, float2 *__restrict__ ghy, float *__restrict__ lam,
                                float2 *__restrict__ yred, unsigned long long *__restrict__ cnt, long long K) {
    const int l = blockIdx.y;
    const long long base = (long long)l * K;
    unsigned long long n = 0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < K; k += (long long)gridDim.x * blockDim.x) {
        const double d = diag[base + k];
        const float2 g = ghy[base + k];
        ghy[base + k] = make_float2(0.f, 0.f);
        float lk = 0.f;
        float2 yk = make_float2(0.f, 0.f);
        if (d > 0.0) {
            const double il = 1.0 / sqrt(d);
            lk = float(il);
            yk = make_float2(float(il * g.x), float(il * g.y));
            ++n;
        }
        lam[base + k] = lk;
        yred[base + k] = yk;
    }
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if ((threadIdx.x & 31) == 0 && n) atomicAdd(cnt + l, n);
}

// The elementwise kernels below take two grid cells per thread and step
// (float4 of complex values, float2 of Lambda; K is even, so every channel's
// grid starts 16-byte aligned) and read every operand unconditionally: off
// the gridded points v', y' and Lambda are zero, so the formulas give zero
// there without a branch, and all loads of a step are independent.

// Reduced dual pre-update: r = v + sigma2 Lambda (H Xhat) - sigma2 y' (r
// replaces v), ||r||^2 per channel.  u (the normal-pass output) is zeroed by
// dr_apply_kernel: a store that does not wait for the load of the same line
// stalls the load/store queue behind that line's miss.
__global__ void __launch_bounds__(256) dr_dual_kernel(const float4 *__restrict__ u,
                                                      float4 *__restrict__ v, const float4 *__restrict__ yred,
                                                      const float2 *__restrict__ lam, float sigma2,
                                                      double *__restrict__ norm2, long long K2h) {
    __shared__ double s_red[8];
    const int l = blockIdx.y;
    const long long base = (long long)l * K2h;
    float acc = 0.f, cmp = 0.f;                     // compensated FP32 per thread, FP64 across threads
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < K2h; k += (long long)gridDim.x * blockDim.x) {
        const long long i = base + k;
        const float4 uu = u[i], vv = v[i], yy = yred[i];
        const float2 lk = lam[i];
        const float sa = sigma2 * lk.x, sb = sigma2 * lk.y;
        float4 r;
        r.x = fmaf(sa, uu.x, fmaf(-sigma2, yy.x, vv.x));
        r.y = fmaf(sa, uu.y, fmaf(-sigma2, yy.y, vv.y));
        r.z = fmaf(sb, uu.z, fmaf(-sigma2, yy.z, vv.z));
        r.w = fmaf(sb, uu.w, fmaf(-sigma2, yy.w, vv.w));
        v[i] = r;
        const float q = fmaf(r.x, r.x, fmaf(r.y, r.y, fmaf(r.z, r.z, r.w * r.w)));
        const float yv = q - cmp, t = acc + yv;
        cmp = (t - acc) - yv;
        acc = t;
    }
    double d = double(acc) - double(cmp);
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w];
        if (t != 0.0) atomicAdd(norm2 + l, t);
    }
}

// l2-ball factor per channel: scale = 1 - min(1, sigma2 eps' / ||r||); norm2 <- 0.
__global__ void dr_scale_kernel(double *norm2, const double *eps, float *scale, int L, double sigma2) {
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= L) return;
    const double nr = sqrt(norm2[l]);
    const double m = nr > 0.0 ? fmin(1.0, sigma2 * eps[l] / nr) : 1.0;
    scale[l] = float(1.0 - m);
    norm2[l] = 0.0;
}

// v = scale_l r; w = Lambda v (the input of the adjoint pass); scale NULL: 1.
// u (may be NULL) is zeroed.
__global__ void __launch_bounds__(256) dr_apply_kernel(float4 *__restrict__ v, const float2 *__restrict__ lam,
                                                       const float *__restrict__ scale, float4 *__restrict__ w,
                                                       float4 *__restrict__ u, long long K2h) {
    const int l = blockIdx.y;
    const long long base = (long long)l * K2h;
    const float sc = scale ? scale[l] : 1.f;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < K2h; k += (long long)gridDim.x * blockDim.x) {
        const long long i = base + k;
        float4 vv = v[i];
        const float2 lk = lam[i];
        vv.x *= sc;
        vv.y *= sc;
        vv.z *= sc;
        vv.w *= sc;
        if (scale) v[i] = vv;
        w[i] = make_float4(lk.x * vv.x, lk.x * vv.y, lk.y * vv.z, lk.y * vv.w);
        if (u) u[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

// w = Lambda (a y' + b Lambda u) (u may be NULL).
__global__ void __launch_bounds__(256) dr_combine_kernel(float4 *__restrict__ u, const float4 *__restrict__ yred,
                                                         const float2 *__restrict__ lam, float a, float b,
                                                         float4 *__restrict__ w, long long K2h) {
    const int l = blockIdx.y;
    const long long base = (long long)l * K2h;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < K2h; k += (long long)gridDim.x * blockDim.x) {
        const long long i = base + k;
        const float2 lk = lam[i];
        const float4 uu = u ? u[i] : z4;
        const float4 yy = a != 0.f ? yred[i] : z4;
        const float ba = b * lk.x, bb = b * lk.y;
        w[i] = make_float4(lk.x * fmaf(a, yy.x, ba * uu.x), lk.x * fmaf(a, yy.y, ba * uu.y),
                           lk.y * fmaf(a, yy.z, bb * uu.z), lk.y * fmaf(a, yy.w, bb * uu.w));
    }
}

// out[l] += sum |y' - Lambda u|^2 over the gridded points.
__global__ void __launch_bounds__(256) dr_resid_norm_kernel(float4 *__restrict__ u, const float4 *__restrict__ yred,
                                                            const float2 *__restrict__ lam, double *__restrict__ out,
                                                            long long K2h) {
    __shared__ double s_red[8];
    const int l = blockIdx.y;
    const long long base = (long long)l * K2h;
    double acc = 0.0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < K2h; k += (long long)gridDim.x * blockDim.x) {
        const long long i = base + k;
        const float4 uu = u[i], yy = yred[i];
        const float2 lk = lam[i];
        const double r0 = double(yy.x) - double(lk.x) * uu.x, r1 = double(yy.y) - double(lk.x) * uu.y;
        const double r2 = double(yy.z) - double(lk.y) * uu.z, r3 = double(yy.w) - double(lk.y) * uu.w;
        acc += r0 * r0 + r1 * r1 + r2 * r2 + r3 * r3;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_red[w];
        if (t != 0.0) atomicAdd(out + l, t);
    }
}

// Grid of the elementwise kernels: CTAs per channel for `n` items per
// channel, capped at whole waves (as many CTAs as the SMs hold at once for
// this kernel, split evenly over the channels; a partial extra wave would
// double the time of a bandwidth-bound pass).
template <typename Kern>
dim3 grid_cells(const fhs_problem *p, Kern kern, long long n) {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        sms = 152;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 256, 0) != cudaSuccess || occ < 1) occ = 1;
    const int L = p->L > 0 ? p->L : 1;
    long long per = (long long)sms * occ / L;
    if (per < 1) per = 1;
    long long g = (n + 255) / 256;
    if (g > per) g = per;
    if (g < 1) g = 1;
    return dim3(unsigned(g), unsigned(L));
}

}  // namespace

cudaError_t launch_dr_diag(fhs_problem *p, double *diag, cudaStream_t s) {
    if (p->Mtot == 0) return cudaSuccess;
    long long g = (p->Mtot + kWarps - 1) / kWarps;
    if (g > 152LL * 64) g = 152LL * 64;
    dr_diag_kernel<<<unsigned(g), 256, 0, s>>>(p->meta, p->fptr, p->gfac, p->d_seg_off, p->n_seg, p->B, p->rank,
                                              p->Mtot, p->K1, p->K2, p->K, diag);
    p->n_launch += 1;
    return cudaGetLastError();
}

cudaError_t launch_dr_setup(fhs_problem *p, const double *diag, float2 *ghy, unsigned long long *cnt,
                            cudaStream_t s) {
    dr_setup_kernel<<<grid_cells(p, dr_setup_kernel, p->K), 256, 0, s>>>(diag, ghy, p->dr_lam, p->dr_y, cnt, p->K);
    p->n_launch += 1;
    return cudaGetLastError();
}

cudaError_t launch_dr_dual(fhs_problem *p, cudaStream_t s) {
    dr_dual_kernel<<<grid_cells(p, dr_dual_kernel, p->K / 2), 256, 0, s>>>(
        f4(p->dr_u), f4(p->dr_v), f4(p->dr_y), f2(p->dr_lam), float(p->sigma2), p->dr_norm2, p->K / 2);
    p->n_launch += 1;
    return cudaGetLastError();
}

cudaError_t launch_dr_finalize(fhs_problem *p, cudaStream_t s) {
    dr_scale_kernel<<<(p->L + 127) / 128, 128, 0, s>>>(p->dr_norm2, p->dr_eps, p->dr_scale, p->L, p->sigma2);
    dr_apply_kernel<<<grid_cells(p, dr_apply_kernel, p->K / 2), 256, 0, s>>>(f4(p->dr_v), f2(p->dr_lam), p->dr_scale,
                                                                          f4(p->dr_w), f4(p->dr_u), p->K / 2);
    p->n_launch += 2;
    return cudaGetLastError();
}

cudaError_t launch_dr_weight(fhs_problem *p, cudaStream_t s) {
    dr_apply_kernel<<<grid_cells(p, dr_apply_kernel, p->K / 2), 256, 0, s>>>(f4(p->dr_v), f2(p->dr_lam), nullptr,
                                                                          f4(p->dr_w), nullptr, p->K / 2);
    p->n_launch += 1;
    return cudaGetLastError();
}

// The two launchers below zero u (when given) after the kernel with a memset:
// zeroing it inside the kernel, right after loading it, stalls the load/store
// queue (see dr_dual_kernel).
cudaError_t launch_dr_resid_norm(fhs_problem *p, double *out, cudaStream_t s) {
    dr_resid_norm_kernel<<<grid_cells(p, dr_resid_norm_kernel, p->K / 2), 256, 0, s>>>(f4(p->dr_u), f4(p->dr_y),
                                                                                    f2(p->dr_lam), out, p->K / 2);
    p->n_launch += 1;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemsetAsync(p->dr_u, 0, sizeof(float2) * p->K * p->L, s);
    return e;
}

cudaError_t launch_dr_combine(fhs_problem *p, float2 *u, float a, float b, float2 *w, cudaStream_t s) {
    dr_combine_kernel<<<grid_cells(p, dr_combine_kernel, p->K / 2), 256, 0, s>>>(f4(u), f4(p->dr_y), f2(p->dr_lam), a, b,
                                                                              f4(w), p->K / 2);
    p->n_launch += 1;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && u) e = cudaMemsetAsync(u, 0, sizeof(float2) * p->K * p->L, s);
    return e;
}

}  // namespace fhs
