// Measurement operator Phi_l = Theta_l G_l F Z (Sec. 2.1, Eq. 1) and the
// data-fidelity dual step of the l2 balls (Eq. 2) on sm_103a.
//
// G in factored box form: every row's support is a T x T box of the
// oversampled grid (KB taps convolved with the w-kernel of its plane,
// Sec. 3.2), and both the KB window and the small-field w-chirp separate over
// the two grid axes, so the row is the outer product g1 (x) g2 of two 1-D
// rows of T taps.  A row keeps its wrapped box corner, T and the 2T factor
// values (16 T bytes instead of 8 T^2 for the entries); the kernels form the
// T^2 products on the fly (the pass over G is in k_binned.cu).  This file
// builds G and holds the grid, reduction and Lanczos helpers around it.
#include "fhs_internal.h"

#include <cstdio>

namespace fhs {

namespace {

constexpr int kWarps = 8;               // warps per CTA for visibility kernels

// Terms of the I0 power series kept: q = (x/2)^2 <= (beta/2)^2 < 87 for
// J <= 8 at 2x oversampling, where the terms beyond k = 35 are below 1e-18 of
// the sum.
constexpr int kI0Terms = 40;
// Intervals of the tabulated KB window over [-J/2, J/2].
constexpr int kKbTab = 4096;

// KB window at offset t, phi(t) = I0(beta sqrt(1 - (2t/J)^2)) / I0(beta), 0
// outside [-J/2, J/2], by cubic Hermite interpolation of a table of its
// values and slopes (tab[n] = {phi(t_n), h phi'(t_n)}, t_n = -J/2 + n h,
// h = J / kKbTab; `scale` = 1 / h).  phi is a power series in t^2 (an entire
// function), so the interpolation error, of order h^4 phi'''' / 384, is about
// 1e-14 of the peak for J <= 8; the cubic runs in FP32 on FP32 nodes (about
// 1e-7 of the peak, the rounding of the stored factors), the position in FP64.
// GB300's FP64 pipe is narrow: this took the G build from a 40-term FP64
// series per tap to a few FP64 operations.
__device__ __forceinline__ double kb_table(double t, int J, const float4 *__restrict__ tab, double scale) {
    const double x = (t + 0.5 * J) * scale;
    if (!(x >= 0.0 && x <= double(kKbTab))) return 0.0;
    const int n = min(int(x), kKbTab - 1);
    // the position in FP64 (t reaches 4096 on the grid), the cubic in FP32: the nodes' values and
    // slopes are at most 1 and the factors are stored in FP32
    const float u = float(x - n), u2 = u * u, u3 = u2 * u;
    const float4 ab = tab[n];                    // {phi_n, h phi'_n, phi_n+1, h phi'_n+1}
    return double(fmaf(2.f * u3 - 3.f * u2 + 1.f, ab.x,
                       fmaf(u3 - 2.f * u2 + u, ab.y, fmaf(3.f * u2 - 2.f * u3, ab.z, (u3 - u2) * ab.w))));
}

__device__ __forceinline__ int seg_of(const long long *seg_off, int n_seg, long long v) {
    int lo = 0, hi = n_seg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (seg_off[mid] <= v) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// One warp per row: KB samples (J per axis, FP64), discrete convolution with
// the w-kernel of the row's plane, whitening; the row of G is the outer
// product g1 (x) g2 of the two 1-D factors, stored as T values of g1 (times
// 1/sigma) followed by T values of g2, in FP32.
//
// With DDE kernels (dde != NULL, ext = kDdeTaps - 1) the row is the 2-D
// convolution of that outer product (Tb = T - ext taps per axis) with the
// row's kDdeTaps x kDdeTaps DDE kernel D (Sec. 3.1).  Splitting the
// convolution over the first DDE axis makes it exact with kDdeTaps separable
// terms: G[a][b] = sum_r A_r[a] B_r[b], A_r[a] = g1[a - r],
// B_r[b] = sum_j D[r][j] g2[b - j] (out-of-range taps zero).  Term r is
// stored at offset 2 T r as T values of A_r followed by T values of B_r.
// gmax[v] bounds the row's entries for the fixed-point scatter: max |g1| max |g2|
// of a single-term row, sum_r max |A_r| max |B_r| of a DDE row.
__global__ void __launch_bounds__(256) build_g_kernel(
    const int2 *__restrict__ meta, const long long *__restrict__ fptr, float2 *__restrict__ gfac,
    const double2 *__restrict__ kap, const short *__restrict__ plane, const double2 *__restrict__ wk,
    const double2 *__restrict__ dde, int ext,
    const long long *__restrict__ seg_off, int n_seg, const double *__restrict__ inv_sigma_seg,
    long long Mtot, int J, const float4 *__restrict__ kbtab, double kbscale, float *__restrict__ gmax) {
    __shared__ double s_kb[kWarps][2][16];
    __shared__ double2 s_g[kWarps][2][16];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long stride = (long long)gridDim.x * kWarps;
    for (long long v = (long long)blockIdx.x * kWarps + warp; v < Mtot; v += stride) {
        const int T = meta[v].y;
        const int Tb = T - ext;
        const int h = (Tb - J) / 2;
        const int S = 2 * h + 1;
        const double2 kp = kap[v];
        const int dim = lane >> 4, i = lane & 15;
        const double kd = dim ? kp.y : kp.x;
        const long long p0 = (long long)floor(kd - 0.5 * J) + 1;
        if (i < J) s_kb[warp][dim][i] = kb_table(kd - double(p0 + i), J, kbtab, kbscale);
        __syncwarp();
        const int pl = plane[v];
        int sg = 0;                              // the row's segment (block), searched once per row
        if (lane == 0) sg = seg_of(seg_off, n_seg, v);
        sg = __shfl_sync(0xffffffffu, sg, 0);
        float gm = 0.f;                          // |factor value| as stored (FP32)
        if (i < Tb) {
            double2 acc = make_double2(0.0, 0.0);
            for (int jj = 0; jj < S; ++jj) {
                const int ti = i + jj - (S - 1);
                if (ti < 0 || ti >= J) continue;
                const double2 c = wk[(pl * 2 + dim) * (2 * kMaxWHalf + 1) + jj];
                const double k = s_kb[warp][dim][ti];
                acc.x += c.x * k;
                acc.y += c.y * k;
            }
            const double f = dim ? 1.0 : inv_sigma_seg[sg];
            acc.x *= f;
            acc.y *= f;
            if (dde) {
                s_g[warp][dim][i] = acc;
            } else {
                const float2 g = make_float2(float(acc.x), float(acc.y));
                gfac[fptr[v] + dim * T + i] = g;
                gm = sqrtf(fmaf(g.x, g.x, g.y * g.y));
            }
        }
        // bound of every entry of a single-term row: max |g1| max |g2| (lanes 0-15: g1, 16-31: g2)
        for (int o = 8; o > 0; o >>= 1) gm = fmaxf(gm, __shfl_xor_sync(0xffffffffu, gm, o));
        const float gm2 = __shfl_sync(0xffffffffu, gm, 16);
        if (lane == 0 && !dde) gmax[v] = gm * gm2;
        if (dde) {
            __syncwarp();
            const double2 *D = dde + v * (kDdeTaps * kDdeTaps);
            for (int e = lane; e < 2 * kDdeTaps * T; e += 32) {
                const int r = e / (2 * T), q = e - r * 2 * T;
                double2 val = make_double2(0.0, 0.0);
                if (q < T) {
                    const int a = q - r;
                    if (a >= 0 && a < Tb) val = s_g[warp][0][a];
                } else {
                    const int bq = q - T;
                    for (int j = 0; j < kDdeTaps; ++j) {
                        const int b = bq - j;
                        if (b < 0 || b >= Tb) continue;
                        const double2 d = D[r * kDdeTaps + j], g = s_g[warp][1][b];
                        val.x += d.x * g.x - d.y * g.y;
                        val.y += d.x * g.y + d.y * g.x;
                    }
                }
                gfac[fptr[v] + e] = make_float2(float(val.x), float(val.y));
            }
            // bound of every entry of the row: sum_r max |A_r| max |B_r| (lane r < kDdeTaps)
            __syncwarp();
            float bt = 0.f;
            if (lane < kDdeTaps) {
                const float2 *f = gfac + fptr[v] + lane * 2 * T;
                float ma = 0.f, mb = 0.f;
                for (int q = 0; q < T; ++q) {
                    ma = fmaxf(ma, sqrtf(fmaf(f[q].x, f[q].x, f[q].y * f[q].y)));
                    mb = fmaxf(mb, sqrtf(fmaf(f[T + q].x, f[T + q].x, f[T + q].y * f[T + q].y)));
                }
                bt = ma * mb;
            }
            for (int o = 4; o > 0; o >>= 1) bt += __shfl_xor_sync(0xffffffffu, bt, o);
            if (lane == 0) gmax[v] = bt;
        }
        __syncwarp();
    }
}

// l2-ball factor per block: m_b = min(1, sigma2 eps_b / ||d_b||), s_b = 1 - m_b.
__global__ void block_finalize_kernel(double *blk_norm2, const double *eps, float *blk_scale, int n_seg,
                                      double sigma2) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_seg) return;
    const double nr = sqrt(blk_norm2[s]);
    const double m = nr > 0.0 ? fmin(1.0, sigma2 * eps[s] / nr) : 1.0;
    blk_scale[s] = float(1.0 - m);
    blk_norm2[s] = 0.0;
}

// The sorted rows' data from the caller's order: kap[v] = omega[perm[v]] K / (2 pi) (grid
// coordinates), plane[v] = cplane[perm[v]], y[v] = y_caller[perm[v]] / sigma_l with l the channel
// of row v (vis_off[l] <= v < vis_off[l + 1]).
__global__ void gather_rows_kernel(const long long *__restrict__ perm, const double2 *__restrict__ omega,
                                   const double2 *__restrict__ ycall, const short *__restrict__ cplane,
                                   const long long *__restrict__ vis_off, int L, const double *__restrict__ sigma,
                                   long long Mtot, int K1, int K2, double2 *__restrict__ kap,
                                   short *__restrict__ plane, float2 *__restrict__ yw) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < Mtot;
         v += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = L - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (vis_off[mid] <= v) lo = mid; else hi = mid - 1;
        }
        const long long i = perm[v];
        const double2 om = omega[i], yy = ycall[i];
        kap[v] = make_double2(om.x * K1 / (2.0 * M_PI), om.y * K2 / (2.0 * M_PI));
        plane[v] = cplane[i];
        const double sg = sigma[lo];
        yw[v] = make_float2(float(yy.x / sg), float(yy.y / sg));
    }
}

// Z: grid[(n mod K)] = x_n s1(n1) s2(n2), a real grid (zero cells elsewhere are left as is).
__global__ void zpad_kernel(const float *__restrict__ x, float *__restrict__ grid, const float *__restrict__ s1,
                            const float *__restrict__ s2, int ny, int nx, int K1, int K2, long long K) {
    const int l = blockIdx.y;
    const long long N = (long long)ny * nx;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        const int i1 = int(p) / nx, i2 = int(p) - i1 * nx;      // 32-bit division: images hold < 2^31 pixels
        int k1 = i1 - ny / 2; k1 += (k1 < 0) ? K1 : 0;
        int k2 = i2 - nx / 2; k2 += (k2 < 0) ? K2 : 0;
        grid[(long long)l * K + (long long)k1 * K2 + k2] = x[(long long)l * N + p] * s1[i1] * s2[i2];
    }
}

// Z^T of a real grid (the C2R output, Re F^H g): x_n = grid[(n mod K)] s1(n1) s2(n2).
__global__ void crop_kernel(const float *__restrict__ grid, float *__restrict__ x, const float *__restrict__ s1,
                            const float *__restrict__ s2, int ny, int nx, int K1, int K2, long long K) {
    const int l = blockIdx.y;
    const long long N = (long long)ny * nx;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        const int i1 = int(p) / nx, i2 = int(p) - i1 * nx;      // 32-bit division: images hold < 2^31 pixels
        int k1 = i1 - ny / 2; k1 += (k1 < 0) ? K1 : 0;
        int k2 = i2 - nx / 2; k2 += (k2 < 0) ? K2 : 0;
        x[(long long)l * N + p] = grid[(long long)l * K + (long long)k1 * K2 + k2] * s1[i1] * s2[i2];
    }
}

__global__ void permute_to_caller_kernel(const float2 *__restrict__ sorted, float2 *__restrict__ caller,
                                         const long long *__restrict__ perm, const long long *__restrict__ chunk_start,
                                         const int *__restrict__ chunk_seg, const float *__restrict__ scale_seg) {
    const int ch = blockIdx.x;
    const float s = scale_seg ? scale_seg[chunk_seg[ch]] : 1.0f;
    for (long long v = chunk_start[ch] + threadIdx.x; v < chunk_start[ch + 1]; v += blockDim.x) {
        const float2 a = sorted[v];
        caller[perm[v]] = make_float2(a.x * s, a.y * s);
    }
}

__global__ void permute_from_caller_kernel(const float2 *__restrict__ caller, float2 *__restrict__ sorted,
                                           const long long *__restrict__ perm, long long M) {
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < M; v += (long long)gridDim.x * blockDim.x)
        sorted[v] = caller[perm[v]];
}

// Power iteration step on every channel: norms[2l] += <x_l, y_l>, norms[2l+1] += ||y_l||^2.
__global__ void __launch_bounds__(256) dots_kernel(const float *__restrict__ x, const float *__restrict__ y,
                                                   long long N, double *__restrict__ out) {
    __shared__ double s_a[8], s_b[8];
    const int l = blockIdx.y;
    double a = 0.0, b = 0.0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        const double xv = x[(long long)l * N + p], yv = y[(long long)l * N + p];
        a += xv * yv;
        b += yv * yv;
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if ((threadIdx.x & 31) == 0) { s_a[threadIdx.x >> 5] = a; s_b[threadIdx.x >> 5] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double sa = 0, sb = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { sa += s_a[w]; sb += s_b[w]; }
        atomicAdd(out + 2 * l, sa);
        atomicAdd(out + 2 * l + 1, sb);
    }
}

__global__ void scale_kernel(const float *__restrict__ y, float *__restrict__ x, long long N,
                             const double *__restrict__ norms) {
    const int l = blockIdx.y;
    const double nb = norms[2 * l + 1];
    const float f = nb > 0.0 ? float(1.0 / sqrt(nb)) : 0.f;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x)
        x[(long long)l * N + p] = y[(long long)l * N + p] * f;
}

// Lanczos three-term recurrence for the largest eigenvalue of
// A_l = Re(Phi_l^H Phi_l), every channel at once (blockIdx.y = channel):
//   w = A v_j - beta_j v_{j-1},  alpha_j = <w, v_j>,  w -= alpha_j v_j,
//   beta_{j+1} = ||w||,  v_{j+1} = w / beta_{j+1}.
// nb2 holds squared norms (beta^2); reductions are FP64.
__device__ __forceinline__ void block_add(double v, double *s_part, double *out) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_part[w];
        atomicAdd(out, t);
    }
}

// Lanczos vector steps, one channel per blockIdx.y, or channel chans[blockIdx.y] of a list.
__global__ void __launch_bounds__(256) lanczos_alpha_kernel(float *__restrict__ y, const float *__restrict__ vprev,
                                                            const float *__restrict__ v, long long N,
                                                            const double *__restrict__ nb2, double *__restrict__ alpha,
                                                            const int *__restrict__ chans) {
    __shared__ double s_part[8];
    const int l = chans ? chans[blockIdx.y] : blockIdx.y;
    const float beta = float(sqrt(nb2[l]));
    double a = 0.0;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x) {
        const long long o = (long long)l * N + q;
        const float w = fmaf(-beta, vprev[o], y[o]);
        y[o] = w;
        a += double(w) * double(v[o]);
    }
    block_add(a, s_part, alpha + l);
}

__global__ void __launch_bounds__(256) lanczos_beta_kernel(float *__restrict__ y, const float *__restrict__ v,
                                                           long long N, const double *__restrict__ alpha,
                                                           double *__restrict__ nb2_next, const int *__restrict__ chans) {
    __shared__ double s_part[8];
    const int l = chans ? chans[blockIdx.y] : blockIdx.y;
    const float a = float(alpha[l]);
    double b = 0.0;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x) {
        const long long o = (long long)l * N + q;
        const float w = fmaf(-a, v[o], y[o]);
        y[o] = w;
        b += double(w) * double(w);
    }
    block_add(b, s_part, nb2_next + l);
}

__global__ void lanczos_next_kernel(const float *__restrict__ y, float *__restrict__ vnext, long long N,
                                    const double *__restrict__ nb2_next, const int *__restrict__ chans) {
    const int l = chans ? chans[blockIdx.y] : blockIdx.y;
    const double nb = nb2_next[l];
    const float f = nb > 0.0 ? float(1.0 / sqrt(nb)) : 0.f;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x)
        vnext[(long long)l * N + q] = y[(long long)l * N + q] * f;
}

// r_m = y_m - phi_m over the sorted visibilities (phi may alias r).
__global__ void vis_residual_kernel(const float2 *__restrict__ y, const float2 *phi, float2 *r, long long M) {
    for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < M; m += (long long)gridDim.x * blockDim.x) {
        const float2 a = y[m], b = phi[m];
        r[m] = make_float2(a.x - b.x, a.y - b.y);
    }
}

// Residual statistics per (channel, block) segment of sorted visibilities:
// stats[3 s] += sum Re r, stats[3 s + 1] += sum Im r, stats[3 s + 2] += sum |r|^2
// with r = y - phi.  Each thread takes a contiguous run of kRun visibilities
// and flushes its FP64 sums whenever the segment changes.
constexpr int kRun = 64;
__global__ void seg_stats_kernel(const float2 *__restrict__ y, const float2 *__restrict__ phi,
                                 const long long *__restrict__ seg_off, int n_seg, long long M,
                                 double *__restrict__ stats) {
    const long long nrun = (M + kRun - 1) / kRun;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nrun;
         t += (long long)gridDim.x * blockDim.x) {
        const long long m0 = t * kRun, m1 = m0 + kRun < M ? m0 + kRun : M;
        int sg = seg_of(seg_off, n_seg, m0);
        double sr = 0.0, si = 0.0, s2 = 0.0;
        for (long long m = m0; m < m1; ++m) {
            while (m >= seg_off[sg + 1]) {
                if (s2 != 0.0 || sr != 0.0 || si != 0.0) {
                    atomicAdd(stats + 3 * sg, sr);
                    atomicAdd(stats + 3 * sg + 1, si);
                    atomicAdd(stats + 3 * sg + 2, s2);
                }
                sr = si = s2 = 0.0;
                ++sg;
            }
            const float2 a = y[m], b = phi[m];
            const double rr = double(a.x) - b.x, ri = double(a.y) - b.y;
            sr += rr;
            si += ri;
            s2 += rr * rr + ri * ri;
        }
        if (s2 != 0.0 || sr != 0.0 || si != 0.0) {
            atomicAdd(stats + 3 * sg, sr);
            atomicAdd(stats + 3 * sg + 1, si);
            atomicAdd(stats + 3 * sg + 2, s2);
        }
    }
}

// x_l *= f_l on every pixel of channel l (blockIdx.y = channel).
__global__ void chan_scale_kernel(float *__restrict__ x, long long N, const float *__restrict__ f) {
    const int l = blockIdx.y;
    const float a = f[l];
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x)
        x[(long long)l * N + q] *= a;
}

inline int grid_for(long long n, int threads, int cap = 152 * 16) {
    long long g = (n + threads - 1) / threads;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return int(g);
}

}  // namespace

cudaError_t launch_build_g(fhs_problem *p, const double2 *kap, const short *plane, const double2 *wk_table,
                           const double2 *dde, int ext, const double *inv_sigma_seg, cudaStream_t s) {
    // the KB table: phi and h phi' at kKbTab + 1 nodes, by the I0 series (in q = (beta/2)^2 (1 - (2t/J)^2),
    // dq/dt = -2 beta^2 t / J^2), normalised by I0(beta)
    const int J = p->J;
    const double beta = kb_beta(J, 2.0), inv_i0b = 1.0 / bessel_i0(beta), h = double(J) / kKbTab;
    std::vector<double2> tab(kKbTab + 1);
    for (int n = 0; n <= kKbTab; ++n) {
        const double t = -0.5 * J + n * h, r = 1.0 - (2.0 * t / J) * (2.0 * t / J);
        const double q = 0.25 * beta * beta * (r > 0.0 ? r : 0.0);
        double f = 0.0, df = 0.0, ck = 1.0, qk = 1.0;          // sum c_k q^k, sum k c_k q^(k-1)
        for (int k = 0; k < kI0Terms; ++k) {
            if (k) ck /= double(k) * double(k);
            if (k) df += k * ck * qk;                           // qk = q^(k-1) here
            f += ck * (k ? qk * q : 1.0);
            if (k) qk *= q;
        }
        tab[n] = make_double2(f * inv_i0b, df * (-2.0 * beta * beta * t / (double(J) * J)) * h * inv_i0b);
    }
    // interval n as one 16-byte entry: both nodes' values and slopes, in FP32
    std::vector<float4> tab4(kKbTab);
    for (int n = 0; n < kKbTab; ++n)
        tab4[n] = make_float4(float(tab[n].x), float(tab[n].y), float(tab[n + 1].x), float(tab[n + 1].y));
    float4 *d_tab = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&d_tab), sizeof(float4) * tab4.size(), s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(d_tab, tab4.data(), sizeof(float4) * tab4.size(), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        build_g_kernel<<<grid_for(p->Mtot, kWarps, 152 * 64), 256, 0, s>>>(
            p->meta, p->fptr, p->gfac, kap, plane, wk_table, dde, ext, p->d_seg_off, p->n_seg, inv_sigma_seg,
            p->Mtot, J, d_tab, 1.0 / h, p->gmax);
        p->n_launch += 1;
        e = cudaGetLastError();
    }
    // the copy's host source must outlive it: wait before tab goes out of scope
    const cudaError_t e2 = cudaStreamSynchronize(s);
    cudaFreeAsync(d_tab, s);
    return e != cudaSuccess ? e : e2;
}

cudaError_t launch_gather_rows(fhs_problem *p, const double2 *omega, const double2 *ycall, const short *cplane,
                               const long long *vis_off, const double *sigma, double2 *kap, short *plane,
                               cudaStream_t s) {
    if (p->Mtot == 0) return cudaSuccess;
    gather_rows_kernel<<<grid_for(p->Mtot, 256, 152 * 32), 256, 0, s>>>(p->perm, omega, ycall, cplane, vis_off, p->L,
                                                                        sigma, p->Mtot, p->K1, p->K2, kap, plane,
                                                                        p->y);
    p->n_launch += 1;
    return cudaGetLastError();
}

cudaError_t launch_zpad(fhs_problem *p, const float *x, float *grid, cudaStream_t s) {
    dim3 g(grid_for(p->N, 256, 512), p->L);
    zpad_kernel<<<g, 256, 0, s>>>(x, grid, p->s1, p->s2, p->ny, p->nx, p->K1, p->K2, p->K);
    p->n_launch += 1;
    return cudaGetLastError();
}

cudaError_t launch_zpad_channel(fhs_problem *p, const float *x, float *grid, int l, cudaStream_t s) {
    zpad_kernel<<<dim3(grid_for(p->N, 256, 512), 1), 256, 0, s>>>(x + (long long)l * p->N, grid + (long long)l * p->K,
                                                                   p->s1, p->s2, p->ny, p->nx, p->K1, p->K2, p->K);
    p->n_launch += 1;
    return cudaGetLastError();
}

cudaError_t launch_crop_channel(fhs_problem *p, const float *grid, float *x, int l, cudaStream_t s) {
    crop_kernel<<<dim3(grid_for(p->N, 256, 512), 1), 256, 0, s>>>(grid + (long long)l * p->K, x + (long long)l * p->N,
                                                                   p->s1, p->s2, p->ny, p->nx, p->K1, p->K2, p->K);
    p->n_launch += 1;
    return cudaGetLastError();
}

cudaError_t launch_crop(fhs_problem *p, const float *grid, float *x, cudaStream_t s) {
    dim3 g(grid_for(p->N, 256, 512), p->L);
    crop_kernel<<<g, 256, 0, s>>>(grid, x, p->s1, p->s2, p->ny, p->nx, p->K1, p->K2, p->K);
    p->n_launch += 1;
    return cudaGetLastError();
}

cudaError_t launch_block_finalize(fhs_problem *p, cudaStream_t s) {
    block_finalize_kernel<<<(p->n_seg + 127) / 128, 128, 0, s>>>(p->blk_norm2, p->eps, p->blk_scale, p->n_seg,
                                                                 p->sigma2);
    p->n_launch += 1;
    return cudaGetLastError();
}

cudaError_t launch_permute_to_caller(fhs_problem *p, const float2 *sorted, float2 *caller, const float *scale_seg,
                                     cudaStream_t s) {
    if (p->n_chunk == 0) return cudaSuccess;
    permute_to_caller_kernel<<<p->n_chunk, 256, 0, s>>>(sorted, caller, p->perm, p->chunk_start, p->chunk_seg,
                                                        scale_seg);
    p->n_launch += 1;
    return cudaGetLastError();
}

cudaError_t launch_permute_from_caller(fhs_problem *p, const float2 *caller, float2 *sorted, cudaStream_t s) {
    if (p->Mtot == 0) return cudaSuccess;
    permute_from_caller_kernel<<<grid_for(p->Mtot, 256), 256, 0, s>>>(caller, sorted, p->perm, p->Mtot);
    p->n_launch += 1;
    return cudaGetLastError();
}

cudaError_t launch_power_dots(fhs_problem *p, const float *x, const float *y, double *out, cudaStream_t s) {
    dim3 g(grid_for(p->N, 256, 256), p->L);
    dots_kernel<<<g, 256, 0, s>>>(x, y, p->N, out);
    p->n_launch += 1;
    return cudaGetLastError();
}

cudaError_t launch_power_scale(fhs_problem *p, const float *y, float *x, const double *norms, cudaStream_t s) {
    dim3 g(grid_for(p->N, 256, 512), p->L);
    scale_kernel<<<g, 256, 0, s>>>(y, x, p->N, norms);
    p->n_launch += 1;
    return cudaGetLastError();
}

cudaError_t launch_vis_residual(fhs_problem *p, const float2 *phi, float2 *r, cudaStream_t s) {
    if (p->Mtot == 0) return cudaSuccess;
    vis_residual_kernel<<<grid_for(p->Mtot, 256), 256, 0, s>>>(p->y, phi, r, p->Mtot);
    p->n_launch += 1;
    return cudaGetLastError();
}

cudaError_t launch_seg_stats(fhs_problem *p, const float2 *phi, double *stats, cudaStream_t s) {
    if (p->Mtot == 0) return cudaSuccess;
    seg_stats_kernel<<<grid_for((p->Mtot + kRun - 1) / kRun, 256), 256, 0, s>>>(p->y, phi, p->d_seg_off, p->n_seg,
                                                                               p->Mtot, stats);
    p->n_launch += 1;
    return cudaGetLastError();
}

cudaError_t launch_chan_scale(fhs_problem *p, float *x, const float *f, cudaStream_t s) {
    dim3 g(grid_for(p->N, 256, 512), p->L);
    chan_scale_kernel<<<g, 256, 0, s>>>(x, p->N, f);
    p->n_launch += 1;
    return cudaGetLastError();
}

cudaError_t launch_lanczos_step(fhs_problem *p, float *y, float *vprev, const float *v, double *alpha_j,
                                double *nb2_j, cudaStream_t s, const int *chans, int nch) {
    dim3 g(grid_for(p->N, 256, 256), chans ? nch : p->L);
    if (g.y == 0) return cudaSuccess;
    lanczos_alpha_kernel<<<g, 256, 0, s>>>(y, vprev, v, p->N, nb2_j, alpha_j, chans);
    lanczos_beta_kernel<<<g, 256, 0, s>>>(y, v, p->N, alpha_j, nb2_j + p->L, chans);
    lanczos_next_kernel<<<g, 256, 0, s>>>(y, vprev, p->N, nb2_j + p->L, chans);
    p->n_launch += 3;
    return cudaGetLastError();
}

}  // namespace fhs
