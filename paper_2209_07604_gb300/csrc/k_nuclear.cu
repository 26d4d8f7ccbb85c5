// Faceted low-rankness prior (Sec. 2.2.2): weighted nuclear-norm dual step of
// every spatio-spectral facet through its L_c x L_c Gram matrix.
//
//   Z_q = P_q + sigma0 S_q xbar               (facet pixels x L_c channels)
//   G_q = Z_q^T Z_q = V diag(s^2) V^T          (FP32 products, FP64 sums; FP64 Jacobi)
//   P_q <- Z_q - SVT(Z_q, mu_bar w) = Z_q V diag(min(1, mu_bar w_i / s_i)) V^T
//
// The Gram contraction reads L_c floats per pixel and does L_c(L_c+1)/2 FMAs
// with them: L_c/2 flop per byte, far below the tensor-core ridge, so it runs
// on the FP32 pipes and is bounded by HBM bandwidth.
#include "fhs_internal.h"

namespace fhs {

namespace {

constexpr int kPix = 2048;          // facet pixels per CTA in the apply kernels and the 32-channel Gram
// Facet pixels per CTA of the register-triangle Gram (L_c <= 16): 32 per thread, so that the
// reduction of the triangle across the CTA (warp shuffles and FP64 atomics) is amortised over
// enough pixels.
constexpr int kGramPix = 8192;

// AccT = float in the iteration (FP32 products, FP64 across threads: small
// singular values are not needed accurately there, they pass the SVT
// unchanged); AccT = double for the reweighting Gram of x, whose weights
// upsilon_bar / (upsilon_bar + s_i) need the small singular values too.
template <int MAXLC, typename AccT>
__global__ void __launch_bounds__(256) gram_kernel(const float *__restrict__ P, const float *__restrict__ img,
                                                   const int4 *__restrict__ facets, const long long *__restrict__ nuc_off,
                                                   int Q, int C, int Lc, int nx, long long N, float s, bool with_dual,
                                                   double *__restrict__ gram) {
    constexpr int NP = MAXLC * (MAXLC + 1) / 2;
    __shared__ double s_red[NP];
    const int cq = blockIdx.y;
    const int c = cq / Q, q = cq - c * Q;
    const int4 f = facets[q];
    const int wy = f.y - f.x, wx = f.w - f.z;
    const long long npix = (long long)wy * wx;
    const long long p0 = (long long)blockIdx.x * kGramPix;
    if (p0 >= npix) return;
    const long long p1 = min(npix, p0 + kGramPix);
    const float *Pq = P + nuc_off[cq];
    AccT acc[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] = AccT(0);
    for (long long pp = p0 + threadIdx.x; pp < p1; pp += blockDim.x) {
        const int py = int(pp) / wx, px = int(pp) - py * wx;     // 32-bit division: facets hold < 2^31 pixels
        const long long o = (long long)(f.x + py) * nx + (f.z + px);
        AccT z[MAXLC];
#pragma unroll
        for (int j = 0; j < MAXLC; ++j) {
            z[j] = AccT(0);
            if (j < Lc) {
                const float xv = img[(long long)(c + j * C) * N + o];
                z[j] = with_dual ? fmaf(s, xv, Pq[(long long)j * npix + pp]) : xv;
            }
        }
        int k = 0;
#pragma unroll
        for (int i = 0; i < MAXLC; ++i)
#pragma unroll
            for (int j = i; j < MAXLC; ++j, ++k) acc[k] = fma(z[i], z[j], acc[k]);
    }
    for (int k = threadIdx.x; k < NP; k += blockDim.x) s_red[k] = 0.0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        AccT v = acc[k];            // warp sum in the accumulation type, FP64 across warps
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&s_red[k], double(v));
    }
    __syncthreads();
    int k = 0;
    double *G = gram + (long long)cq * Lc * Lc;
    for (int i = 0; i < MAXLC; ++i)
        for (int j = i; j < MAXLC; ++j, ++k)
            if (threadIdx.x == (k & 255) && i < Lc && j < Lc) atomicAdd(&G[i * Lc + j], s_red[k]);
}

// L_c in (16, 32]: the per-thread triangle no longer fits in registers.  The
// CTA stages kSub pixels x L_c channels of Z in shared memory (loads coalesced
// along pixels); every lane of a warp then accumulates a 4 x 8 block of the
// 32 x 32 Gram over the warp's pixels.
constexpr int kSub = 128;

template <typename AccT>
__global__ void __launch_bounds__(256) gram32_kernel(const float *__restrict__ P, const float *__restrict__ img,
                                                     const int4 *__restrict__ facets,
                                                     const long long *__restrict__ nuc_off, int Q, int C, int Lc,
                                                     int nx, long long N, float s, bool with_dual,
                                                     double *__restrict__ gram) {
    __shared__ float s_z[32][kSub + 1];
    __shared__ double s_red[32 * 32];
    __shared__ long long s_o[kSub];           // image offset of each pixel of the sub-chunk
    const int cq = blockIdx.y;
    const int c = cq / Q, q = cq - c * Q;
    const int4 f = facets[q];
    const int wx = f.w - f.z;
    const long long npix = (long long)(f.y - f.x) * wx;
    const long long p0 = (long long)blockIdx.x * kPix;
    if (p0 >= npix) return;
    const long long p1 = min(npix, p0 + kPix);
    const float *Pq = P + nuc_off[cq];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) s_red[e] = 0.0;
    // lane (bi, bj) = (lane / 4, lane % 4) accumulates rows 4 bi .. 4 bi + 3 and columns
    // 8 bj .. 8 bj + 7 of the Gram: 12 shared loads (conflict-free: the row stride kSub + 1
    // puts channel j of pixel t in bank (j + t) % 32) for 32 products per pixel
    const int bi = lane >> 2, bj = lane & 3;
    AccT acc[4][8];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[r][q] = AccT(0);
    for (long long sb = p0; sb < p1; sb += kSub) {
        const int nsub = int(min((long long)kSub, p1 - sb));
        __syncthreads();                         // the previous sub-chunk is consumed
        if (threadIdx.x < kSub) {
            const long long pp = sb + threadIdx.x;
            const int py = int(pp) / wx, px = int(pp) - py * wx;     // 32-bit division: facets hold < 2^31 pixels
            s_o[threadIdx.x] = (long long)(f.x + py) * nx + (f.z + px);
        }
        __syncthreads();
        for (int e = threadIdx.x; e < 32 * kSub; e += blockDim.x) {
            const int j = e / kSub, t = e - j * kSub;
            float v = 0.f;
            if (j < Lc && t < nsub) {
                const float xv = img[(long long)(c + j * C) * N + s_o[t]];
                v = with_dual ? fmaf(s, xv, Pq[(long long)j * npix + sb + t]) : xv;
            }
            s_z[j][t] = v;
        }
        __syncthreads();
        for (int t = warp; t < nsub; t += blockDim.x >> 5) {
            AccT zr[4], zc[8];
#pragma unroll
            for (int r = 0; r < 4; ++r) zr[r] = AccT(s_z[4 * bi + r][t]);
#pragma unroll
            for (int q = 0; q < 8; ++q) zc[q] = AccT(s_z[8 * bj + q][t]);
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[r][q] = fma(zr[r], zc[q], acc[r][q]);
        }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 8; ++q) atomicAdd(&s_red[(4 * bi + r) * 32 + 8 * bj + q], double(acc[r][q]));
    __syncthreads();
    double *G = gram + (long long)cq * Lc * Lc;
    for (int e = threadIdx.x; e < Lc * Lc; e += blockDim.x) {
        const int i = e / Lc, j = e - i * Lc;
        if (j >= i) atomicAdd(&G[e], s_red[i * 32 + j]);
    }
}

// Symmetric eigen-decomposition of one L_c x L_c Gram per warp: cyclic Jacobi
// in FP64 with a round-robin ordering, so each round applies L_c/2 disjoint
// rotations at once (columns first, then rows: disjoint Givens rotations
// commute).  Bounded sweeps.  Then either the SVT mixing matrix
// M = V diag(min(1, mu_bar w_i / s_i)) V^T or the reweighting weights.
// Four warps (four matrices of at most 16 x 16) per CTA; larger matrices go
// to eig32_kernel.
// eigv (n x n per matrix, n = L_c rounded up to even), when not NULL, holds
// the eigenvectors found at the previous call and receives the new ones: the
// sweeps start from V0^T G V0, which is nearly diagonal when the facet changes
// little between iterations, so far fewer sweeps reach the same tolerance.
template <int NMAX>
__global__ void __launch_bounds__(NMAX == 16 ? 128 : 32) eig_kernel(double *__restrict__ gram,
                                                                    float *__restrict__ mix,
                                                                    float *__restrict__ wnuc, int n_mat, int Lc,
                                                                    double mu_bar, double upsilon_bar,
                                                                    bool reweight, double *__restrict__ eigv,
                                                                    double *__restrict__ svals) {
    constexpr int kEigWarps = NMAX == 16 ? 4 : 1;
    __shared__ double s_a[kEigWarps][NMAX][NMAX + 1];
    __shared__ double s_v[kEigWarps][NMAX][NMAX + 1];
    __shared__ double s_t[kEigWarps][NMAX][NMAX + 1];
    __shared__ double s_cs[kEigWarps][NMAX / 2], s_sn[kEigWarps][NMAX / 2];
    __shared__ int s_p[kEigWarps][NMAX / 2], s_q[kEigWarps][NMAX / 2];
    __shared__ int s_ord[kEigWarps][NMAX];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cq = blockIdx.x * kEigWarps + w;
    if (cq >= n_mat) return;
    double(*a)[NMAX + 1] = s_a[w];
    double(*V)[NMAX + 1] = s_v[w];
    double *G = gram + (long long)cq * Lc * Lc;
    const int n = Lc + (Lc & 1);                 // even size: a padded row/column stays zero
    for (int e = lane; e < n * n; e += 32) {
        const int i = e / n, j = e - (e / n) * n;
        double v = 0.0;
        if (i < Lc && j < Lc) v = (j >= i) ? G[i * Lc + j] : G[j * Lc + i];
        a[i][j] = v;
        V[i][j] = (i == j) ? 1.0 : 0.0;
    }
    __syncwarp();
    for (int e = lane; e < Lc * Lc; e += 32) G[e] = 0.0;   // ready for the next accumulation
    double *Vg = eigv ? eigv + (long long)cq * n * n : nullptr;
    if (Vg) {
        // T = A V0, then A = V0^T T; V = V0
        double(*T)[NMAX + 1] = s_t[w];
        for (int e = lane; e < n * n; e += 32) V[e / n][e % n] = Vg[e];
        __syncwarp();
        for (int e = lane; e < n * n; e += 32) {
            const int i = e / n, j = e - (e / n) * n;
            double t = 0.0;
            for (int k = 0; k < n; ++k) t = fma(a[i][k], V[k][j], t);
            T[i][j] = t;
        }
        __syncwarp();
        for (int e = lane; e < n * n; e += 32) {
            const int i = e / n, j = e - (e / n) * n;
            double t = 0.0;
            for (int k = 0; k < n; ++k) t = fma(V[k][i], T[k][j], t);
            a[i][j] = t;
        }
        __syncwarp();
    }
    const int half = n / 2;
    for (int sweep = 0; sweep < 40; ++sweep) {
        double off = 0.0, dia = 0.0;
        for (int e = lane; e < n * n; e += 32) {
            const int i = e / n, j = e - (e / n) * n;
            const double x = a[i][j];
            if (i == j) dia += x * x; else off += x * x;
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            dia += __shfl_xor_sync(0xffffffffu, dia, o);
        }
        if (off <= 1e-28 * dia || off == 0.0) break;
        for (int round = 0; round < n - 1; ++round) {
            // round-robin pairing: position 0 fixed, the others rotate
            if (lane < half) {
                const int k = lane;
                int pa = (k == 0) ? 0 : 1 + (k - 1 + round) % (n - 1);
                int pb = 1 + (n - 2 - k + round) % (n - 1);
                const int p = min(pa, pb), q = max(pa, pb);
                const double apq = a[p][q];
                double cs = 1.0, sn = 0.0;
                if (apq != 0.0) {
                    const double theta = (a[q][q] - a[p][p]) / (2.0 * apq);
                    const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                    cs = 1.0 / sqrt(t * t + 1.0);
                    sn = t * cs;
                }
                s_p[w][k] = p;
                s_q[w][k] = q;
                s_cs[w][k] = cs;
                s_sn[w][k] = sn;
            }
            __syncwarp();
            // columns: A <- A J, V <- V J
            for (int e = lane; e < half * n; e += 32) {
                const int k = e / n, r = e - k * n;
                const int p = s_p[w][k], q = s_q[w][k];
                const double cs = s_cs[w][k], sn = s_sn[w][k];
                const double arp = a[r][p], arq = a[r][q];
                a[r][p] = cs * arp - sn * arq;
                a[r][q] = sn * arp + cs * arq;
                const double vrp = V[r][p], vrq = V[r][q];
                V[r][p] = cs * vrp - sn * vrq;
                V[r][q] = sn * vrp + cs * vrq;
            }
            __syncwarp();
            // rows: A <- J^T A
            for (int e = lane; e < half * n; e += 32) {
                const int k = e / n, c = e - k * n;
                const int p = s_p[w][k], q = s_q[w][k];
                const double cs = s_cs[w][k], sn = s_sn[w][k];
                const double apc = a[p][c], aqc = a[q][c];
                a[p][c] = cs * apc - sn * aqc;
                a[q][c] = sn * apc + cs * aqc;
            }
            __syncwarp();
        }
    }
    if (Vg)
        for (int e = lane; e < n * n; e += 32) Vg[e] = V[e / n][e % n];
    if (lane == 0) {                          // eigenvalues descending (padding excluded)
        int *ord = s_ord[w];
        for (int i = 0; i < Lc; ++i) ord[i] = i;
        for (int i = 0; i < Lc; ++i)
            for (int j = i + 1; j < Lc; ++j)
                if (a[ord[j]][ord[j]] > a[ord[i]][ord[i]]) {
                    const int t = ord[i]; ord[i] = ord[j]; ord[j] = t;
                }
    }
    __syncwarp();
    const int *ord = s_ord[w];
    float *wv = wnuc + (long long)cq * Lc;
    if (svals) {                              // singular values only, descending
        if (lane < Lc) svals[(long long)cq * Lc + lane] = sqrt(fmax(a[ord[lane]][ord[lane]], 0.0));
        return;
    }
    if (reweight) {
        if (lane < Lc) {
            const double sv = sqrt(fmax(a[ord[lane]][ord[lane]], 0.0));
            wv[lane] = float(upsilon_bar / (upsilon_bar + sv));
        }
        return;
    }
    __shared__ double s_f[kEigWarps][NMAX];
    if (lane < Lc) {
        const double sv = sqrt(fmax(a[ord[lane]][ord[lane]], 0.0));
        const double thr = mu_bar * double(wv[lane]);
        s_f[w][lane] = (sv > thr) ? thr / sv : 1.0;
    }
    __syncwarp();
    float *M = mix + (long long)cq * Lc * Lc;
    for (int e = lane; e < Lc * Lc; e += 32) {
        const int i = e / Lc, j = e - (e / Lc) * Lc;
        double m = 0.0;
        for (int k = 0; k < Lc; ++k) m += V[i][ord[k]] * s_f[w][k] * V[j][ord[k]];
        M[e] = float(m);
    }
}

// The same eigen-decomposition for 16 < L_c <= 32 by a CTA of kEig32Threads
// threads per matrix (one warp took 1.7 ms for 64 matrices of 32 x 32: each
// round's dependent FP64 updates ran 16 deep per lane).  Same rotations, same
// order, same outputs as eig_kernel<32>.
constexpr int kEig32Threads = 128;

__global__ void __launch_bounds__(kEig32Threads) eig32_kernel(double *__restrict__ gram, float *__restrict__ mix,
                                                              float *__restrict__ wnuc, int n_mat, int Lc,
                                                              double mu_bar, double upsilon_bar, bool reweight,
                                                              double *__restrict__ eigv, double *__restrict__ svals) {
    constexpr int NMAX = 32, NT = kEig32Threads;
    __shared__ double a[NMAX][NMAX + 1];
    __shared__ double V[NMAX][NMAX + 1];
    __shared__ double Tm[NMAX][NMAX + 1];
    __shared__ double s_cs[NMAX / 2], s_sn[NMAX / 2];
    __shared__ int s_p[NMAX / 2], s_q[NMAX / 2];
    __shared__ int s_ord[NMAX];
    __shared__ double s_red[2][NT / 32];
    __shared__ double s_f[NMAX];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int cq = blockIdx.x;
    if (cq >= n_mat) return;
    double *G = gram + (long long)cq * Lc * Lc;
    const int n = Lc + (Lc & 1);
    for (int e = t; e < n * n; e += NT) {
        const int i = e / n, j = e - (e / n) * n;
        double v = 0.0;
        if (i < Lc && j < Lc) v = (j >= i) ? G[i * Lc + j] : G[j * Lc + i];
        a[i][j] = v;
        V[i][j] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    for (int e = t; e < Lc * Lc; e += NT) G[e] = 0.0;   // ready for the next accumulation
    double *Vg = eigv ? eigv + (long long)cq * n * n : nullptr;
    if (Vg) {
        for (int e = t; e < n * n; e += NT) V[e / n][e % n] = Vg[e];
        __syncthreads();
        for (int e = t; e < n * n; e += NT) {
            const int i = e / n, j = e - (e / n) * n;
            double x = 0.0;
            for (int k = 0; k < n; ++k) x = fma(a[i][k], V[k][j], x);
            Tm[i][j] = x;
        }
        __syncthreads();
        for (int e = t; e < n * n; e += NT) {
            const int i = e / n, j = e - (e / n) * n;
            double x = 0.0;
            for (int k = 0; k < n; ++k) x = fma(V[k][i], Tm[k][j], x);
            a[i][j] = x;
        }
        __syncthreads();
    }
    const int half = n / 2;
    for (int sweep = 0; sweep < 40; ++sweep) {
        double off = 0.0, dia = 0.0;
        for (int e = t; e < n * n; e += NT) {
            const int i = e / n, j = e - (e / n) * n;
            const double x = a[i][j];
            if (i == j) dia += x * x; else off += x * x;
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            dia += __shfl_xor_sync(0xffffffffu, dia, o);
        }
        if (lane == 0) {
            s_red[0][w] = off;
            s_red[1][w] = dia;
        }
        __syncthreads();
        off = dia = 0.0;
        for (int k = 0; k < NT / 32; ++k) {
            off += s_red[0][k];
            dia += s_red[1][k];
        }
        __syncthreads();                          // s_red is rewritten by the next sweep
        if (off <= 1e-28 * dia || off == 0.0) break;
        for (int round = 0; round < n - 1; ++round) {
            if (t < half) {
                const int k = t;
                int pa = (k == 0) ? 0 : 1 + (k - 1 + round) % (n - 1);
                int pb = 1 + (n - 2 - k + round) % (n - 1);
                const int p = min(pa, pb), q = max(pa, pb);
                const double apq = a[p][q];
                double cs = 1.0, sn = 0.0;
                if (apq != 0.0) {
                    const double theta = (a[q][q] - a[p][p]) / (2.0 * apq);
                    const double tt = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                    cs = 1.0 / sqrt(tt * tt + 1.0);
                    sn = tt * cs;
                }
                s_p[k] = p;
                s_q[k] = q;
                s_cs[k] = cs;
                s_sn[k] = sn;
            }
            __syncthreads();
            for (int e = t; e < half * n; e += NT) {        // columns: A <- A J, V <- V J
                const int k = e / n, r = e - k * n;
                const int p = s_p[k], q = s_q[k];
                const double cs = s_cs[k], sn = s_sn[k];
                const double arp = a[r][p], arq = a[r][q];
                a[r][p] = cs * arp - sn * arq;
                a[r][q] = sn * arp + cs * arq;
                const double vrp = V[r][p], vrq = V[r][q];
                V[r][p] = cs * vrp - sn * vrq;
                V[r][q] = sn * vrp + cs * vrq;
            }
            __syncthreads();
            for (int e = t; e < half * n; e += NT) {        // rows: A <- J^T A
                const int k = e / n, c = e - k * n;
                const int p = s_p[k], q = s_q[k];
                const double cs = s_cs[k], sn = s_sn[k];
                const double apc = a[p][c], aqc = a[q][c];
                a[p][c] = cs * apc - sn * aqc;
                a[q][c] = sn * apc + cs * aqc;
            }
            __syncthreads();
        }
    }
    if (Vg)
        for (int e = t; e < n * n; e += NT) Vg[e] = V[e / n][e % n];
    if (t == 0) {                             // eigenvalues descending (padding excluded)
        for (int i = 0; i < Lc; ++i) s_ord[i] = i;
        for (int i = 0; i < Lc; ++i)
            for (int j = i + 1; j < Lc; ++j)
                if (a[s_ord[j]][s_ord[j]] > a[s_ord[i]][s_ord[i]]) {
                    const int x = s_ord[i]; s_ord[i] = s_ord[j]; s_ord[j] = x;
                }
    }
    __syncthreads();
    float *wv = wnuc + (long long)cq * Lc;
    if (svals) {                              // singular values only, descending
        if (t < Lc) svals[(long long)cq * Lc + t] = sqrt(fmax(a[s_ord[t]][s_ord[t]], 0.0));
        return;
    }
    if (reweight) {
        if (t < Lc) {
            const double sv = sqrt(fmax(a[s_ord[t]][s_ord[t]], 0.0));
            wv[t] = float(upsilon_bar / (upsilon_bar + sv));
        }
        return;
    }
    if (t < Lc) {
        const double sv = sqrt(fmax(a[s_ord[t]][s_ord[t]], 0.0));
        const double thr = mu_bar * double(wv[t]);
        s_f[t] = (sv > thr) ? thr / sv : 1.0;
    }
    __syncthreads();
    float *M = mix + (long long)cq * Lc * Lc;
    for (int e = t; e < Lc * Lc; e += NT) {
        const int i = e / Lc, j = e - (e / Lc) * Lc;
        double m = 0.0;
        for (int k = 0; k < Lc; ++k) m += V[i][s_ord[k]] * s_f[k] * V[j][s_ord[k]];
        M[e] = float(m);
    }
}

// P_q <- (P_q + sigma0 S_q xbar) M_q, one thread per facet pixel.
template <int MAXLC>
__global__ void __launch_bounds__(256) apply_kernel(float *__restrict__ P, const float *__restrict__ img,
                                                    const int4 *__restrict__ facets,
                                                    const long long *__restrict__ nuc_off, const float *__restrict__ mix,
                                                    int Q, int C, int Lc, int nx, long long N, float s) {
    __shared__ float sM[MAXLC * MAXLC];
    const int cq = blockIdx.y;
    const int c = cq / Q, q = cq - c * Q;
    const int4 f = facets[q];
    const int wy = f.y - f.x, wx = f.w - f.z;
    const long long npix = (long long)wy * wx;
    const long long p0 = (long long)blockIdx.x * kPix;
    if (p0 >= npix) return;
    const long long p1 = min(npix, p0 + kPix);
    for (int k = threadIdx.x; k < Lc * Lc; k += blockDim.x) sM[k] = mix[(long long)cq * Lc * Lc + k];
    __syncthreads();
    float *Pq = P + nuc_off[cq];
    for (long long pp = p0 + threadIdx.x; pp < p1; pp += blockDim.x) {
        const int py = int(pp) / wx, px = int(pp) - py * wx;     // 32-bit division: facets hold < 2^31 pixels
        const long long o = (long long)(f.x + py) * nx + (f.z + px);
        float z[MAXLC];
#pragma unroll
        for (int j = 0; j < MAXLC; ++j)
            z[j] = (j < Lc) ? fmaf(s, img[(long long)(c + j * C) * N + o], Pq[(long long)j * npix + pp]) : 0.f;
#pragma unroll(MAXLC > 16 ? 2 : MAXLC)
        for (int j = 0; j < MAXLC; ++j) {
            if (j < Lc) {
                float r = 0.f;
#pragma unroll
                for (int i = 0; i < MAXLC; ++i)
                    if (i < Lc) r = fmaf(z[i], sM[i * Lc + j], r);
                Pq[(long long)j * npix + pp] = r;
            }
        }
    }
}

// P_q <- (P_q + sigma0 S_q xbar) M_q for more than 8 channels: a thread
// accumulates its pixel's (at most 32) outputs, taking z_i one channel at a
// time and adding z_i times row i of M (padded to 32 columns: eight 16-byte
// shared loads per 32 products).  The per-output form above takes 128-254
// registers at 16-32 channels.
__global__ void __launch_bounds__(256, 3) apply_wide_kernel(float *__restrict__ P, const float *__restrict__ img,
                                                            const int4 *__restrict__ facets,
                                                            const long long *__restrict__ nuc_off,
                                                            const float *__restrict__ mix, int Q, int C, int Lc,
                                                            int nx, long long N, float s) {
    __shared__ __align__(16) float sM[32 * 32];
    const int cq = blockIdx.y;
    const int c = cq / Q, q = cq - c * Q;
    const int4 f = facets[q];
    const int wy = f.y - f.x, wx = f.w - f.z;
    const long long npix = (long long)wy * wx;
    const long long p0 = (long long)blockIdx.x * kPix;
    if (p0 >= npix) return;
    const long long p1 = min(npix, p0 + kPix);
    for (int k = threadIdx.x; k < 32 * 32; k += blockDim.x) {
        const int i = k >> 5, j = k & 31;
        sM[k] = (i < Lc && j < Lc) ? mix[(long long)cq * Lc * Lc + i * Lc + j] : 0.f;
    }
    __syncthreads();
    float *Pq = P + nuc_off[cq];
    for (long long pp = p0 + threadIdx.x; pp < p1; pp += blockDim.x) {
        const int py = int(pp) / wx, px = int(pp) - py * wx;     // 32-bit division: facets hold < 2^31 pixels
        const long long o = (long long)(f.x + py) * nx + (f.z + px);
        float acc[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] = 0.f;
#pragma unroll 2
        for (int i = 0; i < Lc; ++i) {
            const float zi = fmaf(s, img[(long long)(c + i * C) * N + o], Pq[(long long)i * npix + pp]);
            const float4 *mr = reinterpret_cast<const float4 *>(&sM[i * 32]);
#pragma unroll
            for (int jq = 0; jq < 8; ++jq) {
                const float4 m = mr[jq];
                acc[4 * jq] = fmaf(zi, m.x, acc[4 * jq]);
                acc[4 * jq + 1] = fmaf(zi, m.y, acc[4 * jq + 1]);
                acc[4 * jq + 2] = fmaf(zi, m.z, acc[4 * jq + 2]);
                acc[4 * jq + 3] = fmaf(zi, m.w, acc[4 * jq + 3]);
            }
        }
#pragma unroll
        for (int j = 0; j < 32; ++j)
            if (j < Lc) Pq[(long long)j * npix + pp] = acc[j];
    }
}

}  // namespace

template <typename AccT>
static cudaError_t gram_dispatch(fhs_problem *p, const float *img, bool with_dual, cudaStream_t s) {
    long long maxpix = 0;
    for (const Facet &f : p->facets) maxpix = std::max<long long>(maxpix, (long long)(f.y1 - f.y0) * (f.x1 - f.x0));
    dim3 g(int((maxpix + kPix - 1) / kPix), p->C * p->Q);
    const dim3 gt(int((maxpix + kGramPix - 1) / kGramPix), p->C * p->Q);
    const float s0 = with_dual ? float(p->sigma0) : 1.f;
#define FHS_GRAM(M) gram_kernel<M, AccT><<<gt, 256, 0, s>>>(p->P, img, p->d_facets, p->nuc_off, p->Q, p->C, p->Lc, \
                                                           p->nx, p->N, s0, with_dual, p->gram)
    if (p->Lc <= 2) FHS_GRAM(2);
    else if (p->Lc <= 4) FHS_GRAM(4);
    else if (p->Lc <= 8) FHS_GRAM(8);
    else if (p->Lc <= 16) FHS_GRAM(16);
    else if (p->Lc <= 32)
        gram32_kernel<AccT><<<g, 256, 0, s>>>(p->P, img, p->d_facets, p->nuc_off, p->Q, p->C, p->Lc, p->nx, p->N, s0,
                                              with_dual, p->gram);
    else return cudaErrorInvalidValue;
#undef FHS_GRAM
    p->n_launch += 1;
    return cudaGetLastError();
}

cudaError_t launch_nuclear_gram(fhs_problem *p, const float *img, bool with_dual, bool fp64, cudaStream_t s) {
    // the dual step's Gram in FP32 (or FP64) products; the reweighting Gram of x in FP64
    return fp64 ? gram_dispatch<double>(p, img, with_dual, s) : gram_dispatch<float>(p, img, with_dual, s);
}

cudaError_t launch_nuclear_eig(fhs_problem *p, bool reweight, cudaStream_t s) {
    const int n = p->C * p->Q;
    double *v0 = reweight ? nullptr : p->eigv;     // the reweighting Gram (of x) starts cold
    if (p->Lc <= 16)
        eig_kernel<16><<<(n + 3) / 4, 128, 0, s>>>(p->gram, p->mix, p->wnuc, n, p->Lc, p->prm.mu_bar,
                                                  p->prm.upsilon_bar, reweight, v0, nullptr);
    else
        eig32_kernel<<<n, kEig32Threads, 0, s>>>(p->gram, p->mix, p->wnuc, n, p->Lc, p->prm.mu_bar,
                                                 p->prm.upsilon_bar, reweight, v0, nullptr);
    p->n_launch += 1;
    return cudaGetLastError();
}

cudaError_t launch_nuclear_svals(fhs_problem *p, double *svals, cudaStream_t s) {
    const int n = p->C * p->Q;
    if (p->Lc <= 16)
        eig_kernel<16><<<(n + 3) / 4, 128, 0, s>>>(p->gram, p->mix, p->wnuc, n, p->Lc, 0.0, 1.0, true, nullptr,
                                                  svals);
    else
        eig32_kernel<<<n, kEig32Threads, 0, s>>>(p->gram, p->mix, p->wnuc, n, p->Lc, 0.0, 1.0, true, nullptr, svals);
    p->n_launch += 1;
    return cudaGetLastError();
}

cudaError_t launch_nuclear_apply(fhs_problem *p, cudaStream_t s) {
    long long maxpix = 0;
    for (const Facet &f : p->facets) maxpix = std::max<long long>(maxpix, (long long)(f.y1 - f.y0) * (f.x1 - f.x0));
    dim3 g(int((maxpix + kPix - 1) / kPix), p->C * p->Q);
    const float s0 = float(p->sigma0);
    if (p->Lc <= 2)
        apply_kernel<2><<<g, 256, 0, s>>>(p->P, p->Xbar, p->d_facets, p->nuc_off, p->mix, p->Q, p->C, p->Lc, p->nx, p->N, s0);
    else if (p->Lc <= 4)
        apply_kernel<4><<<g, 256, 0, s>>>(p->P, p->Xbar, p->d_facets, p->nuc_off, p->mix, p->Q, p->C, p->Lc, p->nx, p->N, s0);
    else if (p->Lc <= 8)
        apply_kernel<8><<<g, 256, 0, s>>>(p->P, p->Xbar, p->d_facets, p->nuc_off, p->mix, p->Q, p->C, p->Lc, p->nx, p->N, s0);
    else if (p->Lc <= 32)
        apply_wide_kernel<<<g, 256, 0, s>>>(p->P, p->Xbar, p->d_facets, p->nuc_off, p->mix, p->Q, p->C, p->Lc, p->nx,
                                             p->N, s0);
    else
        return cudaErrorInvalidValue;
    p->n_launch += 1;
    return cudaGetLastError();
}

}  // namespace fhs
