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

constexpr int kPix = 2048;          // facet pixels per CTA in the Gram / apply kernels

template <int MAXLC>
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
    const long long p0 = (long long)blockIdx.x * kPix;
    if (p0 >= npix) return;
    const long long p1 = min(npix, p0 + kPix);
    const float *Pq = P + nuc_off[cq];
    float acc[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) acc[k] = 0.f;
    for (long long pp = p0 + threadIdx.x; pp < p1; pp += blockDim.x) {
        const int py = int(pp / wx), px = int(pp - (long long)py * wx);
        const long long o = (long long)(f.x + py) * nx + (f.z + px);
        float z[MAXLC];
#pragma unroll
        for (int j = 0; j < MAXLC; ++j) {
            z[j] = 0.f;
            if (j < Lc) {
                const float xv = img[(long long)(c + j * C) * N + o];
                z[j] = with_dual ? fmaf(s, xv, Pq[(long long)j * npix + pp]) : xv;
            }
        }
        int k = 0;
#pragma unroll
        for (int i = 0; i < MAXLC; ++i)
#pragma unroll
            for (int j = i; j < MAXLC; ++j, ++k) acc[k] = fmaf(z[i], z[j], acc[k]);
    }
    for (int k = threadIdx.x; k < NP; k += blockDim.x) s_red[k] = 0.0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        float v = acc[k];
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

// Symmetric eigen-decomposition of one Gram per thread (cyclic Jacobi, FP64,
// bounded sweeps), then either the SVT mixing matrix or the reweighting weights.
__global__ void eig_kernel(double *__restrict__ gram, float *__restrict__ mix, float *__restrict__ wnuc, int n_mat,
                           int Lc, double mu_bar, double upsilon_bar, bool reweight) {
    const int cq = blockIdx.x * blockDim.x + threadIdx.x;
    if (cq >= n_mat) return;
    double a[kMaxLc][kMaxLc], V[kMaxLc][kMaxLc];
    double *G = gram + (long long)cq * Lc * Lc;
    for (int i = 0; i < Lc; ++i)
        for (int j = 0; j < Lc; ++j) {
            a[i][j] = (j >= i) ? G[i * Lc + j] : G[j * Lc + i];
            V[i][j] = (i == j) ? 1.0 : 0.0;
        }
    for (int i = 0; i < Lc * Lc; ++i) G[i] = 0.0;        // ready for the next accumulation
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = 0.0, dia = 0.0;
        for (int i = 0; i < Lc; ++i) {
            dia += a[i][i] * a[i][i];
            for (int j = i + 1; j < Lc; ++j) off += a[i][j] * a[i][j];
        }
        if (off <= 1e-30 * dia || off == 0.0) break;
        for (int pp = 0; pp < Lc - 1; ++pp)
            for (int qq = pp + 1; qq < Lc; ++qq) {
                const double apq = a[pp][qq];
                if (apq == 0.0) continue;
                const double theta = (a[qq][qq] - a[pp][pp]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
                for (int k = 0; k < Lc; ++k) {
                    const double akp = a[k][pp], akq = a[k][qq];
                    a[k][pp] = cs * akp - sn * akq;
                    a[k][qq] = sn * akp + cs * akq;
                }
                for (int k = 0; k < Lc; ++k) {
                    const double apk = a[pp][k], aqk = a[qq][k];
                    a[pp][k] = cs * apk - sn * aqk;
                    a[qq][k] = sn * apk + cs * aqk;
                }
                for (int k = 0; k < Lc; ++k) {
                    const double vkp = V[k][pp], vkq = V[k][qq];
                    V[k][pp] = cs * vkp - sn * vkq;
                    V[k][qq] = sn * vkp + cs * vkq;
                }
            }
    }
    // eigenvalues descending with their vectors
    int order[kMaxLc];
    for (int i = 0; i < Lc; ++i) order[i] = i;
    for (int i = 0; i < Lc; ++i)
        for (int j = i + 1; j < Lc; ++j)
            if (a[order[j]][order[j]] > a[order[i]][order[i]]) {
                const int t = order[i]; order[i] = order[j]; order[j] = t;
            }
    float *w = wnuc + (long long)cq * Lc;
    double fac[kMaxLc];
    for (int i = 0; i < Lc; ++i) {
        const double sv = sqrt(fmax(a[order[i]][order[i]], 0.0));
        if (reweight) {
            w[i] = float(upsilon_bar / (upsilon_bar + sv));
        } else {
            const double thr = mu_bar * double(w[i]);
            fac[i] = (sv > thr) ? thr / sv : 1.0;
        }
    }
    if (reweight) return;
    float *M = mix + (long long)cq * Lc * Lc;
    for (int i = 0; i < Lc; ++i)
        for (int j = 0; j < Lc; ++j) {
            double m = 0.0;
            for (int k = 0; k < Lc; ++k) m += V[i][order[k]] * fac[k] * V[j][order[k]];
            M[i * Lc + j] = float(m);
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
        const int py = int(pp / wx), px = int(pp - (long long)py * wx);
        const long long o = (long long)(f.x + py) * nx + (f.z + px);
        float z[MAXLC];
#pragma unroll
        for (int j = 0; j < MAXLC; ++j)
            z[j] = (j < Lc) ? fmaf(s, img[(long long)(c + j * C) * N + o], Pq[(long long)j * npix + pp]) : 0.f;
#pragma unroll
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

}  // namespace

cudaError_t launch_nuclear_gram(fhs_problem *p, const float *img, bool with_dual, cudaStream_t s) {
    long long maxpix = 0;
    for (const Facet &f : p->facets) maxpix = std::max<long long>(maxpix, (long long)(f.y1 - f.y0) * (f.x1 - f.x0));
    dim3 g(int((maxpix + kPix - 1) / kPix), p->C * p->Q);
    const float s0 = with_dual ? float(p->sigma0) : 1.f;
    if (p->Lc <= 2)
        gram_kernel<2><<<g, 256, 0, s>>>(p->P, img, p->d_facets, p->nuc_off, p->Q, p->C, p->Lc, p->nx, p->N, s0, with_dual, p->gram);
    else if (p->Lc <= 4)
        gram_kernel<4><<<g, 256, 0, s>>>(p->P, img, p->d_facets, p->nuc_off, p->Q, p->C, p->Lc, p->nx, p->N, s0, with_dual, p->gram);
    else if (p->Lc <= 8)
        gram_kernel<8><<<g, 256, 0, s>>>(p->P, img, p->d_facets, p->nuc_off, p->Q, p->C, p->Lc, p->nx, p->N, s0, with_dual, p->gram);
    else if (p->Lc <= 16)
        gram_kernel<16><<<g, 256, 0, s>>>(p->P, img, p->d_facets, p->nuc_off, p->Q, p->C, p->Lc, p->nx, p->N, s0, with_dual, p->gram);
    else
        return cudaErrorInvalidValue;
    p->n_launch += 1;
    return cudaGetLastError();
}

cudaError_t launch_nuclear_eig(fhs_problem *p, bool reweight, cudaStream_t s) {
    const int n = p->C * p->Q;
    eig_kernel<<<(n + 63) / 64, 64, 0, s>>>(p->gram, p->mix, p->wnuc, n, p->Lc, p->prm.mu_bar, p->prm.upsilon_bar,
                                           reweight);
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
    else if (p->Lc <= 16)
        apply_kernel<16><<<g, 256, 0, s>>>(p->P, p->Xbar, p->d_facets, p->nuc_off, p->mix, p->Q, p->C, p->Lc, p->nx, p->N, s0);
    else
        return cudaErrorInvalidValue;
    p->n_launch += 1;
    return cudaGetLastError();
}

}  // namespace fhs
