// Primal step of the PDFB iteration (Sec. 2.2.3) fused with the gathers of
// the three adjoint terms and the zero-padding of the next forward FFT:
//
//   a    = Re(Z^T F^H g_data) + A_sara + sum_{q covering n} P_q(n)
//          (Re F^H g_data is the C2R transform of the folded adjoint grid)
//   x+   = max(0, x - tau a)             (non-negativity, Eq. 2)
//   xbar = 2 x+ - x,   grid_in[(n mod K)] = xbar s1 s2   (Z for the next F)
//   ||x+ - x||^2 and ||x+||^2 in FP64 for the relative-change test.
#include "fhs_internal.h"

namespace fhs {

namespace {

__global__ void __launch_bounds__(256) primal_kernel(
    float *__restrict__ X, float *__restrict__ Xbar, const float *__restrict__ A_sara,
    const float *__restrict__ grid_adj, float *__restrict__ grid_in, const float *__restrict__ s1,
    const float *__restrict__ s2, const float *__restrict__ P, const int4 *__restrict__ facets,
    const long long *__restrict__ nuc_off, const short *__restrict__ rf, const short *__restrict__ rc,
    const short *__restrict__ cf, const short *__restrict__ cc, int qx, int Q, int C, int ny, int nx, int K1,
    int K2, long long K, float tau, bool use_sara, bool use_nuc, double *__restrict__ red) {
    __shared__ double s_a[8], s_b[8];
    const int l = blockIdx.y;
    const int c = l % C, j = l / C;
    const long long N = (long long)ny * nx;
    // channel bases once; row offsets hoisted out of the column loop
    float *Xl = X + (long long)l * N, *Xbl = Xbar + (long long)l * N;
    const float *Al = A_sara + (long long)l * N;
    const float *gal = grid_adj + (long long)l * K;
    float *gil = grid_in + (long long)l * K;
    // compensated FP32 per thread, FP64 across threads
    float num = 0.f, cnum = 0.f, den = 0.f, cden = 0.f;
    // one image row per CTA step (row-uniform terms hoisted), columns over the threads
    for (int i1 = blockIdx.x; i1 < ny; i1 += gridDim.x) {
        int k1 = i1 - ny / 2;
        k1 += (k1 < 0) ? K1 : 0;
        const float s1r = s1[i1];
        const int r0 = use_nuc ? rf[i1] : 0, nr = use_nuc ? rc[i1] : 0;
        const long long grow = (long long)k1 * K2, irow = (long long)i1 * nx;
        for (int i2 = threadIdx.x; i2 < nx; i2 += blockDim.x) {
            int k2 = i2 - nx / 2;
            k2 += (k2 < 0) ? K2 : 0;
            const float sc = s1r * s2[i2];
            float a = gal[grow + k2] * sc;
            const long long o = irow + i2;
            if (use_sara) a += Al[o];
            if (use_nuc) {
                const int c0 = cf[i2], ncol = cc[i2];
                for (int ry = 0; ry < nr; ++ry)
                    for (int rx = 0; rx < ncol; ++rx) {
                        const int q = (r0 + ry) * qx + (c0 + rx);
                        const int4 f = facets[q];
                        const int fw = f.w - f.z;
                        a += P[nuc_off[c * Q + q] + (long long)j * ((f.y - f.x) * fw) + (i1 - f.x) * fw + (i2 - f.z)];
                    }
            }
            const float x = Xl[o];
            const float xp = fmaxf(0.f, fmaf(-tau, a, x));
            const float xb = 2.f * xp - x;
            Xl[o] = xp;
            Xbl[o] = xb;
            gil[grow + k2] = xb * sc;
            const float dx = xp - x;
            {
                const float yv = fmaf(dx, dx, -cnum), t = num + yv;
                cnum = (t - num) - yv;
                num = t;
            }
            {
                const float yv = fmaf(xp, xp, -cden), t = den + yv;
                cden = (t - den) - yv;
                den = t;
            }
        }
    }
    double dn = double(num) - double(cnum), dd = double(den) - double(cden);
    for (int o = 16; o > 0; o >>= 1) {
        dn += __shfl_xor_sync(0xffffffffu, dn, o);
        dd += __shfl_xor_sync(0xffffffffu, dd, o);
    }
    if ((threadIdx.x & 31) == 0) { s_a[threadIdx.x >> 5] = dn; s_b[threadIdx.x >> 5] = dd; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += s_a[w]; b += s_b[w]; }
        atomicAdd(red, a);
        atomicAdd(red + 1, b);
    }
}

}  // namespace

cudaError_t launch_primal(fhs_problem *p, cudaStream_t s) {
    long long g = p->ny;                 // one row per CTA (rows of a channel are independent)
    if (g > 1024) g = 1024;
    const bool use_sara = p->prm.mu > 0.0;
    const bool use_nuc = p->prm.mu_bar > 0.0;
    primal_kernel<<<dim3(int(g), p->L), 256, 0, s>>>(
        p->X, p->Xbar, p->A_sara, p->adj_real, p->grid_in, p->s1, p->s2, p->P, p->d_facets, p->nuc_off,
        p->cov_row_first, p->cov_row_cnt, p->cov_col_first, p->cov_col_cnt, p->prm.qx, p->Q, p->C, p->ny, p->nx,
        p->K1, p->K2, p->K, float(p->tau), use_sara, use_nuc, p->red);
    p->n_launch += 1;
    return cudaGetLastError();
}

}  // namespace fhs
