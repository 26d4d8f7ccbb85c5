// SARA dictionary Psi^dagger = (1/3)[I; W_db1; ...; W_db8] and its adjoint,
// and the weighted l21 dual step (Sec. 2.2.2, average joint sparsity).
//
// The faceted transform of the paper equals the global one exactly (each
// coefficient is owned by one facet, whose window holds all its inputs); on
// one GPU the facets become CTA tiles: each CTA stages its tile plus the
// filter halo in shared memory (zero extension outside the image) and writes
// only the coefficients it owns, so nothing is computed twice beyond the halo.
// One level, one axis: c[k] = sum_i f[i] a[2k+1-i], k < floor((n+F-1)/2).
#include "fhs_internal.h"

#include <cstring>
#include <mutex>
#include <string>

namespace fhs {

namespace {

constexpr int ATY = 16, ATX = 32;                   // analysis output tile (coefficients)
constexpr int AIN_Y = 2 * ATY + kMaxF - 2;          // staged input rows
constexpr int AIN_X = 2 * ATX + kMaxF - 2;          // staged input cols
constexpr int STY = 32, STX = 64;                   // synthesis output tile (samples, even)
constexpr int SB_Y = (STY + kMaxF - 2) / 2;         // staged band rows
constexpr int SB_X = (STX + kMaxF - 2) / 2;         // staged band cols

// One analysis level of basis db_P on the staged tile: x-filter then y-filter
// with compile-time filter length F = 2P, writing the four subbands at level
// j (details to coef, LL to `ll_out`, row stride mx).  The staged input row r
// holds image row 2 k0y + 2 - kMaxF + r, so output k uses rows 2k+kMaxF-1-i.
//
// Register blocking: a thread of the x-filter computes kAnaNX adjacent outputs
// of one row from 2 (kAnaNX - 1) + F staged inputs held in registers (instead
// of F loads per output), and the warp's threads take consecutive rows (odd
// row stride: no bank conflicts); a thread of the y-filter computes kAnaNY
// outputs of one column the same way.
constexpr int kAnaNX = 4, kAnaNY = 2;
template <int P>
__device__ __forceinline__ void analysis_tile_t(const SaraConst &c, int j, int k0y, int k0x,
                                                float (*sin_)[AIN_X + 1], float (*slo)[ATX + 1],
                                                float (*shi)[ATX + 1], float *coef_l, float *ll_out,
                                                float ll_scale) {
    constexpr int F = 2 * P;
    constexpr int R0 = kMaxF - F;                    // first staged row this filter reaches
    constexpr int NR = AIN_Y - R0;                   // staged rows the y-filter reads
    constexpr int WX = 2 * (kAnaNX - 1) + F, WY = 2 * (kAnaNY - 1) + F;
    float h[F], g[F];
#pragma unroll
    for (int i = 0; i < F; ++i) {
        h[i] = c.h[P][i];
        g[i] = c.g[P][i];
    }
    const int my = c.ny[P][j], mx = c.nx[P][j];
    for (int idx = threadIdx.x; idx < NR * (ATX / kAnaNX); idx += blockDim.x) {
        const int r = R0 + idx % NR, kx0 = (idx / NR) * kAnaNX;
        const float *src = &sin_[r][2 * kx0 + R0];     // src[2n+F-1-i] = input of output kx0+n, tap i
        float a[WX];
#pragma unroll
        for (int t = 0; t < WX; ++t) a[t] = src[t];
#pragma unroll
        for (int n = 0; n < kAnaNX; ++n) {
            float lo = 0.f, hi = 0.f;
#pragma unroll
            for (int i = 0; i < F; ++i) {
                lo = fmaf(h[i], a[2 * n + F - 1 - i], lo);
                hi = fmaf(g[i], a[2 * n + F - 1 - i], hi);
            }
            slo[r][kx0 + n] = lo;
            shi[r][kx0 + n] = hi;
        }
    }
    __syncthreads();
    const long long bs = (long long)my * mx;
    for (int idx = threadIdx.x; idx < (ATY / kAnaNY) * ATX; idx += blockDim.x) {
        const int kx = idx % ATX, ky0 = (idx / ATX) * kAnaNY;
        const int r1 = 2 * ky0 + R0;                   // row of tap i = F-1 of output ky0
        float lo[WY], hi[WY];
#pragma unroll
        for (int t = 0; t < WY; ++t) {
            lo[t] = slo[r1 + t][kx];
            hi[t] = shi[r1 + t][kx];
        }
        const int gx = k0x + kx;
#pragma unroll
        for (int m = 0; m < kAnaNY; ++m) {
            float ll = 0.f, lh = 0.f, hl = 0.f, hh = 0.f;
#pragma unroll
            for (int i = 0; i < F; ++i) {
                const float vl = lo[2 * m + F - 1 - i], vh = hi[2 * m + F - 1 - i];
                ll = fmaf(h[i], vl, ll);
                lh = fmaf(h[i], vh, lh);
                hl = fmaf(g[i], vl, hl);
                hh = fmaf(g[i], vh, hh);
            }
            const int gy = k0y + ky0 + m;
            if (gy < my && gx < mx) {
                float *d = coef_l + c.off_det[P][j] + (long long)gy * mx + gx;
                d[0] = lh * kSaraScale;
                d[bs] = hl * kSaraScale;
                d[2 * bs] = hh * kSaraScale;
                ll_out[(long long)gy * mx + gx] = ll * ll_scale;
            }
        }
    }
    __syncthreads();
}

// Level 1 of every Daubechies basis (and the Dirac basis) from one staged tile
// of the image: the image is read once for all nine bases.
template <int P>
__device__ __forceinline__ void analysis_l1_basis(const SaraConst &c, int l, int k0y, int k0x,
                                                  float (*sin_)[AIN_X + 1], float (*slo)[ATX + 1],
                                                  float (*shi)[ATX + 1], float *coef_l, float *tmp) {
    if (k0y >= c.ny[P][1] || k0x >= c.nx[P][1]) return;
    float *ll_out = (c.levels == 1) ? coef_l + c.off_ll[P] : tmp + (long long)l * c.n_tmp + c.off_tmp[P][1];
    analysis_tile_t<P>(c, 1, k0y, k0x, sin_, slo, shi, coef_l, ll_out, c.levels == 1 ? kSaraScale : 1.f);
}

__global__ void __launch_bounds__(256) analysis_l1_kernel(const __grid_constant__ SaraConst c,
                                                          const float *__restrict__ x, float *__restrict__ coef,
                                                          float *__restrict__ tmp) {
    __shared__ float sin_[AIN_Y][AIN_X + 1];
    __shared__ float slo[AIN_Y][ATX + 1];
    __shared__ float shi[AIN_Y][ATX + 1];
    const int l = blockIdx.z;
    const int k0y = blockIdx.y * ATY, k0x = blockIdx.x * ATX;
    const int ny = c.img_ny, nx = c.img_nx;
    const long long N = (long long)ny * nx;
    const float *xl = x + (long long)l * N;
    float *coef_l = coef + (long long)l * c.n_coef;
    const int r0 = 2 * k0y + 2 - kMaxF, c0 = 2 * k0x + 2 - kMaxF;
    for (int idx = threadIdx.x; idx < AIN_Y * AIN_X; idx += blockDim.x) {
        const int r = idx / AIN_X, cc = idx - r * AIN_X;
        const int gy = r0 + r, gx = c0 + cc;
        sin_[r][cc] = (gy >= 0 && gy < ny && gx >= 0 && gx < nx) ? xl[(long long)gy * nx + gx] : 0.f;
    }
    __syncthreads();
    // Dirac basis: pixels [2 k0, 2 k0 + 2 tile) of this CTA (tiles partition the image).
    for (int idx = threadIdx.x; idx < 4 * ATY * ATX; idx += blockDim.x) {
        const int ry = idx / (2 * ATX), rx = idx - ry * (2 * ATX);
        const int gy = 2 * k0y + ry, gx = 2 * k0x + rx;
        if (gy < ny && gx < nx) coef_l[(long long)gy * nx + gx] = sin_[ry + kMaxF - 2][rx + kMaxF - 2] * kSaraScale;
    }
    analysis_l1_basis<1>(c, l, k0y, k0x, sin_, slo, shi, coef_l, tmp);
    analysis_l1_basis<2>(c, l, k0y, k0x, sin_, slo, shi, coef_l, tmp);
    analysis_l1_basis<3>(c, l, k0y, k0x, sin_, slo, shi, coef_l, tmp);
    analysis_l1_basis<4>(c, l, k0y, k0x, sin_, slo, shi, coef_l, tmp);
    analysis_l1_basis<5>(c, l, k0y, k0x, sin_, slo, shi, coef_l, tmp);
    analysis_l1_basis<6>(c, l, k0y, k0x, sin_, slo, shi, coef_l, tmp);
    analysis_l1_basis<7>(c, l, k0y, k0x, sin_, slo, shi, coef_l, tmp);
    analysis_l1_basis<8>(c, l, k0y, k0x, sin_, slo, shi, coef_l, tmp);
}

// Staging of a level j >= 2 input tile for db_P: only the rows and columns
// from kMaxF - 2P on, which its filters reach (zero outside the band).
template <int P>
__device__ __forceinline__ void analysis_stage_t(const float *__restrict__ in, int ny, int nx, int r0, int c0,
                                                 float (*sin_)[AIN_X + 1]) {
    constexpr int R0 = kMaxF - 2 * P, NY = AIN_Y - R0, NX = AIN_X - R0;
    for (int idx = threadIdx.x; idx < NY * NX; idx += blockDim.x) {
        const int r = R0 + idx / NX, cc = R0 + idx % NX;
        const int gy = r0 + r, gx = c0 + cc;
        // 32-bit offsets: an approximation band holds well under 2^31 samples
        sin_[r][cc] = (gy >= 0 && gy < ny && gx >= 0 && gx < nx) ? in[gy * nx + gx] : 0.f;
    }
    __syncthreads();
}

// Level j >= 2 of basis p from its level j-1 approximation.
__global__ void __launch_bounds__(256) analysis_lj_kernel(const __grid_constant__ SaraConst c, int j,
                                                          float *__restrict__ coef, float *__restrict__ tmp) {
    __shared__ float sin_[AIN_Y][AIN_X + 1];
    __shared__ float slo[AIN_Y][ATX + 1];
    __shared__ float shi[AIN_Y][ATX + 1];
    const int p = 1 + blockIdx.z % kNumDb;
    const int l = blockIdx.z / kNumDb;
    const int k0y = blockIdx.y * ATY, k0x = blockIdx.x * ATX;
    if (k0y >= c.ny[p][j] || k0x >= c.nx[p][j]) return;
    const int ny = c.ny[p][j - 1], nx = c.nx[p][j - 1];
    const float *in = tmp + (long long)l * c.n_tmp + c.off_tmp[p][j - 1];
    float *coef_l = coef + (long long)l * c.n_coef;
    const int r0 = 2 * k0y + 2 - kMaxF, c0 = 2 * k0x + 2 - kMaxF;
    const bool last = (j == c.levels);
    float *ll_out = last ? coef_l + c.off_ll[p] : tmp + (long long)l * c.n_tmp + c.off_tmp[p][j];
    const float lls = last ? kSaraScale : 1.f;
    switch (p) {
        case 1:
            analysis_stage_t<1>(in, ny, nx, r0, c0, sin_);
            analysis_tile_t<1>(c, j, k0y, k0x, sin_, slo, shi, coef_l, ll_out, lls);
            break;
        case 2:
            analysis_stage_t<2>(in, ny, nx, r0, c0, sin_);
            analysis_tile_t<2>(c, j, k0y, k0x, sin_, slo, shi, coef_l, ll_out, lls);
            break;
        case 3:
            analysis_stage_t<3>(in, ny, nx, r0, c0, sin_);
            analysis_tile_t<3>(c, j, k0y, k0x, sin_, slo, shi, coef_l, ll_out, lls);
            break;
        case 4:
            analysis_stage_t<4>(in, ny, nx, r0, c0, sin_);
            analysis_tile_t<4>(c, j, k0y, k0x, sin_, slo, shi, coef_l, ll_out, lls);
            break;
        case 5:
            analysis_stage_t<5>(in, ny, nx, r0, c0, sin_);
            analysis_tile_t<5>(c, j, k0y, k0x, sin_, slo, shi, coef_l, ll_out, lls);
            break;
        case 6:
            analysis_stage_t<6>(in, ny, nx, r0, c0, sin_);
            analysis_tile_t<6>(c, j, k0y, k0x, sin_, slo, shi, coef_l, ll_out, lls);
            break;
        case 7:
            analysis_stage_t<7>(in, ny, nx, r0, c0, sin_);
            analysis_tile_t<7>(c, j, k0y, k0x, sin_, slo, shi, coef_l, ll_out, lls);
            break;
        default:
            analysis_stage_t<8>(in, ny, nx, r0, c0, sin_);
            analysis_tile_t<8>(c, j, k0y, k0x, sin_, slo, shi, coef_l, ll_out, lls);
            break;
    }
}

// Adjoint of one level of db_P for an STY x STX tile of a_{j-1} at (m0y, m0x)
// (both even).  Polyphase: outputs 2q and 2q+1 use the same band samples
// k0 + q + t, t < F/2, with the odd and the even taps respectively
// (a[m] = sum_k f[2k+1-m] band[k]).  Adds this thread's outputs to acc[8]:
// slot pairs s < 4 give rows 2 qy and 2 qy + 1 of column rx (synth_slot).
//
// Register blocking as in the analysis: an x-step thread computes kSynNQ
// adjacent q of one band row from H + kSynNQ - 1 samples per band (rows
// taken by consecutive threads, odd row strides), and a y-step thread
// computes its four adjacent qy of one column from H + 3 samples per array.
constexpr int kSynNQ = 4;

__device__ __forceinline__ void cp_async4(float *dst, const float *src, bool valid) {
    // 4-byte asynchronous copy to shared memory; zero-filled when !valid (nothing is read)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(static_cast<uint32_t>(
                     __cvta_generic_to_shared(dst))),
                 "l"(src), "r"(valid ? 4 : 0)
                 : "memory");
}

// Stage the four level-j bands of db_P that an STY x STX output tile at
// (m0y, m0x) reaches into sb (zero outside the band).  ASYNC: by cp.async
// (the caller commits and waits), otherwise by plain loads.
template <int P, bool ASYNC>
__device__ __forceinline__ void synthesis_stage_t(const SaraConst &c, int j, int m0y, int m0x, const float *coef_l,
                                                  const float *ll_in, float (*sb)[SB_Y][SB_X + 2]) {
    constexpr int H = P;
    const int my = c.ny[P][j], mx = c.nx[P][j];
    const long long bs = (long long)my * mx;
    const int k0y = m0y / 2, k0x = m0x / 2;
    constexpr int NBY = STY / 2 + H - 1, NBX = STX / 2 + H - 1;   // band samples reached
    const float *det = coef_l + c.off_det[P][j];
    for (int idx = threadIdx.x; idx < NBY * NBX; idx += blockDim.x) {
        const int r = idx / NBX, cc = idx - r * NBX;
        const int ky = k0y + r, kx = k0x + cc;
        const bool in = ky < my && kx < mx;
        const long long o = in ? (long long)ky * mx + kx : 0;
        if (ASYNC) {
            cp_async4(&sb[0][r][cc], ll_in + o, in);    // LL  (y lo, x lo)
            cp_async4(&sb[1][r][cc], det + o, in);      // LH  (y lo, x hi)
            cp_async4(&sb[2][r][cc], det + bs + o, in); // HL  (y hi, x lo)
            cp_async4(&sb[3][r][cc], det + 2 * bs + o, in);
        } else {
            sb[0][r][cc] = in ? ll_in[o] : 0.f;
            sb[1][r][cc] = in ? det[o] : 0.f;
            sb[2][r][cc] = in ? det[bs + o] : 0.f;
            sb[3][r][cc] = in ? det[2 * bs + o] : 0.f;
        }
    }
}

// Adjoint of one level of db_P for an STY x STX tile of a_{j-1} from the
// staged bands sb.  Polyphase: outputs 2q and 2q+1 use the same band samples
// k0 + q + t, t < F/2, with the odd and the even taps respectively
// (a[m] = sum_k f[2k+1-m] band[k]).  Adds this thread's outputs to acc[8]:
// slot pairs s < 4 give rows 2 qy and 2 qy + 1 of column rx (synth_slot).
//
// Register blocking as in the analysis: an x-step thread computes kSynNQ
// adjacent q of one band row from H + kSynNQ - 1 samples per band (rows
// taken by consecutive threads, odd row strides), and a y-step thread
// computes its four adjacent qy of one column from H + 3 samples per array.
template <int P>
__device__ __forceinline__ void synthesis_compute_t(const SaraConst &c, float (*sb)[SB_Y][SB_X + 2],
                                                    float (*su)[SB_Y][STX + 1], float *acc) {
    constexpr int F = 2 * P, H = P;
    constexpr int NBY = STY / 2 + H - 1;
    float h[F], g[F];
#pragma unroll
    for (int i = 0; i < F; ++i) {
        h[i] = c.h[P][i];
        g[i] = c.g[P][i];
    }
    // x: u_lo = synth(LL, h) + synth(LH, g); u_hi = synth(HL, h) + synth(HH, g)
    constexpr int WQ = H + kSynNQ - 1;
    for (int idx = threadIdx.x; idx < NBY * (STX / 2 / kSynNQ); idx += blockDim.x) {
        const int r = idx % NBY, q0 = (idx / NBY) * kSynNQ;
        float a0[WQ], a1[WQ], a2[WQ], a3[WQ];
#pragma unroll
        for (int t = 0; t < WQ; ++t) {
            a0[t] = sb[0][r][q0 + t];
            a1[t] = sb[1][r][q0 + t];
            a2[t] = sb[2][r][q0 + t];
            a3[t] = sb[3][r][q0 + t];
        }
#pragma unroll
        for (int n = 0; n < kSynNQ; ++n) {
            float le = 0.f, lo = 0.f, he = 0.f, ho = 0.f;
#pragma unroll
            for (int t = 0; t < H; ++t) {
                le = fmaf(h[2 * t + 1], a0[n + t], fmaf(g[2 * t + 1], a1[n + t], le));
                lo = fmaf(h[2 * t], a0[n + t], fmaf(g[2 * t], a1[n + t], lo));
                he = fmaf(h[2 * t + 1], a2[n + t], fmaf(g[2 * t + 1], a3[n + t], he));
                ho = fmaf(h[2 * t], a2[n + t], fmaf(g[2 * t], a3[n + t], ho));
            }
            su[0][r][2 * (q0 + n)] = le;
            su[0][r][2 * (q0 + n) + 1] = lo;
            su[1][r][2 * (q0 + n)] = he;
            su[1][r][2 * (q0 + n) + 1] = ho;
        }
    }
    __syncthreads();
    {
        const int rx = threadIdx.x % STX, qy0 = (threadIdx.x / STX) * 4;
        float ul[H + 3], uh[H + 3];
#pragma unroll
        for (int t = 0; t < H + 3; ++t) {
            ul[t] = su[0][qy0 + t][rx];
            uh[t] = su[1][qy0 + t][rx];
        }
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            float e = 0.f, o = 0.f;
#pragma unroll
            for (int t = 0; t < H; ++t) {
                e = fmaf(h[2 * t + 1], ul[s + t], fmaf(g[2 * t + 1], uh[s + t], e));
                o = fmaf(h[2 * t], ul[s + t], fmaf(g[2 * t], uh[s + t], o));
            }
            acc[2 * s] += e;
            acc[2 * s + 1] += o;
        }
    }
    __syncthreads();
}


template <int P>
__device__ __forceinline__ void synthesis_tile_t(const SaraConst &c, int j, int m0y, int m0x, const float *coef_l,
                                                 const float *ll_in, float (*sb)[SB_Y][SB_X + 2],
                                                 float (*su)[SB_Y][STX + 1], float *acc) {
    synthesis_stage_t<P, false>(c, j, m0y, m0x, coef_l, ll_in, sb);
    __syncthreads();
    synthesis_compute_t<P>(c, sb, su, acc);
}

__device__ __forceinline__ void synthesis_tile(const SaraConst &c, int p, int j, int m0y, int m0x,
                                               const float *coef_l, const float *ll_in,
                                               float (*sb)[SB_Y][SB_X + 2], float (*su)[SB_Y][STX + 1],
                                               float *acc) {
    switch (p) {
        case 1: synthesis_tile_t<1>(c, j, m0y, m0x, coef_l, ll_in, sb, su, acc); break;
        case 2: synthesis_tile_t<2>(c, j, m0y, m0x, coef_l, ll_in, sb, su, acc); break;
        case 3: synthesis_tile_t<3>(c, j, m0y, m0x, coef_l, ll_in, sb, su, acc); break;
        case 4: synthesis_tile_t<4>(c, j, m0y, m0x, coef_l, ll_in, sb, su, acc); break;
        case 5: synthesis_tile_t<5>(c, j, m0y, m0x, coef_l, ll_in, sb, su, acc); break;
        case 6: synthesis_tile_t<6>(c, j, m0y, m0x, coef_l, ll_in, sb, su, acc); break;
        case 7: synthesis_tile_t<7>(c, j, m0y, m0x, coef_l, ll_in, sb, su, acc); break;
        default: synthesis_tile_t<8>(c, j, m0y, m0x, coef_l, ll_in, sb, su, acc); break;
    }
}

// Output sample of slot s of this thread: (row, col) offsets in the tile
// (column threadIdx % STX, band rows qy0 .. qy0 + 3 with qy0 = 4 (threadIdx / STX),
// even and odd output row of each).
__device__ __forceinline__ void synth_slot(int s, int &ry, int &rx) {
    ry = 2 * ((threadIdx.x / STX) * 4 + (s >> 1)) + (s & 1);
    rx = threadIdx.x % STX;
}

// Synthesis kernels run four CTAs per SM (at most 64 registers: the
// register-blocked sample windows and the eight accumulators fit without
// spills; the band staging is latency-bound and the occupancy hides it).
// Levels j >= 2: reconstruct a_{j-1} of basis p into tmp.
__global__ void __launch_bounds__(256, 4) synthesis_lj_kernel(const __grid_constant__ SaraConst c, int j,
                                                           const float *__restrict__ coef, float *__restrict__ tmp) {
    __shared__ float sb[4][SB_Y][SB_X + 2];
    __shared__ float su[2][SB_Y][STX + 1];
    const int p = 1 + blockIdx.z % kNumDb;
    const int l = blockIdx.z / kNumDb;
    const int m0y = blockIdx.y * STY, m0x = blockIdx.x * STX;
    const int oy = c.ny[p][j - 1], ox = c.nx[p][j - 1];
    if (m0y >= oy || m0x >= ox) return;
    const float *coef_l = coef + (long long)l * c.n_coef;
    const bool last = (j == c.levels);
    const float *ll_in = last ? coef_l + c.off_ll[p] : tmp + (long long)l * c.n_tmp + c.off_tmp[p][j];
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    synthesis_tile(c, p, j, m0y, m0x, coef_l, ll_in, sb, su, acc);
    float *out = tmp + (long long)l * c.n_tmp + c.off_tmp[p][j - 1];
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        int ry, rx;
        synth_slot(s, ry, rx);
        const int gy = m0y + ry, gx = m0x + rx;
        if (gy < oy && gx < ox) out[(long long)gy * ox + gx] = acc[s];
    }
}

// Level 1 of all bases plus the Dirac basis, summed into the image: x = (1/3) sum.
// The bands of basis P + 1 are staged by cp.async into the second buffer
// while basis P is synthesised from the first.
__global__ void __launch_bounds__(256, 4) synthesis_l1_kernel(const __grid_constant__ SaraConst c,
                                                           const float *__restrict__ coef, const float *__restrict__ tmp,
                                                           float *__restrict__ x) {
    __shared__ float sb[2][4][SB_Y][SB_X + 2];
    __shared__ float su[2][SB_Y][STX + 1];
    const int l = blockIdx.z;
    const int m0y = blockIdx.y * STY, m0x = blockIdx.x * STX;
    const int ny = c.img_ny, nx = c.img_nx;
    const float *coef_l = coef + (long long)l * c.n_coef;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#define FHS_SYN_LL(P) ((c.levels == 1) ? coef_l + c.off_ll[P] : tmp + (long long)l * c.n_tmp + c.off_tmp[P][1])
#define FHS_SYN_STAGE(P)                                                                                   \
    synthesis_stage_t<P, true>(c, 1, m0y, m0x, coef_l, FHS_SYN_LL(P), sb[(P) & 1]);                         \
    asm volatile("cp.async.commit_group;" ::: "memory")
#define FHS_SYN_STEP(P)                                                                                    \
    asm volatile("cp.async.wait_group 0;" ::: "memory");                                                   \
    __syncthreads();                                                                                       \
    FHS_SYN_STAGE(P + 1);                                                                                  \
    synthesis_compute_t<P>(c, sb[(P) & 1], su, acc)
    FHS_SYN_STAGE(1);
    FHS_SYN_STEP(1);
    FHS_SYN_STEP(2);
    FHS_SYN_STEP(3);
    FHS_SYN_STEP(4);
    FHS_SYN_STEP(5);
    FHS_SYN_STEP(6);
    FHS_SYN_STEP(7);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    synthesis_compute_t<8>(c, sb[0], su, acc);
#undef FHS_SYN_STEP
#undef FHS_SYN_STAGE
#undef FHS_SYN_LL
#pragma unroll
    for (int s = 0; s < 8; ++s) {
        int ry, rx;
        synth_slot(s, ry, rx);
        const int gy = m0y + ry, gx = m0x + rx;
        if (gy < ny && gx < nx) {
            const long long o = (long long)gy * nx + gx;
            x[(long long)l * ny * nx + o] = (acc[s] + coef_l[o]) * kSaraScale;
        }
    }
}

// Weighted l21 dual step, one thread per (sub-cube, coefficient):
// z_l = W_l + sigma1 A_l over the sub-cube's channels, W_l = z_l min(1, mu w / ||z||).
template <int MAXLC>
__global__ void __launch_bounds__(256) l21_dual_kernel(float *__restrict__ W, const float *__restrict__ A,
                                                       const float *__restrict__ w21, long long n_coef, int C, int Lc,
                                                       float sigma1, float mu) {
    const int c = blockIdx.y;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n_coef;
         r += (long long)gridDim.x * blockDim.x) {
        float z[MAXLC];
        float n2 = 0.f;
#pragma unroll
        for (int jj = 0; jj < MAXLC; ++jj) {
            if (jj < Lc) {
                const long long o = (long long)(c + jj * C) * n_coef + r;
                z[jj] = fmaf(sigma1, A[o], W[o]);
                n2 = fmaf(z[jj], z[jj], n2);
            }
        }
        const float thr = mu * w21[(long long)c * n_coef + r];
        const float nr = sqrtf(n2);
        const float f = (nr > thr) ? thr / nr : 1.f;
#pragma unroll
        for (int jj = 0; jj < MAXLC; ++jj)
            if (jj < Lc) W[(long long)(c + jj * C) * n_coef + r] = z[jj] * f;
    }
}

// The same step for sub-cubes of more than 8 channels, without holding the
// row in registers: a first sweep over the channels forms ||z||^2, a second
// forms z again (its loads hit the caches) and writes z min(1, mu w / ||z||).
// Holding the row took 128 registers a thread at 16 channels and 254 at 32
// (16 and 8 warps per SM).
__global__ void __launch_bounds__(256) l21_dual_wide_kernel(float *__restrict__ W, const float *__restrict__ A,
                                                            const float *__restrict__ w21, long long n_coef, int C,
                                                            int Lc, float sigma1, float mu) {
    const int c = blockIdx.y;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n_coef;
         r += (long long)gridDim.x * blockDim.x) {
        float n2 = 0.f;
#pragma unroll 8
        for (int jj = 0; jj < Lc; ++jj) {
            const long long o = (long long)(c + jj * C) * n_coef + r;
            const float z = fmaf(sigma1, A[o], W[o]);
            n2 = fmaf(z, z, n2);
        }
        const float thr = mu * w21[(long long)c * n_coef + r];
        const float nr = sqrtf(n2);
        const float f = (nr > thr) ? thr / nr : 1.f;
#pragma unroll 8
        for (int jj = 0; jj < Lc; ++jj) {
            const long long o = (long long)(c + jj * C) * n_coef + r;
            W[o] = fmaf(sigma1, A[o], W[o]) * f;
        }
    }
}

// Log-sum weights w_r = upsilon / (upsilon + ||(Psi^dagger X)_r||) per sub-cube.
__global__ void __launch_bounds__(256) l21_reweight_kernel(const float *__restrict__ A, float *__restrict__ w21,
                                                           long long n_coef, int C, int Lc, double upsilon) {
    const int c = blockIdx.y;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n_coef;
         r += (long long)gridDim.x * blockDim.x) {
        double n2 = 0.0;
        for (int jj = 0; jj < Lc; ++jj) {
            const double a = A[(long long)(c + jj * C) * n_coef + r];
            n2 += a * a;
        }
        w21[(long long)c * n_coef + r] = float(upsilon / (upsilon + sqrt(n2)));
    }
}

inline int cdiv(long long a, long long b) { return int((a + b - 1) / b); }

// out[c] += sum_r ||(A_l[r])_{l in sub-cube c}||_2 (unweighted l21 norm, FP64).
__global__ void __launch_bounds__(256) l21_norm_kernel(const float *__restrict__ A, long long n_coef, int C, int Lc,
                                                       double *__restrict__ out) {
    __shared__ double s_part[8];
    const int c = blockIdx.y;
    double acc = 0.0;
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n_coef;
         r += (long long)gridDim.x * blockDim.x) {
        double n2 = 0.0;
        for (int jj = 0; jj < Lc; ++jj) {
            const double a = A[(long long)(c + jj * C) * n_coef + r];
            n2 += a * a;
        }
        acc += sqrt(n2);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_part[w];
        atomicAdd(out + c, t);
    }
}

}  // namespace

// Layout of Psi^dagger for an ny x nx image with `levels` levels: filters,
// level sizes n_{j+1} = floor((n_j + F - 1)/2) and coefficient/temp offsets.
SaraConst sara_layout(int ny, int nx, int levels) {
    SaraConst c;
    std::memset(&c, 0, sizeof c);
    c.levels = levels;
    c.img_ny = ny;
    c.img_nx = nx;
    long long pos = (long long)ny * nx, tpos = 0;
    for (int b = 1; b <= kNumDb; ++b) {
        const std::vector<double> h = daubechies(b);
        const int F = 2 * b;
        c.F[b] = F;
        for (int k = 0; k < F; ++k) {
            c.h[b][k] = float(h[k]);
            c.g[b][k] = float((k & 1) ? -h[F - 1 - k] : h[F - 1 - k]);
        }
        c.ny[b][0] = ny;
        c.nx[b][0] = nx;
        for (int j = 1; j <= levels; ++j) {
            c.ny[b][j] = (c.ny[b][j - 1] + F - 1) / 2;
            c.nx[b][j] = (c.nx[b][j - 1] + F - 1) / 2;
        }
    }
    for (int b = 1; b <= kNumDb; ++b) {
        for (int j = 1; j <= levels; ++j) {
            c.off_det[b][j] = pos;
            pos += 3LL * c.ny[b][j] * c.nx[b][j];
        }
        c.off_ll[b] = pos;
        pos += (long long)c.ny[b][levels] * c.nx[b][levels];
        for (int j = 1; j < levels; ++j) {
            c.off_tmp[b][j] = tpos;
            tpos += (long long)c.ny[b][j] * c.nx[b][j];
        }
    }
    c.n_coef = pos;
    c.n_tmp = tpos > 0 ? tpos : 1;
    return c;
}

cudaError_t launch_sara_analysis(fhs_problem *p, const float *x, float *coef, cudaStream_t s) {
    const SaraConst &c = p->sara;
    int my = 0, mx = 0;
    for (int b = 1; b <= kNumDb; ++b) { my = max(my, c.ny[b][1]); mx = max(mx, c.nx[b][1]); }
    analysis_l1_kernel<<<dim3(cdiv(mx, ATX), cdiv(my, ATY), p->L), 256, 0, s>>>(c, x, coef, p->sara_tmp);
    for (int j = 2; j <= c.levels; ++j) {
        my = mx = 0;
        for (int b = 1; b <= kNumDb; ++b) { my = max(my, c.ny[b][j]); mx = max(mx, c.nx[b][j]); }
        analysis_lj_kernel<<<dim3(cdiv(mx, ATX), cdiv(my, ATY), p->L * kNumDb), 256, 0, s>>>(c, j, coef, p->sara_tmp);
    }
    p->n_launch += c.levels;
    return cudaGetLastError();
}

cudaError_t launch_sara_synthesis(fhs_problem *p, const float *coef, float *x, cudaStream_t s) {
    const SaraConst &c = p->sara;
    for (int j = c.levels; j >= 2; --j) {
        int my = 0, mx = 0;
        for (int b = 1; b <= kNumDb; ++b) { my = max(my, c.ny[b][j - 1]); mx = max(mx, c.nx[b][j - 1]); }
        synthesis_lj_kernel<<<dim3(cdiv(mx, STX), cdiv(my, STY), p->L * kNumDb), 256, 0, s>>>(c, j, coef, p->sara_tmp);
    }
    synthesis_l1_kernel<<<dim3(cdiv(c.img_nx, STX), cdiv(c.img_ny, STY), p->L), 256, 0, s>>>(c, coef, p->sara_tmp, x);
    p->n_launch += c.levels;
    return cudaGetLastError();
}

cudaError_t launch_l21_dual(fhs_problem *p, cudaStream_t s) {
    const long long n = p->sara.n_coef;
    dim3 g(min(cdiv(n, 256), 152 * 8), p->C);
    const float s1 = float(p->sigma1), mu = float(p->prm.mu);
    if (p->Lc <= 2) l21_dual_kernel<2><<<g, 256, 0, s>>>(p->W, p->coef_tmp, p->w21, n, p->C, p->Lc, s1, mu);
    else if (p->Lc <= 4) l21_dual_kernel<4><<<g, 256, 0, s>>>(p->W, p->coef_tmp, p->w21, n, p->C, p->Lc, s1, mu);
    else if (p->Lc <= 8) l21_dual_kernel<8><<<g, 256, 0, s>>>(p->W, p->coef_tmp, p->w21, n, p->C, p->Lc, s1, mu);
    else l21_dual_wide_kernel<<<g, 256, 0, s>>>(p->W, p->coef_tmp, p->w21, n, p->C, p->Lc, s1, mu);
    p->n_launch += 1;
    return cudaGetLastError();
}

cudaError_t launch_l21_norm(fhs_problem *p, const float *A, double *out, cudaStream_t s) {
    const long long n = p->sara.n_coef;
    dim3 g(min(cdiv(n, 256), 152 * 8), p->C);
    l21_norm_kernel<<<g, 256, 0, s>>>(A, n, p->C, p->Lc, out);
    p->n_launch += 1;
    return cudaGetLastError();
}

cudaError_t launch_l21_reweight(fhs_problem *p, cudaStream_t s) {
    const long long n = p->sara.n_coef;
    dim3 g(min(cdiv(n, 256), 152 * 8), p->C);
    l21_reweight_kernel<<<g, 256, 0, s>>>(p->coef_tmp, p->w21, n, p->C, p->Lc, p->prm.upsilon);
    p->n_launch += 1;
    return cudaGetLastError();
}

}  // namespace fhs

// ---------------------------------------------------------------------------
// SARA analysis that allocates nothing.
//
// Its scratch (the level approximations a_1..a_{J-1} of one image, all nine
// bases) lives in a file-scope device array of kNoAllocScratchFloats floats
// (16 MiB), which every GPU that loads the library holds until the process
// exits.  Host code cannot use the array's name as a device address, so the
// address is fetched with cudaGetSymbolAddress once per device, on the first
// call made with that device current, and cached.
// ---------------------------------------------------------------------------
namespace fhs {
namespace {

constexpr long long kNoAllocScratchFloats = 1LL << 22;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchFloats];

std::mutex g_noalloc_mu;
float *g_noalloc_ptr[kNoAllocMaxDevices] = {};

}  // namespace
}  // namespace fhs

extern "C" fhs_status fhs_sara_analysis_noalloc(int32_t ny, int32_t nx, int32_t n_images, int32_t levels,
                                                const float *x_dev, float *coef_dev, void *stream) {
    using namespace fhs;
    if (!x_dev || !coef_dev) {
        set_last_error("fhs_sara_analysis_noalloc: NULL buffer");
        return FHS_ERR_ARG;
    }
    if (ny < 16 || nx < 16 || n_images < 0 || levels < 1 || levels > kMaxLevels) {
        set_last_error("fhs_sara_analysis_noalloc: need ny, nx >= 16, n_images >= 0, 1 <= levels <= 6");
        return FHS_ERR_ARG;
    }
    const SaraConst c = sara_layout(ny, nx, levels);
    if (c.n_tmp > kNoAllocScratchFloats) {
        set_last_error("fhs_sara_analysis_noalloc: image needs " + std::to_string(c.n_tmp) +
                       " scratch floats, more than the static maximum of " +
                       std::to_string(kNoAllocScratchFloats) + " (about 1.4e6 pixels at 4 levels)");
        return FHS_ERR_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
        set_last_error(std::string("fhs_sara_analysis_noalloc: no usable current device: ") + cudaGetErrorString(e));
        return FHS_ERR_CUDA;
    }
    float *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess) {
                set_last_error(std::string("fhs_sara_analysis_noalloc: cudaGetSymbolAddress failed: ") +
                               cudaGetErrorString(e));
                return FHS_ERR_CUDA;
            }
            g_noalloc_ptr[dev] = static_cast<float *>(ptr);
        }
        scratch = g_noalloc_ptr[dev];
    }
    // an error left pending by an earlier CUDA call of this thread would otherwise be read back
    // below as a failure of these launches: report it as what it is
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(std::string("fhs_sara_analysis_noalloc: a CUDA error was pending from an earlier call: ") +
                       cudaGetErrorString(e));
        return FHS_ERR_CUDA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int my = 0, mx = 0;
    for (int b = 1; b <= kNumDb; ++b) { my = max(my, c.ny[b][1]); mx = max(mx, c.nx[b][1]); }
    const long long N = (long long)ny * nx;
    // one image at a time: the scratch holds the approximations of one image
    for (int i = 0; i < n_images; ++i) {
        const float *xi = x_dev + (long long)i * N;
        float *ci = coef_dev + (long long)i * c.n_coef;
        analysis_l1_kernel<<<dim3(cdiv(mx, ATX), cdiv(my, ATY), 1), 256, 0, s>>>(c, xi, ci, scratch);
        for (int j = 2; j <= c.levels; ++j) {
            int ly = 0, lx = 0;
            for (int b = 1; b <= kNumDb; ++b) { ly = max(ly, c.ny[b][j]); lx = max(lx, c.nx[b][j]); }
            analysis_lj_kernel<<<dim3(cdiv(lx, ATX), cdiv(ly, ATY), kNumDb), 256, 0, s>>>(c, j, ci, scratch);
        }
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_last_error(std::string("fhs_sara_analysis_noalloc: launch failed: ") + cudaGetErrorString(e));
        return FHS_ERR_CUDA;
    }
    return FHS_OK;
}
