// The tile-binned pass over G (Sec. 2.1, Eq. 1) in its uses: the data term of
// a PDFB iteration (Eq. 2) as a dual pass (gather + dual pre-update + block
// norms) and a scatter pass, Phi alone, Phi^H alone, and Phi^H Phi for the
// operator-norm estimate.  Rows of G are the outer products g1 (x) g2 of two
// 1-D factors (see k_nufft.cu); rows are sorted by the grid tile of their box
// corner inside each (channel, block) segment.
#include "fhs_internal.h"

#include <cuda.h>
#include <cudaTypedefs.h>

namespace fhs {

namespace {

constexpr int kWarps = 8;               // warps per CTA
// Columns of g2 a gathering thread holds in registers, and the CTAs per SM of
// the gathering passes.  Measured at 1024^2 x 16 channels: 8 and 4 (64
// registers) beat 4 and 5 (48 registers: 9 % slower) and 3 and 6 (40: 21 %):
// narrower chunks pass over the box rows more often than the extra warps hide.
#ifndef FHS_GATHER_COLS
#define FHS_GATHER_COLS 8
#endif
constexpr int kGatherCols = FHS_GATHER_COLS;

__device__ __forceinline__ void red_add_f2(float2 *addr, float2 v) {
    atomicAdd(addr, v);   // sm_90+: vector float2 reduction (red.global.add.v2.f32)
}

// Grid layouts.  Full: [K1][K2] complex.  Half (hs > 0): columns 0..K2/2 of
// each row at a row stride of hs = K2/2 + 1, the layout of the R2C output
// and of the C2R input (cuFFT runs these about 35 % slower with a padded
// row stride, so half grids are not TMA-aligned and their windows are staged
// by per-thread asynchronous copies).
//
// grid(k1, k2) += c.  fold = 0: a full grid.  fold = hs > 0: the half grid
// holds the Hermitian part h(k) = (g(k) + conj g(-k)) / 2 of the sum g, which
// is what the C2R transform needs for Re F^H g: c adds c / 2 at k when
// k2 <= K2/2 and conj(c) / 2 at -k when -k2 mod K2 <= K2/2 (both for k2 = 0
// and k2 = K2/2).
__device__ __forceinline__ void red_grid(float2 *__restrict__ gb, int k1, int k2, int K1, int K2, float re,
                                         float im, int fold) {
    if (!fold) {
        red_add_f2(gb + (long long)k1 * K2 + k2, make_float2(re, im));
        return;
    }
    const int h = K2 >> 1;
    if (k2 <= h) red_add_f2(gb + (long long)k1 * fold + k2, make_float2(0.5f * re, 0.5f * im));
    if (k2 == 0 || k2 >= h) {
        const int m1 = k1 ? K1 - k1 : 0, m2 = k2 ? K2 - k2 : 0;
        red_add_f2(gb + (long long)m1 * fold + m2, make_float2(0.5f * re, -0.5f * im));
    }
}

// X(k1, k2) of a spectrum.  hs = 0: a full grid.  hs > 0: a half grid of a
// real image's spectrum, whose other half follows from X(k) = conj X(-k).
__device__ __forceinline__ float2 spec_at(const float2 *__restrict__ gl, int k1, int k2, int K1, int K2, int hs) {
    if (!hs) return gl[(long long)k1 * K2 + k2];
    if (k2 <= (K2 >> 1)) return gl[(long long)k1 * hs + k2];
    const int m1 = k1 ? K1 - k1 : 0;
    const float2 v = gl[(long long)m1 * hs + (K2 - k2)];
    return make_float2(v.x, -v.y);
}

// The data term of one PDFB iteration (Eq. 2) in two passes over G:
//   dual pass      phi  = G_m . Xhat                    (gather from the forward grid)
//                  d_m  = s_b d_m + sigma2 (phi - y_m)  (= z - sigma2 y, z = v + sigma2 Phi xbar)
//                  ||d_b||^2 per block (compensated FP32, then FP64)
//   (host stream)  s_b = 1 - min(1, sigma2 eps_b / ||d_b||), the block's l2-ball factor
//   scatter pass   grid_l += conj(G_m) s_b d_m           (v_m = s_b d_m)
// The dual is kept as d with the factor s_b applied lazily (v = s_b d).  Two
// passes read G twice but need no per-block adjoint grids and no combine, and
// each pass runs at the occupancy of its own resources.
// Tile-binned form.  A bin holds visibilities of one (channel, block) segment
// whose box corners fall in one kTile x kTile grid tile; every box then lies
// inside the kWin x kWin window at the tile origin.  The CTA stages the
// window of the forward grid in shared memory and gathers from it, or
// accumulates conj(G) v with shared-memory atomics and adds the window to the
// channel grid once at the end (one global reduction per cell instead of one
// per G entry).  Bins marked -1 (sparse tiles) take the global path.
constexpr int kWin = kTile + 15;        // boxes have T <= 16
// The staged forward window holds its even and its odd rows in two boxes of
// kBoxH rows x kBoxW cells (a TMA box row must be a multiple of 16 bytes):
// grids are read as rows of pairs of rows, whose stride is a multiple of 16
// bytes even when a row's is not (a half grid's K2/2 + 1 cells).
constexpr int kBoxW = 48;
constexpr int kBoxH = (kWin + 1) / 2;
constexpr int kBoxCells = kBoxW * kBoxH;
static_assert(kBoxW >= kWin + 1 && kBoxW % 2 == 0, "window box width");
// Window cell (rr, cc), rows and columns relative to the tile origin.  Direct
// (MIR = false): cell (rr, cc) of the grid, the odd rows shifted right by sh
// (the odd box starts one cell early when the grid's row stride is odd).
// MIR: the window lies in the half of a Hermitian spectrum that is not
// stored, and the boxes hold the conjugate-symmetric block, cell (rr, cc) at
// row kBoxH - 1 - rr / 2 and column kWin - 1 + sh (rr odd) - cc of its box: the
// gather reads such a window's rows backwards and conjugated.
template <bool MIR>
__device__ __forceinline__ const float2 *win_cell(const float2 *s_grid, int rr, int cc, int sh) {
    const int p = rr & 1, j = rr >> 1;
    if (!MIR) return s_grid + p * kBoxCells + j * kBoxW + cc + sh * p;
    return s_grid + p * kBoxCells + (kBoxH - 1 - j) * kBoxW + (kWin - 1 + sh * p) - cc;
}
template <bool MIR>
__device__ __forceinline__ float2 win_ld(const float2 *q, int t) {
    if (!MIR) return q[t];
    const float2 v = q[-t];
    return make_float2(v.x, -v.y);
}
// Row stride (in 32-bit words) of the adjoint window planes.  56 = 24 mod 32:
// box rows 1, 2 and 3 below a row start 24, 16 and 8 banks further on, so
// four rows of at most 8 adjacent cells, or two rows 2 apart of at most 16
// adjacent cells, fall in disjoint banks (the scatter's lane mappings).
constexpr int kAdjS = 56;
static_assert(kAdjS >= kWin && kAdjS % 32 == 24, "adjoint window stride");
#ifndef FHS_BIN_MAX
#define FHS_BIN_MAX 384
#endif
constexpr int kBinMax = FHS_BIN_MAX;    // visibilities per bin (host splits longer runs)
// The fixed-point scatter window (below) converts each part of a contribution
// to an integer of magnitude at most 2^22 and adds at most kBinMax of them to a
// cell; the sum stays inside int32 only while kBinMax <= 511.
static_assert(kBinMax <= 511, "the fixed-point scatter window overflows int32 for bins above 511 rows");
static_assert(kBinMax <= 65536, "row offsets of a bin");
// Pieces of a bin: runs of rows of one data block each (a tile's rows of all
// blocks of a channel share one bin); the host merges blocks only while B <= kMaxPieces.
constexpr int kMaxPieces = int(kBinMaxPieces);
static_assert(kMaxPieces <= 32, "a bin's pieces are scanned by one warp");
static_assert((2 * kWin * kAdjS) % 4 == 0 && kWin <= 64, "window zeroed by 16-byte stores, flushed 64 columns per warp step");

// Factors of one row for one warp: lane t < T holds g1[t], lane 16 + t holds
// g2[t]; the other lanes hold 0.
__device__ __forceinline__ float2 load_factors(const float2 *__restrict__ f, int T, int lane) {
    const int half = lane >> 4, col = lane & 15;
    float2 r = make_float2(0.f, 0.f);
    if (col < T) r = __ldcs(f + half * T + col);
    return r;
}

// Modes of the pass: kDual (the data term's dual pass), kGather (Phi only:
// vis_bin[i] = G_i . Xhat), kScatter (Phi^H only, and the data term's scatter
// pass: grid += conj(G_i) vis_bin[i]) and kNormal (G^H G in one pass:
// grid += conj(G_i) (G_i . Xhat), for the operator-norm estimate).
enum { kDual = 0, kGather = 1, kScatter = 2, kNormal = 3 };

constexpr float kFixMagic = 12582912.f;          // 1.5 * 2^23
constexpr unsigned kFixMagicBits = 0x4B400000u;  // its bit pattern
constexpr int kFixBits = 22;                     // contributions are scaled below 2^22

// Scatter of rows i = i0, i0 + kWarps, ... of one bin by one warp,
// grid += conj(G_i) s_d[i].  DENSE: the box lies in the shared window (shared
// atomics); otherwise global reductions.
//
// Row G_i = g1 (x) g2 over the T x T box; lane t < T holds g1[t] and lane
// 16 + t holds g2[t].  A lane adds conj(g1[t1]) (conj(g2[col]) d) to cell
// (t1, col) of the box for the box rows t1 of its mapping:
//  - T <= 8: lane (g, col) = (lane / 8, lane % 8) takes rows t1 = g, g + 4:
//    four box rows per step, ceil(T / 4) steps;
//  - T > 8: lane (h, col) = (lane / 16, lane % 16) takes rows
//    t1 = 4 j + 2 h + e at step 2 j + e: two box rows 2 apart per step.
// With the window's row stride kAdjS both mappings touch 32 distinct banks
// per step.  The next row's factors are loaded while the current row is
// scattered.
//
// FIXED (dense bins): the window accumulates in 32-bit fixed point, with
// native integer shared atomics (a float shared atomic costs about 3.5 times
// as much).  With e = S conj(g2[col]) d formed once per row, the real part
// of S conj(g1) e is rounded to an integer by two FMAs on 1.5 * 2^23:
// fma(g1x, er, fma(g1y, ei, 1.5 * 2^23)) lands in [2^23, 2^24], whose unit is
// 1, so the low mantissa bits hold the integer (each FMA rounds once: at most
// one unit of error), and the bit pattern less the magic's is the integer;
// likewise the imaginary part.  S = 2^(22 - e) with bound < 2^e and bound >=
// |every contribution of the bin|, so each part is at most 2^22 in magnitude
// and a cell's sums of at most kBinMax of them stay inside int32.  (Packing
// both parts in one 64-bit atomic, im 2^32 + re, halves the atomics but was
// measured 20-30 % slower.)  A lane whose cell lies outside its row's box
// (t1 >= T or col >= T) holds a zero factor, so in fixed point it adds
// exactly 0 to a cell that still lies in the window (corner offsets below
// kTile = 32, t1 and col below 16: both below kWin = 47) instead of branching
// around the atomics.

// cell ib += conj(g1) e, with e = conj(g2) d already formed (and scaled by S
// in fixed point).  The window is two planes (real, imaginary) of kWin x kAdjS
// 32-bit words: integers in fixed point, floats otherwise.
template <bool DENSE, bool FIXED>
__device__ __forceinline__ void scatter_cell(int *s_win, int ib, float2 *__restrict__ gb,
                                             int gk1, int gk2, int K1, int K2, int fold, float g1x, float g1y,
                                             float er, float ei) {
    if (DENSE && FIXED) {
        const float re = fmaf(g1x, er, fmaf(g1y, ei, kFixMagic));
        const float im = fmaf(g1x, ei, fmaf(-g1y, er, kFixMagic));
        atomicAdd(s_win + ib, int(__float_as_uint(re) - kFixMagicBits));
        atomicAdd(s_win + kWin * kAdjS + ib, int(__float_as_uint(im) - kFixMagicBits));
    } else {
        const float pr = fmaf(g1x, er, g1y * ei), pi = fmaf(g1x, ei, -g1y * er);
        if (DENSE) {
            float *s_re = reinterpret_cast<float *>(s_win);
            atomicAdd(s_re + ib, pr);
            atomicAdd(s_re + kWin * kAdjS + ib, pi);
        } else {
            red_grid(gb, gk1, gk2, K1, K2, pr, pi, fold);
        }
    }
}

// cell ib += (pr, pi), a contribution already formed (scaled by fs in fixed
// point here: one rounding).
template <bool DENSE, bool FIXED>
__device__ __forceinline__ void scatter_value(int *s_win, int ib, float2 *__restrict__ gb,
                                              int gk1, int gk2, int K1, int K2, int fold, float pr, float pi,
                                              float fs) {
    if (DENSE && FIXED) {
        const float re = fmaf(pr, fs, kFixMagic), im = fmaf(pi, fs, kFixMagic);
        atomicAdd(s_win + ib, int(__float_as_uint(re) - kFixMagicBits));
        atomicAdd(s_win + kWin * kAdjS + ib, int(__float_as_uint(im) - kFixMagicBits));
    } else if (DENSE) {
        float *s_re = reinterpret_cast<float *>(s_win);
        atomicAdd(s_re + ib, pr);
        atomicAdd(s_re + kWin * kAdjS + ib, pi);
    } else {
        red_grid(gb, gk1, gk2, K1, K2, pr, pi, fold);
    }
}

template <bool DENSE, bool FIXED>
__device__ __forceinline__ void scatter_rows(int i0, int nv, int lane, const int2 *s_meta, const int *s_off,
                                             const float2 *s_d, const float2 *__restrict__ fbin, int *s_win,
                                             int wy0, int wx0, float2 *__restrict__ gb, int K1, int K2, float fs,
                                             int fold) {
    constexpr unsigned FULL = 0xffffffffu;
    float2 fac = make_float2(0.f, 0.f);
    if (i0 < nv) fac = load_factors(fbin + s_off[i0], s_meta[i0].y, lane);
    for (int i = i0; i < nv; i += kWarps) {
        const int in = i + kWarps;
        float2 fnx = make_float2(0.f, 0.f);
        if (in < nv) fnx = load_factors(fbin + s_off[in], s_meta[in].y, lane);
        const int2 m = s_meta[i];
        const int T = m.y;
        const int c1 = m.x & 0xffff, c2 = (int)((unsigned)m.x >> 16);
        const float dr = s_d[i].x, di = s_d[i].y;
        if (T <= 8) {                                // warp-uniform: one row per warp
            const int g = lane >> 3, col = lane & 7;
            const bool cin = col < T;
            const float g2x = __shfl_sync(FULL, fac.x, 16 + col), g2y = __shfl_sync(FULL, fac.y, 16 + col);
            // e = conj(g2[col]) d; cell (t1, col) += conj(g1[t1]) e
            float er = fmaf(g2x, dr, g2y * di), ei = fmaf(g2x, di, -g2y * dr);
            if (FIXED) {
                er *= fs;
                ei *= fs;
            }
            int ib = 0, k2 = 0;
            if (DENSE) {
                ib = (c1 - wy0 + g) * kAdjS + (c2 - wx0 + col);
            } else {
                k2 = c2 + col;
                k2 -= (k2 >= K2) ? K2 : 0;
            }
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                if (4 * k >= T) break;                   // warp-uniform
                const int t1 = 4 * k + g;
                const float g1x = __shfl_sync(FULL, fac.x, t1), g1y = __shfl_sync(FULL, fac.y, t1);
                if ((DENSE && FIXED) || (cin && t1 < T)) {   // fixed point: the other cells add 0
                    int kk = 0;
                    if (!DENSE) {
                        kk = c1 + t1;
                        kk -= (kk >= K1) ? K1 : 0;
                    }
                    scatter_cell<DENSE, FIXED>(s_win, ib + 4 * k * kAdjS, gb, kk, k2, K1, K2, fold, g1x, g1y, er,
                                               ei);
                }
            }
        } else {
            const int half = lane >> 4, col = lane & 15;
            const bool cin = col < T;
            const float g2x = __shfl_sync(FULL, fac.x, 16 + col), g2y = __shfl_sync(FULL, fac.y, 16 + col);
            float er = fmaf(g2x, dr, g2y * di), ei = fmaf(g2x, di, -g2y * dr);
            if (FIXED) {
                er *= fs;
                ei *= fs;
            }
            int ib = 0, k2 = 0;
            if (DENSE) {
                ib = (c1 - wy0 + 2 * half) * kAdjS + (c2 - wx0 + col);
            } else {
                k2 = c2 + col;
                k2 -= (k2 >= K2) ? K2 : 0;
            }
            // steps: two per complete block of 4 box rows, then 1 or 2 for the remainder
            const int n = 2 * (T >> 2) + min(T & 3, 2);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if (k >= n) break;                       // warp-uniform
                const int dt = 4 * (k >> 1) + (k & 1);   // t1 = dt + 2 half
                const int t1 = dt + 2 * half;
                const float g1x = __shfl_sync(FULL, fac.x, t1), g1y = __shfl_sync(FULL, fac.y, t1);
                if ((DENSE && FIXED) || (cin && t1 < T)) {   // fixed point: the other cells add 0
                    int kk = 0;
                    if (!DENSE) {
                        kk = c1 + t1;
                        kk -= (kk >= K1) ? K1 : 0;
                    }
                    scatter_cell<DENSE, FIXED>(s_win, ib + dt * kAdjS, gb, kk, k2, K1, K2, fold, g1x, g1y, er,
                                               ei);
                }
            }
        }
        fac = fnx;
    }
}

// Scatter of the rows of a bin whose rows all have at most 8 taps, two rows
// per warp step: the warp's rows i0, i0 + kWarps, ... are taken in pairs
// (i, i + kWarps); half v = lane / 16 takes row i + v kWarps, lane
// (g, col) = ((lane / 8) % 2, lane % 8) its cells (t1, col) for box rows
// t1 = g, g + 2, ...  Lanes 16 v + t hold g1[t] and lanes 16 v + 8 + t hold
// g2[t] of the half's row.  The two box rows of a half's step lie 24 banks
// apart (rows of 8 cells, no conflict); the two halves' rows are unrelated
// (at most 2-way conflicts).  Per row, half the per-row work of scatter_rows.
template <bool DENSE, bool FIXED>
__device__ __forceinline__ void scatter_pairs(int i0, int nv, int lane, const int2 *s_meta, const int *s_off,
                                              const float2 *s_d, const float2 *__restrict__ fbin, int *s_win,
                                              int wy0, int wx0, float2 *__restrict__ gb, int K1, int K2, float fs,
                                              int fold) {
    constexpr unsigned FULL = 0xffffffffu;
    const int v = lane >> 4, g = (lane >> 3) & 1, col = lane & 7, hi = g;
    auto load = [&](int r) -> float2 {
        float2 x = make_float2(0.f, 0.f);
        if (r < nv) {
            const int T = s_meta[r].y;
            if (col < T) x = __ldcs(fbin + s_off[r] + hi * T + col);
        }
        return x;
    };
    float2 fac = load(i0 + v * kWarps);
    for (int i = i0; i < nv; i += 2 * kWarps) {
        const int r = i + v * kWarps;                // this half's row (may be past the end)
        const float2 fnx = load(r + 2 * kWarps);
        int T = 0, c1 = wy0, c2 = wx0;              // past the end: cells of the window, adding 0
        float dr = 0.f, di = 0.f;
        if (r < nv) {
            const int2 m = s_meta[r];
            T = m.y;
            c1 = m.x & 0xffff;
            c2 = (int)((unsigned)m.x >> 16);
            dr = s_d[r].x;
            di = s_d[r].y;
        }
        const bool cin = col < T;
        const int Tm = __reduce_max_sync(FULL, T);
        const float g2x = __shfl_sync(FULL, fac.x, 16 * v + 8 + col);
        const float g2y = __shfl_sync(FULL, fac.y, 16 * v + 8 + col);
        // e = conj(g2[col]) d; cell (t1, col) += conj(g1[t1]) e
        float er = fmaf(g2x, dr, g2y * di), ei = fmaf(g2x, di, -g2y * dr);
        if (FIXED) {
            er *= fs;
            ei *= fs;
        }
        int ib = 0, k2 = 0;
        if (DENSE) {
            ib = (c1 - wy0 + g) * kAdjS + (c2 - wx0 + col);
        } else {
            k2 = c2 + col;
            k2 -= (k2 >= K2) ? K2 : 0;
        }
        auto step = [&](int k) {
            const int t1 = 2 * k + g;
            const float g1x = __shfl_sync(FULL, fac.x, 16 * v + t1), g1y = __shfl_sync(FULL, fac.y, 16 * v + t1);
            if ((DENSE && FIXED) || (cin && t1 < T)) {   // fixed point: the other cells add 0
                int kk = 0;
                if (!DENSE) {
                    kk = c1 + t1;
                    kk -= (kk >= K1) ? K1 : 0;
                }
                scatter_cell<DENSE, FIXED>(s_win, ib + 2 * k * kAdjS, gb, kk, k2, K1, K2, fold, g1x, g1y, er,
                                           ei);
            }
        };
        // warp-uniform: rows of 7 or 8 taps (most rows without w-terms) take all four steps with no
        // test between them (branches were 13 % of the pass's instructions)
        if (Tm > 6) {
#pragma unroll
            for (int k = 0; k < 4; ++k) step(k);
        } else {
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                if (2 * k >= Tm) break;                  // warp-uniform
                step(k);
            }
        }
        fac = fnx;
    }
}

// Scatter of rows with 1 < R <= kDdeTaps separable terms (DDE rows, see
// k_nufft.cu): one row per warp as in scatter_rows; each lane sums
// conj(A_r[t1]) conj(B_r[col]) d over the terms in registers and adds each of
// its cells once.
template <bool DENSE, bool FIXED>
__device__ __forceinline__ void scatter_rows_rank(int i0, int nv, int lane, int R, const int2 *s_meta,
                                                  const int *s_off, const float2 *s_d,
                                                  const float2 *__restrict__ fbin, int *s_win,
                                                  int wy0, int wx0, float2 *__restrict__ gb, int K1, int K2,
                                                  float fs, int fold) {
    constexpr unsigned FULL = 0xffffffffu;
    const int half = lane >> 4, col = lane & 15;
    for (int i = i0; i < nv; i += kWarps) {
        const int2 m = s_meta[i];
        const int T = m.y;
        const int c1 = m.x & 0xffff, c2 = (int)((unsigned)m.x >> 16);
        const bool cin = col < T;
        const int n = 2 * (T >> 2) + min(T & 3, 2);      // steps over the box rows (as in scatter_rows)
        const float dr = s_d[i].x, di = s_d[i].y;
        float accr[8], acci[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) accr[k] = acci[k] = 0.f;
        // all terms' factors are loaded before the first is used (one memory latency per row)
        float2 facs[kDdeTaps];
#pragma unroll
        for (int r = 0; r < kDdeTaps; ++r)
            facs[r] = r < R ? load_factors(fbin + s_off[i] + r * 2 * T, T, lane) : make_float2(0.f, 0.f);
#pragma unroll
        for (int r = 0; r < kDdeTaps; ++r) {
            if (r >= R) break;
            const float2 fac = facs[r];
            const float g2x = __shfl_sync(FULL, fac.x, 16 + col), g2y = __shfl_sync(FULL, fac.y, 16 + col);
            const float er = fmaf(g2x, dr, g2y * di), ei = fmaf(g2x, di, -g2y * dr);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                if (k >= n) break;
                const int t1 = 4 * (k >> 1) + (k & 1) + 2 * half;
                const float g1x = __shfl_sync(FULL, fac.x, t1), g1y = __shfl_sync(FULL, fac.y, t1);
                accr[k] = fmaf(g1x, er, fmaf(g1y, ei, accr[k]));
                acci[k] = fmaf(g1x, ei, fmaf(-g1y, er, acci[k]));
            }
        }
        int k2 = 0;
        if (!DENSE) {
            k2 = c2 + col;
            k2 -= (k2 >= K2) ? K2 : 0;
        }
        // accumulator k holds box row 4 (k / 2) + k % 2 + 2 half: the two halves' rows of one step
        // are 2 apart, 16 banks at the window's row stride kAdjS (no conflicts)
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            if (k >= n) break;
            const int t1 = 4 * (k >> 1) + (k & 1) + 2 * half;
            if ((DENSE && FIXED) || (cin && t1 < T)) {   // fixed point: the other cells add 0
                int kk = 0;
                if (!DENSE) {
                    kk = c1 + t1;
                    kk -= (kk >= K1) ? K1 : 0;
                }
                const int ib = DENSE ? (c1 - wy0 + t1) * kAdjS + (c2 - wx0 + col) : 0;
                scatter_value<DENSE, FIXED>(s_win, ib, gb, kk, k2, K1, K2, fold, accr[k], acci[k], fs);
            }
        }
    }
}

// Columns [C0, C0 + CW) of the gather of one row by one lane:
// sum_t1 g1[t1] sum_t2 g2[t2] X[c1+t1][c2+t2], with g2 of those columns in
// registers (zero beyond T).
template <int C0, int CW, bool DENSE, bool MIR>
__device__ __forceinline__ void gather_cols(const float2 *__restrict__ f, int T, int t_lo, int t_hi, int c1, int c2,
                                            const float2 *s_grid, int wy0, int wx0, int sh,
                                            const float2 *__restrict__ gl, int K1, int K2, int hs, float &ar,
                                            float &ai) {
    float2 g2[CW];
#pragma unroll
    for (int t = 0; t < CW; ++t) g2[t] = (C0 + t < T) ? __ldg(f + T + C0 + t) : make_float2(0.f, 0.f);
    int k2[DENSE ? 1 : CW];
    if (!DENSE) {
#pragma unroll
        for (int t = 0; t < CW; ++t) {
            k2[t] = c2 + C0 + t;
            k2[t] -= (k2[t] >= K2) ? K2 : 0;
        }
    }
    for (int t1 = t_lo; t1 < t_hi; ++t1) {
        const float2 a = __ldg(f + t1);
        float br = 0.f, bi = 0.f;
        if (DENSE) {
            const float2 *row = win_cell<MIR>(s_grid, c1 - wy0 + t1, c2 - wx0 + C0, sh);
#pragma unroll
            for (int t2 = 0; t2 < CW; ++t2) {
                const float2 x = win_ld<MIR>(row, t2);
                br = fmaf(g2[t2].x, x.x, fmaf(-g2[t2].y, x.y, br));
                bi = fmaf(g2[t2].x, x.y, fmaf(g2[t2].y, x.x, bi));
            }
        } else {
            int k1 = c1 + t1;
            k1 -= (k1 >= K1) ? K1 : 0;
#pragma unroll
            for (int t2 = 0; t2 < CW; ++t2) {
                const float2 x = spec_at(gl, k1, k2[t2], K1, K2, hs);
                br = fmaf(g2[t2].x, x.x, fmaf(-g2[t2].y, x.y, br));
                bi = fmaf(g2[t2].x, x.y, fmaf(g2[t2].y, x.x, bi));
            }
        }
        ar = fmaf(a.x, br, fmaf(-a.y, bi, ar));
        ai = fmaf(a.x, bi, fmaf(a.y, br, ai));
    }
}

// Gather of one row by one lane: phi = sum_t1 g1[t1] sum_t2 g2[t2] X[c1+t1][c2+t2],
// rows t1 in [t_lo, t_hi) (g1 is zero outside).  TT >= T is the warp's
// largest side rounded to a compiled size; each entry costs one load of X and
// four FMAs with every lane busy and no reduction across lanes.  Sides above 8
// take two passes over the rows (8 columns of g2 in registers at a time, under
// the 64-register cap).
template <int C0, int TT, bool DENSE, bool MIR>
__device__ __forceinline__ void gather_chunks(const float2 *__restrict__ f, int T, int t_lo, int t_hi, int c1,
                                              int c2, const float2 *s_grid, int wy0, int wx0, int sh,
                                              const float2 *__restrict__ gl, int K1, int K2, int hs, float &ar,
                                              float &ai) {
    constexpr int CW = (TT - C0 < kGatherCols) ? TT - C0 : kGatherCols;
    gather_cols<C0, CW, DENSE, MIR>(f, T, t_lo, t_hi, c1, c2, s_grid, wy0, wx0, sh, gl, K1, K2, hs, ar, ai);
    if constexpr (C0 + CW < TT)
        gather_chunks<C0 + CW, TT, DENSE, MIR>(f, T, t_lo, t_hi, c1, c2, s_grid, wy0, wx0, sh, gl, K1, K2, hs, ar,
                                               ai);
}

// Gather of a row whose side is exactly TT (at most 8) from the shared
// window: the row's 2 TT factors are loaded at once, two per 16-byte load (a
// row's factors start on a 16-byte boundary: offsets are multiples of 2 T
// values of 8 bytes), and every loop is unrolled, so the row waits for one
// memory latency.
template <int TT, bool MIR>
__device__ __forceinline__ float2 gather_exact(const float2 *__restrict__ f, int c1, int c2, const float2 *s_grid,
                                               int wy0, int wx0, int sh) {
    static_assert(TT <= 8, "exact-side gather");
    float2 g[2 * TT];
    const float4 *f4 = reinterpret_cast<const float4 *>(f);
#pragma unroll
    for (int k = 0; k < TT; ++k) {
        const float4 q = __ldg(f4 + k);
        g[2 * k] = make_float2(q.x, q.y);
        g[2 * k + 1] = make_float2(q.z, q.w);
    }
    float ar = 0.f, ai = 0.f;
#pragma unroll
    for (int t1 = 0; t1 < TT; ++t1) {
        const float2 *row = win_cell<MIR>(s_grid, c1 - wy0 + t1, c2 - wx0, sh);
        float br = 0.f, bi = 0.f;
#pragma unroll
        for (int t2 = 0; t2 < TT; ++t2) {
            const float2 x = win_ld<MIR>(row, t2);
            const float2 b = g[TT + t2];
            br = fmaf(b.x, x.x, fmaf(-b.y, x.y, br));
            bi = fmaf(b.x, x.y, fmaf(b.y, x.x, bi));
        }
        const float2 a = g[t1];
        ar = fmaf(a.x, br, fmaf(-a.y, bi, ar));
        ai = fmaf(a.x, bi, fmaf(a.y, br, ai));
    }
    return make_float2(ar, ai);
}

template <int TT, bool DENSE, bool MIR>
__device__ __forceinline__ float2 gather_lane(const float2 *__restrict__ f, int T, int t_lo, int t_hi, int c1,
                                              int c2, const float2 *s_grid, int wy0, int wx0, int sh,
                                              const float2 *__restrict__ gl, int K1, int K2, int hs) {
    float ar = 0.f, ai = 0.f;
    gather_chunks<0, TT, DENSE, MIR>(f, T, t_lo, t_hi, c1, c2, s_grid, wy0, wx0, sh, gl, K1, K2, hs, ar, ai);
    return make_float2(ar, ai);
}

// Gather of a row with R separable terms (term r at offset 2 T r).  With
// R > 1 (DDE rows) the first factor of term r is the base factor shifted by
// r, nonzero only on rows [r, r + T - R + 1), so the other rows are skipped.
template <int TT, bool DENSE, bool MIR>
__device__ __forceinline__ float2 gather_terms(const float2 *__restrict__ f, int T, int R, int c1, int c2,
                                               const float2 *s_grid, int wy0, int wx0, int sh,
                                               const float2 *__restrict__ gl, int K1, int K2, int hs) {
    if (R == 1) return gather_lane<TT, DENSE, MIR>(f, T, 0, T, c1, c2, s_grid, wy0, wx0, sh, gl, K1, K2, hs);
    const int Tb = T - R + 1;
    float2 phi = make_float2(0.f, 0.f);
#pragma unroll 1
    for (int r = 0; r < R; ++r) {
        const float2 t =
            gather_lane<TT, DENSE, MIR>(f + r * 2 * T, T, r, r + Tb, c1, c2, s_grid, wy0, wx0, sh, gl, K1, K2, hs);
        phi.x += t.x;
        phi.y += t.y;
    }
    return phi;
}

// Phase 1 of a bin: one row per thread (rows are sorted by T inside each tile
// run, so a warp's rows mostly share T).  kDual: the data-dual pre-update
// d = s_b d + sigma2 (phi - y) (s_b of the row's block) into s_d and the
// output, |d|^2 into s_n2 for the block norms; kGather: phi to the output;
// kNormal: phi into s_d for the scatter.  s_off: each row's factor offset
// from fbin, s_v: its visibility index, s_pc: its piece (block) in the bin.
template <int MODE, bool DENSE, bool MIR>
__device__ __forceinline__ void gather_phase(int nv, int R, const int2 *s_meta, const int *s_off,
                                             const long long *s_v,
                                             const float2 *s_y, float2 *s_d, float *s_n2,
                                             const float2 *__restrict__ fbin, const float2 *s_grid,
                                             int wy0, int wx0, int sh, const float2 *__restrict__ gl, int K1, int K2,
                                             int hs,
                                             float sigma2, float2 *__restrict__ dvis) {
    const int nvr = (nv + 31) & ~31;                 // whole warps: the max below takes every lane
    for (int i = threadIdx.x; i < nvr; i += blockDim.x) {
        const bool valid = i < nv;
        int T = 0, c1 = wy0, c2 = wx0;                   // past the end: the window origin, nothing read
        const float2 *f = fbin;
        if (valid) {
            const int2 m = s_meta[i];
            T = m.y;
            c1 = m.x & 0xffff;
            c2 = (int)((unsigned)m.x >> 16);
            f = fbin + s_off[i];
        }
        const int tm = __reduce_max_sync(0xffffffffu, T);
        // every valid row of the warp has side tm (7 or 8), one term, window in shared memory
        const bool exact = DENSE && R == 1 && (tm == 7 || tm == 8) &&
                           __reduce_min_sync(0xffffffffu, valid ? T : 16) == tm;
        float2 phi;
        if (exact) {
            // rows past the end take no part (the exact gather reads every cell of its box)
            phi = make_float2(0.f, 0.f);
            if (valid)
                phi = tm == 7 ? gather_exact<7, MIR>(f, c1, c2, s_grid, wy0, wx0, sh)
                              : gather_exact<8, MIR>(f, c1, c2, s_grid, wy0, wx0, sh);
        }
        else if (tm <= 4) phi = gather_terms<4, DENSE, MIR>(f, T, R, c1, c2, s_grid, wy0, wx0, sh, gl, K1, K2, hs);
        else if (tm <= 7) phi = gather_terms<7, DENSE, MIR>(f, T, R, c1, c2, s_grid, wy0, wx0, sh, gl, K1, K2, hs);
        else if (tm <= 9) phi = gather_terms<9, DENSE, MIR>(f, T, R, c1, c2, s_grid, wy0, wx0, sh, gl, K1, K2, hs);
        else if (tm <= 11) phi = gather_terms<11, DENSE, MIR>(f, T, R, c1, c2, s_grid, wy0, wx0, sh, gl, K1, K2, hs);
        else if (tm <= 13) phi = gather_terms<13, DENSE, MIR>(f, T, R, c1, c2, s_grid, wy0, wx0, sh, gl, K1, K2, hs);
        else phi = gather_terms<16, DENSE, MIR>(f, T, R, c1, c2, s_grid, wy0, wx0, sh, gl, K1, K2, hs);
        if (!valid) continue;
        if (MODE == kDual) {
            const float2 dold = s_d[i];
            const float2 sy = s_y[i];
            const float sc = s_n2[i];                 // the row's block factor s_b, staged by this thread
            const float dr = fmaf(sc, dold.x, fmaf(sigma2, phi.x, -sy.x));
            const float di = fmaf(sc, dold.y, fmaf(sigma2, phi.y, -sy.y));
            dvis[s_v[i]] = make_float2(dr, di);
            s_d[i] = make_float2(dr, di);
            s_n2[i] = fmaf(dr, dr, di * di);
        } else if (MODE == kGather) {
            dvis[s_v[i]] = phi;
        } else {
            s_d[i] = phi;
        }
    }
}

// Window staging by the tensor memory accelerator: two 3-D boxes (kBoxW x
// kBoxH row pairs x 1 channel: the window's even rows and its odd rows) of
// the forward grid into shared memory, completion counted on one mbarrier.
// Used for windows that do not wrap around the grid edge (wrapped windows,
// and those that straddle the stored half of a half grid, take per-thread
// copies).
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void window_tma(float2 *dst, const CUtensorMap *tmap, int x0, int y0, int x1, int y1,
                                           int z, uint64_t *bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(int(sizeof(float2) * 2 * kBoxCells))
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x0), "r"(y0), "r"(z), "r"(smem_addr(bar))
        : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(smem_addr(dst + kBoxCells)), "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x1), "r"(y1), "r"(z),
          "r"(smem_addr(bar))
        : "memory");
}

// Bounded wait for phase 0 of the window barrier: at most max_polls polls
// (each try_wait may suspend the thread for a hardware-defined interval);
// false if it gave up.  With `err` given it also gives up once another CTA
// has recorded a timeout there (checked every 4096 polls), so that a failure
// costs the launch one wait limit, not one per CTA.
constexpr int kWindowPolls = 1 << 24;
__device__ __forceinline__ bool window_wait(uint64_t *bar, int max_polls = kWindowPolls, const int *err = nullptr) {
    const uint32_t a = smem_addr(bar);
    for (int it = 0; it < max_polls; ++it) {
        if (err && (it & 4095) == 4095 && *reinterpret_cast<const volatile int *>(err) != 0) return false;
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(a)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// CTAs per SM of the gathering passes (4: 64 registers, what the 8-column
// chunks need without spills).  Problems whose rows nearly all have at most 8
// taps (no w-terms) run the dual and gather passes at 5 (48 registers, no
// spills): 8 % faster there, 10 % slower on rows of up to 16 taps.
#ifndef FHS_GATHER_MIN_BLOCKS
#define FHS_GATHER_MIN_BLOCKS 4
#endif
constexpr int kGatherMinBlocks = FHS_GATHER_MIN_BLOCKS;
constexpr int kGatherMinBlocksNarrow = 5;
// MODE kDual: dvis is the data dual d (read and written), grid the forward
// grid, blk_scale the factors s_b of the previous iteration, blk_norm2 receives
// ||d_b||^2.  kGather: dvis receives Phi x, grid is the forward grid.
// kScatter: dvis holds the visibilities, scaled by blk_scale[segment] when
// blk_scale is given (the data term's v = s_b d), grid_out the per-channel
// output grids.  kNormal: grid is the forward grid, grid_out the per-channel
// output grids, dvis unused.
// MULTI: rows of R > 1 separable terms (DDE rows); otherwise R is 1 and the
// term loops compile away.  Multi-term rows keep 3 CTAs per SM (80 registers:
// their term accumulators spill under the 64-register cap); the single-term
// scatter pass runs 6 CTAs per SM (40 registers, no spills: 3.5 % faster than
// 5, while 8 spills).
// NARROW: the occupancy of problems whose rows nearly all have at most 8 taps (the same code).
template <int MODE, bool MULTI, bool NARROW = false>
__global__ void __launch_bounds__(256, MULTI ? 3
                                             : (MODE == kScatter ? 6
                                                                 : (NARROW ? kGatherMinBlocksNarrow : kGatherMinBlocks)))
    degrid_grid_binned_kernel(
    const int2 *__restrict__ meta, const long long *__restrict__ fptr, const float2 *__restrict__ gfac,
    const float2 *__restrict__ y, float2 *__restrict__ dvis, int slots,
    const long long *__restrict__ bin_fbase, const long long *__restrict__ piece_start, const int *__restrict__ piece_len, const int *__restrict__ piece_blk,
    const int *__restrict__ bin_chan, const int *__restrict__ bin_tile, int ntx, int B,
    const float *__restrict__ blk_scale, double *__restrict__ blk_norm2, const float2 *__restrict__ grid,
    float2 *__restrict__ grid_out, long long in_cs, int in_hs, long long out_cs, int K1, int K2, float sigma2,
    int R_, const __grid_constant__ CUtensorMap tmap, int use_tma, const float *__restrict__ gmax, int allow_fixed,
    int fold, int bin0, int *__restrict__ err) {
    const int R = MULTI ? R_ : 1;
    __shared__ alignas(128) float2 s_grid[2 * kBoxCells];   // forward window: even rows, then odd rows
    __shared__ alignas(8) uint64_t s_bar;
    __shared__ alignas(16) int s_win[2 * kWin * kAdjS];   // adjoint window planes, row stride kAdjS
    __shared__ int2 s_meta[kBinMax];
    __shared__ int s_off[kBinMax];        // factor offset of each row from the bin's base
    __shared__ long long s_v[kBinMax];    // visibility (sorted) index of each row
    __shared__ unsigned char s_pc[kBinMax];  // piece of the bin each row belongs to
    __shared__ float2 s_y[kBinMax];       // sigma2 * y
    __shared__ float2 s_d[kBinMax];
    __shared__ float s_n2[kBinMax];       // |d|^2 of each row (block norms)
    __shared__ long long s_pstart[kMaxPieces];
    __shared__ int s_pcum[kMaxPieces + 1];
    __shared__ int s_pblk[kMaxPieces];
    __shared__ double s_pnb[kMaxPieces];  // block norm of each piece
    __shared__ int s_bound, s_bad;        // fixed-point scatter: bin bound (float bits), non-finite flag
    __shared__ int s_tmax;                // largest box side of the bin (scatter)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bin = bin0 + blockIdx.x;
    const int l = bin_chan[bin];
    const int tile = bin_tile[bin];
    // input grid: channel stride in_cs, full (in_hs = 0) or half layout; output grid: channel stride
    // out_cs, full, or half with the folded adjoint (fold = its row stride)
    const float2 *gl = grid + (long long)l * in_cs;
    float2 *gb = (MODE == kScatter || MODE == kNormal) ? grid_out + (long long)l * out_cs : nullptr;
    const bool dense = tile >= 0;
    int wy0 = 0, wx0 = 0;
    if (dense) {
        wy0 = (tile / ntx) * kTile;
        wx0 = (tile % ntx) * kTile;
    }
    // the window by TMA, issued first so that it overlaps the staging of the rows, when it does not
    // wrap: directly when it lies in the stored columns, or (half grids) as the conjugate-symmetric
    // block when it lies wholly in the other half.  The grid is read as rows of pairs of rows (row
    // stride rs, 2 rs per pair): the even rows' box at column x0, the odd rows' at rs + x0 less sh
    // (x coordinates even: 16-byte aligned).
    const int rs = in_hs ? in_hs : K2, sh = rs & 1, hcol = K2 >> 1;
    bool tma = false, mir = false;
    int bx0 = 0, by0 = 0, bx1 = 0, by1 = 0;
    if (MODE != kScatter && use_tma && dense && wy0 + kWin <= K1) {
        if (wx0 + kWin - 1 <= (in_hs ? hcol : K2 - 1)) {
            tma = true;
            bx0 = wx0;
            bx1 = rs + wx0 - sh;
            by0 = by1 = wy0 >> 1;
        } else if (in_hs && wx0 > hcol && wx0 + kWin <= K2 && wy0 > 0) {
            // rows K1 - wy0 - rr, columns K2 - wx0 - cc: both in range, no wrap
            tma = mir = true;
            bx0 = K2 - wx0 - (kWin - 1);
            bx1 = rs + K2 - wx0 - (kWin - 1) - sh;
            by0 = ((K1 - wy0) >> 1) - (kBoxH - 1);
            by1 = ((K1 - wy0) >> 1) - kBoxH;
        }
    }
    const int wsh = tma ? sh : 0;                  // odd-row shift of the window layout
    if (tma && threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&s_bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        window_tma(s_grid, &tmap, bx0, by0, bx1, by1, l, &s_bar);
    }
    // otherwise by per-thread asynchronous 8-byte copies, issued now for the same overlap; cells of
    // a half grid's other half come from -k (conjugated once they have arrived)
    const bool acopy = MODE != kScatter && dense && !tma;
    if (acopy) {
        // one window row per warp step, its cells over the lanes (row terms computed once)
        const int h = K2 >> 1;
        for (int r = warp; r < kWin; r += kWarps) {
            int k1 = wy0 + r;
            while (k1 >= K1) k1 -= K1;
            const float2 *rd = gl + (long long)k1 * (in_hs ? in_hs : K2);          // row k1
            const float2 *rm = gl + (long long)(k1 ? K1 - k1 : 0) * in_hs + K2;    // row -k1, + K2
            const uint32_t dst = smem_addr(&s_grid[(r & 1) * kBoxCells + (r >> 1) * kBoxW]);
            for (int c = lane; c < kWin; c += 32) {
                int k2 = wx0 + c;
                while (k2 >= K2) k2 -= K2;
                const float2 *src = (!in_hs || k2 <= h) ? rd + k2 : rm - k2;
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst + 8u * c), "l"(src) : "memory");
            }
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    // the bin's pieces: runs of rows of one block each, in the order of their blocks.  Warp 0 loads
    // the slots and scans their lengths by shuffles (slots <= kMaxPieces <= 32): one barrier
    // between the slot loads and the rows' loads
    const long long pp0 = (long long)bin * slots;
    const long long fb = bin_fbase[bin];       // factor offset of the bin's first row (the smallest)
    const int np = slots;                     // pieces of length 0 in unused slots
    if (warp == 0) {
        int len = 0;
        if (lane < np) {
            s_pstart[lane] = piece_start[pp0 + lane];
            s_pblk[lane] = piece_blk[pp0 + lane];
            s_pnb[lane] = 0.0;
            len = piece_len[pp0 + lane];
        }
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, len, o);
            if (lane >= o) len += t;
        }
        if (lane < np) s_pcum[lane + 1] = len;
        if (lane == 0) {
            s_pcum[0] = 0;
            s_bound = 0;
            s_bad = 0;
            s_tmax = 0;
        }
    }
    __syncthreads();
    const int nv = s_pcum[np];
    int tmax = 0;                        // largest box side among this thread's rows
    for (int i = threadIdx.x; i < nv; i += blockDim.x) {
        int q = 0;
        while (i >= s_pcum[q + 1]) ++q;
        const long long v = s_pstart[q] + (i - s_pcum[q]);
        const int2 mv = meta[v];
        s_meta[i] = mv;
        tmax = max(tmax, mv.y);
        s_off[i] = int(fptr[v] - fb);
        s_pc[i] = (unsigned char)q;
        if (MODE == kDual || MODE == kGather) s_v[i] = v;
        // the block factor s_b of the row's block, loaded with the row (not before the barrier)
        const float vsc = ((MODE == kDual || MODE == kScatter) && blk_scale) ? blk_scale[l * B + s_pblk[q]] : 1.f;
        if (MODE == kDual) {
            const float2 yy = y[v];
            s_y[i] = make_float2(sigma2 * yy.x, sigma2 * yy.y);
            s_d[i] = dvis[v];
            s_n2[i] = vsc;                    // read (then replaced by |d|^2) by this thread's gather
        }
        if (MODE == kScatter) {
            const float2 dd = dvis[v];
            s_d[i] = make_float2(vsc * dd.x, vsc * dd.y);
        }
        if ((MODE == kScatter || MODE == kNormal) && dense && allow_fixed) s_n2[i] = gmax[v];
    }
    if (MODE == kScatter || MODE == kNormal) {
        tmax = __reduce_max_sync(0xffffffffu, tmax);
        if (lane == 0 && tmax > 0) atomicMax(&s_tmax, tmax);
    }
    if (dense && MODE != kGather && MODE != kDual) {
        int4 *w4 = reinterpret_cast<int4 *>(s_win);
        for (int i = threadIdx.x; i < 2 * kWin * kAdjS / 4; i += blockDim.x) w4[i] = make_int4(0, 0, 0, 0);
    }
    if (acopy) asm volatile("cp.async.wait_all;" ::: "memory");
    // A thread gathers the rows it staged (row i by thread i mod blockDim), so the gathers wait on no
    // barrier for them, and the TMA window is waited for on its mbarrier (initialised before the
    // barrier above).  The scatter's warps take other threads' rows and the zeroed window, and the
    // per-thread window copies fill cells that other threads read: those wait here.
    if (MODE == kScatter || acopy) __syncthreads();
    if (tma && !window_wait(&s_bar, kWindowPolls, err)) {
        // the copy did not complete in time: record it, then wait once more (bounded) so that
        // no copy into this CTA's shared memory is still in flight when it moves on
        if (threadIdx.x == 0) atomicExch(err, 2);
        window_wait(&s_bar, kWindowPolls, err);
    }
    // conjugate the window's cells that came from -k (columns past K2/2 of a half grid)
    if (acopy && in_hs && wx0 + kWin - 1 > (K2 >> 1)) {
        for (int r = warp; r < kWin; r += kWarps)
            for (int c = lane; c < kWin; c += 32) {
                int k2 = wx0 + c;
                while (k2 >= K2) k2 -= K2;
                float2 &x = s_grid[(r & 1) * kBoxCells + (r >> 1) * kBoxW + c];
                if (k2 > (K2 >> 1)) x.y = -x.y;
            }
        __syncthreads();
    }
    const float2 *fbin = gfac + fb;
    // phase 1: gathers, one row per thread
    if (MODE != kScatter) {
        if (dense && mir)
            gather_phase<MODE, true, true>(nv, R, s_meta, s_off, s_v, s_y, s_d, s_n2, fbin, s_grid, wy0,
                                           wx0, wsh, gl, K1, K2, in_hs, sigma2, dvis);
        else if (dense)
            gather_phase<MODE, true, false>(nv, R, s_meta, s_off, s_v, s_y, s_d, s_n2, fbin, s_grid, wy0,
                                            wx0, wsh, gl, K1, K2, in_hs, sigma2, dvis);
        else
            gather_phase<MODE, false, false>(nv, R, s_meta, s_off, s_v, s_y, s_d, s_n2, fbin, s_grid,
                                             wy0, wx0, wsh, gl, K1, K2, in_hs, sigma2, dvis);
    }
    // phase 2: scatters of conj(G_i) s_d[i], one row per warp
    bool fixed = false;
    float fs = 1.f, finv = 1.f;
    if (MODE == kScatter || MODE == kNormal) {
        if (MODE == kNormal) __syncthreads();        // s_d holds the gathered values
        // fixed point in the scatter when the caller allows it (Phi^H, the data term's scatter pass,
        // the normal-mode pass of the norm estimate); the passes of the data reduction keep the
        // float atomics: their output is weighted by Lambda and the faint, sparsely covered cells
        // need their own relative precision, which a quantum set by the bin's brightest
        // contribution does not give
        if (dense && allow_fixed) {
            // the bin's bound of |contribution|: max_i |s_d[i]| max|g1_i| max|g2_i|
            float m = 0.f;
            bool bad = false;
            for (int i = threadIdx.x; i < nv; i += blockDim.x) {
                const float2 d = s_d[i];
                bad |= !(isfinite(d.x) && isfinite(d.y));
                m = fmaxf(m, sqrtf(fmaf(d.x, d.x, d.y * d.y)) * s_n2[i]);    // s_n2: the rows' bounds here
            }
            if (m > 0.f) atomicMax(&s_bound, __float_as_int(m));   // non-negative floats order as integers
            if (bad) s_bad = 1;
            __syncthreads();
            const float bound = __int_as_float(s_bound);
            int e = 0;
            if (bound > 0.f) frexpf(bound, &e);             // bound < 2^e
            // fixed point unless a value is not finite or the bin is so faint (bound < 2^-100)
            // that 2^(22 - e) would overflow: those bins keep the float atomics
            if (!s_bad && isfinite(bound) && e >= -100) {
                fixed = true;
                fs = ldexpf(1.f, kFixBits - e);
                finv = ldexpf(1.f, e - kFixBits);
            }
        }
        if (MULTI) {
            if (dense && fixed)
                scatter_rows_rank<true, true>(warp, nv, lane, R, s_meta, s_off, s_d, fbin, s_win, wy0, wx0, gb,
                                              K1, K2, fs, fold);
            else if (dense)
                scatter_rows_rank<true, false>(warp, nv, lane, R, s_meta, s_off, s_d, fbin, s_win, wy0, wx0, gb,
                                               K1, K2, fs, fold);
            else
                scatter_rows_rank<false, false>(warp, nv, lane, R, s_meta, s_off, s_d, fbin, s_win, wy0, wx0, gb,
                                                K1, K2, fs, fold);
        } else if (s_tmax <= 8) {
            // every row of the bin has at most 8 taps: two rows per warp step
            if (dense && fixed)
                scatter_pairs<true, true>(warp, nv, lane, s_meta, s_off, s_d, fbin, s_win, wy0, wx0, gb, K1, K2,
                                          fs, fold);
            else if (dense)
                scatter_pairs<true, false>(warp, nv, lane, s_meta, s_off, s_d, fbin, s_win, wy0, wx0, gb, K1, K2,
                                           fs, fold);
            else
                scatter_pairs<false, false>(warp, nv, lane, s_meta, s_off, s_d, fbin, s_win, wy0, wx0, gb, K1,
                                            K2, fs, fold);
        } else if (dense && fixed)
            scatter_rows<true, true>(warp, nv, lane, s_meta, s_off, s_d, fbin, s_win, wy0, wx0, gb, K1, K2, fs, fold);
        else if (dense)
            scatter_rows<true, false>(warp, nv, lane, s_meta, s_off, s_d, fbin, s_win, wy0, wx0, gb, K1, K2, fs, fold);
        else
            scatter_rows<false, false>(warp, nv, lane, s_meta, s_off, s_d, fbin, s_win, wy0, wx0, gb, K1, K2,
                                       fs, fold);
    }
    if (MODE != kDual) {
        if ((MODE == kScatter || MODE == kNormal) && dense) {
            __syncthreads();
            // a box starts in the tile and spans at most s_tmax cells: only the window's first
            // kTile + s_tmax - 1 rows and columns can hold a contribution (one window row per warp
            // step, its cells over the lanes)
            const int ext = min(kWin, kTile + s_tmax - 1);
            int k2a = wx0 + lane, k2b = wx0 + lane + 32;
            while (k2a >= K2) k2a -= K2;
            while (k2b >= K2) k2b -= K2;
            for (int r = warp; r < ext; r += kWarps) {
                int k1 = wy0 + r;
                while (k1 >= K1) k1 -= K1;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int c = lane + 32 * h;
                    if (c >= ext) break;
                    float re, im;
                    if (fixed) {
                        const int ir = s_win[r * kAdjS + c], ii = s_win[kWin * kAdjS + r * kAdjS + c];
                        re = float(ir) * finv;                    // exact scaling by a power of two
                        im = float(ii) * finv;
                    } else {
                        const float *s_re = reinterpret_cast<const float *>(s_win);
                        re = s_re[r * kAdjS + c];
                        im = s_re[kWin * kAdjS + r * kAdjS + c];
                    }
                    if (re != 0.f || im != 0.f) red_grid(gb, k1, h ? k2b : k2a, K1, K2, re, im, fold);
                }
            }
        }
        return;
    }
    // block norms ||d_b||^2: the rows are ordered by piece (one block each), so every 32 rows
    // reduce in FP32 per piece (segmented, towards the first row of each piece), then in FP64
    __syncthreads();
    for (int base = warp * 32; base < nv; base += blockDim.x) {
        const int i = base + lane;
        const bool ok = i < nv;
        float v = ok ? s_n2[i] : 0.f;
        const int pc = ok ? int(s_pc[i]) : -1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float t = __shfl_down_sync(0xffffffffu, v, o);
            const int q = __shfl_down_sync(0xffffffffu, pc, o);
            if (lane + o < 32 && q == pc) v += t;
        }
        const int prev = __shfl_up_sync(0xffffffffu, pc, 1);
        if (ok && (lane == 0 || prev != pc)) atomicAdd(&s_pnb[pc], double(v));
    }
    __syncthreads();
    if (threadIdx.x < np && s_pnb[threadIdx.x] != 0.0)
        atomicAdd(blk_norm2 + l * B + s_pblk[threadIdx.x], s_pnb[threadIdx.x]);
}

// Test aid for the failure path: one thread waits, with the window wait of
// the pass over G, on an mbarrier that expects one arrival that never comes.
// The wait gives up after max_polls polls and records the code a timed-out
// window copy records (2); the kernel then returns.  Nothing is copied, so no
// transfer can be in flight when the CTA exits.
__global__ void unsatisfied_wait_kernel(int max_polls, int *__restrict__ err) {
    __shared__ alignas(8) uint64_t s_bar;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&s_bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0 && !window_wait(&s_bar, max_polls)) atomicExch(err, 2);
}

}  // namespace

cudaError_t launch_unsatisfied_wait(fhs_problem *p, int max_polls, cudaStream_t s) {
    unsatisfied_wait_kernel<<<1, 32, 0, s>>>(max_polls, p->dev_err);
    p->n_launch += 1;
    return cudaGetLastError();
}

// Tensor map of a [L][K1][row stride] complex grid (full: K2, half: hs) for
// the window staging, viewed as [L][K1 / 2][2 x row stride] (pairs of rows:
// the pair stride is a multiple of 16 bytes); 8-byte elements, box kBoxW x
// kBoxH x 1.  The encoder comes from the driver entry point; ok = 0
// (per-thread staging) if it is unavailable or refuses the map.
struct WindowMap {
    CUtensorMap map;
    int ok = 0;
};

static WindowMap window_map(const fhs_problem *p, const float2 *grid, bool half) {
    static PFN_cuTensorMapEncodeTiled_v12000 enc = [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            fn = nullptr;
        }
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }();
    WindowMap w{};
    const int rs = half ? p->HS : p->K2;
    if (!enc || !grid || p->K1 < kWin || p->K1 % 2 != 0 || 2 * rs < kBoxW) return w;
    const cuuint64_t dims[3] = {cuuint64_t(2) * rs, cuuint64_t(p->K1 / 2), cuuint64_t(p->L)};
    const cuuint64_t strides[2] = {cuuint64_t(2) * rs * sizeof(float2), cuuint64_t(p->K1) * rs * sizeof(float2)};
    const cuuint32_t box[3] = {cuuint32_t(kBoxW), cuuint32_t(kBoxH), 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    w.ok = enc(&w.map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<float2 *>(grid), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    return w;
}

// One launch of the pass over G in mode MODE, one CTA per bin.
template <int MODE>
// in_half: the input grid is a half grid (a forward spectrum); fold: the output is the folded
// adjoint in a half grid (otherwise a full grid).
// Bins [bin0, bin0 + nbin) (all with nbin < 0).
cudaError_t launch_pass(fhs_problem *p, const float2 *y, float2 *dvis, const float *blk_scale, double *blk_norm2,
                        const float2 *grid, bool in_half, float2 *grid_out, bool fold, float sigma2,
                        const WindowMap &tm, int allow_fixed, cudaStream_t s, int bin0 = 0, int nbin = -1) {
    if (nbin < 0) nbin = p->n_bin;
    if (nbin == 0) return cudaSuccess;
    const long long in_cs = in_half ? p->KH : p->K, out_cs = fold ? p->KH : p->K;
    auto kern = p->rank > 1 ? degrid_grid_binned_kernel<MODE, true> : degrid_grid_binned_kernel<MODE, false>;
    if constexpr (MODE == kDual || MODE == kGather)
        if (p->rank == 1 && p->narrow_rows) kern = degrid_grid_binned_kernel<MODE, false, true>;
    kern<<<nbin, 256, 0, s>>>(
        p->meta, p->fptr, p->gfac, y, dvis, p->bin_slots, p->bin_fbase, p->piece_start, p->piece_len, p->piece_blk,
        p->bin_chan, p->bin_tile, p->ntx, p->B, blk_scale, blk_norm2, grid, grid_out, in_cs, in_half ? p->HS : 0,
        out_cs, p->K1, p->K2, sigma2, p->rank, tm.map, tm.ok, p->gmax, allow_fixed, fold ? p->HS : 0, bin0,
        p->dev_err);
    p->n_launch += 1;
    return cudaGetLastError();
}

cudaError_t launch_degrid(fhs_problem *p, const float2 *grid, float2 *vis_sorted, cudaStream_t s) {
    if (p->n_bin == 0) return cudaSuccess;
    return launch_pass<kGather>(p, nullptr, vis_sorted, nullptr, nullptr, grid, true, nullptr, false, 0.f,
                                window_map(p, grid, true), 0, s);
}

cudaError_t launch_grid(fhs_problem *p, const float2 *vis_sorted, float2 *grid, cudaStream_t s, bool fixed,
                        bool fold) {
    return launch_pass<kScatter>(p, nullptr, const_cast<float2 *>(vis_sorted), nullptr, nullptr, nullptr, false,
                                 grid, fold, 0.f, WindowMap{}, fixed ? 1 : 0, s);
}

cudaError_t launch_normal(fhs_problem *p, const float2 *grid, bool in_half, float2 *grid_out, cudaStream_t s,
                          bool fixed, bool fold, int bin0, int nbin) {
    if (p->n_bin == 0) return cudaSuccess;
    return launch_pass<kNormal>(p, nullptr, nullptr, nullptr, nullptr, grid, in_half, grid_out, fold, 0.f,
                                window_map(p, grid, in_half), fixed ? 1 : 0, s, bin0, nbin);
}

// The data term in two passes: the dual pre-update with the block norms
// (kDual), then, once the l2-ball factors s_b are known, the scatter of
// s_b d into the channel grids (kScatter with blk_scale), with no per-block
// grids to combine.
cudaError_t launch_data_dual(fhs_problem *p, cudaStream_t s) {
    if (p->n_bin == 0) return cudaSuccess;
    return launch_pass<kDual>(p, p->y, p->dvis, p->blk_scale, p->blk_norm2, p->grid_work, true, nullptr, false,
                              float(p->sigma2), window_map(p, p->grid_work, true), 0, s);
}

cudaError_t launch_data_scatter(fhs_problem *p, cudaStream_t s) {
    return launch_pass<kScatter>(p, nullptr, p->dvis, p->blk_scale, nullptr, nullptr, false, p->grid_work, true, 0.f,
                                 WindowMap{}, 1, s);
}

}  // namespace fhs
