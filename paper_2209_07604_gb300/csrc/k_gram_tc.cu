// Facet Gram matrices of the nuclear-norm dual step (Sec. 2.2.2) on the
// 5th-generation tensor cores: G_q = Z_q^T Z_q with Z_q = P_q + sigma0 S_q xbar
// (facet pixels x L_c channels), inputs rounded to TF32 or BF16, products
// accumulated in FP32 in tensor memory, CTA partial sums added in FP64.
//
// One CTA takes kPixTc pixels of one (sub-cube, facet).  Its four warps write
// Z for a stage of pixels into shared memory in the K-major core-matrix
// layout (8 rows x 16 bytes per core matrix; K = pixels, rows = channels);
// one thread issues tcgen05.mma with A = Z^T (M = 128 rows, channels >= L_c
// kept zero) and B = the same rows as Z (N = 32), D in TMEM; a commit to an
// mbarrier per stage frees the stage for the next fill (two stages).  Every
// wait is bounded: on a timeout the kernel records an error, skips the rest
// and still releases its tensor memory.
#include "fhs_internal.h"

#include <cstdint>
#include <cuda_bf16.h>

namespace fhs {

namespace {

constexpr int kPixTc = 2048;               // facet pixels per CTA
constexpr int kStageBytes = 128 * 128;     // 128 rows x 128 bytes of K per stage
constexpr int kTcThreads = 128;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor, no swizzle, K-major: LBO = byte distance of
// core matrices adjacent in K, SBO = of 8-row groups adjacent in M/N.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);
    d |= static_cast<uint64_t>((lbo >> 4) & 0x3FFFu) << 16;
    d |= static_cast<uint64_t>((sbo >> 4) & 0x3FFFu) << 32;
    d |= static_cast<uint64_t>(1) << 46;     // descriptor version of tcgen05
    return d;                                // base offset 0, swizzle none
}

// Instruction descriptor: D F32, A and B of format fmt (TF32 = 2 for
// kind::tf32, BF16 = 1 for kind::f16), both K-major, M x N.
__host__ __device__ constexpr uint32_t instr_desc(uint32_t fmt, uint32_t M, uint32_t N) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    for (int it = 0; it < (1 << 22); ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

template <int KIND>   // 0: kind::tf32, 1: kind::f16 (BF16 inputs)
__device__ __forceinline__ void umma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    if (KIND == 0)
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
            : "memory");
    else
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
            : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 TMEM lanes x 32 columns of 32 bits: lane i of the warp receives row
// (lane base + i), columns [col, col + 32).
__device__ __forceinline__ void tmem_ld_32x32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t to_tf32(float v) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
    return r;
}

// KIND 0: TF32, 32 pixels per stage (4 pixels per 16-byte core row);
// KIND 1: BF16, 64 pixels per stage (8 per core row).  Four MMAs per stage
// (K = 8 TF32 or 16 BF16 values = two core matrices each).
template <int KIND>
__global__ void __launch_bounds__(kTcThreads) gram_tc_kernel(const float *__restrict__ P, const float *__restrict__ img,
                                                            const int4 *__restrict__ facets,
                                                            const long long *__restrict__ nuc_off, int Q, int C,
                                                            int Lc, int nx, long long N, float s0,
                                                            double *__restrict__ gram, int *__restrict__ err) {
    constexpr int KS = KIND == 0 ? 32 : 64;             // pixels per stage
    __shared__ __align__(1024) uint8_t s_stage[2][kStageBytes];
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    const int cq = blockIdx.y;
    const int c = cq / Q, q = cq - c * Q;
    const int4 f = facets[q];
    const int wx = f.w - f.z;
    const int npix = (f.y - f.x) * wx;
    const int p0 = blockIdx.x * kPixTc;
    if (p0 >= npix) return;                              // before any TMEM is held
    const int p1 = min(npix, p0 + kPixTc);
    const int n_stage = (p1 - p0 + KS - 1) / KS;
    const float *Pq = P + nuc_off[cq];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // zero both stages (rows >= 32 stay zero: the padding of M = 128)
    for (int e = tid; e < 2 * kStageBytes / 16; e += kTcThreads)
        reinterpret_cast<uint4 *>(&s_stage[0][0])[e] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        mbar_init(&s_bar[0]);
        mbar_init(&s_bar[1]);
        s_fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" ::"r"(smem_u32(&s_tmem))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = s_tmem;
    constexpr uint32_t idesc = instr_desc(KIND == 0 ? 2u : 1u, 128u, 32u);

    // Thread (warp w, lane) owns channel row j = 8 w + lane / 4 of every stage
    // and the 16-byte slot lane % 4 of each K column kq: TF32 pixels
    // 4 kq + lane % 4, BF16 pixels 8 kq + 2 (lane % 4) + {0, 1}.  Two register
    // sets take turns: the global loads of stage it + 1 are in flight while
    // stage it is written and its MMAs are issued.
    constexpr int VPT = KIND == 0 ? 8 : 16;             // values per thread per stage
    const int j = (warp << 3) | (lane >> 2);
    const bool jv = j < Lc;
    const float *imgj = img + (long long)(c + (jv ? j : 0) * C) * N;
    const float *Pj = Pq + (long long)(jv ? j : 0) * npix;
    auto load_stage = [&](int it, float (&v)[VPT]) {
        const int pb = p0 + it * KS;
        int py = pb / wx, px = pb - (pb / wx) * wx;   // facet coordinates of the stage's first pixel
        int k_prev = 0;
#pragma unroll
        for (int i = 0; i < VPT; ++i) {
            const int k = KIND == 0 ? ((i << 2) | (lane & 3)) : (((i >> 1) << 3) | ((lane & 3) << 1) | (i & 1));
            px += k - k_prev;
            k_prev = k;
            while (px >= wx) {
                px -= wx;
                ++py;
            }
            const int pp = pb + k;
            float x = 0.f;
            if (jv && pp < p1) {
                const long long o = (long long)(f.x + py) * nx + (f.z + px);
                x = fmaf(s0, __ldg(imgj + o), __ldg(Pj + pp));
            }
            v[i] = x;
        }
    };
    // one stage: wait until the MMAs that last read buffer it & 1 are done,
    // write the stage from registers, issue its four MMAs and commit
    auto process = [&](int it, const float (&v)[VPT]) -> bool {
        const int st = it & 1;
        if (it >= 2) {
            if (!mbar_wait(&s_bar[st], uint32_t(((it - 2) >> 1) & 1))) {
                if (lane == 0) atomicExch(&s_fail, 1);
            }
            __syncthreads();
            if (s_fail) return false;
        }
        // core matrix (row group warp, K column kq), row j & 7, slot lane & 3:
        // byte warp*1024 + kq*128 + lane*4
        uint8_t *buf = s_stage[st];
#pragma unroll
        for (int kq = 0; kq < 8; ++kq) {
            uint32_t word;
            if (KIND == 0) {
                word = to_tf32(v[kq]);
            } else {
                const __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * kq], v[2 * kq + 1]);
                word = *reinterpret_cast<const uint32_t *>(&b);
            }
            *reinterpret_cast<uint32_t *>(buf + warp * 1024 + kq * 128 + lane * 4) = word;
        }
        fence_async_smem();
        fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            fence_after_sync();
            const uint32_t base = smem_u32(buf);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint64_t d = smem_desc(base + k * 256, 128, 1024);
                umma<KIND>(tmem, d, d, idesc, (it > 0 || k > 0) ? 1u : 0u);
            }
            umma_commit(&s_bar[st]);
        }
        return true;
    };
    float ra[VPT], rb[VPT];
    load_stage(0, ra);
    bool ok = true;
    for (int it = 0; it < n_stage && ok; it += 2) {
        if (it + 1 < n_stage) load_stage(it + 1, rb);
        ok = process(it, ra);
        if (!ok || it + 1 >= n_stage) break;
        if (it + 2 < n_stage) load_stage(it + 2, ra);
        ok = process(it + 1, rb);
    }
    // the last commit covers every MMA issued before it
    if (ok) {
        const int last = n_stage - 1;
        if (!mbar_wait(&s_bar[last & 1], uint32_t((last >> 1) & 1))) atomicExch(&s_fail, 1);
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (s_fail) {
        if (tid == 0) atomicExch(err, 1);
    } else if (warp == 0) {
        uint32_t r[32];
        tmem_ld_32x32(tmem, r);                           // lane i: row i = channel i
        double *G = gram + (long long)cq * Lc * Lc;
#pragma unroll
        for (int jj = 0; jj < 32; ++jj)
            if (lane < Lc && jj >= lane && jj < Lc) atomicAdd(&G[lane * Lc + jj], double(__uint_as_float(r[jj])));
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(tmem) : "memory");
    }
}

}  // namespace

cudaError_t launch_nuclear_gram_tc(fhs_problem *p, int precision, cudaStream_t s) {
    long long maxpix = 0;
    for (const Facet &f : p->facets) maxpix = std::max<long long>(maxpix, (long long)(f.y1 - f.y0) * (f.x1 - f.x0));
    dim3 g(int((maxpix + kPixTc - 1) / kPixTc), p->C * p->Q);
    const float s0 = float(p->sigma0);
    if (precision == FHS_GRAM_TF32)
        gram_tc_kernel<0><<<g, kTcThreads, 0, s>>>(p->P, p->Xbar, p->d_facets, p->nuc_off, p->Q, p->C, p->Lc, p->nx,
                                                   p->N, s0, p->gram, p->dev_err);
    else if (precision == FHS_GRAM_BF16)
        gram_tc_kernel<1><<<g, kTcThreads, 0, s>>>(p->P, p->Xbar, p->d_facets, p->nuc_off, p->Q, p->C, p->Lc, p->nx,
                                                   p->N, s0, p->gram, p->dev_err);
    else
        return cudaErrorInvalidValue;
    p->n_launch += 1;
    return cudaGetLastError();
}

}  // namespace fhs
