// tcgen05 building blocks shared by the tensor-core kernels (gint_tc.cu, gint_dm.cu): PTX
// wrappers for mbarriers, MMA issue and commit, TMEM loads, asynchronous copies; the split
// precision schemes and the canonical K-major no-swizzle shared-memory operand layout.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cstdint>

#include "gint_device.cuh"

namespace gint {

constexpr int kLBO = 144;         // bytes between core matrices along K
constexpr int kTmemCols = 512;

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(kLBO >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("{ .reg .b64 st; mbarrier.arrive.shared::cta.b64 st, [%0]; }" ::"r"(su32(bar)) : "memory");
}

constexpr uint32_t kWaitHintNs = 200000;   // longest single suspension of a waiting thread (0.2 ms)

// bounded wait on the phase with the given parity; false if the budget ran out
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long budget)
{
    const uint32_t a = su32(bar);
    const long long t0 = clock64();
    while (true) {
        uint32_t ok;
        // the thread is suspended until the phase completes or the hint (nanoseconds) runs out,
        // so a waiting warp takes no issue slots from the working ones
        asm volatile("{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; selp.u32 %0, 1, 0, p; }"
                     : "=r"(ok)
                     : "r"(a), "r"(parity), "r"(kWaitHintNs)
                     : "memory");
        if (ok) return true;
        if (clock64() - t0 > budget) return false;
    }
}

// the mbarrier's current phase also waits for `bytes` more bytes of asynchronous copies
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
}

// bulk copy global -> shared (both 16-byte aligned, bytes a multiple of 16) that completes the
// transaction bytes on `bar`
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     su32(dst)),
                 "l"(src), "r"(bytes), "r"(su32(bar))
                 : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                 : "memory");
}

template <bool F16KIND>
__device__ __forceinline__ void umma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    if constexpr (F16KIND)
        asm volatile("{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p; }" ::"r"(d),
                     "l"(a), "l"(b), "r"(idesc), "r"(acc));
    else
        asm volatile("{ .reg .pred p; setp.ne.b32 p, %4, 0; tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p; }" ::"r"(d),
                     "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// asynchronous global -> shared copies (completion: cp_async_wait_all + a barrier)
__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(su32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(su32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_group1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// FP64 add to global memory without a return value (the scatters never read the old value)
__device__ __forceinline__ void red_add_f64(double *a, double v)
{
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(a), "d"(v) : "memory");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void named_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t addr, float *v)
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 16 TMEM columns of the warp's 32 lanes; complete after tmem_wait_ld()
__device__ __forceinline__ void tmem_ld16_async(uint32_t addr, uint32_t *r)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                 : "r"(addr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tmem_st16(uint32_t addr, const float *v)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(addr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                 "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
                 "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
                 "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
                 "r"(__float_as_uint(v[15]))
                 : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// ------------------------------------------------------------------ precision schemes
// CG elements = 16 bytes per core-matrix row; KCM core matrices per row per pipeline chunk, so a
// chunk is 32 K values (points for vlocal, orbitals for rho) in every scheme.  RSTAGES / VSTAGES:
// operand stages in the rho/force and vlocal kernels (one stage suffices when the next chunk's
// orbital evaluation, which precedes the stage rewrite, covers the chunk's MMAs; measured).
// PA/PB: operand term of product q, packed one nibble per product.
// HALF: fp16 terms (FMT 0), whose narrow exponent range needs the power-of-two operand
// scaling of scale_for(); the other schemes keep FP32's exponent range and use no scaling.
struct TF32x3W {  // hi + lo TF32 terms, products hi.hi + hi.lo + lo.hi
    static constexpr int CG = 4, NT = 2, NPROD = 3, KCM = 8;
    static constexpr int RSTAGES = 1;
    static constexpr int VSTAGES = 1;
    static constexpr bool F16 = false, HALF = false;
    static constexpr uint32_t FMT = 2, PA = 0x100, PB = 0x010;
};
struct BF16x3W {  // hi + lo BF16 terms, the same three products
    static constexpr int CG = 8, NT = 2, NPROD = 3, KCM = 4;
    static constexpr int RSTAGES = 2;
    static constexpr int VSTAGES = 1;
    static constexpr bool F16 = true, HALF = false;
    static constexpr uint32_t FMT = 1, PA = 0x100, PB = 0x010;
};
struct BF16x6W {  // hi + mid + lo BF16 terms, the six products of total order <= 2
    static constexpr int CG = 8, NT = 3, NPROD = 6, KCM = 4;
    static constexpr int RSTAGES = 1;
    static constexpr int VSTAGES = 1;
    static constexpr bool F16 = true, HALF = false;
    static constexpr uint32_t FMT = 1, PA = 0x210100, PB = 0x012010;
};
struct FP16x3W {  // hi + lo fp16 terms (11-bit significands, as TF32), the three products
    static constexpr int CG = 8, NT = 2, NPROD = 3, KCM = 4;
    static constexpr int RSTAGES = 2;
    static constexpr int VSTAGES = 2;
    static constexpr bool F16 = true, HALF = true;
    static constexpr uint32_t FMT = 0, PA = 0x100, PB = 0x010;
};

// Power of two s with m * s < 2^14 (1 if m is zero or not finite): the fp16 operands are
// scaled by it so that their largest terms sit just below 2^14, products below 2^28, and the
// low terms of values down to 2^-17 of the largest stay normal numbers.
__device__ __forceinline__ float scale_for(float m)
{
    if (!(m > 0.f) || !(m < 3.0e38f)) return 1.f;
    int e;
    frexpf(m, &e);   // m < 2^e
    return ldexpf(1.f, 14 - e);
}
__host__ __device__ constexpr int term(uint32_t packed, int q) { return (int)((packed >> (4 * q)) & 0xF); }

__device__ __forceinline__ float tf32_rna(float x)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// split CG consecutive FP32 values into NT terms and store each as one 16-byte chunk
template <class S>
__device__ __forceinline__ void split_store(const float *x, unsigned char *const *dst)
{
    if constexpr (!S::F16) {
        float4 hi, lo;
        float *h = &hi.x, *l = &lo.x;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            h[i] = tf32_rna(x[i]);
            l[i] = tf32_rna(x[i] - h[i]);
        }
        *reinterpret_cast<float4 *>(dst[0]) = hi;
        *reinterpret_cast<float4 *>(dst[1]) = lo;
    } else {
        // two elements per conversion: term k of elements 2i, 2i + 1 is one packed pair (the
        // lower address holds element 2i); r - term is exact in FP32
        uint4 t[S::NT];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float a = x[2 * i], b = x[2 * i + 1];
#pragma unroll
            for (int k = 0; k < S::NT; ++k) {
                uint32_t w;
                if constexpr (S::HALF) {
                    const __half2 h = __floats2half2_rn(a, b);
                    const float2 f = __half22float2(h);
                    a -= f.x;
                    b -= f.y;
                    w = *reinterpret_cast<const uint32_t *>(&h);
                } else {
                    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
                    const float2 f = __bfloat1622float2(h);
                    a -= f.x;
                    b -= f.y;
                    w = *reinterpret_cast<const uint32_t *>(&h);
                }
                (&t[k].x)[i] = w;
            }
        }
#pragma unroll
        for (int k = 0; k < S::NT; ++k) *reinterpret_cast<uint4 *>(dst[k]) = t[k];
    }
}

template <class S>
__device__ __forceinline__ void zero_store(unsigned char *const *dst)
{
#pragma unroll
    for (int k = 0; k < S::NT; ++k) *reinterpret_cast<uint4 *>(dst[k]) = make_uint4(0, 0, 0, 0);
}

// byte offset of core-matrix row (row, kc) in an operand array
template <class S>
__device__ __forceinline__ int cm_off(int row, int kc)
{
    constexpr int SBO = S::KCM * kLBO;
    return (row >> 3) * SBO + kc * kLBO + (row & 7) * 16;
}

template <class S>
constexpr int arr_bytes(int rows)
{
    return (rows / 8) * S::KCM * kLBO;
}

template <class S>
__host__ __device__ constexpr uint32_t idesc(int M, int N)
{
    return (1u << 4) | (S::FMT << 7) | (S::FMT << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// FP32 -> FP64 with integer operations (exact for normal numbers; subnormals flush to 0)
__device__ __forceinline__ double f2d(float f)
{
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xFF;
    if (e == 0) return 0.0;
    if (e == 0xFF) return (double)f;
    const uint64_t bits = ((uint64_t)(u & 0x80000000u) << 32) | ((uint64_t)(e + 896u) << 52) |
                          ((uint64_t)(u & 0x7FFFFFu) << 29);
    return __longlong_as_double((long long)bits);
}


// Role-uniform bounded wait: thread 0 of the role waits, the outcome is shared through `flag`.
// The callers pass another barrier of the same role between two calls, so every thread has
// read the flag before thread 0 writes it again.
__device__ __forceinline__ bool role_wait(uint64_t *bar, uint32_t parity, const Plan &P, int rtid, volatile int *flag,
                                          int barid, int nthr)
{
    if (rtid == 0) {
        bool ok = !aborted(P) && mbar_wait(bar, parity, P.spin_limit);
        if (!ok) report_timeout(P);
        *flag = ok ? 0 : 1;
    }
    named_sync(barid, nthr);
    return *flag == 0;
}

}  // namespace gint
