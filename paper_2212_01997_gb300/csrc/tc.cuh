// tcgen05 / bulk-copy / mbarrier primitives shared by the split-precision
// recursion kernels (inline PTX for sm_103a), and the FP16/BF16 hi-lo split.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace {

// iterations of a bounded mbarrier wait before it reports a timeout
constexpr uint32_t TC_WAIT_LIMIT = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t desc_bits(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05; layout: no swizzle
    return d;
}

// kind::f16 instruction descriptor: D FP32, A/B FP16 (fmt 0) or BF16 (fmt 1),
// A K-major, B MN-major (bit 16), M = 128, N = n.
__device__ __forceinline__ uint32_t make_idesc(int fmt, int neg_a, int n) {
    return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)neg_a << 13) |
           (1u << 16) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ void fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// orders this thread's generic global writes before later async-proxy
// (bulk copy) reads of them
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// one bulk copy global -> shared of `bytes` (multiple of 16, both addresses
// 16-byte aligned), completing on the mbarrier's transaction count
__device__ __forceinline__ void bulk_g2s(uint32_t sdst, const void* gsrc, uint32_t bytes, uint32_t mbar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(sdst),
        "l"(gsrc), "r"(bytes), "r"(mbar)
        : "memory");
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase) {
    for (uint32_t it = 0; it < TC_WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            "selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

// waits for every tcgen05.ld this thread issued
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// two 16-column loads (e.g. the same chunk of two slots) behind one wait
__device__ __forceinline__ void tmem_ld16x2(uint32_t ta, uint32_t tb, float (&u)[16], float (&w)[16]) {
    uint32_t r[16], q[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(ta));
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
        "%12, %13, %14, %15}, [%16];"
        : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]),
          "=r"(q[7]), "=r"(q[8]), "=r"(q[9]), "=r"(q[10]), "=r"(q[11]), "=r"(q[12]), "=r"(q[13]),
          "=r"(q[14]), "=r"(q[15])
        : "r"(tb));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    // the registers are defined only after the wait: pin every use behind it
#pragma unroll
    for (int j = 0; j < 16; ++j) asm volatile("" : "+r"(r[j]), "+r"(q[j]));
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        u[j] = __uint_as_float(r[j]);
        w[j] = __uint_as_float(q[j]);
    }
}

// one column per RHS of a block: NC single-column loads (columns cols[q],
// q < nc; the others repeat cols[0]) behind one wait.  Warp-uniform columns.
template <int NC>
__device__ __forceinline__ void tmem_ld_cols(uint32_t base, const int32_t* cols, int nc, float (&v)[NC]) {
    uint32_t r[NC];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
        const uint32_t col = (uint32_t)cols[q < nc ? q : 0];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r[q]) : "r"(base + col));
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < NC; ++q) {
        asm volatile("" : "+r"(r[q]));
        v[q] = __uint_as_float(r[q]);
    }
}

// completes every tcgen05.st this thread issued
__device__ __forceinline__ void tmem_wait_st() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// hi/lo split of a pair of values: hi = rn(x), lo = rn(x - hi), packed.
// x - hi (exact) comes from one mixed-precision FMA per value, hi x (-1) + x
// with the 16-bit hi operand read directly, instead of a conversion back to
// FP32 and a subtraction.
__device__ __forceinline__ void split_pair(float x0, float x1, int fmt, uint32_t& hi, uint32_t& lo) {
    float d0, d1;
    if (fmt == 0) {
        asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(x1), "f"(x0));
        asm("{.reg .b16 l, h, m;\n mov.b32 {l, h}, %2;\n mov.b16 m, 0xBC00;\n"
            " fma.rn.f32.f16 %0, l, m, %3;\n fma.rn.f32.f16 %1, h, m, %4;}"
            : "=f"(d0), "=f"(d1) : "r"(hi), "f"(x0), "f"(x1));
        asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(d1), "f"(d0));
    } else {
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(x1), "f"(x0));
        asm("{.reg .b16 l, h, m;\n mov.b32 {l, h}, %2;\n mov.b16 m, 0xBF80;\n"
            " fma.rn.f32.bf16 %0, l, m, %3;\n fma.rn.f32.bf16 %1, h, m, %4;}"
            : "=f"(d0), "=f"(d1) : "r"(hi), "f"(x0), "f"(x1));
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(d1), "f"(d0));
    }
}

// hi parts of a pair (rn), packed
__device__ __forceinline__ uint32_t hi_pair(float x0, float x1, int fmt) {
    if (fmt == 0) {
        const __half2 h = __floats2half2_rn(x0, x1);
        return *(const uint32_t*)&h;
    }
    const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
    return *(const uint32_t*)&h;
}

// float -> double by integer operations (exact; FP32 subnormals flush to
// zero).  Keeps the conversions off GB300's narrow FP64 pipe.
__device__ __forceinline__ double f2d(float x) {
    const uint32_t u = __float_as_uint(x);
    const uint32_t e = (u >> 23) & 0xffu;
    const uint64_t sign = (uint64_t)(u >> 31) << 63;
    const uint64_t ex = e == 0u ? 0ull : (e == 255u ? (0x7ffull << 52) : (uint64_t)(e + 896u) << 52);
    const uint64_t man = e == 0u ? 0ull : (uint64_t)(u & 0x7fffffu) << 29;
    return __longlong_as_double((long long)(sign | ex | man));
}

// unevaluated float pairs (hi + lo): error-free sum (Knuth), pair sum
struct FF {
    float hi, lo;
};

__device__ __forceinline__ FF two_sum(float a, float b) {
    const float t = a + b;
    const float bv = t - a;
    return {t, (a - (t - bv)) + (b - bv)};
}

__device__ __forceinline__ FF ff_add(FF a, FF b) {
    const FF t = two_sum(a.hi, b.hi);
    const float e = t.lo + (a.lo + b.lo);
    const float h = t.hi + e;
    return {h, e - (h - t.hi)};
}

__device__ __forceinline__ FF ff_neg(FF a) { return {-a.hi, -a.lo}; }

// 8-column TMEM loads (32 lanes x 8 columns per warp), issued without a wait
__device__ __forceinline__ void tmem_ld8_issue(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7])
                 : "r"(taddr));
}

__device__ __forceinline__ void pin8(uint32_t (&r)[8]) {
#pragma unroll
    for (int j = 0; j < 8; ++j) asm volatile("" : "+r"(r[j]));
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float (&v)[8]) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                 "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7]))
                 : "memory");
}

}  // namespace
