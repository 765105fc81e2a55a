// Inline-PTX building blocks for the tcgen05 kernels (sm_100 family, sm_103a):
// mbarriers with bounded waits, bulk and tensor (TMA) async copies, TMEM
// allocation and access, UMMA descriptors and issue, FP16/BF16 packing and the
// MUFU unit phasor.  Shared by k_tc.cu and k_kr.cu.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace psf {
namespace tc {

constexpr unsigned long long kTimeoutNs = 2000000000ull;

static __device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

static __device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

static __device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
                 : "memory");
}

// try_wait; with a nonzero suspend-time hint the waiting thread is parked (no issue
// slots) until the phase completes or about `hint_ns` elapse.  Measured on GB300,
// parked waits beat polling for every role of this kernel (polling warps take
// issue slots from the generators).
static __device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    if (hint_ns) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
            : "memory");
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
    }
    return ok != 0;
}
static constexpr uint32_t kSleepNs = 1000000u;

static __device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase of `bar` with the given parity.  Returns false if the CTA is
// aborting or the wall-clock limit expired (then the abort flag and the global
// error flag are raised).
static __device__ __forceinline__ bool wait_bounded(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                             int *err, uint32_t hint_ns = kSleepNs) {
    if (mbar_try_wait(bar, parity, hint_ns)) return true;
    const unsigned long long t0 = globaltimer();
    for (;;) {
        if (mbar_try_wait(bar, parity, hint_ns)) return true;
        if (*abort_flag) return false;
        if (globaltimer() - t0 > kTimeoutNs) {
            *abort_flag = 1;
            if (err) atomicExch(err, 1);
            return false;
        }
    }
}

static __device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                     smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// Bulk (non-tensor) async copy global -> shared, completing `bytes` on `bar`.
// Both addresses 16-byte aligned, size a multiple of 16.
static __device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

static __device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
static __device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
static __device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

static __device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
}
static __device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
static __device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, kind::f16, one CTA.
static __device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on `bar` once all previously issued tcgen05.mma of this thread complete.
static __device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 32 TMEM lanes x 16 consecutive 32-bit columns -> 16 registers per thread.
static __device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), version 1 (sm_100 family).
static __device__ __forceinline__ uint64_t desc_sw128(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// Instruction descriptor, kind::f16: FP32 accumulator, FP16 (0) or BF16 (1)
// operands, both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
static __host__ __device__ constexpr uint32_t idesc_f16(int M, int N, int bf16) {
    return (1u << 4) | ((uint32_t)bf16 << 7) | ((uint32_t)bf16 << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

// Byte offset of the 32-bit (re, im) pair `kp` (0..31) of row `row` in a K-major
// 128-byte-swizzled tile: 16-byte chunk index XOR (row mod 8).
static __device__ __forceinline__ uint32_t sw128_pair_offset(int row, int kp) {
    return (uint32_t)row * 128u + ((uint32_t)(((kp >> 2) ^ (row & 7))) << 4) + ((uint32_t)(kp & 3) << 2);
}

template <int BF16>
static __device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    if (BF16) {
        __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
        return *reinterpret_cast<uint32_t *>(&h);
    } else {
        __half2 h = __floats2half2_rn(lo, hi);
        return *reinterpret_cast<uint32_t *>(&h);
    }
}

template <int BF16>
static __device__ __forceinline__ float2 unpack2(uint32_t v) {
    if (BF16) {
        const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162 *>(&v);
        return __bfloat1622float2(h);
    } else {
        const __half2 h = *reinterpret_cast<const __half2 *>(&v);
        return __half22float2(h);
    }
}

// Low parts of a pair packed by pack2 (split precision): each value minus its 16-bit
// rounding (exact in FP32), rounded to 16 bits again.
template <int BF16>
static __device__ __forceinline__ uint32_t pack2_lo(float lo, float hi, uint32_t packed) {
    const float2 r = unpack2<BF16>(packed);
    return pack2<BF16>(lo - r.x, hi - r.y);
}

static __device__ __forceinline__ uint32_t pow2_cols(int n) {
    uint32_t c = 32;
    while ((int)c < n) c <<= 1;
    return c;
}

// exp(2 pi i x) via the MUFU sine/cosine of the reduced argument (|error| ~ 1e-6).
static __device__ __forceinline__ float2 cis_turns(float x) {
    const float f = x - rintf(x);
    float s, c;
    __sincosf(6.28318530717958647f * f, &s, &c);
    return make_float2(c, s);
}

static __device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}


// Four 8x8 b16 matrices from registers to shared memory.  Lane t holds, per matrix,
// the 32-bit pair at matrix row t/4, columns 2(t%4), 2(t%4)+1; lanes 8m..8m+7 give
// the 16-byte row addresses of matrix m.  With one K-major 128-byte operand row per
// matrix, lane t's pair is K' elements (2t, 2t+1) of that row: one instruction
// stores four operand rows of one 32-visibility stage.
static __device__ __forceinline__ void stmatrix_x4(uint32_t saddr, uint32_t v0, uint32_t v1, uint32_t v2,
                                                   uint32_t v3) {
    asm volatile("stmatrix.sync.aligned.m8n8.x4.shared.b16 [%0], {%1, %2, %3, %4};" ::"r"(saddr), "r"(v0), "r"(v1),
                 "r"(v2), "r"(v3)
                 : "memory");
}

// Per-lane stmatrix addresses for the four rows q, q+8, q+16, q+24 (q = 0..7) of a
// 32-row block of a K-major 128-byte-swizzled tile: lane t addresses matrix t/8
// (row q + 8 (t/8)), 16-byte chunk t%8, swizzled by XOR with the row index mod 8 (= q).
static __device__ __forceinline__ void stmatrix_offsets(int lane, uint32_t (&off)[8]) {
    const uint32_t m = (uint32_t)lane >> 3, a = (uint32_t)lane & 7u;
#pragma unroll
    for (int q = 0; q < 8; ++q) off[q] = (uint32_t)q * 128u + m * 1024u + ((a ^ (uint32_t)q) << 4);
}

// 2-D tiled TMA load of one box into shared memory, completing on `bar`.
static __device__ __forceinline__ void tma_load_2d(void *dst, const void *tmap, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// 16 consecutive 32-bit TMEM columns of 32 lanes <- 16 registers per thread.
static __device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15, %16};" ::"r"(taddr),
        "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
        "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
        "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
        "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
        "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
        "r"(__float_as_uint(v[15]))
        : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

}  // namespace tc
}  // namespace psf
