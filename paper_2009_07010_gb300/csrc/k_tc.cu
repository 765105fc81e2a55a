// tcgen05 (5th-generation tensor core) contraction of the smeared PSF, sm_103a.
//
// One CTA computes one 128 x ncols output tile of one cutout over a contiguous
// range of visibilities (split-K), as the real GEMM of Eqs. 21-22 in separable form:
//   P[j][i] = sum_k Re( c_k[j] a_k[i] ),   c_k[j] = w_k exp(2 pi i v_k dm_j),
//                                          a_k[i] = exp(2 pi i u_k dl_i),
//   A'[j][2k] = Re c, A'[j][2k+1] = Im c,  B'[i][2k] = Re a, B'[i][2k+1] = -Im a,
//   P = A' B'^T  with K' = 2K (FP16 or BF16 operands, FP32 accumulation in TMEM).
//
// Warp roles (736 threads):
//   warps 0-15  operand generators (four groups on stages s mod 4, two chains per warp
//               and stage): per pipeline stage of 32 visibilities each lane
//               owns one visibility and walks a 32-row recurrence chain
//               (seed and step from the MUFU sin/cos of the reduced phase, then
//               complex multiplication), writing FP16/BF16 pairs straight into the
//               128-byte-swizzled K-major shared-memory layout the MMA reads;
//   warps 20, 22  TMEM allocation and the tcgen05.mma issue: with NISS = 2 (tiles of at
//               most 128 columns) warp 20 issues the even stages and warp 22 the odd
//               ones, each into accumulators of its own, so that one issuer's barrier
//               wait (an mbarrier round trip during which a lone issuer leaves the
//               tensor core idle) overlaps the other issuer's MMAs; with NISS = 1
//               warp 20 issues every stage;
//   warp 21     the uv/w input ring: one bulk copy pair per stage, refilled when the
//               generator group of the stage has read it (`in_empty`);
//   warps 16-19 drain: every kDrainStages stages the issuers switch to their second
//               TMEM accumulator while these warps read the first ones (tcgen05.ld),
//               add them and add the sum into the CTA's FP32 partial tile in global
//               memory.  Short TMEM accumulation runs bound the tensor-core rounding
//               growth.  In split precision each add into the running sum is an
//               error-free TwoSum whose rounding error goes back into the drained
//               accumulator, on which the issuer's next range in that buffer
//               accumulates (compensated summation, the correction carried by the
//               tensor core).
// Stages are handed over with mbarriers (input copies -> generators: `in_full`,
// generators -> input warp: `in_empty`, generators -> MMA: `full`, MMA commit ->
// generators: `empty`, MMA commit -> drain: `acc_full`, drain -> MMA: `acc_empty`).
// An issuing thread does nothing per stage but wait, issue and commit: MMA issue
// blocks the thread, so its serial latency bounds the stage rate.  Every wait is bounded by a wall-clock limit; on
// expiry the CTA raises the plan's error flag, stops all roles, waits (bounded) for
// its bulk copies and issued MMAs and frees TMEM.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "psf_internal.cuh"
#include "tc_ptx.cuh"

namespace psf {
namespace {
using namespace tc;

constexpr int kInStages = 16;      // per-visibility input (uv, w) ring depth
constexpr int kKS = 32;            // complex visibilities per stage (K' = 64 = one 128 B row)
constexpr int kGenWarps = 16;      // four groups of 4; group g generates stages s = g (mod 4)
constexpr int kGroupWarps = 4;
constexpr int kGroups = kGenWarps / kGroupWarps;
// A group waiting for slot reuse (stage s - S consumed) must find the slot's previous
// phase (stage s - 2S) already consumed, or the parity test of the barrier aliases;
// that holds when the group's previous stage s - kGroups waited for stage
// s - kGroups - S >= s - 2S, i.e. kGroups <= S for every ring depth S used (4, 6, 8).
static_assert(kGroups <= 4, "generator groups must not exceed the smallest operand ring depth");
static_assert(kGroups <= kInStages, "generator groups must not exceed the input ring depth");
constexpr int kDrainWarp0 = 16;
constexpr int kMmaWarp = 20;
constexpr int kInWarp = 21;
constexpr int kMma2Warp = 22;
constexpr int kThreads = 23 * 32;
constexpr int kDrainStages = 64;   // stages accumulated in TMEM between drains
// Split precision: the tensor core's FP32 accumulation loses about 2^-24.5 of the running
// value per added MMA (measured: the error of a cutout grows with the MMAs accumulated
// between drains, 64-stage runs of 12 MMAs left ~1e-5), so the runs are 8 stages and the
// drain warps keep the running sum in TMEM.
//
// Running sums of nearly equal terms (a coherent pixel such as the PSF peak, where every
// range adds about the same value) do not round at random: the sum sits on its own ulp
// grid and each add rounds the same way, so plain FP32 adds drift by up to ulp/2 per
// range (about 1.5e-5 of the peak over 1500 ranges).  Every add is therefore a TwoSum,
// s + v = t + e exactly, and e is written into the drained accumulator; the issuer's first
// MMA of the next range in that buffer keeps it (accumulate) instead of clearing it.
constexpr int kDrainStagesSplit = 8;

// t = fl(a + b) and the exact rounding error e (a + b = t + e), any magnitudes (Knuth).
__device__ __forceinline__ void two_sum(float a, float b, float &t, float &e) {
    t = a + b;
    const float bp = t - a;
    e = (a - (t - bp)) + (b - bp);
}
constexpr int kATileBytes = 128 * 128;
// One 32-row twiddle chain of one visibility (this lane), rows r = 0..31 of `base`:
// value(r) = [w] exp(2 pi i theta (n0 + r)), written as an FP16/BF16 (re, im) pair at
// the lane's K-major swizzled slot.  The chain runs as eight interleaved 4-row pieces
// (seeds at r = 0, 4, ..., 28) held in four packed FP32x2 pairs, so each step is four
// independent packed complex multiplications, and the eight rows of a step leave in
// two stmatrix.
// MIRROR: the chain also writes the complex conjugate of row r at row R0 - r (mbase =
// tile + R0 * 128 with R0 a multiple of 8; the packed pair's imaginary half is the
// high 16 bits, so conjugation is a sign-bit XOR), and with `tail` the conjugate of
// the value one step past the last row at `tail_addr` (row 0 of the tile).
// CPLX: each row value z is also written as (-Im z, Re z) at row r of base + mbase
// (the second half of a doubled B tile: with z = conj(a) these rows give the
// imaginary part of the contraction).
// SPLIT: every value is also written as its low part (value - rounded value, rounded
// to 16 bits) at the same position lo_off bytes further on (the lo tile of a split
// precision stage); conjugation of the low part is the same sign-bit XOR.
// The step exp(2 pi i theta) of a chain and its 4-, 8- and 16-row strides (squarings):
// shared by the chains of one visibility that have the same theta.
struct ChainSteps {
    float2 st, s4, s8, s16;
};
__device__ __forceinline__ ChainSteps chain_steps(float theta) {
    ChainSteps S;
    S.st = cis_turns(theta);
    const float2 s2 = cmulf(S.st, S.st);
    S.s4 = cmulf(s2, s2);
    S.s8 = cmulf(S.s4, S.s4);
    S.s16 = cmulf(S.s8, S.s8);
    return S;
}

template <int BF16, bool MIRROR = false, bool CPLX = false, bool SPLIT = false>
__device__ __forceinline__ void gen_chain32_s(const ChainSteps &S, uint32_t base, const uint32_t (&off)[8],
                                              float theta, int n0, float2 wk, bool weighted, uint32_t mbase = 0,
                                              bool tail = false, uint32_t tail_addr = 0, uint32_t lo_off = 0) {
    // eight interleaved 4-row pieces: rows q + 4p (p = 0..7) at step q = 0..3.  Two
    // sine/cosine evaluations per chain (row 0 and the step, the latter in S); the piece
    // seeds follow by complex multiplication with the 4- and 16-row strides (squarings
    // of the step), which keeps the MUFU pipe to 4 instructions per 32 rows.
    const float2 st = S.st, s4 = S.s4, s8 = S.s8, s16 = S.s16;
    float2 z[8];
    z[0] = cis_turns(theta * (float)n0);
    if (weighted) z[0] = cmulf(z[0], wk);
    z[1] = cmulf(z[0], s4);
    z[2] = cmulf(z[0], s8);
    z[3] = cmulf(z[1], s8);
#pragma unroll
    for (int pc = 4; pc < 8; ++pc) z[pc] = cmulf(z[pc - 4], s16);
    // packed pairs: P0 = rows (q, q+16), P1 = (q+8, q+24), P2 = (q+4, q+20), P3 = (q+12, q+28)
    float2 re[4], im[4];
    re[0] = make_float2(z[0].x, z[4].x); im[0] = make_float2(z[0].y, z[4].y);
    re[1] = make_float2(z[2].x, z[6].x); im[1] = make_float2(z[2].y, z[6].y);
    re[2] = make_float2(z[1].x, z[5].x); im[2] = make_float2(z[1].y, z[5].y);
    re[3] = make_float2(z[3].x, z[7].x); im[3] = make_float2(z[3].y, z[7].y);
    const float2 sr = make_float2(st.x, st.x), si = make_float2(st.y, st.y), nsi = make_float2(-st.y, -st.y);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        // rows q, q+8, q+16, q+24 and rows q+4, q+12, q+20, q+28
        // matrix m of a mirrored store at offset q' writes row R0 - (q' + 8 m), chunk
        // (lane mod 8) swizzled with (-q') mod 8
        constexpr uint32_t kConj = 0x80000000u;
        const uint32_t ln = threadIdx.x & 31u, ca = ln & 7u;
        {
            const uint32_t v0 = pack2<BF16>(re[0].x, im[0].x), v1 = pack2<BF16>(re[1].x, im[1].x);
            const uint32_t v2 = pack2<BF16>(re[0].y, im[0].y), v3 = pack2<BF16>(re[1].y, im[1].y);
            // without mirroring the row addresses are recomputed from the lane (cheaper than
            // holding eight offsets at this kernel's register budget)
            const uint32_t addr = MIRROR ? base + off[q]
                                         : base + (((threadIdx.x >> 3) & 3u) << 10) + (uint32_t)q * 128u +
                                               (((threadIdx.x & 7u) ^ (uint32_t)q) << 4);
            stmatrix_x4(addr, v0, v1, v2, v3);
            uint32_t l0 = 0u, l1 = 0u, l2 = 0u, l3 = 0u;
            if (SPLIT) {
                l0 = pack2_lo<BF16>(re[0].x, im[0].x, v0);
                l1 = pack2_lo<BF16>(re[1].x, im[1].x, v1);
                l2 = pack2_lo<BF16>(re[0].y, im[0].y, v2);
                l3 = pack2_lo<BF16>(re[1].y, im[1].y, v3);
                stmatrix_x4(addr + lo_off, l0, l1, l2, l3);
            }
            if (MIRROR) {
                const uint32_t maddr = mbase - (ln >> 3) * 1024u - (uint32_t)q * 128u + ((ca ^ ((8u - q) & 7u)) << 4);
                stmatrix_x4(maddr, v0 ^ kConj, v1 ^ kConj, v2 ^ kConj, v3 ^ kConj);
                if (SPLIT) stmatrix_x4(maddr + lo_off, l0 ^ kConj, l1 ^ kConj, l2 ^ kConj, l3 ^ kConj);
            }
            if (CPLX)
                stmatrix_x4(base + mbase + (((threadIdx.x >> 3) & 3u) << 10) + (uint32_t)q * 128u +
                                (((threadIdx.x & 7u) ^ (uint32_t)q) << 4),
                            pack2<BF16>(-im[0].x, re[0].x), pack2<BF16>(-im[1].x, re[1].x),
                            pack2<BF16>(-im[0].y, re[0].y), pack2<BF16>(-im[1].y, re[1].y));
        }
        {
            const uint32_t v4 = pack2<BF16>(re[2].x, im[2].x), v5 = pack2<BF16>(re[3].x, im[3].x);
            const uint32_t v6 = pack2<BF16>(re[2].y, im[2].y), v7 = pack2<BF16>(re[3].y, im[3].y);
            const uint32_t addr = MIRROR ? base + off[q + 4]
                                         : base + (((threadIdx.x >> 3) & 3u) << 10) + (uint32_t)(q + 4) * 128u +
                                               (((threadIdx.x & 7u) ^ (uint32_t)(q + 4)) << 4);
            stmatrix_x4(addr, v4, v5, v6, v7);
            uint32_t l4 = 0u, l5 = 0u, l6 = 0u, l7 = 0u;
            if (SPLIT) {
                l4 = pack2_lo<BF16>(re[2].x, im[2].x, v4);
                l5 = pack2_lo<BF16>(re[3].x, im[3].x, v5);
                l6 = pack2_lo<BF16>(re[2].y, im[2].y, v6);
                l7 = pack2_lo<BF16>(re[3].y, im[3].y, v7);
                stmatrix_x4(addr + lo_off, l4, l5, l6, l7);
            }
            if (MIRROR) {
                const uint32_t maddr =
                    mbase - (ln >> 3) * 1024u - (uint32_t)(q + 4) * 128u + ((ca ^ ((4u - q) & 7u)) << 4);
                stmatrix_x4(maddr, v4 ^ kConj, v5 ^ kConj, v6 ^ kConj, v7 ^ kConj);
                if (SPLIT) stmatrix_x4(maddr + lo_off, l4 ^ kConj, l5 ^ kConj, l6 ^ kConj, l7 ^ kConj);
            }
            if (CPLX)
                stmatrix_x4(base + mbase + (((threadIdx.x >> 3) & 3u) << 10) + (uint32_t)(q + 4) * 128u +
                                (((threadIdx.x & 7u) ^ (uint32_t)(q + 4)) << 4),
                            pack2<BF16>(-im[2].x, re[2].x), pack2<BF16>(-im[3].x, re[3].x),
                            pack2<BF16>(-im[2].y, re[2].y), pack2<BF16>(-im[3].y, re[3].y));
        }
        if (q < 3) {
#pragma unroll
            for (int pp = 0; pp < 4; ++pp) {
                const float2 t = __fmul2_rn(im[pp], nsi), u = __fmul2_rn(im[pp], sr);
                im[pp] = __ffma2_rn(re[pp], si, u);
                re[pp] = __ffma2_rn(re[pp], sr, t);
            }
        }
    }
    if (MIRROR && tail) {   // row 32 = piece 7 (row 31, the .y half of pair 3) one step on
        const float r32 = re[3].y * st.x - im[3].y * st.y, i32 = re[3].y * st.y + im[3].y * st.x;
        const uint32_t lane = threadIdx.x & 31u;
        // row 0: chunk lane / 4 (unswizzled), pair lane mod 4
        const uint32_t h = pack2<BF16>(r32, -i32);
        asm volatile("st.shared.b32 [%0], %1;" ::"r"(tail_addr + lane * 4u), "r"(h) : "memory");
        if (SPLIT)
            asm volatile("st.shared.b32 [%0], %1;" ::"r"(tail_addr + lo_off + lane * 4u),
                         "r"(pack2_lo<BF16>(r32, -i32, h))
                         : "memory");
    }
}

template <int BF16, bool MIRROR = false, bool CPLX = false, bool SPLIT = false>
__device__ __forceinline__ void gen_chain32(uint32_t base, const uint32_t (&off)[8], float theta, int n0, float2 wk,
                                            bool weighted, uint32_t mbase = 0, bool tail = false,
                                            uint32_t tail_addr = 0, uint32_t lo_off = 0) {
    gen_chain32_s<BF16, MIRROR, CPLX, SPLIT>(chain_steps(theta), base, off, theta, n0, wk, weighted, mbase, tail,
                                             tail_addr, lo_off);
}

// Two real-weight copies of one conjugate-symmetric 32-row chain of unweighted twiddles
// (the fused uv + image-plane form): the value z(r) of row R0 + r is stored as
// (wa z) at base + r rows and (wb z) at base + half_off + r rows, each with its
// conjugate at the mirrored row R0 - r (mbase, mbase + half_off); with `tail` the
// conjugates of (wa, wb) x the value one step past the last row go to row 0 of each
// half (tail_addr, tail_addr + half_off).
template <int BF16>
__device__ __forceinline__ void gen_chain32_dual(uint32_t base, uint32_t mbase, uint32_t half_off, float theta,
                                                 int n0, float wa, float wb, bool tail, uint32_t tail_addr) {
    const float2 st = cis_turns(theta);
    float2 z[8];
    z[0] = cis_turns(theta * (float)n0);
    const float2 s2 = cmulf(st, st), s4 = cmulf(s2, s2), s8 = cmulf(s4, s4), s16 = cmulf(s8, s8);
    z[1] = cmulf(z[0], s4);
    z[2] = cmulf(z[0], s8);
    z[3] = cmulf(z[1], s8);
#pragma unroll
    for (int pc = 4; pc < 8; ++pc) z[pc] = cmulf(z[pc - 4], s16);
    float2 re[4], im[4];
    re[0] = make_float2(z[0].x, z[4].x); im[0] = make_float2(z[0].y, z[4].y);
    re[1] = make_float2(z[2].x, z[6].x); im[1] = make_float2(z[2].y, z[6].y);
    re[2] = make_float2(z[1].x, z[5].x); im[2] = make_float2(z[1].y, z[5].y);
    re[3] = make_float2(z[3].x, z[7].x); im[3] = make_float2(z[3].y, z[7].y);
    const float2 sr = make_float2(st.x, st.x), si = make_float2(st.y, st.y), nsi = make_float2(-st.y, -st.y);
    constexpr uint32_t kConj = 0x80000000u;
    const uint32_t ln = threadIdx.x & 31u, ca = ln & 7u;
    const uint32_t lrow = (((threadIdx.x >> 3) & 3u) << 10);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float2 wv = h ? make_float2(wb, wb) : make_float2(wa, wa);
            const uint32_t ho = h ? half_off : 0u;
#pragma unroll
            for (int m = 0; m < 2; ++m) {   // matrices of rows q + 8 m' (m = 0) and q + 4 + 8 m' (m = 1)
                const float2 ra = __fmul2_rn(re[2 * m], wv), ia = __fmul2_rn(im[2 * m], wv);
                const float2 rb = __fmul2_rn(re[2 * m + 1], wv), ib = __fmul2_rn(im[2 * m + 1], wv);
                const uint32_t v0 = pack2<BF16>(ra.x, ia.x), v1 = pack2<BF16>(rb.x, ib.x);
                const uint32_t v2 = pack2<BF16>(ra.y, ia.y), v3 = pack2<BF16>(rb.y, ib.y);
                const uint32_t qq = (uint32_t)(q + 4 * m);
                stmatrix_x4(base + ho + lrow + qq * 128u + ((ca ^ qq) << 4), v0, v1, v2, v3);
                stmatrix_x4(mbase + ho - lrow - qq * 128u + ((ca ^ ((8u - qq) & 7u)) << 4), v0 ^ kConj, v1 ^ kConj,
                            v2 ^ kConj, v3 ^ kConj);
            }
        }
        if (q < 3) {
#pragma unroll
            for (int pp = 0; pp < 4; ++pp) {
                const float2 t = __fmul2_rn(im[pp], nsi), u = __fmul2_rn(im[pp], sr);
                im[pp] = __ffma2_rn(re[pp], si, u);
                re[pp] = __ffma2_rn(re[pp], sr, t);
            }
        }
    }
    if (tail) {   // row 32 = piece 7 (row 31, the .y half of pair 3) one step on
        const float r32 = re[3].y * st.x - im[3].y * st.y, i32 = re[3].y * st.y + im[3].y * st.x;
        asm volatile("st.shared.b32 [%0], %1;" ::"r"(tail_addr + ln * 4u), "r"(pack2<BF16>(wa * r32, -wa * i32))
                     : "memory");
        asm volatile("st.shared.b32 [%0], %1;" ::"r"(tail_addr + half_off + ln * 4u),
                     "r"(pack2<BF16>(wb * r32, -wb * i32))
                     : "memory");
    }
}

struct SmemLayout {
    uint32_t a_off, b_off, in_off, bar_off, bytes;
};

constexpr uint32_t kInSlotBytes = kKS * 16;   // uv (8 B) + w (8 B) per visibility

// Operand ring depth for a tile width: as many 128-row A + ncols-row B stages as fit
// in ~192 KB (4 at 256 columns, 6 at 128, 8 at <= 64); split precision stages hold hi
// and lo tiles of both operands (3 at 128 columns, 4 at <= 64; tiles of at most 128
// columns).
__host__ __device__ constexpr int stages_for(int ncols_max, int split = 0) {
    return split ? (ncols_max > 64 ? 3 : 4) : (ncols_max > 128 ? 4 : (ncols_max > 64 ? 6 : 8));
}

__host__ __device__ inline SmemLayout smem_layout(int ncols_max, int kStages, uint32_t in_slot = kInSlotBytes,
                                                  int split = 0) {
    SmemLayout L;
    const uint32_t bt = (uint32_t)ncols_max * 128u;
    L.a_off = 0;
    L.b_off = kStages * kATileBytes * (1 + split);
    L.in_off = L.b_off + kStages * ((bt + 1023u) / 1024u * 1024u) * (1 + split);
    L.bar_off = L.in_off + kInStages * in_slot;
    L.bytes = L.bar_off + 512;   // 2 S + 2 kInStages + 8 barriers (<= 56 x 8 B), TMEM address, abort flag
    return L;
}

// MIR: 1 = the weights of the launch are real, so whole-cutout tiles may use the
// conjugate-symmetric generation (a separate instance keeps its register pressure out
// of the complex-weight kernel); 2 = real weights and every tile of the launch spans
// a whole 64- or 128-pixel cutout (no unmirrored path compiled in); 4 = the fused uv +
// image-plane form on such tiles: the A operand holds the unweighted column twiddles,
// the B operand (2 N rows) the row twiddles times the Method 1 weights (rows 0 .. N-1)
// and times the Method 2 weights (rows N .. 2N-1), so one N = 2 ncols MMA yields both
// cutouts side by side in TMEM (w2: second weight rows; part2: offset of the second
// cutout's partial sums from `partial`); 5 = complex output: A as in mode 0, B of 2 ncols
// rows = the conjugated row twiddles (a_r, -a_i) and then (a_i, a_r), so the two halves
// of the accumulator are the real and the imaginary parts of the cutout.
//
// SPLIT = 1 (split precision, MIR 0-2, tiles of at most 128 columns): every operand
// value x is held as hi = rnd16(x) and lo = rnd16(x - hi) in two tiles of the stage, and
// each stage issues A_hi B_hi + A_hi B_lo + A_lo B_hi into the same accumulator (the
// lo x lo term is below the 16-bit rounding of the lo parts).  The stages are twice as
// large, so the ring holds 3 or 4 of them and as many generator groups run.
template <int BF16, int kStages, int NISS, int MIR, int SPLIT = 0>
__global__ void __launch_bounds__(kThreads, 1)
    k_psf_tc(const float2 *__restrict__ uv, const float2 *__restrict__ w, int64_t ldw,
             const TcItem *__restrict__ items, int ncols_max, float cell, float *__restrict__ partial,
             int64_t split_stride, int *err, const float2 *__restrict__ w2, int64_t part2) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    // 1024-byte alignment of the operand tiles (swizzle atoms)
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    constexpr int kBMul = (MIR == 4 || MIR == 5) ? 2 : 1;           // B rows per output column
    constexpr uint32_t kSlot = (MIR == 4) ? kKS * 24 : kInSlotBytes;   // uv, w (, w2) per visibility
    // generator groups: one per stage of the ring at most (see kGroups)
    constexpr int kGrp0 = kStages < kGroups ? kStages : kGroups;
    // With two issuers the group count must be even: a group that waits for the release
    // of stage s - S relies on its previous stage's wait (for stage s - kGrp - S) having
    // seen stage s - 2S released, which only follows when both stages belong to the same
    // issuer (each issuer commits in order, the two do not order each other).  An
    // instance with five groups aliased the parity test and gave up its bounded waits.
    constexpr int kGrp = (NISS == 2) ? (kGrp0 & ~1) : kGrp0;
    static_assert(NISS == 1 || kGrp % 2 == 0, "two issuers need an even number of generator groups");
    static_assert(kGrp <= kStages, "generator groups must not exceed the operand ring depth");
    static_assert(!SPLIT || MIR <= 2, "split precision covers the plain and mirrored real-weight forms");
    // Two issuers take alternate stages; with an even ring depth every slot (and its release
    // barrier) then belongs to one issuer.  An odd depth makes the two issuing threads commit
    // alternately to the same release barrier, and such launches (3 stages, two issuers)
    // gave up bounded waits in about one launch in eight on GB300 with the protocol reading
    // correctly; two issuers are therefore only used with even depths.
    static_assert(NISS == 1 || kStages % 2 == 0, "two MMA issuers need an even operand ring depth");
    constexpr int kRange = SPLIT ? kDrainStagesSplit : kDrainStages;   // stages per accumulation run
    const SmemLayout L = smem_layout(kBMul * ncols_max, kStages, kSlot, SPLIT);
    uint64_t *full = (uint64_t *)(smem + L.bar_off);
    uint64_t *empty = full + kStages;
    uint64_t *in_full = empty + kStages;
    uint64_t *in_empty = in_full + kInStages;
    uint64_t *acc_full = in_empty + kInStages;   // [issuer][buffer]
    uint64_t *acc_empty = acc_full + 4;          // [buffer], shared by the issuers
    uint64_t *done_bar = acc_empty + 2;          // [issuer]
    uint32_t *s_tmem = (uint32_t *)(done_bar + 2);
    volatile int *s_abort = (volatile int *)(s_tmem + 1);
    volatile int no_abort = 0;   // teardown waits ignore the abort flag

    const TcItem it = items[blockIdx.x];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ncols = it.ncols;
    const uint32_t bt_stride = ((uint32_t)(kBMul * ncols_max) * 128u + 1023u) / 1024u * 1024u;   // one B tile
    const uint32_t b_stage = bt_stride * (1 + SPLIT);                  // hi (and lo) B tiles of a stage
    constexpr uint32_t kAStage = kATileBytes * (1 + SPLIT);
    const uint32_t acc_cols = pow2_cols(kBMul * ncols_max);
    const int nst = (it.k1 - it.k0 + kKS - 1) / kKS;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], kGroupWarps);
            mbar_init(&empty[s], 1);
        }
        for (int s = 0; s < kInStages; ++s) {
            mbar_init(&in_full[s], 1);
            mbar_init(&in_empty[s], kGroupWarps);
        }
        for (int a = 0; a < 4; ++a) mbar_init(&acc_full[a], 1);
        for (int a = 0; a < 2; ++a) mbar_init(&acc_empty[a], 4);
        for (int a = 0; a < 2; ++a) mbar_init(&done_bar[a], 1);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // accumulator (issuer q, buffer b) at TMEM column (2 q + b) acc_cols
    // accumulators (issuer, buffer) and, with split precision, the running sum
    const uint32_t tmem_cols = pow2_cols((2 * NISS + SPLIT) * (int)acc_cols);
    if (warp == kMmaWarp) {
        tmem_alloc(s_tmem, tmem_cols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;

    if (warp < kGrp * kGroupWarps) {
        // ------------------------------------------------------------ generators
        const int grp = warp / kGroupWarps, gw = warp % kGroupWarps;
        const int half = it.N / 2;
        // Conjugate symmetry about the cutout centre (pixel offsets (r - N/2) cell):
        // row N - r of the row twiddles holds the conjugate of row r, and so do the
        // column twiddles when the weights are real (uv and image-plane methods).  For
        // a tile that spans a whole cutout of 64 or 128 pixels only rows N/2 .. N-1 are
        // generated; rows 1 .. N/2 are their conjugates and row 0 the conjugate of the
        // value one step past row N-1.
        const bool mirror = (MIR == 2) || (MIR == 4) || (MIR == 1 && it.j0 == 0 && it.i0 == 0 && it.ncols == it.N && it.N <= 128 && (it.N & 63) == 0);
        // 32-row chains of the A (128 rows) and B tiles (complex output: A rows past the
        // cutout are skipped)
        const int nA = mirror ? it.N / 64 : (MIR == 5 ? min(4, (it.N - it.j0 + 31) / 32) : 4);
        const int nB = mirror ? it.N / 64 : ncols / 32;
        uint32_t off8[8];
        stmatrix_offsets(lane, off8);
        for (int s_i = grp; s_i < nst; s_i += kGrp) {
            const int slot = s_i % kStages;
            const uint32_t ph = (uint32_t)(s_i / kStages) & 1u;
            const int islot = s_i % kInStages;
            bool ok = wait_bounded(&in_full[islot], (uint32_t)(s_i / kInStages) & 1u, s_abort, err);
            if (!__all_sync(0xffffffffu, ok)) break;   // warp-uniform exit
            const float2 *in_uv = (const float2 *)(smem + L.in_off + islot * kSlot);
            const float2 uvk = in_uv[lane];
            const bool kin = it.k0 + s_i * kKS + lane < it.k1;
            const float2 wk = kin ? in_uv[kKS + lane] : make_float2(0.f, 0.f);
            const float w2k = (MIR == 4 && kin) ? in_uv[2 * kKS + lane].x : 0.f;
            __syncwarp();
            if (lane == 0) mbar_arrive(&in_empty[islot]);   // the input slot may be refilled
            if (s_i >= kStages) {
                ok = wait_bounded(&empty[slot], ph ^ 1u, s_abort, err);
                if (!__all_sync(0xffffffffu, ok)) break;
            }
            const uint32_t a_tile = smem_u32(smem + L.a_off + slot * kAStage);
            const uint32_t b_tile = smem_u32(smem + L.b_off + slot * b_stage);
            if (MIR == 0 && !SPLIT && nA == 4 && nB == 4) {
                // complex weights on a full 128 x 128 tile: warps 0-1 take two A chains each
                // (rows 64 gw .. 64 gw + 63), warps 2-3 two B chains each, so the two chains
                // of a warp share one theta and its step phasors
                const bool isA = gw < 2;
                const int c0 = 2 * (gw & 1);
                const float th = isA ? uvk.y * cell : -uvk.x * cell;
                const ChainSteps S = chain_steps(th);
#pragma unroll 1
                for (int c = c0; c < c0 + 2; ++c) {
                    if (isA)
                        gen_chain32_s<BF16, false, false, SPLIT>(S, a_tile + c * 32 * 128, off8, th,
                                                                 it.j0 + c * 32 - half, wk, true, 0, false, 0,
                                                                 (uint32_t)kATileBytes);
                    else
                        gen_chain32_s<BF16, false, false, SPLIT>(S, b_tile + c * 32 * 128, off8, th,
                                                                 it.i0 + c * 32 - half, wk, false, 0, false, 0,
                                                                 bt_stride);
                }
            } else
            for (int ch = gw; ch < nA + nB; ch += kGroupWarps) {
                if (MIR == 5) {   // A: weighted column twiddles; B: row twiddles, real and imaginary halves
                    if (ch < nA)
                        gen_chain32<BF16>(a_tile + ch * 32 * 128, off8, uvk.y * cell, it.j0 + ch * 32 - half, wk, true);
                    else
                        gen_chain32<BF16, false, true>(b_tile + (ch - nA) * 32 * 128, off8, -uvk.x * cell,
                                                       it.i0 + (ch - nA) * 32 - half, wk, false,
                                                       (uint32_t)ncols * 128u);
                } else if (MIR == 4) {   // A: unweighted column twiddles; B: weighted row twiddles, both halves
                    const bool isA = ch < nA;
                    const int c = isA ? ch : ch - nA;
                    const int R0 = half + 32 * c;
                    if (isA)
                        gen_chain32<BF16, true>(a_tile + (uint32_t)R0 * 128u, off8, uvk.y * cell, 32 * c, wk, false,
                                                a_tile + (uint32_t)(it.N - R0) * 128u, c == nA - 1, a_tile);
                    else
                        gen_chain32_dual<BF16>(b_tile + (uint32_t)R0 * 128u, b_tile + (uint32_t)(it.N - R0) * 128u,
                                               (uint32_t)it.N * 128u, -uvk.x * cell, 32 * c, wk.x, w2k, c == nB - 1,
                                               b_tile);
                } else if (mirror) {   // rows R0 .. R0+31 (R0 = N/2 + 32 c) and their mirrors N - R0 - r
                    const bool isA = ch < nA;
                    const int c = isA ? ch : ch - nA;
                    const int R0 = half + 32 * c;
                    const uint32_t tile = isA ? a_tile : b_tile;
                    gen_chain32<BF16, true, false, SPLIT>(tile + (uint32_t)R0 * 128u, off8,
                                                          isA ? uvk.y * cell : -uvk.x * cell, 32 * c, wk, isA,
                                                          tile + (uint32_t)(it.N - R0) * 128u, c == nA - 1, tile,
                                                          isA ? (uint32_t)kATileBytes : bt_stride);
                } else if (ch < nA) {   // weighted column twiddles c_k[j], rows j = j0 + 32 ch + r
                    gen_chain32<BF16, false, false, SPLIT>(a_tile + ch * 32 * 128, off8, uvk.y * cell,
                                                           it.j0 + ch * 32 - half, wk, true, 0, false, 0,
                                                           (uint32_t)kATileBytes);
                } else {                // conjugated row twiddles (a_r, -a_i), rows i = i0 + 32 (ch - nA) + r
                    gen_chain32<BF16, false, false, SPLIT>(b_tile + (ch - nA) * 32 * 128, off8, -uvk.x * cell,
                                                           it.i0 + (ch - nA) * 32 - half, wk, false, 0, false, 0,
                                                           bt_stride);
                }
            }
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&full[slot]);
        }
    } else if (warp == kMmaWarp || (NISS == 2 && warp == kMma2Warp)) {
        // ------------------------------------------------------------ MMA issue
        // Issuer q takes the stages s = q (mod NISS); with an even ring depth every
        // slot belongs to one issuer.  Accumulation range d covers stages
        // [d kRange, (d + 1) kRange) and uses buffer b = d mod 2.
        if (lane == 0) {
            const int q = (warp == kMmaWarp) ? 0 : 1;
            // The MMA issue blocks this thread until the tensor core takes the
            // instruction, so the per-stage path is kept short: slot, phase and range
            // by increment, descriptors by adding the slot offset to the 14-bit address
            // field (shared addresses < 256 KB cannot carry out of it).
            const uint32_t idesc = idesc_f16(128, kBMul * ncols, BF16);
            const uint64_t ad0 = desc_sw128(smem_u32(smem + L.a_off));
            const uint64_t bd0 = desc_sw128(smem_u32(smem + L.b_off));
            int slot = q, r = q, d = 0;
            uint32_t ph = 0;
            for (int s_i = q; s_i < nst; s_i += NISS) {
                if (!wait_bounded(&full[slot], ph, s_abort, err)) break;
                const int b = d & 1;
                if (r == q && d >= 2 &&   // first own stage of a range: the buffer's last drain is done
                    !wait_bounded(&acc_empty[b], (uint32_t)((d >> 1) - 1) & 1u, s_abort, err))
                    break;
                tc_fence_after();
                const uint64_t ad = ad0 + (uint64_t)(slot * (kAStage >> 4));
                const uint64_t bd = bd0 + (uint64_t)(slot * (b_stage >> 4));
                const uint32_t dt = tmem + (uint32_t)(2 * q + b) * acc_cols;
                // K' = 16 per MMA = 32 bytes (descriptor units of 16 B: +2) of the 128-byte row
                // a range's first MMA clears the buffer, except issuer 0's from range 2 on:
                // the drain has left the compensation of the running sum there
                if (r == q) umma_f16(dt, ad, bd, idesc, (SPLIT && q == 0 && d >= 2) ? 1u : 0u);
                else umma_f16(dt, ad, bd, idesc, 1u);
                umma_f16(dt, ad + 2, bd + 2, idesc, 1u);
                umma_f16(dt, ad + 4, bd + 4, idesc, 1u);
                umma_f16(dt, ad + 6, bd + 6, idesc, 1u);
                if (SPLIT) {   // A_hi B_lo, then A_lo B_hi
                    const uint64_t bl = bd + (uint64_t)(bt_stride >> 4), al = ad + (uint64_t)(kATileBytes >> 4);
#pragma unroll
                    for (int kk = 0; kk < 8; kk += 2) umma_f16(dt, ad + kk, bl + kk, idesc, 1u);
#pragma unroll
                    for (int kk = 0; kk < 8; kk += 2) umma_f16(dt, al + kk, bd + kk, idesc, 1u);
                }
                umma_commit(&empty[slot]);
                r += NISS;
                if (r >= kRange || s_i + NISS >= nst) umma_commit(&acc_full[2 * q + b]);
                if (r >= kRange) {
                    r -= kRange;
                    ++d;
                }
                slot += NISS;
                if (slot >= kStages) {
                    slot -= kStages;
                    ph ^= 1u;
                }
            }
            // all issued MMAs complete before TMEM is released (waited for even after
            // an abort; the wait is still time-limited)
            umma_commit(&done_bar[q]);
            wait_bounded(&done_bar[q], 0, &no_abort, err);
        }
        __syncwarp();
    } else if (warp == kInWarp) {
        // ------------------------------------------------------------ input ring
        // stage s's uv and w (256 B each) into slot s % kInStages, once the generator
        // group of stage s - kInStages has read that slot
        if (lane == 0) {
            const float2 *wp = w + (int64_t)it.slot * ldw;
            int issued = 0;
            for (int s_i = 0; s_i < nst; ++s_i) {
                const int islot = s_i % kInStages;
                if (s_i >= kInStages &&
                    !wait_bounded(&in_empty[islot], (uint32_t)(s_i / kInStages - 1) & 1u, s_abort, err))
                    break;
                uint8_t *dst = smem + L.in_off + islot * kSlot;
                const int32_t kb = it.k0 + s_i * kKS;
                mbar_arrive_expect_tx(&in_full[islot], kSlot);
                bulk_g2s(dst, uv + kb, kKS * 8, &in_full[islot]);
                bulk_g2s(dst + kKS * 8, wp + kb, kKS * 8, &in_full[islot]);
                if (MIR == 4) bulk_g2s(dst + kKS * 16, w2 + (int64_t)it.slot * ldw + kb, kKS * 8, &in_full[islot]);
                issued = s_i + 1;
            }
            // every copy has landed before the CTA exits (the last use of each slot)
            for (int s_i = max(0, issued - kInStages); s_i < issued; ++s_i)
                wait_bounded(&in_full[s_i % kInStages], (uint32_t)(s_i / kInStages) & 1u, &no_abort, err);
        }
        __syncwarp();
    } else if (warp == kMma2Warp) {
        // second issuer, idle with one issuer (NISS == 1): it must not join the drain
        // warps (lane quarters 0-3, four arrivals per accumulator release)
    } else if (warp < kGenWarps) {
        // generator warps beyond the ring depth's groups (split precision): idle
    } else {
        // ------------------------------------------------------------ drain
        // The partial cutout is stored transposed (element (j, i) at i N + j), so the 32
        // lanes of a warp (32 consecutive rows j, one column per access) touch one
        // contiguous 128-byte line.
        const int q = warp - kDrainWarp0;          // TMEM lane quarter (warp % 4)
        const int j = it.j0 + q * 32 + lane;       // output row (m offset index)
        float *dst = partial + (int64_t)it.split * split_stride + it.out_off + (int64_t)it.i0 * it.N + j;
        const int64_t cstride = it.N;
        const bool row_ok = j < it.N;
        const int ncol_valid = min(ncols, it.N - it.i0);
        float *dst2 = dst + part2;   // second cutout of the fused form
        if (nst == 0) {
            if (row_ok)
                for (int c = 0; c < ncol_valid; ++c) {
                    dst[c * cstride] = 0.f;
                    if (kBMul == 2) dst2[c * cstride] = 0.f;
                }
        }
        const int ndrain = (nst + kRange - 1) / kRange;
        // split precision: running sum of the drained ranges in TMEM columns after the
        // accumulators
        const uint32_t tsum = tmem + ((uint32_t)(q * 32) << 16) + 2u * NISS * acc_cols;
        for (int d = 0; d < ndrain; ++d) {
            const int b = d & 1;
            // issuer 1 has a stage in range d unless the range holds a single stage
            const bool two = (NISS == 2) && (min(nst, (d + 1) * kRange) - d * kRange > 1);
            bool ok = wait_bounded(&acc_full[b], (uint32_t)(d >> 1) & 1u, s_abort, err);
            if (two && ok) ok = wait_bounded(&acc_full[2 + b], (uint32_t)(d >> 1) & 1u, s_abort, err);
            if (!__all_sync(0xffffffffu, ok)) break;   // warp-uniform exit
            tc_fence_after();
            const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)b * acc_cols;
            for (int c0 = 0; c0 < kBMul * ncols; c0 += 16) {
                // fused form: columns ncols .. 2 ncols - 1 are the second cutout
                float *const dd = (kBMul == 2 && c0 >= ncols) ? dst2 : dst;
                const int cb = (kBMul == 2 && c0 >= ncols) ? c0 - ncols : c0;
                float v[16];
                tmem_ld16(ta + (uint32_t)c0, v);
                if (two) {
                    float v2[16];
                    tmem_ld16(ta + 2u * acc_cols + (uint32_t)c0, v2);
#pragma unroll
                    for (int e = 0; e < 16; ++e) v[e] += v2[e];
                }
                if (SPLIT) {
                    float sv[16], cv[16];   // running sum; compensation for the buffer's next range
#pragma unroll
                    for (int e = 0; e < 16; ++e) sv[e] = 0.f;
                    if (d > 0) tmem_ld16(tsum + (uint32_t)c0, sv);
#pragma unroll
                    for (int e = 0; e < 16; ++e) two_sum(sv[e], v[e], v[e], cv[e]);
                    if (d < ndrain - 1) {
                        tmem_st16(tsum + (uint32_t)c0, v);
                    } else if (row_ok) {   // last range: the CTA's sum goes out once
#pragma unroll
                        for (int e = 0; e < 16; ++e)
                            if (cb + e < ncol_valid) dd[(cb + e) * cstride] = v[e];
                    }
                    // issuer 0's buffer b is accumulated on again by range d + 2
                    if (d + 2 < ndrain) tmem_st16(ta + (uint32_t)c0, cv);
                    continue;
                }
                if (row_ok) {
                    // eight loads in flight before their stores (one L2 round trip per eight)
#pragma unroll
                    for (int h = 0; h < 16; h += 8) {
                        float o[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e)
                            o[e] = (d > 0 && cb + h + e < ncol_valid) ? dd[(cb + h + e) * cstride] : 0.f;
#pragma unroll
                        for (int e = 0; e < 8; ++e)
                            if (cb + h + e < ncol_valid) dd[(cb + h + e) * cstride] = o[e] + v[h + e];
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[b]);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kMmaWarp) tmem_dealloc(tmem, tmem_cols);
}

// Self-test: one 128 x n x 64 FP16 GEMM through the same layout, descriptors,
// instruction descriptor and TMEM read-out as the contraction kernel.
__global__ void __launch_bounds__(128, 1)
    k_selftest(const __half *__restrict__ A, const __half *__restrict__ B, float *__restrict__ D, int n,
               int *err) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *a_tile = smem;
    uint8_t *b_tile = smem + kATileBytes;
    uint64_t *bar = (uint64_t *)(smem + kATileBytes + 256 * 128);
    uint32_t *s_tmem = (uint32_t *)(bar + 1);
    volatile int *s_abort = (volatile int *)(s_tmem + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t cols = pow2_cols(n);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        tmem_alloc(s_tmem, cols);
        tmem_relinquish();
    }
    // operands: pairs of FP16 (k' = 2 kp, 2 kp + 1) into the swizzled K-major tiles
    for (int idx = threadIdx.x; idx < 128 * 32; idx += blockDim.x) {
        const int row = idx >> 5, kp = idx & 31;
        *reinterpret_cast<uint32_t *>(a_tile + sw128_pair_offset(row, kp)) =
            *reinterpret_cast<const uint32_t *>(A + row * 64 + 2 * kp);
    }
    for (int idx = threadIdx.x; idx < n * 32; idx += blockDim.x) {
        const int row = idx >> 5, kp = idx & 31;
        *reinterpret_cast<uint32_t *>(b_tile + sw128_pair_offset(row, kp)) =
            *reinterpret_cast<const uint32_t *>(B + row * 64 + 2 * kp);
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;
    if (threadIdx.x == 0) {
        const uint32_t idesc = idesc_f16(128, n, 0);
        const uint64_t ad = desc_sw128(smem_u32(a_tile)), bd = desc_sw128(smem_u32(b_tile));
        for (int kk = 0; kk < 4; ++kk) umma_f16(tmem, ad + 2 * kk, bd + 2 * kk, idesc, kk > 0 ? 1u : 0u);
        umma_commit(bar);
    }
    __syncwarp();
    const bool ok = __all_sync(0xffffffffu, wait_bounded(bar, 0, s_abort, err));
    tc_fence_after();
    if (ok) {
        const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < n; c0 += 16) {
            float v[16];
            tmem_ld16(ta + (uint32_t)c0, v);
            for (int e = 0; e < 16; ++e) D[(warp * 32 + lane) * n + c0 + e] = v[e];
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, cols);
}

// A wait that nothing completes: the bounded-wait path with a caller-given limit.
__global__ void k_wait_timeout(unsigned long long limit_ns, int *err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long t0 = globaltimer();
        for (;;) {
            if (mbar_try_wait(&bar, 0, 100000u)) return;   // never completes
            if (globaltimer() - t0 > limit_ns) {
                atomicExch(err, 1);
                return;
            }
        }
    }
}

}  // namespace

int selftest_timeout(int limit_ms) {
    int *err = nullptr;
    if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) { cudaGetLastError(); return PSF_ENOMEM; }
    cudaError_t e = cudaMemset(err, 0, sizeof(int));
    if (e == cudaSuccess) {
        k_wait_timeout<<<1, 32>>>((unsigned long long)limit_ms * 1000000ull, err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int flag = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&flag, err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(err);
    if (e != cudaSuccess) { cudaGetLastError(); return PSF_ECUDA; }
    return flag ? PSF_ETIMEOUT : PSF_OK;
}

template <int BF16, int S, int NISS, int MIR, int SPLIT = 0>
static cudaError_t launch_tc_t(const DevObs &o, const float2 *w, int64_t ldw, const TcItem *items, int nitems,
                               int ncols_max, float cell, float *partial, int64_t split_stride, int *err,
                               cudaStream_t st, const float2 *w2 = nullptr, int64_t part2 = 0) {
    const SmemLayout L =
        smem_layout((MIR == 4 || MIR == 5 ? 2 : 1) * ncols_max, S, MIR == 4 ? kKS * 24 : kInSlotBytes, SPLIT);
    const size_t bytes = L.bytes + 1024;
    cudaError_t e = cudaFuncSetAttribute(k_psf_tc<BF16, S, NISS, MIR, SPLIT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    k_psf_tc<BF16, S, NISS, MIR, SPLIT><<<nitems, kThreads, bytes, st>>>(o.uv, w, ldw, items, ncols_max, cell,
                                                                          partial, split_stride, err, w2, part2);
    return cudaGetLastError();
}

cudaError_t launch_psf_tc(const DevObs &o, const float2 *w, int64_t ldw, const TcItem *items, int nitems,
                          int ncols_max, int bf16, float cell, int wreal, float *partial, int64_t split_stride,
                          int *err, cudaStream_t st, int split) {
    if (nitems <= 0) return cudaSuccess;
    if (split) {   // tiles of at most 128 columns
        if (ncols_max > 128) return cudaErrorInvalidValue;
        // 3 stages (128 columns): one issuer (twelve MMAs per stage hide its barrier round
        // trip; two issuers need an even depth); 4 stages (<= 64 columns): two issuers
#define PSF_TC_SPLIT(B, SS)                                                                                    \
    if (bf16 == B && stages_for(ncols_max, 1) == SS) {                                                         \
        constexpr int NI = SS % 2 == 0 ? 2 : 1;                                                                \
        if (wreal == 2)                                                                                        \
            return launch_tc_t<B, SS, NI, 2, 1>(o, w, ldw, items, nitems, ncols_max, cell, partial, split_stride, \
                                                err, st);                                                      \
        return wreal ? launch_tc_t<B, SS, NI, 1, 1>(o, w, ldw, items, nitems, ncols_max, cell, partial,        \
                                                    split_stride, err, st)                                     \
                     : launch_tc_t<B, SS, NI, 0, 1>(o, w, ldw, items, nitems, ncols_max, cell, partial,        \
                                                    split_stride, err, st);                                    \
    }
        PSF_TC_SPLIT(0, 3) PSF_TC_SPLIT(0, 4) PSF_TC_SPLIT(1, 3) PSF_TC_SPLIT(1, 4)
#undef PSF_TC_SPLIT
        return cudaErrorInvalidValue;
    }
    const int S = stages_for(ncols_max);
    // two issuers while both double-buffered accumulator pairs fit in TMEM (<= 128 columns)
#define PSF_TC_CASE(B, SS)                                                                                  \
    if (bf16 == B && S == SS) {                                                                             \
        constexpr int NI = SS == 4 ? 1 : 2;                                                                 \
        if (wreal == 2)                                                                                     \
            return launch_tc_t<B, SS, NI, 2>(o, w, ldw, items, nitems, ncols_max, cell, partial, split_stride, \
                                             err, st);                                                      \
        return wreal ? launch_tc_t<B, SS, NI, 1>(o, w, ldw, items, nitems, ncols_max, cell, partial,         \
                                                 split_stride, err, st)                                      \
                     : launch_tc_t<B, SS, NI, 0>(o, w, ldw, items, nitems, ncols_max, cell, partial,         \
                                                 split_stride, err, st);                                     \
    }
    PSF_TC_CASE(0, 4) PSF_TC_CASE(0, 6) PSF_TC_CASE(0, 8) PSF_TC_CASE(1, 4) PSF_TC_CASE(1, 6) PSF_TC_CASE(1, 8)
#undef PSF_TC_CASE
    return cudaErrorInvalidValue;
}

cudaError_t launch_psf_tc_uvimg(const DevObs &o, const float2 *w_uv, const float2 *w_img, int64_t ldw,
                                const TcItem *items, int nitems, int ncols_max, int bf16, float cell, float *partial,
                                int64_t split_stride, int64_t part2, int *err, cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
    if (ncols_max != 64 && ncols_max != 128) return cudaErrorInvalidValue;
    // B tiles of 2 ncols rows: 128 rows -> 6 stages, two issuers; 256 rows -> 4 stages, one
    if (ncols_max == 64)
        return bf16 ? launch_tc_t<1, 6, 2, 4>(o, w_uv, ldw, items, nitems, 64, cell, partial, split_stride, err, st,
                                              w_img, part2)
                    : launch_tc_t<0, 6, 2, 4>(o, w_uv, ldw, items, nitems, 64, cell, partial, split_stride, err, st,
                                              w_img, part2);
    return bf16 ? launch_tc_t<1, 4, 1, 4>(o, w_uv, ldw, items, nitems, 128, cell, partial, split_stride, err, st,
                                          w_img, part2)
                : launch_tc_t<0, 4, 1, 4>(o, w_uv, ldw, items, nitems, 128, cell, partial, split_stride, err, st,
                                          w_img, part2);
}

cudaError_t launch_psf_tc_cplx(const DevObs &o, const float2 *w, int64_t ldw, const TcItem *items, int nitems,
                               int ncols_max, int bf16, float cell, float *partial, int64_t split_stride,
                               int64_t part2, int *err, cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
    if (ncols_max > 128) return cudaErrorInvalidValue;
    // B tiles of 2 ncols rows: <= 128 rows -> 6 stages, two issuers; up to 256 -> 4, one
    if (2 * ncols_max <= 128)
        return bf16 ? launch_tc_t<1, 6, 2, 5>(o, w, ldw, items, nitems, ncols_max, cell, partial, split_stride, err,
                                              st, nullptr, part2)
                    : launch_tc_t<0, 6, 2, 5>(o, w, ldw, items, nitems, ncols_max, cell, partial, split_stride, err,
                                              st, nullptr, part2);
    return bf16 ? launch_tc_t<1, 4, 1, 5>(o, w, ldw, items, nitems, ncols_max, cell, partial, split_stride, err, st,
                                          nullptr, part2)
                : launch_tc_t<0, 4, 1, 5>(o, w, ldw, items, nitems, ncols_max, cell, partial, split_stride, err, st,
                                          nullptr, part2);
}

int selftest_umma(const void *a, const void *b, float *d, int n) {
    int *err = nullptr;
    if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) { cudaGetLastError(); return PSF_ENOMEM; }
    cudaMemset(err, 0, sizeof(int));
    const size_t bytes = kATileBytes + 256 * 128 + 256 + 1024;
    cudaError_t e = cudaFuncSetAttribute(k_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) {
        k_selftest<<<1, 128, bytes>>>((const __half *)a, (const __half *)b, d, n, err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    int flag = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&flag, err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(err);
    if (e != cudaSuccess) { cudaGetLastError(); return PSF_ECUDA; }
    return flag ? PSF_ETIMEOUT : PSF_OK;
}

}  // namespace psf
