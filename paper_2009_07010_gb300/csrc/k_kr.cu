// Batched (Khatri-Rao) tcgen05 contraction: many positions with the same cutout size.
//
//   X[p][q] = sum_k Re( w_{p,k} KR_k[q] ),   KR_k[q] = exp(2 pi i (u_k dl_i + v_k dm_j)),
//   pixel q = j N + i,  w_{p,k} = W_k D_k(l0_p)                         (Eqs. 21-22)
//
// As a real GEMM with K' = 2K: A'[p][2k] = Re w, A'[p][2k+1] = -Im w (the weights,
// precomputed per position chunk into an FP16/BF16 buffer and loaded by 2-D TMA with
// 128-byte swizzle), B'[q][2k] = Re KR, B'[q][2k+1] = Im KR (generated on chip).
// One CTA computes a 128-position x 256-pixel tile over a range of visibilities:
//   warps 0-15   (four groups on stages s mod 4) generate the 256 pixel twiddles of
//                each 32-visibility stage: each
//                lane owns one visibility and walks a 32-pixel run of one cutout row
//                (phasor recurrence along l, seeded from the MUFU sine/cosine of the
//                reduced phase u dl + v dm), FP16/BF16 pairs into the swizzled layout;
//   warp 20      TMA producer of the weight tile of each stage;
//   warp 21      TMEM allocation and the single-thread tcgen05.mma issue
//                (M = 128, N = 256, K = 16);
//   warp 22      the uv input ring (bulk copies), refilled when the generator group
//                of a stage has read its slot;
//   warps 16-19  every kFoldStages stages add the active TMEM accumulator into a
//                running-sum region of TMEM (short FP32 accumulation runs); at the
//                end they add sum + active into the output with global atomics (the
//                output is zeroed first; several visibility ranges of a tile add up).
// Every barrier wait is bounded (2 s); on expiry the CTA raises the error flag, stops,
// waits (bounded) for its copies in flight and issued MMAs and frees TMEM.
#include "psf_internal.cuh"
#include "tc_ptx.cuh"

#include <cuda.h>

#include <algorithm>

namespace psf {
namespace {
using namespace tc;

constexpr int kKrStages = 4;
constexpr int kKrIn = 16;             // uv input ring depth (stages)
constexpr int kKrKS = 32;             // visibilities per stage
constexpr int kKrGenWarps = 16;       // four groups of 4; group g generates stages s = g (mod 4)
constexpr int kKrGroupWarps = 4;
constexpr int kKrGroups = kKrGenWarps / kKrGroupWarps;
constexpr int kKrFoldWarp0 = 16;
constexpr int kKrTmaWarp = 20;
constexpr int kKrMmaWarp = 21;
constexpr int kKrInWarp = 22;
constexpr int kKrThreads = 23 * 32;
constexpr int kKrFoldStages = 64;
// roles that read each item index from the ring: 16 generator warps, 4 fold warps, the
// MMA issuer and the uv ring (one arrival each)
constexpr int kKrItemReaders = kKrGenWarps + 4 + 1 + 1;
// Slot-reuse parity waits stay unambiguous only with at most as many generator groups
// as operand stages (see k_tc.cu).
static_assert(kKrGroups <= kKrStages && kKrGroups <= kKrIn, "generator groups exceed a ring depth");
constexpr uint32_t kKrATile = 128 * 128;   // 128 positions x 64 K' x 2 B
constexpr uint32_t kKrBTile = 256 * 128;   // 256 pixels x 64 K' x 2 B
constexpr uint32_t kKrInSlot = 2 * kKrKS * 8;  // uv per stage (64 visibilities in the real form)
constexpr uint32_t kKrSmemBytes =
    kKrStages * (kKrATile + kKrBTile) + kKrIn * kKrInSlot + 512 + 1024;
static_assert((2 * kKrStages + 2 * kKrIn + 3 + 5) * 8 + 2 * 4 + 8 <= 512, "barrier block exceeds its reserve");

// One 32-pixel run of one visibility (this lane): value(r) = exp(2 pi i (theta (n0 + r) + phi)),
// r = 0..31, as eight interleaved 4-pixel pieces in packed FP32x2 recurrences.
// The step phasor st = exp(2 pi i theta) and its 4-, 8- and 16-row strides depend only on
// the visibility, so the caller forms them once per stage for all runs of its lane.
struct Steps {
    float2 st, s4, s8, s16;
};
__device__ __forceinline__ Steps make_steps(float theta) {
    Steps S;
    S.st = cis_turns(theta);
    const float2 s2 = cmulf(S.st, S.st);
    S.s4 = cmulf(s2, s2);
    S.s8 = cmulf(S.s4, S.s4);
    S.s16 = cmulf(S.s8, S.s8);
    return S;
}

template <int BF16>
__device__ __forceinline__ void gen_run32(uint32_t base, const uint32_t (&off)[8], float theta, int n0, float phi,
                                          const Steps &S) {
    // eight interleaved 4-row pieces: rows q + 4p (p = 0..7) at step q = 0..3; one
    // sine/cosine evaluation per run (row 0), piece seeds by the 4- and 16-row strides
    const float2 st = S.st, s4 = S.s4, s8 = S.s8, s16 = S.s16;
    float2 z[8];
    z[0] = cis_turns(fmaf(theta, (float)n0, phi));
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
        stmatrix_x4(base + off[q], pack2<BF16>(re[0].x, im[0].x), pack2<BF16>(re[1].x, im[1].x),
                    pack2<BF16>(re[0].y, im[0].y), pack2<BF16>(re[1].y, im[1].y));
        stmatrix_x4(base + off[q + 4], pack2<BF16>(re[2].x, im[2].x), pack2<BF16>(re[3].x, im[3].x),
                    pack2<BF16>(re[2].y, im[2].y), pack2<BF16>(re[3].y, im[3].y));
        if (q < 3) {
#pragma unroll
            for (int pp = 0; pp < 4; ++pp) {
                const float2 t = __fmul2_rn(im[pp], nsi), u = __fmul2_rn(im[pp], sr);
                im[pp] = __ffma2_rn(re[pp], si, u);
                re[pp] = __ffma2_rn(re[pp], sr, t);
            }
        }
    }
}

// Real-weight form: lane t owns visibilities 2t and 2t+1 of a 64-visibility stage and
// stores the pair (Re KR_2t, Re KR_2t+1) per pixel; the recurrences are packed across
// the two visibilities, four interleaved 8-pixel pieces.
struct StepsR {   // two visibilities: steps and their 8- and 16-row strides
    float2 sa, sb, a8, a16, b8, b16;
};
__device__ __forceinline__ StepsR make_steps_real(float2 ta) {
    StepsR S;
    S.sa = cis_turns(ta.x);
    S.sb = cis_turns(ta.y);
    const float2 a2 = cmulf(S.sa, S.sa), a4 = cmulf(a2, a2);
    const float2 b2 = cmulf(S.sb, S.sb), b4 = cmulf(b2, b2);
    S.a8 = cmulf(a4, a4);
    S.a16 = cmulf(S.a8, S.a8);
    S.b8 = cmulf(b4, b4);
    S.b16 = cmulf(S.b8, S.b8);
    return S;
}

template <int BF16>
__device__ __forceinline__ void gen_run32_real(uint32_t base, const uint32_t (&off)[8], float2 ta, int n0,
                                               float2 phi, const StepsR &S) {
    // ta = (theta_u of visibility 2t, of 2t+1); phi likewise
    // piece seeds (rows 0, 8, 16, 24) from row 0 and the 8- and 16-row strides
    // (squarings of the step, formed by the caller): two sine/cosine evaluations per run
    const float2 sa = S.sa, sb = S.sb;
    float2 za[4], zb[4];
    za[0] = cis_turns(fmaf(ta.x, (float)n0, phi.x));
    zb[0] = cis_turns(fmaf(ta.y, (float)n0, phi.y));
    za[1] = cmulf(za[0], S.a8);
    za[2] = cmulf(za[0], S.a16);
    za[3] = cmulf(za[1], S.a16);
    zb[1] = cmulf(zb[0], S.b8);
    zb[2] = cmulf(zb[0], S.b16);
    zb[3] = cmulf(zb[1], S.b16);
    float2 re[4], im[4];
#pragma unroll
    for (int pc = 0; pc < 4; ++pc) {
        re[pc] = make_float2(za[pc].x, zb[pc].x);
        im[pc] = make_float2(za[pc].y, zb[pc].y);
    }
    const float2 sr = make_float2(sa.x, sb.x), si = make_float2(sa.y, sb.y), nsi = make_float2(-sa.y, -sb.y);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        // rows q, q+8, q+16, q+24 = pieces 0..3 at step q
        stmatrix_x4(base + off[q], pack2<BF16>(re[0].x, re[0].y), pack2<BF16>(re[1].x, re[1].y),
                    pack2<BF16>(re[2].x, re[2].y), pack2<BF16>(re[3].x, re[3].y));
        if (q < 7) {
#pragma unroll
            for (int pp = 0; pp < 4; ++pp) {
                const float2 t = __fmul2_rn(im[pp], nsi), u = __fmul2_rn(im[pp], sr);
                im[pp] = __ffma2_rn(re[pp], si, u);
                re[pp] = __ffma2_rn(re[pp], sr, t);
            }
        }
    }
}

template <int BF16, int REAL>
__global__ void __launch_bounds__(kKrThreads, 1)
    k_psf_kr(const __grid_constant__ CUtensorMap wmap, const KrItem *__restrict__ items, int nitems,
             int *__restrict__ queue, const float2 *__restrict__ uv, int32_t kchunk0, float cell,
             const int64_t *__restrict__ out_off, float *__restrict__ out, int *err) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *a_base = smem;
    uint8_t *b_base = smem + kKrStages * kKrATile;
    uint8_t *in_base = b_base + kKrStages * kKrBTile;
    uint64_t *full = (uint64_t *)(in_base + kKrIn * kKrInSlot);
    uint64_t *empty = full + kKrStages;
    uint64_t *in_full = empty + kKrStages;
    uint64_t *in_empty = in_full + kKrIn;
    uint64_t *acc_full = in_empty + kKrIn;
    uint64_t *acc_empty = acc_full + 1;
    uint64_t *done_bar = acc_empty + 1;
    uint64_t *item_full = done_bar + 1;    // [2]: the item index of ring slot written
    uint64_t *item_empty = item_full + 2;  // [2]: every role has read it
    uint64_t *item_done = item_empty + 2;  // the fold warps have finished an item
    int *s_item = (int *)(item_done + 1);   // [2]
    uint32_t *s_tmem = (uint32_t *)(s_item + 2);
    volatile int *s_abort = (volatile int *)(s_tmem + 1);
    volatile int no_abort = 0;   // teardown waits ignore the abort flag

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int KS = REAL ? 2 * kKrKS : kKrKS;   // visibilities per stage (64 K' either way)

    if (threadIdx.x == 0) {
        for (int s = 0; s < kKrStages; ++s) {
            mbar_init(&full[s], kKrGroupWarps + 1);
            mbar_init(&empty[s], 1);
        }
        for (int s = 0; s < kKrIn; ++s) {
            mbar_init(&in_full[s], 1);
            mbar_init(&in_empty[s], kKrGroupWarps);
        }
        mbar_init(acc_full, 1);
        mbar_init(acc_empty, 4);
        mbar_init(done_bar, 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(&item_full[b], 1);
            mbar_init(&item_empty[b], kKrItemReaders);
        }
        mbar_init(item_done, 4);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kKrMmaWarp) {
        tmem_alloc(s_tmem, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;   // columns [0, 256): active accumulator, [256, 512): running sum

    // Every role walks the same item sequence from the two-slot ring: the li-th item of
    // this CTA is in slot li & 1; a role reads it, acknowledges (item_empty) and keeps the
    // index in registers.  item < 0 ends the sequence.  Stages and fold ranges are
    // numbered globally across the CTA's items, so the operand rings and the accumulator
    // run on without draining between items.
    auto next_item = [&](int li, bool ack) -> int {
        const int slot = li & 1;
        if (!wait_bounded(&item_full[slot], (uint32_t)(li >> 1) & 1u, s_abort, err)) return -2;
        const int item = *(volatile int *)&s_item[slot];
        if (ack) mbar_arrive(&item_empty[slot]);
        return item;
    };
    auto item_stages = [&](const KrItem &it) { return (it.ke - it.kb + KS - 1) / KS; };

    if (warp < kKrGenWarps) {
        // ------------------------------------------------------------ pixel twiddles
        const int grp = warp / kKrGroupWarps, gw = warp % kKrGroupWarps;
        uint32_t off8[8];
        stmatrix_offsets(lane, off8);
        int g0 = 0;   // global index of the current item's first stage
        bool ok = true;
        for (int li = 0; ok; ++li) {
            int item = -2;
            if (lane == 0) item = next_item(li, true);
            item = __shfl_sync(0xffffffffu, item, 0);
            if (item < 0) { ok = item == -1; break; }
            const KrItem it = items[item];
            const int nst = item_stages(it);
            const int half = it.N / 2;
            // this group's stages of the item: global g = g0 + s with g = grp (mod 4)
            for (int s = ((grp - g0) % kKrGroups + kKrGroups) % kKrGroups; s < nst; s += kKrGroups) {
                const int g = g0 + s;
                const int slot = g % kKrStages;
                const uint32_t ph = (uint32_t)(g / kKrStages) & 1u;
                const int islot = g % kKrIn;
                bool w = wait_bounded(&in_full[islot], (uint32_t)(g / kKrIn) & 1u, s_abort, err);
                if (!__all_sync(0xffffffffu, w)) { ok = false; break; }
                const float2 *in_uv = reinterpret_cast<const float2 *>(in_base + islot * kKrInSlot);
                float2 uva, uvb;
                if (REAL) {
                    uva = in_uv[2 * lane];
                    uvb = in_uv[2 * lane + 1];
                } else {
                    uva = in_uv[lane];
                    uvb = uva;
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&in_empty[islot]);   // the input slot may be refilled
                if (g >= kKrStages) {
                    w = wait_bounded(&empty[slot], ph ^ 1u, s_abort, err);
                    if (!__all_sync(0xffffffffu, w)) { ok = false; break; }
                }
                Steps S;
                StepsR SR;
                if (REAL) SR = make_steps_real(make_float2(uva.x * cell, uvb.x * cell));
                else S = make_steps(uva.x * cell);
                for (int r0 = gw * 32; r0 < it.npx; r0 += kKrGroupWarps * 32) {   // 32-pixel runs of this warp
                    const int q = it.q0 + r0;
                    const int jrow = q / it.N, i0 = q - jrow * it.N;   // inside one cutout row
                    const uint32_t dst = smem_u32(b_base + slot * kKrBTile + r0 * 128);
                    if (REAL)
                        gen_run32_real<BF16>(dst, off8, make_float2(uva.x * cell, uvb.x * cell), i0 - half,
                                             make_float2(uva.y * cell * (float)(jrow - half),
                                                         uvb.y * cell * (float)(jrow - half)),
                                             SR);
                    else
                        gen_run32<BF16>(dst, off8, uva.x * cell, i0 - half, uva.y * cell * (float)(jrow - half), S);
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&full[slot]);
            }
            g0 += nst;
        }
    } else if (warp == kKrTmaWarp) {
        // ------------------------------------------------------------ items and weight tiles
        if (lane == 0) {
            int g = 0;
            for (int li = 0;; ++li) {
                const int islot = li & 1;
                if (li >= 2 && !wait_bounded(&item_empty[islot], (uint32_t)((li >> 1) - 1) & 1u, s_abort, err)) break;
                // Items do not overlap in the pipeline: the next one is published once the
                // fold warps have written the previous one out.  (With overlapping items the
                // twiddle tile of one stage early in a CTA's later items came out wrong in
                // about one item in ten on GB300; the cause was not found, see the design
                // notes.)  The bubble costs a ring fill per item.
                if (li >= 1 && !wait_bounded(item_done, (uint32_t)(li - 1) & 1u, s_abort, err)) break;
                const int idx = atomicAdd(queue, 1);   // largest items first (host order)
                const int item = idx < nitems ? idx : -1;
                s_item[islot] = item;
                mbar_arrive(&item_full[islot]);   // release: the index is visible to the waiters
                if (item < 0) break;
                const KrItem it = items[item];
                const int nst = item_stages(it);
                const int x0 = (REAL ? 1 : 2) * (it.kb - kchunk0);   // K' column of the item's first visibility
                bool stop = false;
                for (int s = 0; s < nst; ++s, ++g) {
                    const int slot = g % kKrStages;
                    const uint32_t ph = (uint32_t)(g / kKrStages) & 1u;
                    if (g >= kKrStages && !wait_bounded(&empty[slot], ph ^ 1u, s_abort, err)) { stop = true; break; }
                    mbar_arrive_expect_tx(&full[slot], kKrATile);
                    tma_load_2d(a_base + slot * kKrATile, &wmap, x0 + s * 2 * kKrKS, it.wrow, &full[slot]);
                }
                if (stop) break;
            }
        }
        __syncwarp();
    } else if (warp == kKrMmaWarp) {
        // ------------------------------------------------------------ MMA issue
        if (lane == 0) {
            // short per-stage issue path (the MMA issue blocks this thread): slot and
            // phase by increment, descriptors by adding the slot offset to the address
            // field, constant accumulate flags
            const uint64_t ad0 = desc_sw128(smem_u32(a_base)), bd0 = desc_sw128(smem_u32(b_base));
            int slot = 0, folds = 0;
            uint32_t ph = 0;
            bool stop = false;
            for (int li = 0; !stop; ++li) {
                const int item = next_item(li, true);
                if (item < 0) break;
                const KrItem it = items[item];
                const int nst = item_stages(it);
                const uint32_t idesc = idesc_f16(128, it.npx, BF16);
                int in_acc = 0;
                for (int s = 0; s < nst; ++s) {
                    if (!wait_bounded(&full[slot], ph, s_abort, err)) { stop = true; break; }
                    if (in_acc == 0 && folds > 0 &&
                        !wait_bounded(acc_empty, (uint32_t)(folds - 1) & 1u, s_abort, err)) { stop = true; break; }
                    tc_fence_after();
                    const uint64_t ad = ad0 + (uint64_t)(slot * (kKrATile >> 4));
                    const uint64_t bd = bd0 + (uint64_t)(slot * (kKrBTile >> 4));
                    if (in_acc == 0) umma_f16(tmem, ad, bd, idesc, 0u);
                    else umma_f16(tmem, ad, bd, idesc, 1u);
                    umma_f16(tmem, ad + 2, bd + 2, idesc, 1u);
                    umma_f16(tmem, ad + 4, bd + 4, idesc, 1u);
                    umma_f16(tmem, ad + 6, bd + 6, idesc, 1u);
                    umma_commit(&empty[slot]);
                    if (++in_acc == kKrFoldStages || s == nst - 1) {
                        umma_commit(acc_full);
                        ++folds;
                        in_acc = 0;
                    }
                    if (++slot == kKrStages) {
                        slot = 0;
                        ph ^= 1u;
                    }
                }
            }
            umma_commit(done_bar);
            wait_bounded(done_bar, 0, &no_abort, err);   // even after an abort (time-limited)
        }
        __syncwarp();
    } else if (warp == kKrInWarp) {
        // ------------------------------------------------------------ uv input ring
        if (lane == 0) {
            int g = 0, issued = 0;
            bool stop = false;
            for (int li = 0; !stop; ++li) {
                const int item = next_item(li, true);
                if (item < 0) break;
                const KrItem it = items[item];
                const int nst = item_stages(it);
                for (int s = 0; s < nst; ++s, ++g) {
                    const int islot = g % kKrIn;
                    if (g >= kKrIn && !wait_bounded(&in_empty[islot], (uint32_t)(g / kKrIn - 1) & 1u, s_abort, err)) {
                        stop = true;
                        break;
                    }
                    mbar_arrive_expect_tx(&in_full[islot], KS * 8);
                    bulk_g2s(in_base + islot * kKrInSlot, uv + it.kb + s * KS, KS * 8, &in_full[islot]);
                    issued = g + 1;
                }
            }
            // every copy has landed before the CTA exits (the last use of each slot)
            for (int q = max(0, issued - kKrIn); q < issued; ++q)
                wait_bounded(&in_full[q % kKrIn], (uint32_t)(q / kKrIn) & 1u, &no_abort, err);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ fold / output
        const int qw = warp - kKrFoldWarp0;          // TMEM lane quarter
        const int row = qw * 32 + lane;              // position row of the tile
        const uint32_t ta = tmem + ((uint32_t)(qw * 32) << 16);
        int F = 0;   // global fold range index
        bool ok = true;
        for (int li = 0; ok; ++li) {
            int item = -2;
            if (lane == 0) item = next_item(li, true);
            item = __shfl_sync(0xffffffffu, item, 0);
            if (item < 0) break;
            const KrItem it = items[item];
            const int nfold = (item_stages(it) + kKrFoldStages - 1) / kKrFoldStages;
            const bool row_ok = row < it.npos;
            float *dst = out + (row_ok ? out_off[it.slot0 + row] : 0) + it.q0;
            for (int f = 0; f < nfold; ++f, ++F) {
                const bool w = wait_bounded(acc_full, (uint32_t)F & 1u, s_abort, err);
                if (!__all_sync(0xffffffffu, w)) { ok = false; break; }
                tc_fence_after();
                const bool last = (f == nfold - 1);
                for (int c0 = 0; c0 < it.npx; c0 += 16) {
                    float v[16];
                    tmem_ld16(ta + (uint32_t)c0, v);
                    if (f > 0) {
                        float sacc[16];
                        tmem_ld16(ta + 256u + (uint32_t)c0, sacc);
#pragma unroll
                        for (int e = 0; e < 16; ++e) v[e] += sacc[e];
                    }
                    if (last) {
                        if (row_ok) {
#pragma unroll
                            for (int e = 0; e < 16; ++e) atomicAdd(dst + c0 + e, v[e]);
                        }
                    } else {
                        tmem_st16(ta + 256u + (uint32_t)c0, v);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(acc_empty);
            }
            __syncwarp();
            if (ok && lane == 0) mbar_arrive(item_done);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kKrMmaWarp) tmem_dealloc(tmem, 512);
}

}  // namespace

template <int BF16, int REAL>
static cudaError_t launch_kr_t(const CUtensorMap *m, const KrItem *items, int nitems, int *queue, int nctas,
                               const float2 *uv, int32_t kchunk0, float cell, const int64_t *out_off, float *out,
                               int *err, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_psf_kr<BF16, REAL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kKrSmemBytes);
    if (e != cudaSuccess) return e;
    k_psf_kr<BF16, REAL><<<nctas, kKrThreads, kKrSmemBytes, st>>>(*m, items, nitems, queue, uv, kchunk0, cell,
                                                                   out_off, out, err);
    return cudaGetLastError();
}

cudaError_t launch_psf_kr(const void *wmap, const KrItem *items, int nitems, int *queue, int nctas, const float2 *uv,
                          int32_t kchunk0, float cell, const int64_t *out_off, float *out, int bf16, int real, int *err,
                          cudaStream_t st) {
    if (nitems <= 0) return cudaSuccess;
    nctas = std::max(1, std::min(nctas, nitems));
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    const CUtensorMap *m = (const CUtensorMap *)wmap;
    if (bf16)
        return real ? launch_kr_t<1, 1>(m, items, nitems, queue, nctas, uv, kchunk0, cell, out_off, out, err, st)
                    : launch_kr_t<1, 0>(m, items, nitems, queue, nctas, uv, kchunk0, cell, out_off, out, err, st);
    return real ? launch_kr_t<0, 1>(m, items, nitems, queue, nctas, uv, kchunk0, cell, out_off, out, err, st)
                : launch_kr_t<0, 0>(m, items, nitems, queue, nctas, uv, kchunk0, cell, out_off, out, err, st);
}

// 2-D tensor map over the FP16/BF16 weight buffer: dim0 = pitch elements (2 KC for
// complex weights, KC for real ones), dim1 = rows; box 64 x 128 elements (one
// 128-byte-swizzled stage of 128 positions).
int make_weight_map(void *map_out, void *w16, int bf16, int64_t pitch_elems, int64_t rows) {
    typedef CUresult (*EncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static EncodeFn fn = nullptr;
    if (!fn) {
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !ptr) {
            cudaGetLastError();
            return PSF_ECUDA;
        }
        fn = (EncodeFn)ptr;
    }
    const cuuint64_t dims[2] = {(cuuint64_t)pitch_elems, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch_elems * 2};
    const cuuint32_t box[2] = {64, 128};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = fn((CUtensorMap *)map_out, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                    w16, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? PSF_OK : PSF_ECUDA;
}

int kr_smem_bytes() { return (int)kKrSmemBytes; }

}  // namespace psf
