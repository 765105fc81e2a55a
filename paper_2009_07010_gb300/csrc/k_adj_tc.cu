// Adjoint (vector-Jacobian product) of the cutout map of Eqs. 21-22 on the tensor cores.
//
// For a cotangent R = dL/dP (packed like the forward output) and positions p of one
// cutout size N, the adjoint needs per (position, visibility)
//   H_pk = sum_q R_p[q] exp(2 pi i (u_k dl_i + v_k dm_j)),   pixel q = j N + i,
// and then dL/dW_k = sum_p Re(D_k(l0_p) H_pk), dL/dl0_p = sum_k W_k Re(dD_k/dl0 H_pk)
// (likewise m0).  H is a GEMM: M = positions, N = visibilities (real and imaginary
// parts), K = pixels, with the pixel twiddles KR_k[q] generated on chip.
//
//   k_adj_r16   R (FP32, packed cutouts) -> a FP16/BF16 matrix [position row][pixel] of
//               one size group (rows padded to 128 with zeros): the TMA-loaded A operand;
//   k_adj_tc    one CTA per SM, looping over (128-position tile, 128-visibility tile)
//               items of a visibility chunk; per item the K loop runs over the N^2
//               pixels in 64-pixel stages.  Warps 0-15 (four groups on stages s mod 4):
//               each lane of a group owns one visibility of the item and writes its
//               twiddles for the stage's 64 pixels -- two 32-pixel runs along a cutout
//               row, phasor recurrences from a MUFU seed per run -- as the B operand rows
//               (Re KR_k: rows 0-127, Im KR_k: rows 128-255; K-major, 128-byte swizzle);
//               warp 20 loads the R tile of each stage by 2-D TMA; warp 21 issues
//               tcgen05.mma (M = 128, N = 256, K = 16) into one of two TMEM accumulators
//               (items alternate); warps 16-19 write the finished accumulator as
//               H[row][k] = (Re, Im) float32 pairs while the next item accumulates;
//   k_adj_fold  grid-stride over the visibilities of the chunk, one thread per visibility
//               at a time: D and its gradient for every position (the decorrelation of
//               the plan's method), dL/dW_k summed over positions (one write per
//               visibility), dL/d(l0, m0) summed per warp in shared memory, then per block;
//   k_adj_sum   the per-block position sums added in float64 (and over chunks).
// Every barrier wait is bounded (2 s); on expiry the CTA raises the error flag, stops,
// waits (bounded) for its copies in flight and issued MMAs and frees TMEM.
#include "decorr.cuh"
#include "tc_ptx.cuh"

#include <cuda.h>

#include <algorithm>

namespace psf {
namespace {
using namespace tc;

constexpr int kAdjS = 4;              // operand ring depth
constexpr int kAdjGroups = 4;         // generator groups (stages s mod 4)
constexpr int kAdjGroupWarps = 4;     // one lane per visibility of the 128-visibility tile
constexpr int kAdjEpiWarp0 = 16;
constexpr int kAdjTmaWarp = 20;
constexpr int kAdjMmaWarp = 21;
constexpr int kAdjThreads = 22 * 32;
static_assert(kAdjGroups <= kAdjS, "generator groups exceed the ring depth");
constexpr uint32_t kAdjATile = 128 * 128;   // 128 positions x 64 pixels x 2 B
constexpr uint32_t kAdjBTile = 256 * 128;   // 256 rows (Re, Im of 128 visibilities) x 64 pixels x 2 B
constexpr uint32_t kAdjSmem = kAdjS * (kAdjATile + kAdjBTile) + 256 + 1024;

// 32 pixels of one cutout row for this lane's visibility, pixel offsets i = i0 .. i0+31:
// z(i) = exp(2 pi i (tu (i0 - N/2 + i') + tv (j - N/2))), written as FP16/BF16 into the
// lane's real row (re_row) and imaginary row (im_row) at the 16-byte chunks c0 .. c0+3
// (8 pixels per chunk).  Four 8-pixel pieces from one MUFU seed, two at a time.
template <int BF16>
__device__ __forceinline__ void adj_run32(uint32_t re_row, uint32_t im_row, int row, int c0, float tu, float tv,
                                          int i0, int j, int half, float2 st, float2 st8, float2 st16) {
    const float2 z0 = cis_turns(fmaf(tu, (float)(i0 - half), tv * (float)(j - half)));
    const float2 sr = make_float2(st.x, st.x), si = make_float2(st.y, st.y), nsi = make_float2(-st.y, -st.y);
    const uint32_t sw = (uint32_t)(row & 7);
    // pieces p = 0..3 start at pixels 8p; pieces (0, 1) and then (2, 3) run packed for FFMA2
#pragma unroll
    for (int pp = 0; pp < 2; ++pp) {
        const float2 za = pp ? cmulf(z0, st16) : z0;
        const float2 zb = cmulf(za, st8);
        float2 re = make_float2(za.x, zb.x), im = make_float2(za.y, zb.y), pre, pim;
        uint32_t wre[2][4], wim[2][4];   // [piece][word]
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            if (q & 1) {
                wre[0][q >> 1] = pack2<BF16>(pre.x, re.x);
                wre[1][q >> 1] = pack2<BF16>(pre.y, re.y);
                wim[0][q >> 1] = pack2<BF16>(pim.x, im.x);
                wim[1][q >> 1] = pack2<BF16>(pim.y, im.y);
            } else {
                pre = re;
                pim = im;
            }
            if (q < 7) {
                const float2 t = __fmul2_rn(im, nsi), u = __fmul2_rn(im, sr);
                im = __ffma2_rn(re, si, u);
                re = __ffma2_rn(re, sr, t);
            }
        }
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const uint32_t off = ((uint32_t)(c0 + 2 * pp + e) ^ sw) << 4;
            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(re_row + off), "r"(wre[e][0]),
                         "r"(wre[e][1]), "r"(wre[e][2]), "r"(wre[e][3])
                         : "memory");
            asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(im_row + off), "r"(wim[e][0]),
                         "r"(wim[e][1]), "r"(wim[e][2]), "r"(wim[e][3])
                         : "memory");
        }
    }
}

template <int BF16>
__global__ void __launch_bounds__(kAdjThreads, 1)
    k_adj_tc(const __grid_constant__ CUtensorMap rmap, int ntile_pos, int ntile_vis, int N, const float2 *__restrict__ uv,
             int32_t kc0, int32_t kcn, float cell, float2 *__restrict__ H, int64_t ldh, int *err) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *a_base = smem;
    uint8_t *b_base = smem + kAdjS * kAdjATile;
    uint64_t *full = (uint64_t *)(b_base + kAdjS * kAdjBTile);
    uint64_t *empty = full + kAdjS;
    uint64_t *acc_full = empty + kAdjS;     // [buffer]
    uint64_t *acc_empty = acc_full + 2;     // [buffer]
    uint64_t *done_bar = acc_empty + 2;
    uint32_t *s_tmem = (uint32_t *)(done_bar + 1);
    volatile int *s_abort = (volatile int *)(s_tmem + 1);
    volatile int no_abort = 0;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nitems = ntile_pos * ntile_vis;
    const int nst = N * N / 64;   // 64-pixel stages per item (N a multiple of 32)
    // this CTA's items: blockIdx.x, blockIdx.x + gridDim.x, ...
    const int my_items = blockIdx.x < nitems ? (nitems - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kAdjS; ++s) {
            mbar_init(&full[s], kAdjGroupWarps + 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 4);
        }
        mbar_init(done_bar, 1);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kAdjMmaWarp) {
        tmem_alloc(s_tmem, 512);   // two 256-column accumulators
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;
    const int half = N / 2;

    if (warp < kAdjGroups * kAdjGroupWarps) {
        // ------------------------------------------------------------ pixel twiddles
        const int grp = warp / kAdjGroupWarps;
        const int vrow = (warp % kAdjGroupWarps) * 32 + lane;   // visibility row of the tile
        int cur_item = -1;
        float tu = 0.f, tv = 0.f;
        float2 st = make_float2(1.f, 0.f), st8 = st, st16 = st;
        for (int g = grp; g < my_items * nst; g += kAdjGroups) {
            const int li = g / nst, s = g - li * nst;
            const int slot = g % kAdjS;
            if (li != cur_item) {   // a new item: this lane's visibility and its pixel step
                cur_item = li;
                const int item = blockIdx.x + li * gridDim.x;
                const int vt = item % ntile_vis;
                const int kk = vt * 128 + vrow;
                const float2 uvk = kk < kcn ? uv[kc0 + kk] : make_float2(0.f, 0.f);
                tu = uvk.x * cell;
                tv = uvk.y * cell;
                st = cis_turns(tu);
                const float2 s2 = cmulf(st, st), s4 = cmulf(s2, s2);
                st8 = cmulf(s4, s4);
                st16 = cmulf(st8, st8);
            }
            if (g >= kAdjS) {
                const bool ok = wait_bounded(&empty[slot], (uint32_t)((g / kAdjS) & 1) ^ 1u, s_abort, err);
                if (!__all_sync(0xffffffffu, ok)) break;
            }
            const uint32_t bt = smem_u32(b_base + slot * kAdjBTile);
            const uint32_t re_row = bt + (uint32_t)vrow * 128u, im_row = bt + (uint32_t)(128 + vrow) * 128u;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int q0 = s * 64 + r * 32;
                const int j = q0 / N, i0 = q0 - j * N;
                adj_run32<BF16>(re_row, im_row, vrow, 4 * r, tu, tv, i0, j, half, st, st8, st16);
            }
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&full[slot]);
        }
    } else if (warp == kAdjTmaWarp) {
        // ------------------------------------------------------------ R tiles
        if (lane == 0) {
            for (int g = 0; g < my_items * nst; ++g) {
                const int li = g / nst, s = g - li * nst;
                const int slot = g % kAdjS;
                if (g >= kAdjS && !wait_bounded(&empty[slot], (uint32_t)((g / kAdjS) & 1) ^ 1u, s_abort, err)) break;
                const int item = blockIdx.x + li * gridDim.x;
                const int pt = item / ntile_vis;
                mbar_arrive_expect_tx(&full[slot], kAdjATile);
                tma_load_2d(a_base + slot * kAdjATile, &rmap, s * 64, pt * 128, &full[slot]);
            }
        }
        __syncwarp();
    } else if (warp == kAdjMmaWarp) {
        // ------------------------------------------------------------ MMA issue
        if (lane == 0) {
            const uint32_t idesc = idesc_f16(128, 256, BF16);
            const uint64_t ad0 = desc_sw128(smem_u32(a_base)), bd0 = desc_sw128(smem_u32(b_base));
            int slot = 0;
            uint32_t ph = 0;
            bool stop = false;
            for (int li = 0; li < my_items && !stop; ++li) {
                const int b = li & 1;
                // the epilogue has read this buffer's previous item (li - 2)
                if (li >= 2 && !wait_bounded(&acc_empty[b], (uint32_t)((li >> 1) - 1) & 1u, s_abort, err)) break;
                const uint32_t dt = tmem + (uint32_t)b * 256u;
                for (int s = 0; s < nst; ++s) {
                    if (!wait_bounded(&full[slot], ph, s_abort, err)) { stop = true; break; }
                    tc_fence_after();
                    const uint64_t ad = ad0 + (uint64_t)(slot * (kAdjATile >> 4));
                    const uint64_t bd = bd0 + (uint64_t)(slot * (kAdjBTile >> 4));
                    if (s == 0) umma_f16(dt, ad, bd, idesc, 0u);
                    else umma_f16(dt, ad, bd, idesc, 1u);
                    umma_f16(dt, ad + 2, bd + 2, idesc, 1u);
                    umma_f16(dt, ad + 4, bd + 4, idesc, 1u);
                    umma_f16(dt, ad + 6, bd + 6, idesc, 1u);
                    umma_commit(&empty[slot]);
                    if (s == nst - 1) umma_commit(&acc_full[b]);
                    if (++slot == kAdjS) {
                        slot = 0;
                        ph ^= 1u;
                    }
                }
            }
            umma_commit(done_bar);
            wait_bounded(done_bar, 0, &no_abort, err);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------------ epilogue: TMEM -> H
        const int qw = warp - kAdjEpiWarp0;   // TMEM lane quarter
        const int row = qw * 32 + lane;       // position row of the tile
        for (int li = 0; li < my_items; ++li) {
            const int b = li & 1;
            const bool ok = wait_bounded(&acc_full[b], (uint32_t)(li >> 1) & 1u, s_abort, err);
            if (!__all_sync(0xffffffffu, ok)) break;
            tc_fence_after();
            const int item = blockIdx.x + li * gridDim.x;
            const int pt = item / ntile_vis, vt = item - pt * ntile_vis;
            float2 *dst = H + (int64_t)(pt * 128 + row) * ldh + (int64_t)vt * 128;
            const uint32_t ta = tmem + ((uint32_t)(qw * 32) << 16) + (uint32_t)b * 256u;
            for (int c0 = 0; c0 < 128; c0 += 16) {
                float vr[16], vi[16];
                tmem_ld16(ta + (uint32_t)c0, vr);
                tmem_ld16(ta + 128u + (uint32_t)c0, vi);
#pragma unroll
                for (int e = 0; e < 16; e += 2)
                    *reinterpret_cast<float4 *>(dst + c0 + e) = make_float4(vr[e], vi[e], vr[e + 1], vi[e + 1]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[b]);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kAdjMmaWarp) tmem_dealloc(tmem, 512);
}

// R of a size group -> FP16/BF16 rows: r16[row][q] = R[offs[row] + q] for row < npos,
// zero for the padding rows up to `rows`.
template <int BF16>
__global__ void __launch_bounds__(256) k_adj_r16(const float *__restrict__ R, const int64_t *__restrict__ offs,
                                                 int npos, int rows, int n2, uint16_t *__restrict__ r16) {
    const int row = blockIdx.y;
    for (int q = 2 * (blockIdx.x * blockDim.x + threadIdx.x); q < n2; q += 2 * gridDim.x * blockDim.x) {
        float a = 0.f, b = 0.f;
        if (row < npos) {
            a = R[offs[row] + q];
            b = R[offs[row] + q + 1];
        }
        *reinterpret_cast<uint32_t *>(r16 + (int64_t)row * n2 + q) = pack2<BF16>(a, b);
    }
    (void)rows;
}

struct AdjPosT {
    float4 L, dLl, dLm;   // direction (l0, m0, n0-1) and its derivatives
};

constexpr int kFoldThreads = 256;
constexpr int kFoldWarps = kFoldThreads / 32;

// Grid-stride over the visibilities k = kc0 + t of the chunk, one thread per visibility
// at a time: D_k(l0_p) and its gradient for every position p of the group,
// dL/dW_k (+)= sum_p Re(D H_pk) (one write per visibility), and per warp the sums of
// W_k Re(dD/dl0 H_pk), W_k Re(dD/dm0 H_pk) in shared memory [warp][p][2]; each block
// writes its per-position totals to partial[block][p][2].
template <bool FAST>
__global__ void __launch_bounds__(kFoldThreads) k_adj_fold(DevObs o, int method, uint32_t flags,
                                                           const AdjPosT *__restrict__ pos, int npos,
                                                           const float2 *__restrict__ H, int64_t ldh, int32_t kc0,
                                                           int32_t kcn, float *__restrict__ gW, int accumulate_gW,
                                                           double *__restrict__ partial) {
    extern __shared__ float red[];   // [kFoldWarps][npos][2]
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int e = threadIdx.x; e < kFoldWarps * npos * 2; e += kFoldThreads) red[e] = 0.f;
    __syncthreads();
    float *myred = red + (int64_t)wid * npos * 2;
    for (int64_t base = (int64_t)blockIdx.x * kFoldThreads; base < kcn; base += (int64_t)gridDim.x * kFoldThreads) {
        const int64_t t = base + threadIdx.x;
        const bool valid = t < kcn;
        const int32_t k = kc0 + (int32_t)(valid ? t : 0);
        const int bin = k / o.nout, r = k - bin * o.nout;
        const float Wk = valid ? o.W[k] : 0.f;
        float gw = 0.f;
        for (int p = 0; p < npos; ++p) {
            float gl = 0.f, gm = 0.f;
            if (valid) {
                const AdjPosT P = pos[p];
                float4 g;
                const float2 D = decorr<true, FAST>(o, method, flags, bin, r, P.L, P.dLl, P.dLm, &g);
                const float2 h = H[(int64_t)p * ldh + t];
                gw += D.x * h.x - D.y * h.y;
                gl = Wk * (g.x * h.x - g.y * h.y);
                gm = Wk * (g.z * h.x - g.w * h.y);
            }
#pragma unroll
            for (int sh = 16; sh > 0; sh >>= 1) {
                gl += __shfl_xor_sync(0xffffffffu, gl, sh);
                gm += __shfl_xor_sync(0xffffffffu, gm, sh);
            }
            if (lane == 0) {   // the warp's only writer of its row
                myred[2 * p] += gl;
                myred[2 * p + 1] += gm;
            }
        }
        if (valid && gW) gW[k] = accumulate_gW ? gW[k] + gw : gw;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < npos * 2; e += kFoldThreads) {
        double s = 0.0;
        for (int w = 0; w < kFoldWarps; ++w) s += red[(int64_t)w * npos * 2 + e];
        partial[(int64_t)blockIdx.x * npos * 2 + e] = s;
    }
}

// The exact method's fold with affine output channels (nu_r = nu_0 + r dnu, the boxcar):
// a thread owns one bin and eight consecutive channels (visibilities k0 .. k0 + 7).  Per
// raw sample s the channel-independent factor f = Dirichlet x sinc of X_s = uvw_s . L0 and
// its derivative are evaluated once, and the channel phasors e_j = exp(-2 pi i nu_j ds / c)
// follow by the recurrence e_{j+1} = e_j rho, rho = exp(-2 pi i dnu ds / c); the phase's
// derivative is linear in j.  Per channel:
//   D_j = (1/n) sum_s e_j f,   dD_j/dl0 = (1/n) sum_s e_j (df/dX X_l + i (p_0 + j p_d) f),
// then as k_adj_fold.  FAST forms (MUFU sine/cosine after exact argument reduction) for
// the values, the accurate derivatives of the sinc and the Dirichlet kernel.
__global__ void __launch_bounds__(kFoldThreads) k_adj_fold_exact8(DevObs o, const AdjPosT *__restrict__ pos, int npos,
                                                                  const float2 *__restrict__ H, int64_t ldh,
                                                                  int32_t kc0, int32_t kcn, float *__restrict__ gW,
                                                                  int accumulate_gW, double *__restrict__ partial) {
    extern __shared__ float red[];   // [kFoldWarps][npos][2]
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int e = threadIdx.x; e < kFoldWarps * npos * 2; e += kFoldThreads) red[e] = 0.f;
    __syncthreads();
    float *myred = red + (int64_t)wid * npos * 2;
    const int64_t ngrp = (kcn + 7) / 8;
    for (int64_t base = (int64_t)blockIdx.x * kFoldThreads; base < ngrp; base += (int64_t)gridDim.x * kFoldThreads) {
        const int64_t gi = base + threadIdx.x;
        const bool valid = gi < ngrp;
        const int32_t t0 = (int32_t)(valid ? gi * 8 : 0);     // chunk-relative first visibility
        const int32_t k0 = kc0 + t0;                          // kc0 and nout are multiples of 8
        const int bin = k0 / o.nout, r0 = k0 - bin * o.nout;
        const float4 ub = o.bin_ubar[bin];
        const int2 sm = o.bin_samp[bin];
        const float4 ch = o.chan[r0];
        const float nu0 = ch.x, dnu = o.dnu_ch, inv = 1.0f / (float)sm.y;
        float Wk[8], gw[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            Wk[j] = (valid && t0 + j < kcn) ? o.W[k0 + j] : 0.f;
            gw[j] = 0.f;
        }
        for (int p = 0; p < npos; ++p) {
            float gl = 0.f, gm = 0.f;
            if (valid) {
                const AdjPosT P = pos[p];
                const float Xbar = dot3(ub, P.L), Xbl = dot3(ub, P.dLl), Xbm = dot3(ub, P.dLm);
                float Dr[8], Di[8], Lr[8], Li[8], Mr[8], Mi[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) { Dr[j] = Di[j] = Lr[j] = Li[j] = Mr[j] = Mi[j] = 0.f; }
                for (int s = 0; s < sm.y; ++s) {
                    const float4 d = o.samp[sm.x + s];
                    const float ds = dot3(d, P.L), dsl = dot3(d, P.dLl), dsm = dot3(d, P.dLm);
                    const float Xs = Xbar + ds, Xl = Xbl + dsl, Xm = Xbm + dsm;
                    const float a = ch.z * Xs * kInvC, y = ch.w * Xs * kInvC;
                    const float dir = dirichlet_fast(o.favg, a), sc = sincpi_fast(y);
                    const float f = dir * sc;
                    const float df = (ddirichlet(o.favg, a) * ch.z * sc + dir * dsincpi(y) * ch.w) * kInvC;
                    const float al = df * Xl, am = df * Xm;                           // real parts
                    const float pl0 = -2.0f * kPiF * nu0 * dsl * kInvC * f, pdl = -2.0f * kPiF * dnu * dsl * kInvC * f;
                    const float pm0 = -2.0f * kPiF * nu0 * dsm * kInvC * f, pdm = -2.0f * kPiF * dnu * dsm * kInvC * f;
                    float es, ec, rs, rc;
                    sincospi2_fast(-nu0 * ds * kInvC, &es, &ec);
                    sincospi2_fast(-dnu * ds * kInvC, &rs, &rc);
                    float er = ec, ei = es;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        Dr[j] = fmaf(er, f, Dr[j]);
                        Di[j] = fmaf(ei, f, Di[j]);
                        const float bl = fmaf((float)j, pdl, pl0), bm = fmaf((float)j, pdm, pm0);   // imaginary parts
                        // e (al + i bl)
                        Lr[j] += er * al - ei * bl;
                        Li[j] += er * bl + ei * al;
                        Mr[j] += er * am - ei * bm;
                        Mi[j] += er * bm + ei * am;
                        const float tr = er * rc - ei * rs;
                        ei = er * rs + ei * rc;
                        er = tr;
                    }
                }
                const float4 *hp = reinterpret_cast<const float4 *>(H + (int64_t)p * ldh + t0);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 h = hp[q];   // channels 2q, 2q + 1
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int j = 2 * q + e;
                        const float hr = e ? h.z : h.x, hi = e ? h.w : h.y;
                        gw[j] += (Dr[j] * hr - Di[j] * hi) * inv;
                        gl += Wk[j] * (Lr[j] * hr - Li[j] * hi) * inv;
                        gm += Wk[j] * (Mr[j] * hr - Mi[j] * hi) * inv;
                    }
                }
            }
#pragma unroll
            for (int sh = 16; sh > 0; sh >>= 1) {
                gl += __shfl_xor_sync(0xffffffffu, gl, sh);
                gm += __shfl_xor_sync(0xffffffffu, gm, sh);
            }
            if (lane == 0) {
                myred[2 * p] += gl;
                myred[2 * p + 1] += gm;
            }
        }
        if (valid && gW) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (t0 + j < kcn) gW[k0 + j] = accumulate_gW ? gW[k0 + j] + gw[j] : gw[j];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < npos * 2; e += kFoldThreads) {
        double s = 0.0;
        for (int w = 0; w < kFoldWarps; ++w) s += red[(int64_t)w * npos * 2 + e];
        partial[(int64_t)blockIdx.x * npos * 2 + e] = s;
    }
}

// g_lm[2 idx[p] + d] (+)= sum over blocks of partial[block][p][d], in float64.
__global__ void __launch_bounds__(256) k_adj_sum(const double *__restrict__ partial, int nblk, int npos,
                                                 const int32_t *__restrict__ idx, int accumulate,
                                                 double *__restrict__ g_lm) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= npos * 2) return;
    double s = 0.0;
    for (int c = 0; c < nblk; ++c) s += partial[(int64_t)c * npos * 2 + e];
    const int64_t o = 2 * (int64_t)idx[e >> 1] + (e & 1);
    g_lm[o] = accumulate ? g_lm[o] + s : s;
}

}  // namespace

int adj_tc_smem_bytes() { return (int)kAdjSmem; }

cudaError_t launch_adj_r16(const float *R, const int64_t *offs, int npos, int rows, int n2, int bf16, void *r16,
                           cudaStream_t st) {
    dim3 grid((unsigned)std::max(1, std::min(64, (n2 / 2 + 255) / 256)), (unsigned)rows);
    if (bf16) k_adj_r16<1><<<grid, 256, 0, st>>>(R, offs, npos, rows, n2, (uint16_t *)r16);
    else k_adj_r16<0><<<grid, 256, 0, st>>>(R, offs, npos, rows, n2, (uint16_t *)r16);
    return cudaGetLastError();
}

cudaError_t launch_adj_tc(const void *rmap, int ntile_pos, int ntile_vis, int N, const float2 *uv, int32_t kc0,
                          int32_t kcn, float cell, float2 *H, int64_t ldh, int bf16, int nsm, int *err,
                          cudaStream_t st) {
    const int nitems = ntile_pos * ntile_vis;
    if (nitems <= 0) return cudaSuccess;
    const int grid = std::min(nitems, nsm);
    const CUtensorMap *m = (const CUtensorMap *)rmap;
    cudaError_t e;
    if (bf16) {
        e = cudaFuncSetAttribute(k_adj_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAdjSmem);
        if (e != cudaSuccess) return e;
        k_adj_tc<1><<<grid, kAdjThreads, kAdjSmem, st>>>(*m, ntile_pos, ntile_vis, N, uv, kc0, kcn, cell, H, ldh, err);
    } else {
        e = cudaFuncSetAttribute(k_adj_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAdjSmem);
        if (e != cudaSuccess) return e;
        k_adj_tc<0><<<grid, kAdjThreads, kAdjSmem, st>>>(*m, ntile_pos, ntile_vis, N, uv, kc0, kcn, cell, H, ldh, err);
    }
    return cudaGetLastError();
}

int adj_fold_max_pos() { return 1024; }
int adj_fold_blocks(int nsm) { return 4 * nsm; }

cudaError_t launch_adj_fold(const DevObs &o, int method, uint32_t flags, const void *pos, int npos, const float2 *H,
                            int64_t ldh, int32_t kc0, int32_t kcn, float *gW, int accumulate_gW, double *partial,
                            const int32_t *idx, double *g_lm, int accumulate_lm, int fast, int nsm, cudaStream_t st) {
    if (npos <= 0 || npos > adj_fold_max_pos()) return cudaErrorInvalidValue;
    const int nblk = adj_fold_blocks(nsm);
    const size_t smem = (size_t)kFoldWarps * npos * 2 * sizeof(float);
    cudaError_t e;
    // H rows of 8-visibility groups read as float4 pairs: ldh, kc0 multiples of 8
    if (fast && method == kExact && o.chan_affine && o.nout % 8 == 0 && kc0 % 8 == 0 && ldh % 8 == 0) {
        e = cudaFuncSetAttribute(k_adj_fold_exact8, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_adj_fold_exact8<<<nblk, kFoldThreads, smem, st>>>(o, (const AdjPosT *)pos, npos, H, ldh, kc0, kcn, gW,
                                                           accumulate_gW, partial);
    } else if (fast) {
        e = cudaFuncSetAttribute(k_adj_fold<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_adj_fold<true><<<nblk, kFoldThreads, smem, st>>>(o, method, flags, (const AdjPosT *)pos, npos, H, ldh, kc0,
                                                          kcn, gW, accumulate_gW, partial);
    } else {
        e = cudaFuncSetAttribute(k_adj_fold<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_adj_fold<false><<<nblk, kFoldThreads, smem, st>>>(o, method, flags, (const AdjPosT *)pos, npos, H, ldh,
                                                           kc0, kcn, gW, accumulate_gW, partial);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_adj_sum<<<(npos * 2 + 255) / 256, 256, 0, st>>>(partial, nblk, npos, idx, accumulate_lm, g_lm);
    return cudaGetLastError();
}

}  // namespace psf
