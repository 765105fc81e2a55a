// Smearing weights w_{p,k} = W_k D_k(l0_p), the FP32 CUDA-core contraction and the
// float64 reduction of split-K partial cutouts.
//
// Weights (Eqs. 13, 35, 44): one thread per (position, visibility), streamed over
// visibilities with coalesced 16-byte loads of the bin records.
//
// FP32 contraction (Eqs. 21-22 as a separable DFT): a CTA owns a 64 x 64 pixel tile
// of one cutout and a contiguous range of visibilities; the tile body (twiddle chains
// from float-float seed phases, 4 x 4 pixel blocks per thread, compensated FP32 sums)
// is fp32t::tile_sum, and split-K partials are added in float64, so the path meets
// 1e-6 relative.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "decorr.cuh"
#include "fp32_tile.cuh"

namespace psf {

// --------------------------------------------------------------- weights
template <bool FAST>
__global__ void __launch_bounds__(256) k_weights(DevObs o, int method, uint32_t flags,
                                                 const float4 *__restrict__ pos, int32_t k0,
                                                 int32_t kn, float2 *__restrict__ w, int64_t ldw) {
    // grid-stride over the visibilities (a few waves of blocks rather than one thread
    // per visibility: the per-visibility work is a handful of loads and sines)
    const int p = blockIdx.y;
    const float4 L = pos[p];
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int32_t kk = blockIdx.x * blockDim.x + threadIdx.x; kk < kn; kk += gridDim.x * blockDim.x) {
        const int32_t k = k0 + kk;
        const int bin = k / o.nout;
        const int r = k - bin * o.nout;
        float2 D = decorr<false, FAST>(o, method, flags, bin, r, L, z, z, nullptr);
        const float Wk = o.W[k];
        w[(int64_t)p * ldw + kk] = make_float2(Wk * D.x, Wk * D.y);
    }
}

// Sums over the raw samples of one bin for the eight affine channels r0 .. r0 + 7 of a
// thread: S_j = sum_s f_s exp(-2 pi i (nu_r0 + j dnu) ds_s / c), f_s the channel-
// independent factor (the raw channels' Dirichlet kernel times their sinc, Eq. 13 with
// a boxcar), held as packed FP32 pairs (S_j, S_j+4): per sample three phasors (j = 0,
// j = 4 and the step) and three packed complex steps.
__device__ __forceinline__ void exact8_sums(const DevObs &o, float4 ub, int2 sm, float4 ch, float4 L,
                                            float2 (&re)[4], float2 (&im)[4]) {
#pragma unroll
    for (int j = 0; j < 4; ++j) { re[j] = make_float2(0.f, 0.f); im[j] = make_float2(0.f, 0.f); }
    const float Xbar = dot3(ub, L);
    for (int s = 0; s < sm.y; ++s) {
        const float4 d = o.samp[sm.x + s];
        const float ds = dot3(d, L);
        const float Xs = Xbar + ds;
        const float f = dirichlet_fast(o.favg, ch.z * Xs * kInvC) * sincpi_fast(ch.w * Xs * kInvC);
        float es, ec, e4s, e4c, rs, rc;
        sincospi2_fast(-ch.x * ds * kInvC, &es, &ec);
        sincospi2_fast(-(ch.x + 4.0f * o.dnu_ch) * ds * kInvC, &e4s, &e4c);
        sincospi2_fast(-o.dnu_ch * ds * kInvC, &rs, &rc);
        float2 er = make_float2(ec * f, e4c * f), ei = make_float2(es * f, e4s * f);
        const float2 rc2 = make_float2(rc, rc), rs2 = make_float2(rs, rs), nrs2 = make_float2(-rs, -rs);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            re[j] = __fadd2_rn(re[j], er);
            im[j] = __fadd2_rn(im[j], ei);
            if (j < 3) {
                const float2 t = __fmul2_rn(ei, nrs2), u = __fmul2_rn(ei, rc2);
                ei = __ffma2_rn(er, rs2, u);
                er = __ffma2_rn(er, rc2, t);
            }
        }
    }
}

// Exact-method weights of the tensor-core paths (FP32 (Re w, Im w) per position row,
// MUFU sine/cosine after exact argument reduction) by the per-bin channel recurrence
// of k_weights16_exact8: a thread owns eight consecutive channels of one bin, and per
// raw sample three phasors and a packed complex recurrence (exact8_sums) replace eight.
__global__ void __launch_bounds__(256) k_weights_exact8(DevObs o, const float4 *__restrict__ pos, int32_t k0,
                                                        int32_t kn, float2 *__restrict__ w, int64_t ldw) {
    const int p = blockIdx.y;
    const float4 L = pos[p];
    for (int32_t g = blockIdx.x * blockDim.x + threadIdx.x; (int64_t)g * 8 < kn; g += gridDim.x * blockDim.x) {
        const int32_t kk0 = 8 * g;
        const int32_t kb = k0 + kk0;   // k0 and nout are multiples of 8: one bin per group
        const int bin = kb / o.nout;
        const int r0 = kb - bin * o.nout;
        const float4 ub = o.bin_ubar[bin];
        const int2 sm = o.bin_samp[bin];
        const float4 ch = o.chan[r0];
        float2 re[4], im[4];
        exact8_sums(o, ub, sm, ch, L, re, im);
        const float inv = 1.0f / (float)sm.y;
        float2 *dst = w + (int64_t)p * ldw + kk0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float sr = (j < 4) ? re[j].x : re[j - 4].y, si = (j < 4) ? im[j].x : im[j - 4].y;
            const float Wk = (kk0 + j < kn) ? o.W[kb + j] : 0.f;
            if (kk0 + j < kn) dst[j] = make_float2(Wk * sr * inv, Wk * si * inv);
        }
    }
}

cudaError_t launch_weights(const DevObs &o, int method, uint32_t flags, const float4 *pos, int npos,
                           int32_t k0, int32_t kn, float2 *w, int64_t ldw, int fast, cudaStream_t st) {
    if (npos <= 0 || kn <= 0) return cudaSuccess;
    static int nsm = 0;   // SM count of the first device used (only sizes the grid)
    if (nsm == 0 && cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess) {
        cudaGetLastError();
        nsm = 152;
    }
    const int64_t blocks = std::min<int64_t>((kn + 255) / 256, (int64_t)nsm * 16 / std::max(1, std::min(npos, 16)));
    dim3 grid((unsigned)std::max<int64_t>(1, blocks), npos);
    if (fast && method == kExact && o.chan_affine && o.nout % 8 == 0 && k0 % 8 == 0) {
        const int64_t b8 = std::min<int64_t>((kn / 8 + 255) / 256 + 1, (int64_t)nsm * 16 / std::max(1, std::min(npos, 16)));
        k_weights_exact8<<<dim3((unsigned)std::max<int64_t>(1, b8), npos), 256, 0, st>>>(o, pos, k0, kn, w, ldw);
        return cudaGetLastError();
    }
    if (fast) k_weights<true><<<grid, 256, 0, st>>>(o, method, flags, pos, k0, kn, w, ldw);
    else k_weights<false><<<grid, 256, 0, st>>>(o, method, flags, pos, k0, kn, w, ldw);
    return cudaGetLastError();
}

// --------------------------------------------------------------- FP16/BF16 weights
// Weights of a position chunk for the batched tensor-core contraction: row r holds
// position slot_of_row[r] (zeros for padding rows, slot < 0) as (Re w, -Im w) pairs
// at column pair (k - kc0); columns at or beyond kcn are zero.  The weights are
// rounded to 16 bits, so the fast sine/cosine forms are used.
// One thread per visibility (column) and a block of kRowsPerBlock position rows: the
// visibility's records (bin, channel, weight, raw samples) are loaded once and reused
// for every row; each warp writes 32 consecutive columns of one row at a time.
constexpr int kRowsPerBlock = 32;

// Rounding of the weights to 16 bits.  Round-to-nearest is biased on these data: with
// natural weights most values W_k D_k sit just below the power of two W_k (small
// decorrelation), where every one rounds up, and a PSF peak sums them coherently (a bias
// of ~1e-5 of the peak over 2e8 visibilities).  Stochastic rounding (cvt.rs) is unbiased:
// the random bits, a hash of (position, visibility), make the rounding errors average out
// like independent ones.  The hash is deterministic, so a call is reproducible.
__device__ __forceinline__ uint32_t sr_bits(uint32_t slot, uint32_t k) {
    uint32_t h = k * 0x9E3779B1u ^ (slot + 0x7F4A7C15u) * 0x85EBCA77u;
    h ^= h >> 16;
    h *= 0x7FEB352Du;
    h ^= h >> 15;
    h *= 0x846CA68Bu;
    h ^= h >> 16;
    return h;
}

// (x, y) -> packed 16-bit pair, x in the low half (the layout of __floats2half2_rn)
template <int BF16>
__device__ __forceinline__ uint32_t pack_sr(float x, float y, uint32_t rbits) {
    uint32_t d;
    if (BF16) asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(y), "f"(x), "r"(rbits));
    else asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(y), "f"(x), "r"(rbits));
    return d;
}

template <int BF16>
__global__ void __launch_bounds__(256) k_weights16(DevObs o, int method, uint32_t flags,
                                                   const float4 *__restrict__ pos,
                                                   const int32_t *__restrict__ slot_of_row, int rows, int32_t kc0,
                                                   int32_t kcn, int64_t kpitch, uint32_t *__restrict__ w16) {
    const int32_t kk = blockIdx.x * blockDim.x + threadIdx.x;
    if (kk >= kpitch) return;
    const int row0 = blockIdx.y * kRowsPerBlock;
    const bool valid = kk < kcn;
    const int32_t k = kc0 + (valid ? kk : 0);
    const int bin = k / o.nout;
    const int r = k - bin * o.nout;
    const float Wk = valid ? o.W[k] : 0.f;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int row = row0; row < min(rows, row0 + kRowsPerBlock); ++row) {
        const int slot = slot_of_row[row];
        float2 w = make_float2(0.f, 0.f);
        if (slot >= 0 && valid) {
            const float2 D = decorr<false, true>(o, method, flags, bin, r, pos[slot], z, z, nullptr);
            w = make_float2(Wk * D.x, Wk * D.y);
        }
        w16[(int64_t)row * kpitch + kk] = pack_sr<BF16>(w.x, -w.y, sr_bits((uint32_t)slot, (uint32_t)k));
    }
}

// Real weights (Methods 1 and 2, no windows): one FP16/BF16 value W_k D_k per
// visibility; a thread owns the visibility pair (2 kp, 2 kp + 1) of a row (kpitch2 pairs
// per row).  Both methods are D = sinc(A) sinc(B) with arguments that are, per
// visibility, fixed forms in the position: Method 1 (Eq. 35) A = a . L and B = b . L
// with a = (uvw(t_e) - uvw(t_s)) nu_r / c and b = ubar Dnu_r / c; Method 2 (Eqs. 38-44)
// A = a . L with a = omega_E Dt (udot, vdot, 0) and B = f |(l0, m0)| with
// f = (Dnu_r / nu_r) |(u, v)|.  The thread forms a, b, f once for its two visibilities
// (decorr_uv / decorr_img do the same per call) and each position costs two dot
// products and two sincs.
template <int BF16>
__global__ void __launch_bounds__(256) k_weights16_real(DevObs o, int method, uint32_t flags,
                                                        const float4 *__restrict__ pos,
                                                        const int32_t *__restrict__ slot_of_row, int rows,
                                                        int32_t kc0, int32_t kcn, int64_t kpitch2,
                                                        uint32_t *__restrict__ w16) {
    const int32_t kp = blockIdx.x * blockDim.x + threadIdx.x;
    if (kp >= kpitch2) return;
    const int row0 = blockIdx.y * kRowsPerBlock;
    float4 a[2], b[2];   // A = a . L; B = b . L (Method 1) or b.x |(l0, m0)| (Method 2)
    float Wk[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int32_t kk = 2 * kp + e;
        const bool valid = kk < kcn;
        const int32_t k = kc0 + (valid ? kk : 0);
        const int bin = k / o.nout;
        const int r = k - bin * o.nout;
        Wk[e] = valid ? o.W[k] : 0.f;
        const float4 ub = o.bin_ubar[bin];
        const float4 ch = o.chan[r];
        if (method == kUV) {
            const float4 ed = o.bin_edge[bin];
            const float sa = ch.x * kInvC, sb = ch.y * kInvC;
            a[e] = make_float4(ed.x * sa, ed.y * sa, ed.z * sa, 0.f);
            b[e] = make_float4(ub.x * sb, ub.y * sb, ub.z * sb, 0.f);
        } else {
            const float sc = ch.x * kInvC;
            const float u = ub.x * sc, v = ub.y * sc;
            const float uvlen = sqrtf(u * u + v * v);
            float udot = -v, vdot = u;
            if (flags & PSF_IMG_LITERAL_THETA) {
                const float th = (v != 0.0f) ? atanf(u / v) : (u >= 0.0f ? 0.5f * kPiF : -0.5f * kPiF);
                float st, ct;
                sincosf(th, &st, &ct);
                udot = -uvlen * st;
                vdot = uvlen * ct;
            }
            const float wdt = (float)kOmegaE * ub.w;
            a[e] = make_float4(wdt * udot, wdt * vdot, 0.f, 0.f);
            b[e] = make_float4(ch.y / ch.x * uvlen, 0.f, 0.f, 0.f);
        }
    }
    for (int row = row0; row < min(rows, row0 + kRowsPerBlock); ++row) {
        const int slot = slot_of_row[row];
        float wv[2] = {0.f, 0.f};
        if (slot >= 0) {
            const float4 P = pos[slot];
            const float rho = sqrtf(P.x * P.x + P.y * P.y);
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const float A = dot3(a[e], P);
                const float B = (method == kUV) ? dot3(b[e], P) : b[e].x * rho;
                if (Wk[e] != 0.f) wv[e] = Wk[e] * sincpi_fast(A) * sincpi_fast(B);
            }
        }
        w16[(int64_t)row * kpitch2 + kp] = pack_sr<BF16>(wv[0], wv[1], sr_bits((uint32_t)slot, (uint32_t)(kc0 + 2 * kp)));
    }
}

// Exact weights, eight output channels of one bin per thread (affine channels, the
// group count nout a multiple of 8).  Per raw sample only the factor
// exp(-2 pi i nu_r ds / c) depends on the channel r; with nu_r = nu_r0 + j dnu it is
// e0 rho^j, e0 = exp(-2 pi i nu_r0 ds / c), rho = exp(-2 pi i dnu ds / c), so a sample
// costs three phasors (e0, e4 and rho) and a recurrence of packed FP32 pairs (channels j
// and j + 4 together) instead of eight.  The channel-independent factor
// is the Dirichlet kernel of the raw channels times their sinc (Eq. 13, boxcar).
template <int BF16>
__global__ void __launch_bounds__(256) k_weights16_exact8(DevObs o, uint32_t flags, const float4 *__restrict__ pos,
                                                          const int32_t *__restrict__ slot_of_row, int rows,
                                                          int32_t kc0, int32_t kcn, int64_t kpitch,
                                                          uint32_t *__restrict__ w16) {
    const int32_t g = blockIdx.x * blockDim.x + threadIdx.x;   // group of 8 columns
    if ((int64_t)g * 8 >= kpitch) return;
    const int row0 = blockIdx.y * kRowsPerBlock;
    const int32_t kk0 = 8 * g;
    const bool valid = kk0 < kcn;   // kcn is a multiple of nout, hence of 8, unless the tail
    const int32_t k0 = kc0 + (valid ? kk0 : 0);
    const int bin = k0 / o.nout;
    const int r0 = k0 - bin * o.nout;
    const float4 ub = o.bin_ubar[bin];
    const int2 sm = o.bin_samp[bin];
    const float4 ch = o.chan[r0];
    float Wk[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) Wk[j] = (valid && kk0 + j < kcn) ? o.W[k0 + j] : 0.f;
    const float inv = 1.0f / (float)sm.y;
    for (int row = row0; row < min(rows, row0 + kRowsPerBlock); ++row) {
        const int slot = slot_of_row[row];
        // channels j and j + 4 as packed FP32 pairs: re[j] = (Re S_j, Re S_j+4), ...
        float2 re[4], im[4];
        if (slot >= 0 && valid) {
            exact8_sums(o, ub, sm, ch, pos[slot], re, im);
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) { re[j] = make_float2(0.f, 0.f); im[j] = make_float2(0.f, 0.f); }
        }
        uint32_t packed[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float sr = (j < 4) ? re[j].x : re[j - 4].y, si = (j < 4) ? im[j].x : im[j - 4].y;
            const float wr = Wk[j] * sr * inv, wi = Wk[j] * si * inv;
            packed[j] = pack_sr<BF16>(wr, -wi, sr_bits((uint32_t)slot, (uint32_t)(k0 + j)));
        }
        uint4 *dst = reinterpret_cast<uint4 *>(w16 + (int64_t)row * kpitch + kk0);
        dst[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
        dst[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
    }
}

cudaError_t launch_weights16(const DevObs &o, int method, uint32_t flags, const float4 *pos,
                             const int32_t *slot_of_row, int rows, int32_t kc0, int32_t kcn, int64_t kpitch,
                             int bf16, void *w16, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    if (method == kExact && o.chan_affine && o.nout % 8 == 0 && kc0 % 8 == 0 && kpitch % 8 == 0) {
        const unsigned gy = (unsigned)((rows + kRowsPerBlock - 1) / kRowsPerBlock);
        dim3 grid((unsigned)((kpitch / 8 + 255) / 256), gy);
        if (bf16)
            k_weights16_exact8<1><<<grid, 256, 0, st>>>(o, flags, pos, slot_of_row, rows, kc0, kcn, kpitch,
                                                        (uint32_t *)w16);
        else
            k_weights16_exact8<0><<<grid, 256, 0, st>>>(o, flags, pos, slot_of_row, rows, kc0, kcn, kpitch,
                                                        (uint32_t *)w16);
        return cudaGetLastError();
    }
    const unsigned gy = (unsigned)((rows + kRowsPerBlock - 1) / kRowsPerBlock);
    if (method != kExact && !o.win) {   // real weights: kpitch pairs per row hold 2 kpitch visibilities
        const int64_t kp2 = kpitch / 2;
        dim3 grid((unsigned)((kp2 + 255) / 256), gy);
        if (bf16)
            k_weights16_real<1><<<grid, 256, 0, st>>>(o, method, flags, pos, slot_of_row, rows, kc0, kcn, kp2,
                                                      (uint32_t *)w16);
        else
            k_weights16_real<0><<<grid, 256, 0, st>>>(o, method, flags, pos, slot_of_row, rows, kc0, kcn, kp2,
                                                      (uint32_t *)w16);
        return cudaGetLastError();
    }
    dim3 grid((unsigned)((kpitch + 255) / 256), gy);
    if (bf16)
        k_weights16<1><<<grid, 256, 0, st>>>(o, method, flags, pos, slot_of_row, rows, kc0, kcn, kpitch,
                                             (uint32_t *)w16);
    else
        k_weights16<0><<<grid, 256, 0, st>>>(o, method, flags, pos, slot_of_row, rows, kc0, kcn, kpitch,
                                             (uint32_t *)w16);
    return cudaGetLastError();
}

// Zero the listed cutouts (outputs that are accumulated with atomics).
__global__ void __launch_bounds__(256) k_zero_cutouts(float *__restrict__ out, const int64_t *__restrict__ offs,
                                                      const int32_t *__restrict__ npix) {
    const int p = blockIdx.y;
    const int64_t n2 = (int64_t)npix[p] * npix[p];
    float *dst = out + offs[p];
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n2; q += (int64_t)gridDim.x * blockDim.x)
        dst[q] = 0.f;
}

cudaError_t launch_zero_cutouts(float *out, const int64_t *offs, const int32_t *npix, int npos, cudaStream_t st) {
    if (npos <= 0) return cudaSuccess;
    k_zero_cutouts<<<dim3(16, npos), 256, 0, st>>>(out, offs, npix);
    return cudaGetLastError();
}

// --------------------------------------------------------------- FP32 contraction
// One CTA per (64 x 64 tile, visibility range); the tile body is fp32t::tile_sum.
__global__ void __launch_bounds__(256) k_psf_fp32(const float2 *__restrict__ uv, const float2 *__restrict__ uv_lo,
                                                  const float2 *__restrict__ w, int64_t ldw, int32_t nvis,
                                                  const Tile *__restrict__ tiles, int32_t kper, float2 cell,
                                                  float *__restrict__ partial, int64_t split_stride) {
    __shared__ __align__(16) float2 sa[fp32t::kKC][fp32t::kT];   // row (l) twiddles
    __shared__ __align__(16) float2 sc[fp32t::kKC][fp32t::kT];   // weighted column (m) twiddles
    const Tile t = tiles[blockIdx.x];
    const int split = blockIdx.y;
    const int32_t kbeg = split * kper;
    const int32_t kend = min(nvis, kbeg + kper);
    const float2 *wp = w + (int64_t)t.slot * ldw;
    float tot[4][4];
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int a = 0; a < 4; ++a) tot[b][a] = 0.f;
    fp32t::tile_sum(uv, uv_lo, kbeg, kend, t.N, t.i0, t.j0, cell, [&](int32_t k) { return wp[k]; }, sa, sc, tot);
    fp32t::tile_store(partial + (int64_t)split * split_stride + t.out_off, t.N, t.i0, t.j0, tot);
}

cudaError_t launch_psf_fp32(const DevObs &o, const float2 *w, int64_t ldw, const Tile *tiles, int ntiles,
                            int nsplit, int32_t kper, double cell, float *partial, int64_t split_stride,
                            cudaStream_t st) {
    if (ntiles <= 0) return cudaSuccess;
    dim3 grid(ntiles, nsplit);
    k_psf_fp32<<<grid, 256, 0, st>>>(o.uv, o.uv_lo, w, ldw, o.nvis, tiles, kper, fp32t::cell_pair(cell), partial,
                                     split_stride);
    return cudaGetLastError();
}

// --------------------------------------------------------------- FP32 FMA rate
// Denominator of the FP32 path's roofline: every thread runs kFmaChains independent
// chains x <- x c + b (|c| < 1, so the values stay bounded), as scalar FMAs or as packed
// pairs (fma.rn.f32x2, one instruction for two FMAs).  The last values are written so
// that nothing is optimised away.
constexpr int kFmaChains = 16;

template <int PACKED>
__global__ void __launch_bounds__(256) k_fma_rate(int iters, float seed, float *__restrict__ out) {
    const float b = seed * 1e-3f + 1e-9f * threadIdx.x, c = 0.999f - 1e-7f * blockIdx.x;
    float r = 0.f;
    if (PACKED) {
        unsigned long long x[kFmaChains], bb, cc;
        asm("mov.b64 %0, {%1, %1};" : "=l"(bb) : "f"(b));
        asm("mov.b64 %0, {%1, %1};" : "=l"(cc) : "f"(c));
#pragma unroll
        for (int j = 0; j < kFmaChains; ++j) {
            const float v = seed + j;
            asm("mov.b64 %0, {%1, %2};" : "=l"(x[j]) : "f"(v), "f"(-v));
        }
#pragma unroll 4
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int j = 0; j < kFmaChains; ++j) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[j]) : "l"(cc), "l"(bb));
#pragma unroll
        for (int j = 0; j < kFmaChains; ++j) {
            float lo, hi;
            asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[j]));
            r += lo + hi;
        }
    } else {
        float x[kFmaChains];
#pragma unroll
        for (int j = 0; j < kFmaChains; ++j) x[j] = seed + j;
#pragma unroll 8
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int j = 0; j < kFmaChains; ++j) x[j] = fmaf(x[j], c, b);
#pragma unroll
        for (int j = 0; j < kFmaChains; ++j) r += x[j];
    }
    out[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = r;
}

int selftest_fma_rate(int packed, double *flops_per_s) {
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return PSF_ECUDA;
    const int blocks = nsm * 8, threads = 256, iters = 1 << 15;
    float *out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = PSF_OK;
    double best = 0.0;
    if (cudaMalloc(&out, sizeof(float) * blocks * threads) != cudaSuccess) return PSF_ENOMEM;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        rc = PSF_ECUDA;
    } else {
        for (int rep = 0; rep < 4 && rc == PSF_OK; ++rep) {   // the first launch is warm-up
            cudaEventRecord(e0, st);
            if (packed) k_fma_rate<1><<<blocks, threads, 0, st>>>(iters, 1.0f + rep, out);
            else k_fma_rate<0><<<blocks, threads, 0, st>>>(iters, 1.0f + rep, out);
            cudaEventRecord(e1, st);
            float ms = 0.f;
            if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                rc = PSF_ECUDA;
                break;
            }
            const double flops = 2.0 * (packed ? 2 : 1) * kFmaChains * (double)iters * blocks * threads;
            if (rep > 0 && ms > 0.f) best = std::max(best, flops / (ms * 1e-3));
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    cudaFree(out);
    if (rc == PSF_OK) *flops_per_s = best;
    return rc;
}

// --------------------------------------------------------------- split reduction
// One block row per position; the partial sums of each pixel are added in float64
// in split order (deterministic).  Partials use chunk-local packed offsets, the
// output the caller's offsets.
__global__ void __launch_bounds__(256) k_reduce(const float *__restrict__ partial, int nsplit,
                                                int64_t stride, const int64_t *__restrict__ loc_offs,
                                                const int64_t *__restrict__ out_offs,
                                                const int32_t *__restrict__ npix, int transposed,
                                                float *__restrict__ out) {
    const int p = blockIdx.y;
    const int N = npix[p];
    const int64_t n2 = (int64_t)N * N;
    const float *src = partial + loc_offs[p];
    float *dst = out + out_offs[p];
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n2; q += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int sp = 0; sp < nsplit; ++sp) s += (double)src[(int64_t)sp * stride + q];
        // transposed partials hold (j, i) at q = i N + j
        const int64_t o = transposed ? (q % N) * N + q / N : q;
        dst[o] = (float)s;
    }
}

cudaError_t launch_reduce(const float *partial, int nsplit, int64_t stride, const int64_t *loc_offs,
                          const int64_t *out_offs, const int32_t *npix, int npos, int transposed, float *out,
                          cudaStream_t st) {
    if (npos <= 0) return cudaSuccess;
    dim3 grid(64, npos);
    k_reduce<<<grid, 256, 0, st>>>(partial, nsplit, stride, loc_offs, out_offs, npix, transposed, out);
    return cudaGetLastError();
}

// --------------------------------------------------------------- binning (plan build)
// One thread per averaging bin: baseline b (binary search in bin_first), bin tau of its
// tavg[b] raw samples s0 = tau tavg[b] ...  Eq. 12's bin centre is the mean of the raw
// uvw, summed in sample order in float64 and divided by n; the edge delta (Eq. 33) is
// uvw(last) - uvw(first) scaled by n / (n - 1) (the bin's full width), or for a single
// sample the central difference of the neighbouring samples; the raw samples are kept as
// float32 offsets from the centre.  The same float64 operations in the same order as a
// host loop, so the records are bit-identical to host binning.
__global__ void __launch_bounds__(256) k_bin(const double *__restrict__ uvw, int ntime, int nbl,
                                             const int32_t *__restrict__ tavg, const int32_t *__restrict__ bin_first,
                                             const int64_t *__restrict__ samp_first, double dt_raw,
                                             float4 *__restrict__ bin_ubar, double2 *__restrict__ bin_uv64,
                                             float4 *__restrict__ bin_edge, int2 *__restrict__ bin_samp,
                                             float4 *__restrict__ samp) {
    const int32_t bin = blockIdx.x * blockDim.x + threadIdx.x;
    if (bin >= bin_first[nbl]) return;
    int lo = 0, hi = nbl;   // bin_first[lo] <= bin < bin_first[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (bin_first[mid] <= bin) lo = mid; else hi = mid;
    }
    const int b = lo, n = tavg[b];
    const int64_t tau = bin - bin_first[b];
    const int64_t s0 = tau * n;
    const double *ub = uvw + (size_t)b * ntime * 3;
    double mean[3] = {0, 0, 0}, edge[3] = {0, 0, 0};
    for (int64_t s = s0; s < s0 + n; ++s)
        for (int d = 0; d < 3; ++d) mean[d] += ub[s * 3 + d];
    for (int d = 0; d < 3; ++d) mean[d] /= n;
    if (n >= 2) {
        for (int d = 0; d < 3; ++d) edge[d] = __dmul_rn(ub[(s0 + n - 1) * 3 + d] - ub[s0 * 3 + d], (double)n) / (double)(n - 1);
    } else if (ntime >= 2) {
        const int64_t sa = s0 > 0 ? s0 - 1 : s0, sb = s0 < ntime - 1 ? s0 + 1 : s0;
        for (int d = 0; d < 3; ++d) edge[d] = (ub[sb * 3 + d] - ub[sa * 3 + d]) / (double)(sb - sa);
    }
    const int64_t rec = samp_first[b] + tau * n;
    bin_ubar[bin] = make_float4((float)mean[0], (float)mean[1], (float)mean[2], (float)(n * dt_raw));
    bin_uv64[bin] = make_double2(mean[0], mean[1]);
    bin_edge[bin] = make_float4((float)edge[0], (float)edge[1], (float)edge[2], 0.f);
    bin_samp[bin] = make_int2((int)rec, n);
    for (int s = 0; s < n; ++s) {
        const double *u = ub + (s0 + s) * 3;
        samp[rec + s] = make_float4((float)(u[0] - mean[0]), (float)(u[1] - mean[1]), (float)(u[2] - mean[2]), 0.f);
    }
}

cudaError_t launch_bin(const double *uvw, int ntime, int nbl, const int32_t *tavg, const int32_t *bin_first,
                       const int64_t *samp_first, int64_t nbin, double dt_raw, float4 *bin_ubar, double2 *bin_uv64,
                       float4 *bin_edge, int2 *bin_samp, float4 *samp, cudaStream_t st) {
    if (nbin <= 0) return cudaSuccess;
    k_bin<<<(unsigned)((nbin + 255) / 256), 256, 0, st>>>(uvw, ntime, nbl, tavg, bin_first, samp_first, dt_raw,
                                                           bin_ubar, bin_uv64, bin_edge, bin_samp, samp);
    return cudaGetLastError();
}

// --------------------------------------------------------------- per-visibility tables
// uv[k] + uv_lo[k] = ubar (x, y) nu_r / c in wavelengths, formed in float64 from the bin
// means and channel frequencies and split into a rounded float pair; W[k] = tavg * favg
// when no weights are given.
__global__ void __launch_bounds__(256) k_fill_vis(DevObs o, const double2 *__restrict__ bin_uv64,
                                                  const double2 *__restrict__ chan64, float2 *__restrict__ uv,
                                                  float2 *__restrict__ uv_lo, float *__restrict__ W, int natural) {
    const int32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= o.nvis) return;
    const int bin = k / o.nout;
    const int r = k - bin * o.nout;
    const double2 ub = bin_uv64[bin];
    const double nu = chan64[r].x;
    const double u = ub.x * nu / kCLight, v = ub.y * nu / kCLight;
    const float uh = (float)u, vh = (float)v;
    uv[k] = make_float2(uh, vh);
    uv_lo[k] = make_float2((float)(u - (double)uh), (float)(v - (double)vh));
    if (natural) W[k] = (float)(o.bin_samp[bin].y * o.favg);
}

cudaError_t launch_fill_vis(const DevObs &o, const double2 *bin_uv64, const double2 *chan64, float2 *uv,
                            float2 *uv_lo, float *W, int natural, cudaStream_t st) {
    k_fill_vis<<<(o.nvis + 255) / 256, 256, 0, st>>>(o, bin_uv64, chan64, uv, uv_lo, W, natural);
    return cudaGetLastError();
}

}  // namespace psf
