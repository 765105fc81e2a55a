// FP32 CUDA-core contraction of one 64 x 64 pixel tile of a cutout over a range of
// visibilities (Eqs. 21-22 as a separable DFT), shared by the FP32 path (weights read
// from a buffer) and the allocation-free entry point (weights evaluated inline).
//
// Per chunk of 32 visibilities the CTA stages the row twiddles a_k[i] = exp(2 pi i u_k dl_i)
// and the weighted column twiddles c_k[j] = w_k exp(2 pi i v_k dm_j) in shared memory, then
// every thread accumulates a 4 x 4 pixel block of Re(c a) with two FMAs per term.  Sums
// stay short in FP32 (one chunk) and are folded into a compensated (Kahan) total.
//
// Phase accuracy.  A pixel phase u_k (i - N/2) cell reaches tens of turns, so forming it
// in FP32 leaves ~2^-24 relative, i.e. several 1e-6 rad, of error in every term -- more
// than the 1e-6 bound allows when a cutout sums only tens of visibilities.  The phase is
// therefore carried as a float-float pair: u_k = u_hi + u_lo (both rounded from the
// float64 bin centre), cell = cell_hi + cell_lo, the product by the exact-error FMA
// identity, and the whole turns are removed exactly (x - rint(x)) before anything is
// rounded; each visibility's chains of twiddles start from such seeds every 8 pixels.
#pragma once

#include "decorr.cuh"

namespace psf {
namespace fp32t {

constexpr int kT = 64;     // tile edge (pixels)
constexpr int kKC = 32;    // visibilities per shared-memory chunk
constexpr int kSeg = 16;   // twiddles per generator thread (two chains of 8)
constexpr int kChain = 8;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// (x_hi + x_lo) (c_hi + c_lo) as an unevaluated pair (hi, lo): hi = fl(x_hi c_hi), lo its
// rounding error (exact by FMA) plus the cross terms (the lo x lo term is below 2^-48).
__device__ __forceinline__ float2 ff_mul(float xh, float xl, float ch, float cl) {
    const float p = xh * ch;
    const float e = fmaf(xh, ch, -p);
    return make_float2(p, fmaf(xh, cl, fmaf(xl, ch, e)));
}

// Fractional part of th * n in turns, in [-1/2, 1/2] up to one rounding (|n| < 2^24): the
// product's high part loses its whole turns exactly before the low parts are added.
__device__ __forceinline__ float ff_turns(float2 th, int n) {
    const float fn = (float)n;
    const float p = th.x * fn;
    const float e = fmaf(th.x, fn, -p);
    const float r = p - rintf(p);   // exact: |p - rint(p)| <= 1/2 with p's spacing
    return r + fmaf(th.y, fn, e);
}

// exp(2 pi i t), t in turns
__device__ __forceinline__ float2 cis_acc(float t) {
    float s, c;
    sincospif(2.0f * t, &s, &c);
    return make_float2(c, s);
}

// Adds to tot[b][a] the sum over k in [kbeg, kend) of Re(c_k[j] a_k[i]) for the pixel
// block of this thread (rows j = j0 + 4 ty + b, columns i = i0 + 4 tx + a, 16 x 16
// threads), with w_k = wfn(k).  Called by all 256 threads of the block.
template <class WFn>
__device__ __forceinline__ void tile_sum(const float2 *__restrict__ uv, const float2 *__restrict__ uv_lo,
                                         int32_t kbeg, int32_t kend, int N, int i0, int j0, float2 cell, WFn wfn,
                                         float2 (&sa)[kKC][kT], float2 (&sc)[kKC][kT], float (&tot)[4][4]) {
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    // generator role: visibility lane gk of the chunk, 16-twiddle segment gs (0-3 rows, 4-7 cols)
    const int gk = tid & 31, gs = tid >> 5;
    const int half = N / 2;
    const int seg_first = (gs & 3) * kSeg;
    const int n_first = (gs < 4 ? i0 : j0) + seg_first - half;   // pixel offset index of the chain start

    float acc[4][4], cmp[4][4];
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int a = 0; a < 4; ++a) { acc[b][a] = 0.f; cmp[b][a] = 0.f; }

    for (int32_t kc = kbeg; kc < kend; kc += kKC) {
        const int32_t k = kc + gk;
        float2 s0 = make_float2(0.f, 0.f), s1 = s0, step = make_float2(1.f, 0.f);
        if (k < kend) {
            const float2 uh = uv[k], ul = uv_lo[k];
            const float2 th = gs < 4 ? ff_mul(uh.x, ul.x, cell.x, cell.y) : ff_mul(uh.y, ul.y, cell.x, cell.y);
            s0 = cis_acc(ff_turns(th, n_first));
            s1 = cis_acc(ff_turns(th, n_first + kChain));
            step = cis_acc(ff_turns(th, 1));
            if (gs >= 4) {
                const float2 wk = wfn(k);
                s0 = cmul(s0, wk);
                s1 = cmul(s1, wk);
            }
        }
        __syncthreads();   // previous chunk consumed
        float2 *dst = (gs < 4 ? &sa[gk][seg_first] : &sc[gk][seg_first]);
#pragma unroll
        for (int q = 0; q < kChain; ++q) {
            dst[q] = s0;
            dst[q + kChain] = s1;
            s0 = cmul(s0, step);
            s1 = cmul(s1, step);
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < kKC; ++kk) {
            const float4 a01 = *reinterpret_cast<const float4 *>(&sa[kk][tx * 4]);
            const float4 a23 = *reinterpret_cast<const float4 *>(&sa[kk][tx * 4 + 2]);
            const float4 c01 = *reinterpret_cast<const float4 *>(&sc[kk][ty * 4]);
            const float4 c23 = *reinterpret_cast<const float4 *>(&sc[kk][ty * 4 + 2]);
            const float ar[4] = {a01.x, a01.z, a23.x, a23.z}, ai[4] = {a01.y, a01.w, a23.y, a23.w};
            const float cr[4] = {c01.x, c01.z, c23.x, c23.z}, ci[4] = {c01.y, c01.w, c23.y, c23.w};
#pragma unroll
            for (int b = 0; b < 4; ++b)
#pragma unroll
                for (int a = 0; a < 4; ++a) acc[b][a] = fmaf(cr[b], ar[a], fmaf(-ci[b], ai[a], acc[b][a]));
        }
        // fold the chunk sum into the compensated total
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const float y = acc[b][a] - cmp[b][a];
                const float s = tot[b][a] + y;
                cmp[b][a] = (s - tot[b][a]) - y;
                tot[b][a] = s;
                acc[b][a] = 0.f;
            }
    }
}

// Writes this thread's 4 x 4 block to dst[j * N + i] (pixels inside the cutout only).
__device__ __forceinline__ void tile_store(float *dst, int N, int i0, int j0, const float (&tot)[4][4]) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int j = j0 + ty * 4 + b;
        if (j >= N) continue;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int i = i0 + tx * 4 + a;
            if (i < N) dst[(int64_t)j * N + i] = tot[b][a];
        }
    }
}

// Pixel size as a float pair (hi, lo) with hi + lo = cell to ~2^-48.
inline float2 cell_pair(double cell) {
    const float hi = (float)cell;
    return make_float2(hi, (float)(cell - (double)hi));
}

}  // namespace fp32t
}  // namespace psf
