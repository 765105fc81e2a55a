// Hogbom CLEAN with position-dependent PSFs (Algorithm 2): the per-iteration kernels.
//
// One iteration on the residual image I_D [nm][nl] (pixel (x, y) is the direction
// (l_c + (x - nl/2) cell, m_c + (y - nm/2) cell)):
//   k_clean_argmax  l0 = argmax I_D: every thread folds its pixels into a 64-bit key
//                   (order-preserving bits of the value, then the complement of the
//                   index, so that equal maxima resolve to the first pixel in row-major
//                   order), one atomicMax per block
//   k_clean_prep    one thread: decodes the key, applies the do-while test of the
//                   algorithm (the first iteration always runs, later ones only while the
//                   peak exceeds the threshold, at most max_iter), and writes the
//                   iteration's record: peak pixel and value, and the position record
//                   the gridded PSF kernel reads; clears the other key for the next
//                   iteration
//   (the PSF cutout at l0, by any of the plan's methods)
//   k_clean_sub     I_D -= gain I_D(l0) P / P(l0) on the N x N window around l0 (clipped
//                   to the image); the model gains gain I_D(l0) at l0; the component is
//                   recorded
// Every kernel returns at once when the record says the loop has stopped, so a chunk of
// iterations can be queued ahead and the host reads the record once per chunk.
#include <cuda_runtime.h>

#include "psf_internal.cuh"

namespace psf {
namespace {

__device__ __forceinline__ unsigned int ordered_bits(float v) {
    const unsigned int u = __float_as_uint(v);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

__device__ __forceinline__ float from_ordered(unsigned int o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
    return a > b ? a : b;
}

__global__ void k_clean_argmax(const float *__restrict__ res, int64_t n, const CleanState *__restrict__ st,
                               unsigned long long *__restrict__ key) {
    if (st->done) return;
    unsigned long long best = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k =
            ((unsigned long long)ordered_bits(res[i]) << 32) | (unsigned long long)(0xffffffffu - (unsigned int)i);
        best = umax64(best, k);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) best = umax64(best, __shfl_xor_sync(0xffffffffu, best, o));
    __shared__ unsigned long long wbest[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) wbest[w] = best;
    __syncthreads();
    if (w == 0) {
        best = lane < (int)(blockDim.x >> 5) ? wbest[lane] : 0ull;
#pragma unroll
        for (int o = 16; o; o >>= 1) best = umax64(best, __shfl_xor_sync(0xffffffffu, best, o));
        if (lane == 0) atomicMax(key, best);
    }
}

__global__ void k_clean_prep(const unsigned long long *__restrict__ key, unsigned long long *__restrict__ key_next,
                             CleanState *__restrict__ st, int nl, int nm, double cell, double lc, double mc,
                             float threshold, int max_iter, int literal) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    *key_next = 0ull;
    st->active = 0;
    if (st->done) return;
    if (st->iter >= max_iter) {
        st->done = 1;
        return;
    }
    const unsigned long long k = *key;
    const int pix = (int)(0xffffffffu - (unsigned int)(k & 0xffffffffull));
    const float peak = from_ordered((unsigned int)(k >> 32));
    if (st->iter > 0 && !(peak > threshold)) {
        st->done = 1;
        return;
    }
    st->active = 1;
    st->pix = pix;
    st->peak = peak;
    const int x = pix % nl, y = pix / nl;
    const double l0 = lc + (x - nl / 2) * cell, m0 = mc + (y - nm / 2) * cell;
    const float rho = (float)sqrt(l0 * l0 + m0 * m0);
    st->gpos.c = literal ? make_float4((float)-l0, (float)m0, rho, 0.f) : make_float4((float)m0, (float)-l0, rho, 0.f);
    st->gpos.off = 0;
    st->gpos.pad = 0;
}

__global__ void k_clean_sub(float *__restrict__ res, float *__restrict__ model, const float *__restrict__ P,
                            CleanState *__restrict__ st, int nl, int nm, int N, float gain,
                            int32_t *__restrict__ comp_pix, float *__restrict__ comp_flux) {
    if (!st->active) return;
    const int pix = st->pix;
    const float g = gain * st->peak;
    const float s = g / P[(N / 2) * N + N / 2];
    const int px = pix % nl, py = pix / nl;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (int64_t)N * N;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(q % N), j = (int)(q / N);
        const int x = px + i - N / 2, y = py + j - N / 2;
        if (x >= 0 && x < nl && y >= 0 && y < nm) res[(int64_t)y * nl + x] -= s * P[q];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (model) model[pix] += g;
        if (comp_pix) comp_pix[st->iter] = pix;
        if (comp_flux) comp_flux[st->iter] = g;
        st->iter += 1;
    }
}

}  // namespace

cudaError_t launch_clean_argmax(const float *res, int64_t n, const CleanState *st, unsigned long long *key, int nsm,
                                cudaStream_t s) {
    const int threads = 512;
    const int64_t want = (n + threads - 1) / threads;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)nsm * 4));
    k_clean_argmax<<<grid, threads, 0, s>>>(res, n, st, key);
    return cudaGetLastError();
}

cudaError_t launch_clean_prep(const unsigned long long *key, unsigned long long *key_next, CleanState *st, int nl,
                              int nm, double cell, double lc, double mc, float threshold, int max_iter, int literal,
                              cudaStream_t s) {
    k_clean_prep<<<1, 32, 0, s>>>(key, key_next, st, nl, nm, cell, lc, mc, threshold, max_iter, literal);
    return cudaGetLastError();
}

cudaError_t launch_clean_sub(float *res, float *model, const float *P, CleanState *st, int nl, int nm, int N,
                             float gain, int32_t *comp_pix, float *comp_flux, cudaStream_t s) {
    const int threads = 256;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)N * N + threads - 1) / threads, 64));
    k_clean_sub<<<grid, threads, 0, s>>>(res, model, P, st, nl, nm, N, gain, comp_pix, comp_flux);
    return cudaGetLastError();
}

}  // namespace psf
