// psf_exact_noalloc: the exact smeared PSF of one cutout without any device
// allocation during the call.
//
// Some callers cannot allocate device memory while they compute: code that runs
// inside a CUDA stream capture (cudaMalloc is not a capturable call), real-time or
// embedded pipelines that forbid allocation after start-up, and plug-ins running
// inside a host application whose allocator already owns the device memory.  This
// entry point serves them: it uses only the plan's arrays (allocated earlier by
// psf_plan), the caller's output buffer, and a fixed scratch array that lives in the
// library's image on every device that loads it.
//
// The computation is the FP32 CUDA-core form: per 64 x 64 pixel tile and visibility
// range, the smearing weights W_k D_k are evaluated inline (no weight buffer), the
// twiddles are generated by recurrence, and each (tile, range) partial sum goes to
// the scratch array; a second kernel adds the partials in float64 into the output.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "decorr.cuh"

namespace psf {
namespace {

constexpr int kNaTile = 64;
constexpr int kNaKC = 32;
constexpr int kNaSeg = 16;
constexpr int kNaMaxN = 256;       // largest cutout
constexpr int kNaMaxSplit = 64;    // visibility ranges per tile
constexpr size_t kNaScratchFloats = (size_t)kNaMaxSplit * kNaMaxN * kNaMaxN;   // 16 MiB

// Split-K partial cutouts of the last call, [split][N*N].  Shared by every call on
// a device; every element a call reads back is written earlier in the same call.
static __device__ __align__(256) float g_noalloc_partial[kNaScratchFloats];

__device__ __forceinline__ float2 na_cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__global__ void __launch_bounds__(256) k_noalloc_exact(DevObs o, uint32_t flags, float4 L, int N, float cell,
                                                       int32_t kper, float *__restrict__ partial) {
    __shared__ __align__(16) float2 sa[kNaKC][kNaTile];
    __shared__ __align__(16) float2 sc[kNaKC][kNaTile];
    const int ntx = (N + kNaTile - 1) / kNaTile;
    const int i0 = (blockIdx.x % ntx) * kNaTile, j0 = (blockIdx.x / ntx) * kNaTile;
    const int split = blockIdx.y;
    const int32_t kbeg = split * kper, kend = min(o.nvis, kbeg + kper);
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int gk = tid & 31, gs = tid >> 5;
    const int seg_first = (gs & 3) * kNaSeg;
    const int n_first = (gs < 4 ? i0 : j0) + seg_first - N / 2;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float acc[4][4], tot[4][4], cmp[4][4];
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int a = 0; a < 4; ++a) { acc[b][a] = 0.f; tot[b][a] = 0.f; cmp[b][a] = 0.f; }
    for (int32_t kc = kbeg; kc < kend; kc += kNaKC) {
        const int32_t k = kc + gk;
        float2 seed = make_float2(0.f, 0.f), step = make_float2(1.f, 0.f);
        if (k < kend) {
            const float2 uvk = o.uv[k];
            const float theta = (gs < 4 ? uvk.x : uvk.y) * cell;
            sincospif(2.0f * theta * (float)n_first, &seed.y, &seed.x);
            sincospif(2.0f * theta, &step.y, &step.x);
            if (gs >= 4) {
                const int bin = k / o.nout, r = k - bin * o.nout;
                const float2 D = decorr<false>(o, kExact, flags, bin, r, L, z4, z4, nullptr);
                const float Wk = o.W[k];
                seed = na_cmul(seed, make_float2(Wk * D.x, Wk * D.y));
            }
        }
        __syncthreads();
        float2 *dst = (gs < 4 ? &sa[gk][seg_first] : &sc[gk][seg_first]);
#pragma unroll
        for (int q = 0; q < kNaSeg; ++q) {
            dst[q] = seed;
            seed = na_cmul(seed, step);
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < kNaKC; ++kk) {
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
    float *dst = partial + (size_t)split * N * N;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int j = j0 + ty * 4 + b;
        if (j >= N) continue;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int i = i0 + tx * 4 + a;
            if (i < N) dst[(size_t)j * N + i] = tot[b][a];
        }
    }
}

__global__ void __launch_bounds__(256) k_noalloc_reduce(const float *__restrict__ partial, int nsplit, int n2,
                                                        float *__restrict__ out) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n2; q += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int sp = 0; sp < nsplit; ++sp) s += (double)partial[(size_t)sp * n2 + q];
        out[q] = (float)s;
    }
}

// Device address of the scratch array, looked up once per device.
constexpr int kNaMaxDevices = 64;
std::mutex g_na_mutex;
float *g_na_ptr[kNaMaxDevices] = {};

int scratch_for_current_device(float **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return PSF_ECUDA; }
    if (dev < 0 || dev >= kNaMaxDevices) return PSF_EUNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_partial) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return PSF_ECUDA;
        }
        g_na_ptr[dev] = (float *)ptr;
    }
    *out = g_na_ptr[dev];
    return PSF_OK;
}

}  // namespace
}  // namespace psf

extern "C" int psf_exact_noalloc(psf_plan_t plan, double l0, double m0, int npix, double cell_rad,
                                 float *out_dev, void *cuda_stream) {
    using namespace psf;
    const DevObs *o = plan_devobs(plan);
    if (!o || !out_dev || !(cell_rad > 0.0)) return PSF_EINVAL;
    if (npix < 2 || (npix & 1)) return PSF_EINVAL;
    if (npix > kNaMaxN) return PSF_EUNSUPPORTED;   // beyond the fixed scratch
    const double r2 = l0 * l0 + m0 * m0;
    if (!(r2 < 1.0)) return PSF_EINVAL;
    const uint32_t flags = plan_flags(plan);
    const double n0m1 = (flags & PSF_WTERM) ? -r2 / (1.0 + std::sqrt(1.0 - r2)) : 0.0;
    float *scratch = nullptr;
    int st = scratch_for_current_device(&scratch);
    if (st) return st;
    const int64_t K = o->nvis;
    const int ntiles = ((npix + kNaTile - 1) / kNaTile) * ((npix + kNaTile - 1) / kNaTile);
    int nsplit = (int)std::min<int64_t>(kNaMaxSplit, std::max<int64_t>(1, (K + 4095) / 4096));
    const int32_t kper = (int32_t)(((K + nsplit - 1) / nsplit + 31) / 32 * 32);
    nsplit = (int)((K + kper - 1) / kper);
    if ((size_t)nsplit * npix * npix > kNaScratchFloats) return PSF_EUNSUPPORTED;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const float4 L = make_float4((float)l0, (float)m0, (float)n0m1, 0.f);
    k_noalloc_exact<<<dim3(ntiles, nsplit), 256, 0, s>>>(*o, flags, L, npix, (float)cell_rad, kper, scratch);
    if (cudaGetLastError() != cudaSuccess) return PSF_ECUDA;
    k_noalloc_reduce<<<64, 256, 0, s>>>(scratch, nsplit, npix * npix, out_dev);
    if (cudaGetLastError() != cudaSuccess) return PSF_ECUDA;
    return PSF_OK;
}
