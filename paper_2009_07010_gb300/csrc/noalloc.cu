// psf_exact_noalloc: the exact smeared PSF of one cutout without any device
// allocation during the call.
//
// Some callers cannot allocate device memory while they compute: real-time or
// embedded pipelines that forbid allocation once they have started, and plug-ins
// running inside a host application whose allocator already owns the device memory.
// This entry point serves them: it uses only the plan's arrays (allocated earlier by
// psf_plan), the caller's output buffer, and a fixed scratch array that lives in the
// library's image on every device that loads it.
//
// The computation is the FP32 CUDA-core form (the tile body fp32t::tile_sum of the
// FP32 path): per 64 x 64 pixel tile and visibility range the smearing weights
// W_k D_k are evaluated inline (no weight buffer), each (tile, range) partial sum goes
// to the scratch array, and a second kernel adds the partials in float64 into the
// output.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "decorr.cuh"
#include "fp32_tile.cuh"

namespace psf {
namespace {

constexpr int kNaMaxN = 256;       // largest cutout
constexpr int kNaMaxSplit = 64;    // visibility ranges per tile
constexpr size_t kNaScratchFloats = (size_t)kNaMaxSplit * kNaMaxN * kNaMaxN;   // 16 MiB

// Split-K partial cutouts of the last call, [split][N*N].  Shared by every call on
// a device; every element a call reads back is written earlier in the same call.
static __device__ __align__(256) float g_noalloc_partial[kNaScratchFloats];

__global__ void __launch_bounds__(256) k_noalloc_exact(DevObs o, uint32_t flags, float4 L, int N, float2 cell,
                                                       int32_t kper, float *__restrict__ partial) {
    __shared__ __align__(16) float2 sa[fp32t::kKC][fp32t::kT];
    __shared__ __align__(16) float2 sc[fp32t::kKC][fp32t::kT];
    const int ntx = (N + fp32t::kT - 1) / fp32t::kT;
    const int i0 = (blockIdx.x % ntx) * fp32t::kT, j0 = (blockIdx.x / ntx) * fp32t::kT;
    const int split = blockIdx.y;
    const int32_t kbeg = split * kper, kend = min(o.nvis, kbeg + kper);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float tot[4][4];
#pragma unroll
    for (int b = 0; b < 4; ++b)
#pragma unroll
        for (int a = 0; a < 4; ++a) tot[b][a] = 0.f;
    // the weight W_k D_k(l0) of Eqs. 13 and 21-22, evaluated where the twiddles need it
    auto wfn = [&](int32_t k) {
        const int bin = k / o.nout, r = k - bin * o.nout;
        const float2 D = decorr<false>(o, kExact, flags, bin, r, L, z4, z4, nullptr);
        const float Wk = o.W[k];
        return make_float2(Wk * D.x, Wk * D.y);
    };
    fp32t::tile_sum(o.uv, o.uv_lo, kbeg, kend, N, i0, j0, cell, wfn, sa, sc, tot);
    fp32t::tile_store(partial + (size_t)split * N * N, N, i0, j0, tot);
}

__global__ void __launch_bounds__(256) k_noalloc_reduce(const float *__restrict__ partial, int nsplit, int n2,
                                                        float *__restrict__ out) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n2; q += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int sp = 0; sp < nsplit; ++sp) s += (double)partial[(size_t)sp * n2 + q];
        out[q] = (float)s;
    }
}

// Device address of the scratch array, looked up once per device with that device
// current (in host code the array's name is only a host-side stand-in).
constexpr int kNaMaxDevices = 64;
std::mutex g_na_mutex;
float *g_na_ptr[kNaMaxDevices] = {};

int scratch_for_device(int dev, float **out) {
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
    // the kernel reads the plan's arrays: it must run on the plan's device
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return PSF_ECUDA; }
    if (dev != plan_device(plan)) return PSF_EINVAL;
    const uint32_t flags = plan_flags(plan);
    const double n0m1 = (flags & PSF_WTERM) ? -r2 / (1.0 + std::sqrt(1.0 - r2)) : 0.0;
    float *scratch = nullptr;
    int st = scratch_for_device(dev, &scratch);
    if (st) return st;
    const int64_t K = o->nvis;
    const int nt = (npix + fp32t::kT - 1) / fp32t::kT;
    int nsplit = (int)std::min<int64_t>(kNaMaxSplit, std::max<int64_t>(1, (K + 4095) / 4096));
    const int32_t kper = (int32_t)(((K + nsplit - 1) / nsplit + 31) / 32 * 32);
    nsplit = (int)((K + kper - 1) / kper);
    if ((size_t)nsplit * npix * npix > kNaScratchFloats) return PSF_EUNSUPPORTED;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const float4 L = make_float4((float)l0, (float)m0, (float)n0m1, 0.f);
    k_noalloc_exact<<<dim3(nt * nt, nsplit), 256, 0, s>>>(*o, flags, L, npix, fp32t::cell_pair(cell_rad), kper,
                                                          scratch);
    if (cudaGetLastError() != cudaSuccess) return PSF_ECUDA;
    k_noalloc_reduce<<<64, 256, 0, s>>>(scratch, nsplit, npix * npix, out_dev);
    if (cudaGetLastError() != cudaSuccess) return PSF_ECUDA;
    return PSF_OK;
}
