// Width of PSF cutouts at half maximum along the radial and tangential directions of
// their positions (the size measure of Fig. 3).  One thread per (cutout, direction):
// half maximum = half the centre pixel (the PSF at l0); on each side the profile is
// sampled by bilinear interpolation every quarter pixel until the first sample at or
// below it, and the crossing is interpolated linearly from the previous sample.
#include <cuda_runtime.h>

#include "psf_internal.cuh"

namespace psf {
namespace {

constexpr float kStep = 0.25f;

// Bilinear P(x, y) (column x, row y); false outside [0, N-1]^2.
__device__ __forceinline__ bool bilinear(const float *P, int N, float x, float y, float *v) {
    if (!(x >= 0.f && y >= 0.f && x <= (float)(N - 1) && y <= (float)(N - 1))) return false;
    int i0 = (int)floorf(x), j0 = (int)floorf(y);
    i0 = min(i0, N - 2);
    j0 = min(j0, N - 2);
    const float fx = x - (float)i0, fy = y - (float)j0;
    const float *r0 = P + (int64_t)j0 * N + i0, *r1 = r0 + N;
    *v = (1.f - fx) * (1.f - fy) * r0[0] + fx * (1.f - fy) * r0[1] + (1.f - fx) * fy * r1[0] + fx * fy * r1[1];
    return true;
}

__global__ void k_fwhm(const float *__restrict__ cut, const FwhmItem *__restrict__ items, int npos, double cell,
                       double *__restrict__ out) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * npos) return;
    const int p = t >> 1, dir = t & 1;
    const FwhmItem it = items[p];
    const int N = it.N, c = N / 2;
    const float *P = cut + it.off;
    const float ex = dir ? -it.er_y : it.er_x, ey = dir ? it.er_x : it.er_y;
    const float centre = P[(int64_t)c * N + c], h = 0.5f * centre;
    double width = 0.0;
    for (int side = 0; side < 2; ++side) {
        const float sg = side ? -1.f : 1.f;
        float prev = centre, cross = -1.f;
        for (int k = 1; k <= 8 * N; ++k) {
            const float tt = k * kStep;
            float v;
            if (!bilinear(P, N, (float)c + sg * tt * ex, (float)c + sg * tt * ey, &v)) break;
            if (v <= h) {
                cross = tt - kStep + kStep * (prev - h) / (prev - v);
                break;
            }
            prev = v;
        }
        if (cross < 0.f) {
            width = __longlong_as_double(0x7ff8000000000000ll);   // NaN: the walk left the cutout
            break;
        }
        width += (double)cross;
    }
    out[2 * p + dir] = width * cell;
}

}  // namespace

cudaError_t launch_fwhm(const float *cut, const FwhmItem *items, int npos, double cell, double *out, cudaStream_t s) {
    if (npos <= 0) return cudaSuccess;
    const int threads = 128;
    k_fwhm<<<(2 * npos + threads - 1) / threads, threads, 0, s>>>(cut, items, npos, cell, out);
    return cudaGetLastError();
}

}  // namespace psf
