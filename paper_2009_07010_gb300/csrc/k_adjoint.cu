// Adjoint (vector-Jacobian product) of the cutout map of Eqs. 21-22, FP32 CUDA cores.
//
// For a cotangent R = dL/dP (packed like the forward output):
//   H_pk      = sum_{i,j} R_p[j][i] exp(2 pi i (u_k dl_i + v_k dm_j))
//             = sum_j b_k[j] ( sum_i R_p[j][i] a_k[i] ),
//   dL/dW_k   = sum_p Re( D_k(l0_p) H_pk ),
//   dL/dl0_p  = sum_k W_k Re( dD_k/dl0 (l0_p) H_pk ),   likewise m0.
// The pixel offsets dl_i, dm_j do not depend on l0 (the cutout moves with the
// source), so l0 enters through D_k alone.
//
// A CTA owns a contiguous range of visibilities; each thread owns kAdjT of them.
// For every position and every 32-row block of R (staged transposed in shared
// memory) a thread forms t_j = sum_i R[j][i] a_k[i] for the 32 rows (row twiddles by
// complex recurrence, re-seeded every 32 columns from float-float phases), then adds
// sum_j b_k[j] t_j into H.  After the last block D_k and its gradient are evaluated
// (decorr<true>) and folded into dL/dW_k (registers; written once per call, no
// atomics) and into per-thread position sums, which are reduced over the block and
// written to a per-CTA partial buffer; a second kernel adds the partials in float64.
#include "decorr.cuh"
#include "fp32_tile.cuh"

namespace psf {
namespace {

constexpr int kAdjThreads = 256;
constexpr int kAdjT = 4;        // visibilities per thread
constexpr int kAdjRows = 32;    // rows of R per shared-memory block
constexpr int kAdjMaxN = 512;

__device__ __forceinline__ float2 acmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

struct AdjPos {
    float4 L, dLl, dLm;   // direction (l0, m0, n0-1) and its derivatives
};

__global__ void __launch_bounds__(kAdjThreads) k_adjoint(DevObs o, int method, uint32_t flags,
                                                         const AdjPos *__restrict__ pos,
                                                         const int32_t *__restrict__ npix,
                                                         const int64_t *__restrict__ offs, int npos, float2 cell,
                                                         const float *__restrict__ R, float *__restrict__ gW,
                                                         int accumulate_gW, double *__restrict__ partial) {
    extern __shared__ __align__(16) float RT[];   // [N][kAdjRows], transposed block of R
    __shared__ float red[2][kAdjThreads / 32];
    const int tid = threadIdx.x;
    const int32_t kbase = blockIdx.x * (kAdjThreads * kAdjT);
    float gw[kAdjT];
    int32_t kk[kAdjT];
#pragma unroll
    for (int t = 0; t < kAdjT; ++t) {
        kk[t] = kbase + t * kAdjThreads + tid;
        gw[t] = 0.f;
    }
    for (int p = 0; p < npos; ++p) {
        const int N = npix[p];
        const int half = N / 2;
        const float *Rp = R + offs[p];
        float2 H[kAdjT];
#pragma unroll
        for (int t = 0; t < kAdjT; ++t) H[t] = make_float2(0.f, 0.f);
        for (int j0 = 0; j0 < N; j0 += kAdjRows) {
            __syncthreads();
            for (int e = tid; e < N * kAdjRows; e += kAdjThreads) {
                const int i = e / kAdjRows, jj = e - i * kAdjRows;
                const int j = j0 + jj;
                RT[e] = (j < N) ? Rp[(int64_t)j * N + i] : 0.f;
            }
            __syncthreads();
#pragma unroll
            for (int t = 0; t < kAdjT; ++t) {
                const int32_t k = kk[t];
                if (k >= o.nvis) continue;
                // pixel phases per unit offset as float-float pairs (fp32_tile.cuh): seeds
                // and steps lose their whole turns exactly before rounding
                const float2 uh = o.uv[k], ul = o.uv_lo[k];
                const float2 tu = fp32t::ff_mul(uh.x, ul.x, cell.x, cell.y);
                const float2 tv = fp32t::ff_mul(uh.y, ul.y, cell.x, cell.y);
                const float2 zu = fp32t::cis_acc(fp32t::ff_turns(tu, 1));
                float tre[kAdjRows], tim[kAdjRows];
#pragma unroll
                for (int jj = 0; jj < kAdjRows; ++jj) { tre[jj] = 0.f; tim[jj] = 0.f; }
                for (int i0 = 0; i0 < N; i0 += 32) {
                    float2 a = fp32t::cis_acc(fp32t::ff_turns(tu, i0 - half));
                    const int iend = min(N, i0 + 32);
                    for (int i = i0; i < iend; ++i) {
                        const float4 *row = reinterpret_cast<const float4 *>(RT + i * kAdjRows);
#pragma unroll
                        for (int q = 0; q < kAdjRows / 4; ++q) {
                            const float4 r = row[q];
                            tre[4 * q + 0] = fmaf(r.x, a.x, tre[4 * q + 0]);
                            tim[4 * q + 0] = fmaf(r.x, a.y, tim[4 * q + 0]);
                            tre[4 * q + 1] = fmaf(r.y, a.x, tre[4 * q + 1]);
                            tim[4 * q + 1] = fmaf(r.y, a.y, tim[4 * q + 1]);
                            tre[4 * q + 2] = fmaf(r.z, a.x, tre[4 * q + 2]);
                            tim[4 * q + 2] = fmaf(r.z, a.y, tim[4 * q + 2]);
                            tre[4 * q + 3] = fmaf(r.w, a.x, tre[4 * q + 3]);
                            tim[4 * q + 3] = fmaf(r.w, a.y, tim[4 * q + 3]);
                        }
                        a = acmul(a, zu);
                    }
                }
                float2 b = fp32t::cis_acc(fp32t::ff_turns(tv, j0 - half));
                const float2 zv = fp32t::cis_acc(fp32t::ff_turns(tv, 1));
                float2 h = H[t];
#pragma unroll
                for (int jj = 0; jj < kAdjRows; ++jj) {
                    // h += b * (tre + i tim)
                    h.x = fmaf(b.x, tre[jj], fmaf(-b.y, tim[jj], h.x));
                    h.y = fmaf(b.x, tim[jj], fmaf(b.y, tre[jj], h.y));
                    b = acmul(b, zv);
                }
                H[t] = h;
            }
        }
        // fold H into the gradients
        const AdjPos P = pos[p];
        float gl = 0.f, gm = 0.f;
#pragma unroll
        for (int t = 0; t < kAdjT; ++t) {
            const int32_t k = kk[t];
            if (k >= o.nvis) continue;
            const int bin = k / o.nout, r = k - bin * o.nout;
            float4 g;
            const float2 D = decorr<true>(o, method, flags, bin, r, P.L, P.dLl, P.dLm, &g);
            const float Wk = o.W[k];
            gw[t] += D.x * H[t].x - D.y * H[t].y;
            gl += Wk * (g.x * H[t].x - g.y * H[t].y);
            gm += Wk * (g.z * H[t].x - g.w * H[t].y);
        }
        // block reduction of the position sums
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1) {
            gl += __shfl_xor_sync(0xffffffffu, gl, sh);
            gm += __shfl_xor_sync(0xffffffffu, gm, sh);
        }
        if ((tid & 31) == 0) {
            red[0][tid >> 5] = gl;
            red[1][tid >> 5] = gm;
        }
        __syncthreads();
        if (tid == 0) {
            double sl = 0.0, sm = 0.0;
            for (int w = 0; w < kAdjThreads / 32; ++w) { sl += red[0][w]; sm += red[1][w]; }
            partial[((int64_t)blockIdx.x * npos + p) * 2 + 0] = sl;
            partial[((int64_t)blockIdx.x * npos + p) * 2 + 1] = sm;
        }
    }
#pragma unroll
    for (int t = 0; t < kAdjT; ++t) {
        const int32_t k = kk[t];
        if (k < o.nvis && gW) gW[k] = accumulate_gW ? gW[k] + gw[t] : gw[t];
    }
}

__global__ void __launch_bounds__(256) k_adjoint_reduce(const double *__restrict__ partial, int ncta, int npos,
                                                        double *__restrict__ g_lm) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= npos * 2) return;
    double s = 0.0;
    for (int c = 0; c < ncta; ++c) s += partial[(int64_t)c * npos * 2 + e];
    g_lm[e] = s;
}

}  // namespace

int adjoint_max_n() { return kAdjMaxN; }
int64_t adjoint_ctas(int64_t nvis) { return (nvis + kAdjThreads * kAdjT - 1) / (kAdjThreads * kAdjT); }

cudaError_t launch_adjoint_chunk(const DevObs &o, int method, uint32_t flags, const void *pos, const int32_t *npix,
                                 const int64_t *offs, int npos, int nmax, double cell, const float *R, float *gW,
                                 int accumulate_gW, double *partial, double *g_lm, cudaStream_t st) {
    if (npos <= 0) return cudaSuccess;
    const int64_t ncta = adjoint_ctas(o.nvis);
    const size_t smem = (size_t)nmax * kAdjRows * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(k_adjoint, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_adjoint<<<(unsigned)ncta, kAdjThreads, smem, st>>>(o, method, flags, (const AdjPos *)pos, npix, offs, npos,
                                                         fp32t::cell_pair(cell), R, gW, accumulate_gW, partial);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_adjoint_reduce<<<(npos * 2 + 255) / 256, 256, 0, st>>>(partial, (int)ncta, npos, g_lm);
    return cudaGetLastError();
}

}  // namespace psf
