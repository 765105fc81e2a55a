// Gridded image-plane approximation: Eq. 45 with Algorithm 1 on the cutout's uv grid.
//
// Eq. 45 writes the image-plane approximation as F^-1{F{P} . D}: the effective PSF P
// is transformed once, and per source position only the distortion D of Algorithm 1
// is evaluated on the uv cells before one inverse transform.  Here the grid is the
// N x N Fourier grid of an N x N cutout of pixel size cell: cells du = dv = 1/(N cell),
// cell (a, b) at u = (a - N/2) du, v = (b - N/2) dv, so that the transform pair is the
// N x N DFT of the cutout's pixel grid.
//
// Position independent, once per (N, cell, precision) and kept by the plan:
//   P  the effective PSF, the cutout at the phase centre where every decorrelation
//      is 1 (computed by the visibility-level path of the plan's precision),
//   S  = F{P} / N^2 (k_grid_dft_rows / k_grid_dft_cols, FP64),
//   per cell the W-weighted means of dt_k and dnu_r / nu_r over the visibilities whose
//      nearest cell is this cell or its mirror, modulo N; cells that receive none take
//      the means over all visibilities (k_grid_cells, FP64 sums); the nearest-cell
//      decision a' = floor(u_k N cell + 0.5), u_k = ubar nu_r / c, is taken in FP64
//      with IEEE round-to-nearest operations in exactly that order,
//   the table G[a][b] = (Re S, Im S, alpha, beta), alpha = omega_E dt_c du and
//      beta = (dnu/nu)_c |u_c|, so that Algorithm 1's half phase changes are
//      A = alpha (a' m0 - b' l0) (theta = atan2(v, u); (b' m0 - a' l0) for the literal
//      arctan(u/v)) and B = beta rho (k_grid_table).
// Per pair of positions (k_img_grid): X = S (D_0 + i D_1) with D_p = sinc(A_p) sinc(B_p).
// The cutout is the real part of F^-1{S D}; with S Hermitian that equals F^-1{S D'} where
// D' averages D over each cell and its mirror modulo N, which differs from D only on the
// Nyquist row and column (a' or b' = -N/2, their own mirrors).  S D' is Hermitian, so the
// inverse transform of X has the cutout of position 0 as its real part and that of
// position 1 as its imaginary part.  The N x N inverse FFT runs in
// shared memory as two passes (rows, then columns) of radix R1 x R2 Cooley-Tukey with
// the small DFTs in registers; D is evaluated inside the first stage, and the last stage
// writes both cutouts straight to global memory.
#include <cuda_runtime.h>

#include "psf_internal.cuh"

namespace psf {
namespace {

__device__ __forceinline__ int mod_n(int64_t x, int n) {
    const int64_t r = x % n;
    return (int)(r < 0 ? r + n : r);
}

// ------------------------------------------------------------------ table build

__device__ __forceinline__ void cell_flush(double *acc, int c1, int c2, double sw, double sdt, double sr) {
    if (c1 < 0) return;
    atomicAdd(acc + 3 * c1, sw);
    atomicAdd(acc + 3 * c1 + 1, sdt);
    atomicAdd(acc + 3 * c1 + 2, sr);
    atomicAdd(acc + 3 * c2, sw);
    atomicAdd(acc + 3 * c2 + 1, sdt);
    atomicAdd(acc + 3 * c2 + 2, sr);
}

// One thread per (baseline, output channel): walks the baseline's time bins, whose uv
// track stays in one cell for many consecutive bins, and adds its running sums to the
// cell and its mirror whenever the cell changes.  acc[3 q + (0, 1, 2)] = sum W,
// sum W dt, sum W dnu/nu of cell q = b N + a; glob = the same sums over all visibilities.
__global__ void k_grid_cells(const double2 *__restrict__ bin_uv, const int2 *__restrict__ bin_samp,
                             const int32_t *__restrict__ bin_first, const double2 *__restrict__ chan,
                             const float *__restrict__ W, int nbl, int nout, double dt_raw, int N, double ncell,
                             double *__restrict__ acc, double *__restrict__ glob) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double gw = 0, gdt = 0, gr = 0;
    if (t < (int64_t)nbl * nout) {
        const int b = (int)(t / nout), r = (int)(t % nout);
        const double nu = chan[r].x, rr = __ddiv_rn(chan[r].y, nu);
        int c1 = -1, c2 = -1;
        double sw = 0, sdt = 0, sr = 0;
        const int e = bin_first[b + 1];
        for (int bin = bin_first[b]; bin < e; ++bin) {
            const double2 ub = bin_uv[bin];
            const double u = __ddiv_rn(__dmul_rn(ub.x, nu), kCLight);
            const double v = __ddiv_rn(__dmul_rn(ub.y, nu), kCLight);
            const int64_t ia = (int64_t)floor(__dadd_rn(__dmul_rn(u, ncell), 0.5));
            const int64_t ib = (int64_t)floor(__dadd_rn(__dmul_rn(v, ncell), 0.5));
            const int n1 = mod_n(ib + N / 2, N) * N + mod_n(ia + N / 2, N);
            const double w = (double)W[(int64_t)bin * nout + r];
            const double dt = __dmul_rn((double)bin_samp[bin].y, dt_raw);
            if (n1 != c1) {
                cell_flush(acc, c1, c2, sw, sdt, sr);
                c1 = n1;
                c2 = mod_n(-ib + N / 2, N) * N + mod_n(-ia + N / 2, N);
                sw = sdt = sr = 0;
            }
            sw += w;
            sdt += w * dt;
            sr += w * rr;
            gw += w;
            gdt += w * dt;
            gr += w * rr;
        }
        cell_flush(acc, c1, c2, sw, sdt, sr);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        gw += __shfl_xor_sync(0xffffffffu, gw, o);
        gdt += __shfl_xor_sync(0xffffffffu, gdt, o);
        gr += __shfl_xor_sync(0xffffffffu, gr, o);
    }
    if ((threadIdx.x & 31) == 0 && gw != 0.0) {
        atomicAdd(glob, gw);
        atomicAdd(glob + 1, gdt);
        atomicAdd(glob + 2, gr);
    }
}

// exp(-2 pi i m / N) for m in [0, N), in shared memory.
__device__ __forceinline__ void dft_table(double2 *tw, int N) {
    for (int m = threadIdx.x; m < N; m += blockDim.x) {
        double s, c;
        sincospi(2.0 * m / N, &s, &c);
        tw[m] = make_double2(c, -s);
    }
    __syncthreads();
}

__device__ __forceinline__ int twiddle_index(int x, int y, int N) {
    return mod_n((int64_t)(x - N / 2) * (int64_t)(y - N / 2), N);
}

// Y[j][a] = sum_i P[j][i] exp(-2 pi i (a - N/2)(i - N/2) / N); block j, thread a.
__global__ void k_grid_dft_rows(const float *__restrict__ P, double2 *__restrict__ Y, int N) {
    extern __shared__ double2 tw[];
    dft_table(tw, N);
    const int j = blockIdx.x;
    for (int a = threadIdx.x; a < N; a += blockDim.x) {
        double re = 0, im = 0;
        for (int i = 0; i < N; ++i) {
            const double2 w = tw[twiddle_index(a, i, N)];
            const double p = (double)P[(int64_t)j * N + i];
            re += p * w.x;
            im += p * w.y;
        }
        Y[(int64_t)j * N + a] = make_double2(re, im);
    }
}

// S[b][a] = sum_j Y[j][a] exp(-2 pi i (b - N/2)(j - N/2) / N); block b, thread a.
__global__ void k_grid_dft_cols(const double2 *__restrict__ Y, double2 *__restrict__ S, int N) {
    extern __shared__ double2 tw[];
    dft_table(tw, N);
    const int b = blockIdx.x;
    for (int a = threadIdx.x; a < N; a += blockDim.x) {
        double re = 0, im = 0;
        for (int j = 0; j < N; ++j) {
            const double2 w = tw[twiddle_index(b, j, N)];
            const double2 y = Y[(int64_t)j * N + a];
            re += y.x * w.x - y.y * w.y;
            im += y.x * w.y + y.y * w.x;
        }
        S[(int64_t)b * N + a] = make_double2(re, im);
    }
}

// G[a N + b] = (Re S / N^2, Im S / N^2, omega_E dt_c du, (dnu/nu)_c |u_c|) for cell (a, b).
__global__ void k_grid_table(const double2 *__restrict__ S, const double *__restrict__ acc,
                             const double *__restrict__ glob, int N, double du, float4 *__restrict__ G) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)N * N) return;
    const int a = (int)(q % N), b = (int)(q / N);
    const double sw = acc[3 * q];
    const double gw = glob[0];
    const double dt = sw > 0 ? acc[3 * q + 1] / sw : (gw > 0 ? glob[1] / gw : 0.0);
    const double r = sw > 0 ? acc[3 * q + 2] / sw : (gw > 0 ? glob[2] / gw : 0.0);
    const double ua = (a - N / 2) * du, vb = (b - N / 2) * du;
    const double inv = 1.0 / ((double)N * N);
    G[(int64_t)a * N + b] = make_float4((float)(S[q].x * inv), (float)(S[q].y * inv), (float)(kOmegaE * dt * du),
                                        (float)(r * sqrt(ua * ua + vb * vb)));
}

// ------------------------------------------------------------------ per-position transform

// sinc_pi(x) = sin(pi x) / (pi x) = (-1)^n [sin(pi f) / (pi f)] (f / x), x = n + f, |f| <= 1/2.
// The bracket is its Taylor series in (pi f)^2 to order 12 (truncation error < 5e-10).
__device__ __forceinline__ float sinc_fast(float x) {
    const float n = rintf(x);
    const float f = x - n;
    const float z = f * f;
    float q = fmaf(z, 1.4842879e-4f, -2.3460810e-3f);
    q = fmaf(z, q, 2.6147848e-2f);
    q = fmaf(z, q, -1.9075182e-1f);
    q = fmaf(z, q, 8.1174243e-1f);
    q = fmaf(z, q, -1.6449341f);
    q = fmaf(z, q, 1.0f);
    const int ni = (int)n;
    if (ni != 0) q *= __fdividef(f, x);
    return (ni & 1) ? -q : q;
}

__host__ __device__ constexpr int ilog2(int r) { return r <= 1 ? 0 : 1 + ilog2(r / 2); }

__host__ __device__ constexpr int bitrev(int i, int r) {
    int o = 0;
    for (int b = 1; b < r; b <<= 1) {
        o = (o << 1) | (i & 1);
        i >>= 1;
    }
    return o;
}

// cos and sin of 2 pi e / 16.
__host__ __device__ constexpr float cos16(int e) {
    return e == 0 ? 1.f : e == 1 ? 0.92387953f : e == 2 ? 0.70710678f : e == 3 ? 0.38268343f
         : e == 4 ? 0.f : e == 5 ? -0.38268343f : e == 6 ? -0.70710678f : -0.92387953f;
}
__host__ __device__ constexpr float sin16(int e) {
    return e == 0 ? 0.f : e == 1 ? 0.38268343f : e == 2 ? 0.70710678f : e == 3 ? 0.92387953f
         : e == 4 ? 1.f : e == 5 ? 0.92387953f : e == 6 ? 0.70710678f : 0.38268343f;
}

// v exp(+2 pi i e / R), 0 <= e < R / 2 (a compile-time constant once unrolled).
template <int R>
__device__ __forceinline__ float2 rot(float2 v, int e) {
    const int e16 = e * (16 / R);
    if (e16 == 0) return v;
    if (e16 == 4) return make_float2(-v.y, v.x);
    const float c = cos16(e16), s = sin16(e16);
    return make_float2(v.x * c - v.y * s, v.x * s + v.y * c);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// In-register inverse DFT y[k] = sum_n x[n] exp(+2 pi i n k / R), R in {4, 8, 16}:
// radix-2 decimation in time, natural order in and out.
template <int R>
__device__ __forceinline__ void dft_reg(float2 (&x)[R]) {
    static_assert(R == 4 || R == 8 || R == 16, "radix");
    float2 t[R];
#pragma unroll
    for (int i = 0; i < R; ++i) t[bitrev(i, R)] = x[i];
#pragma unroll
    for (int st = 0; st < ilog2(R); ++st) {
        const int m = 1 << st;
#pragma unroll
        for (int s = 0; s < R; s += 2 * m)
#pragma unroll
            for (int k = 0; k < m; ++k) {
                const float2 u = t[s + k];
                const float2 v = rot<R>(t[s + k + m], k * (R / (2 * m)));
                t[s + k] = make_float2(u.x + v.x, u.y + v.y);
                t[s + k + m] = make_float2(u.x - v.x, u.y - v.y);
            }
    }
#pragma unroll
    for (int i = 0; i < R; ++i) x[i] = t[i];
}

template <int N>
struct GridFft;
template <>
struct GridFft<16> { static constexpr int R1 = 4, R2 = 4, T = 64; };
template <>
struct GridFft<32> { static constexpr int R1 = 8, R2 = 4, T = 128; };
template <>
struct GridFft<64> { static constexpr int R1 = 8, R2 = 8, T = 256; };
template <>
struct GridFft<128> { static constexpr int R1 = 16, R2 = 8, T = 512; };

template <int N>
constexpr int grid_smem_bytes() { return (N * (N + 1) + N) * (int)sizeof(float2); }

// One CTA per pair of positions (grid-stride over pairs).  Shared memory: X [N][N + 1]
// complex (row b = v cell / output row j, column a = u cell / output column i; the pad
// keeps row-wise and column-wise lane patterns free of bank conflicts) and the N
// twiddles exp(+2 pi i m / N).  Cell and pixel index origins are at N/2:
// exp(2 pi i (a - N/2)(i - N/2) / N) = (-1)^(a + i) exp(2 pi i a i / N) for N % 4 == 0,
// so X carries (-1)^(a + b) and the output (-1)^(i + j).
template <int N>
__global__ void __launch_bounds__(GridFft<N>::T) k_img_grid(const float4 *__restrict__ G,
                                                            const GridPair *__restrict__ pairs, int npairs,
                                                            float *__restrict__ out) {
    constexpr int R1 = GridFft<N>::R1, R2 = GridFft<N>::R2, T = GridFft<N>::T, LD = N + 1;
    constexpr int NA = N * R2 / T;   // items (line, n2) per thread in the first stage of a pass
    constexpr int NB = N * R1 / T;   // items (line, k1) per thread in the second stage
    static_assert(R1 * R2 == N && NA * T == N * R2 && NB * T == N * R1, "shape");
    extern __shared__ float2 smem[];
    float2 *X = smem;
    float2 *tw = smem + N * LD;
    for (int m = threadIdx.x; m < N; m += T) {
        float s, c;
        sincospif(2.0f * (float)m / (float)N, &s, &c);
        tw[m] = make_float2(c, s);
    }
    __syncthreads();
    for (int pr = blockIdx.x; pr < npairs; pr += gridDim.x) {
        const GridPair pp = pairs[pr];
        // pass 1 (rows b), stage a: X = S (D_0 + i D_1) (-1)^(a+b) on the cells a = n2 + R2 n1,
        // R1-point DFT over n1, twiddle exp(2 pi i n2 k1 / N), stored at a = n2 + R2 k1
#pragma unroll 1
        for (int q = 0; q < NA; ++q) {
            const int it = threadIdx.x + q * T;
            const int b = it % N, n2 = it / N;
            const float bf = (float)(b - N / 2);
            const float t0 = bf * pp.c0.y, t1 = bf * pp.c1.y;
            float2 x[R1];
#pragma unroll
            for (int n1 = 0; n1 < R1; ++n1) {
                const int a = n2 + R2 * n1;
                const float4 g = __ldg(G + a * N + b);
                const float af = (float)(a - N / 2);
                float e0 = sinc_fast(g.z * fmaf(af, pp.c0.x, t0));
                float e1 = sinc_fast(g.z * fmaf(af, pp.c1.x, t1));
                if (a == 0 || b == 0) {
                    // Nyquist row / column: the cell is its own mirror modulo N, and the real
                    // part of the inverse transform averages D over u and its alias
                    const float ma = a == 0 ? af : -af, mb = b == 0 ? bf : -bf;
                    e0 = 0.5f * (e0 + sinc_fast(g.z * fmaf(ma, pp.c0.x, mb * pp.c0.y)));
                    e1 = 0.5f * (e1 + sinc_fast(g.z * fmaf(ma, pp.c1.x, mb * pp.c1.y)));
                }
                const float d0 = e0 * sinc_fast(g.w * pp.c0.z), d1 = e1 * sinc_fast(g.w * pp.c1.z);
                float xr = g.x * d0 - g.y * d1, xi = g.y * d0 + g.x * d1;
                if ((a + b) & 1) {
                    xr = -xr;
                    xi = -xi;
                }
                x[n1] = make_float2(xr, xi);
            }
            dft_reg<R1>(x);
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1) X[b * LD + n2 + R2 * k1] = cmul(x[k1], tw[n2 * k1]);
        }
        __syncthreads();
        // pass 1, stage b: R2-point DFT over n2 for each (b, k1); output column k1 + R1 k2
        {
            float2 y[NB][R2];
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                const int it = threadIdx.x + q * T;
                const int b = it % N, k1 = it / N;
#pragma unroll
                for (int n2 = 0; n2 < R2; ++n2) y[q][n2] = X[b * LD + R2 * k1 + n2];
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                const int it = threadIdx.x + q * T;
                const int b = it % N, k1 = it / N;
                dft_reg<R2>(y[q]);
#pragma unroll
                for (int k2 = 0; k2 < R2; ++k2) X[b * LD + k1 + R1 * k2] = y[q][k2];
            }
        }
        __syncthreads();
        // pass 2 (columns i), stage a: rows n2 + R2 n1, in place
#pragma unroll 1
        for (int q = 0; q < NA; ++q) {
            const int it = threadIdx.x + q * T;
            const int i = it % N, n2 = it / N;
            float2 x[R1];
#pragma unroll
            for (int n1 = 0; n1 < R1; ++n1) x[n1] = X[(n2 + R2 * n1) * LD + i];
            dft_reg<R1>(x);
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1) X[(n2 + R2 * k1) * LD + i] = cmul(x[k1], tw[n2 * k1]);
        }
        __syncthreads();
        // pass 2, stage b: rows j = k1 + R1 k2 of both cutouts, streamed to global memory
#pragma unroll 1
        for (int q = 0; q < NB; ++q) {
            const int it = threadIdx.x + q * T;
            const int i = it % N, k1 = it / N;
            float2 y[R2];
#pragma unroll
            for (int n2 = 0; n2 < R2; ++n2) y[n2] = X[(R2 * k1 + n2) * LD + i];
            dft_reg<R2>(y);
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) {
                const int j = k1 + R1 * k2;
                const float sg = ((i + j) & 1) ? -1.f : 1.f;
                __stcs(out + pp.off0 + (int64_t)j * N + i, sg * y[k2].x);
                if (pp.off1 >= 0) __stcs(out + pp.off1 + (int64_t)j * N + i, sg * y[k2].y);
            }
        }
        __syncthreads();
    }
}

template <int N>
cudaError_t launch_img_grid_n(const float4 *G, const GridPair *pairs, int npairs, float *out, int nsm,
                              cudaStream_t st) {
    constexpr int smem = grid_smem_bytes<N>();
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_img_grid<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    int per_sm = 1;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_img_grid<N>, GridFft<N>::T, smem);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<int64_t>(npairs, (int64_t)nsm * std::max(1, per_sm) * 8);
    k_img_grid<N><<<grid, GridFft<N>::T, smem, st>>>(G, pairs, npairs, out);
    return cudaGetLastError();
}

}  // namespace

bool img_grid_supported(int N) { return N == 16 || N == 32 || N == 64 || N == 128; }

cudaError_t launch_grid_cells(const double2 *bin_uv, const int2 *bin_samp, const int32_t *bin_first,
                              const double2 *chan, const float *W, int nbl, int nout, double dt_raw, int N,
                              double ncell, double *acc, double *glob, cudaStream_t st) {
    const int64_t n = (int64_t)nbl * nout;
    const int threads = 256;
    k_grid_cells<<<(unsigned)((n + threads - 1) / threads), threads, 0, st>>>(bin_uv, bin_samp, bin_first, chan, W,
                                                                             nbl, nout, dt_raw, N, ncell, acc, glob);
    return cudaGetLastError();
}

cudaError_t launch_grid_dft(const float *P, double2 *Y, double2 *S, int N, cudaStream_t st) {
    const int threads = std::min(N, 256);
    const size_t smem = (size_t)N * sizeof(double2);
    k_grid_dft_rows<<<N, threads, smem, st>>>(P, Y, N);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_grid_dft_cols<<<N, threads, smem, st>>>(Y, S, N);
    return cudaGetLastError();
}

cudaError_t launch_grid_table(const double2 *S, const double *acc, const double *glob, int N, double du,
                              float4 *G, cudaStream_t st) {
    const int64_t n = (int64_t)N * N;
    k_grid_table<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(S, acc, glob, N, du, G);
    return cudaGetLastError();
}

cudaError_t launch_img_grid(const float4 *G, const GridPair *pairs, int npairs, int N, float *out, int nsm,
                            cudaStream_t st) {
    if (npairs <= 0) return cudaSuccess;
    switch (N) {
        case 16: return launch_img_grid_n<16>(G, pairs, npairs, out, nsm, st);
        case 32: return launch_img_grid_n<32>(G, pairs, npairs, out, nsm, st);
        case 64: return launch_img_grid_n<64>(G, pairs, npairs, out, nsm, st);
        case 128: return launch_img_grid_n<128>(G, pairs, npairs, out, nsm, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace psf
