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
//   the table G[b][a] = (Re S, Im S, alpha, beta), alpha = omega_E dt_c du and
//      beta = (dnu/nu)_c |u_c|, so that Algorithm 1's half phase changes are
//      A = alpha (a' m0 - b' l0) (theta = atan2(v, u); (b' m0 - a' l0) for the literal
//      arctan(u/v)) and B = beta rho (k_grid_table).
// Per position (k_img_grid): D = sinc(A) sinc(B) on the cells and the real part of
// F^-1{S D}.  With S Hermitian, that real part is F^-1{S D'} where D' averages D over
// each cell and its mirror modulo N; D' differs from D only on the Nyquist row and
// column (a' or b' = -N/2, their own mirrors).  S D' is Hermitian, so the transform runs
// on half the cells: column transforms over b, then per row a real-output transform
// built from one complex transform of half the length, all in shared memory with the
// small DFTs in registers.
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

// G[b N + a] = (Re S / N^2, Im S / N^2, omega_E dt_c du, (dnu/nu)_c |u_c|) for cell (a, b).
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
    G[q] = make_float4((float)(S[q].x * inv), (float)(S[q].y * inv), (float)(kOmegaE * dt * du),
                                        (float)(r * sqrt(ua * ua + vb * vb)));
}

// ------------------------------------------------------------------ per-position transform

// sinc_pi(x) = sin(pi x) / (pi x) = (-1)^n [sin(pi f) / (pi f)] (f / x), x = n + f, |f| <= 1/2.
// n comes from adding 1.5 * 2^23 (|x| < 2^22), which rounds x to the nearest integer and
// leaves the parity of n in the lowest mantissa bit; the bracket is its Taylor series in
// (pi f)^2 to order 10 (truncation error < 4e-8).
__device__ __forceinline__ float sinc_fast(float x) {
    const float t = x + 12582912.0f;
    const float n = t - 12582912.0f;
    const float f = x - n;
    const float z = f * f;
    float q = fmaf(z, -2.3460810e-3f, 2.6147848e-2f);
    q = fmaf(z, q, -1.9075182e-1f);
    q = fmaf(z, q, 8.1174243e-1f);
    q = fmaf(z, q, -1.6449341f);
    q = fmaf(z, q, 1.0f);
    if (n != 0.0f) q *= __fdividef(f, x);
    return __int_as_float(__float_as_int(q) ^ (__float_as_int(t) << 31));
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

// In-register inverse DFT y[k] = sum_n x[n] exp(+2 pi i n k / R), R in {2, 4, 8, 16}:
// radix-2 decimation in time, natural order in and out.
template <int R>
__device__ __forceinline__ void dft_reg(float2 (&x)[R]) {
    static_assert(R == 2 || R == 4 || R == 8 || R == 16, "radix");
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

// Shapes: the column transforms (length N over b) run as R1 x R2 Cooley-Tukey, the row
// transforms (length M = N/2, the complex core of each real row) as Q1 x Q2; T threads;
// the second stages of both passes take their lines in P parts to bound registers.
template <int N>
struct GridFft;
template <>
struct GridFft<16> { static constexpr int R1 = 4, R2 = 4, Q1 = 4, Q2 = 2, T = 64, P = 1; };
template <>
struct GridFft<32> { static constexpr int R1 = 8, R2 = 4, Q1 = 4, Q2 = 4, T = 128, P = 1; };
template <>
struct GridFft<64> { static constexpr int R1 = 8, R2 = 8, Q1 = 8, Q2 = 4, T = 128, P = 1; };
template <>
struct GridFft<128> { static constexpr int R1 = 16, R2 = 8, Q1 = 8, Q2 = 8, T = 256, P = 2; };

template <int N>
constexpr int grid_smem_bytes() { return (N * (N / 2 + 1) + N) * (int)sizeof(float2); }

template <int N>
constexpr int grid_min_blocks() { return N == 128 ? 3 : N == 64 ? 6 : 8; }

// One CTA per position (grid-stride).  X = (-1)^(a+b) S D' is Hermitian, so only the
// cells a in [0, N/2] are formed, in shared memory Z [N rows][N/2 + 1] (row b, later
// output row j; the odd row stride keeps every lane pattern below free of bank
// conflicts), with the N twiddles exp(+2 pi i m / N).
//   (0) X on the half grid, flat over its cells
//   (1) columns: length-N inverse DFT over b for a in [0, N/2); column 0 carries
//       X[.][0] + i X[.][N/2], whose transforms are both real, and is unpacked into them
//   (2) rows: each row j is Hermitian in a, and its real inverse DFT x is obtained from
//       one length-N/2 complex DFT of C[k] = E[k] + i O[k], E[k] = Z[k] + conj Z[N/2 - k],
//       O[k] = (Z[k] - conj Z[N/2 - k]) exp(2 pi i k / N): it returns x[2n] + i x[2n+1]
//   (3) out[j][i] = (-1)^(i + j) x[i], two floats per store.
// Cell and pixel index origins are at N/2: exp(2 pi i (a - N/2)(i - N/2) / N) =
// (-1)^(a + i) exp(2 pi i a i / N) for N % 4 == 0.
template <int N>
__global__ void __launch_bounds__(GridFft<N>::T, grid_min_blocks<N>())
    k_img_grid(const float4 *__restrict__ G, const GridPos *__restrict__ pos, int npos, float *__restrict__ out) {
    using F = GridFft<N>;
    constexpr int M = N / 2, LD = M + 1, T = F::T, R1 = F::R1, R2 = F::R2, Q1 = F::Q1, Q2 = F::Q2, P = F::P;
    static_assert(R1 * R2 == N && Q1 * Q2 == M && M % P == 0 && N % P == 0, "shape");
    extern __shared__ float2 smem[];
    float2 *Z = smem;
    float2 *tw = smem + N * LD;
    for (int m = threadIdx.x; m < N; m += T) {
        float s, c;
        sincospif(2.0f * (float)m / (float)N, &s, &c);
        tw[m] = make_float2(c, s);
    }
    __syncthreads();
    for (int p = blockIdx.x; p < npos; p += gridDim.x) {
        const GridPos gp = pos[p];
        // (0) X = (-1)^(a+b) S D' on the cells a in [0, M]; D' = D except on the Nyquist
        // row and column, where it is averaged with the mirror cell modulo N.  Columns
        // a < M: a fixed per thread, rows b0, b0 + RS, ... (RS even: the sign is fixed too);
        // column M: one row per thread.
        {
            constexpr int RS = T / M;
            static_assert(T % M == 0 && RS % 2 == 0 && T >= N, "pre-pass shape");
            const int a = threadIdx.x % M, b0 = threadIdx.x / M;
            const float af = (float)(a - M), lin0 = af * gp.c.x, cb = gp.c.y, rho = gp.c.z;
            const float sg = ((a + b0) & 1) ? -1.f : 1.f;
#pragma unroll 4
            for (int b = b0; b < N; b += RS) {
                const float4 g = __ldg(G + b * N + a);
                const float bf = (float)(b - M);
                float e = sinc_fast(g.z * fmaf(bf, cb, lin0));
                if (a == 0 || b == 0) {
                    const float ma = a == 0 ? af : -af, mb = b == 0 ? bf : -bf;
                    e = 0.5f * (e + sinc_fast(g.z * fmaf(ma, gp.c.x, mb * cb)));
                }
                const float d = sg * e * sinc_fast(g.w * rho);
                Z[b * LD + a] = make_float2(g.x * d, g.y * d);
            }
            for (int b = threadIdx.x; b < N; b += T) {
                const float4 g = __ldg(G + b * N + M);
                const float bf = (float)(b - M);
                // a' = 0: the mirror (0, -b') has the same D (D is even), so D' = D here
                float d = sinc_fast(g.z * (bf * cb)) * sinc_fast(g.w * rho);
                if ((M + b) & 1) d = -d;
                Z[b * LD + M] = make_float2(g.x * d, g.y * d);
            }
        }
        __syncthreads();
        // (1a) columns a in [0, M): R1-point DFT over b = n2 + R2 n1, twiddle
        // exp(2 pi i n2 k1 / N), stored in place at rows n2 + R2 k1
#pragma unroll 1
        for (int it = threadIdx.x; it < M * R2; it += T) {
            const int a = it % M, n2 = it / M;
            float2 x[R1];
#pragma unroll
            for (int n1 = 0; n1 < R1; ++n1) {
                const int r = (n2 + R2 * n1) * LD;
                float2 v = Z[r + a];
                if (a == 0) {
                    const float2 w = Z[r + M];
                    v = make_float2(v.x - w.y, v.y + w.x);
                }
                x[n1] = v;
            }
            dft_reg<R1>(x);
#pragma unroll
            for (int k1 = 0; k1 < R1; ++k1) Z[(n2 + R2 * k1) * LD + a] = cmul(x[k1], tw[n2 * k1]);
        }
        __syncthreads();
        // (1b) R2-point DFT over n2 for each (a, k1); output rows j = k1 + R1 k2.  A part's
        // reads all precede its writes; parts touch disjoint columns (column M belongs to
        // the part holding column 0).
#pragma unroll 1
        for (int part = 0; part < P; ++part) {
            constexpr int LA = M / P, NI = LA * R1, K = (NI + T - 1) / T;
            float2 y[K][R2];
#pragma unroll
            for (int q = 0; q < K; ++q) {
                const int it = threadIdx.x + q * T;
                if (it < NI) {
                    const int a = part * LA + it % LA, k1 = it / LA;
#pragma unroll
                    for (int n2 = 0; n2 < R2; ++n2) y[q][n2] = Z[(R2 * k1 + n2) * LD + a];
                }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < K; ++q) {
                const int it = threadIdx.x + q * T;
                if (it < NI) {
                    const int a = part * LA + it % LA, k1 = it / LA;
                    dft_reg<R2>(y[q]);
#pragma unroll
                    for (int k2 = 0; k2 < R2; ++k2) {
                        const int r = (k1 + R1 * k2) * LD;
                        if (a == 0) {
                            Z[r] = make_float2(y[q][k2].x, 0.f);
                            Z[r + M] = make_float2(y[q][k2].y, 0.f);
                        } else {
                            Z[r + a] = y[q][k2];
                        }
                    }
                }
            }
        }
        __syncthreads();
        // (2a) rows j: C[k] for k = n2 + Q2 n1, Q1-point DFT over n1, twiddle
        // exp(2 pi i n2 k1 / M) = tw[2 n2 k1], stored at k = n2 + Q2 k1 (parts = row ranges)
#pragma unroll 1
        for (int part = 0; part < P; ++part) {
            constexpr int LJ = N / P, NI = LJ * Q2, K = (NI + T - 1) / T;
            float2 c[K][Q1];
#pragma unroll
            for (int q = 0; q < K; ++q) {
                const int it = threadIdx.x + q * T;
                if (it < NI) {
                    const int j = part * LJ + it % LJ, n2 = it / LJ;
#pragma unroll
                    for (int n1 = 0; n1 < Q1; ++n1) {
                        const int k = n2 + Q2 * n1;
                        const float2 zk = Z[j * LD + k], zm = Z[j * LD + M - k];
                        const float2 e = make_float2(zk.x + zm.x, zk.y - zm.y);
                        const float2 o = cmul(make_float2(zk.x - zm.x, zk.y + zm.y), tw[k]);
                        c[q][n1] = make_float2(e.x - o.y, e.y + o.x);
                    }
                }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < K; ++q) {
                const int it = threadIdx.x + q * T;
                if (it < NI) {
                    const int j = part * LJ + it % LJ, n2 = it / LJ;
                    dft_reg<Q1>(c[q]);
#pragma unroll
                    for (int k1 = 0; k1 < Q1; ++k1) Z[j * LD + n2 + Q2 * k1] = cmul(c[q][k1], tw[2 * n2 * k1]);
                }
            }
        }
        __syncthreads();
        // (2b) Q2-point DFT over n2 for each (j, k1): y[k1 + Q1 k2] = x[2n] + i x[2n+1],
        // n = k1 + Q1 k2, stored at slot n of row j
#pragma unroll 1
        for (int part = 0; part < P; ++part) {
            constexpr int LJ = N / P, NI = LJ * Q1, K = (NI + T - 1) / T;
            float2 y[K][Q2];
#pragma unroll
            for (int q = 0; q < K; ++q) {
                const int it = threadIdx.x + q * T;
                if (it < NI) {
                    const int j = part * LJ + it % LJ, k1 = it / LJ;
#pragma unroll
                    for (int n2 = 0; n2 < Q2; ++n2) y[q][n2] = Z[j * LD + Q2 * k1 + n2];
                }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < K; ++q) {
                const int it = threadIdx.x + q * T;
                if (it < NI) {
                    const int j = part * LJ + it % LJ, k1 = it / LJ;
                    dft_reg<Q2>(y[q]);
#pragma unroll
                    for (int k2 = 0; k2 < Q2; ++k2) Z[j * LD + k1 + Q1 * k2] = y[q][k2];
                }
            }
        }
        __syncthreads();
        // (3) out[j][2n], out[j][2n + 1] = (-1)^j (Re y[n], -Im y[n]), streamed
        float *o = out + gp.off;
        if ((gp.off & 1) == 0) {
            for (int it = threadIdx.x; it < N * M; it += T) {
                const int j = it / M, n = it % M;
                const float2 y = Z[j * LD + n];
                const float sg = (j & 1) ? -1.f : 1.f;
                __stcs(reinterpret_cast<float2 *>(o + j * N + 2 * n), make_float2(sg * y.x, -sg * y.y));
            }
        } else {
            for (int it = threadIdx.x; it < N * M; it += T) {
                const int j = it / M, n = it % M;
                const float2 y = Z[j * LD + n];
                const float sg = (j & 1) ? -1.f : 1.f;
                __stcs(o + j * N + 2 * n, sg * y.x);
                __stcs(o + j * N + 2 * n + 1, -sg * y.y);
            }
        }
        __syncthreads();
    }
}

template <int N>
cudaError_t launch_img_grid_n(const float4 *G, const GridPos *pos, int npos, float *out, int nsm, cudaStream_t st) {
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
    const int grid = (int)std::min<int64_t>(npos, (int64_t)nsm * std::max(1, per_sm) * 4);
    k_img_grid<N><<<grid, GridFft<N>::T, smem, st>>>(G, pos, npos, out);
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

cudaError_t launch_img_grid(const float4 *G, const GridPos *pos, int npos, int N, float *out, int nsm,
                            cudaStream_t st) {
    if (npos <= 0) return cudaSuccess;
    switch (N) {
        case 16: return launch_img_grid_n<16>(G, pos, npos, out, nsm, st);
        case 32: return launch_img_grid_n<32>(G, pos, npos, out, nsm, st);
        case 64: return launch_img_grid_n<64>(G, pos, npos, out, nsm, st);
        case 128: return launch_img_grid_n<128>(G, pos, npos, out, nsm, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace psf
