// Internal declarations shared by the library's translation units.
// Device-resident plan arrays, per-call batch descriptors and kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "psf.h"

namespace psf {

constexpr double kCLight = 299792458.0;   // m/s
constexpr double kOmegaE = 7.2921150e-5;   // sidereal rate, rad/s (omega_E of Eqs. 38-41)

// Position-independent arrays of a plan, float32, resident in HBM.
// Bins are (baseline, time bin) pairs in plan order; visibility k = bin * nout + r.
struct DevObs {
    int32_t nvis;          // K (averaged visibilities), < 2^31
    int32_t nbin;          // number of (baseline, time bin) pairs
    int32_t nout;          // output channels
    int32_t favg;          // raw channels per output channel
    int32_t uniform;       // 1: raw channels equally spaced with equal widths in every group
    float dt;              // raw sample spacing [s]
    int32_t chan_affine;   // 1: nu_r = nu_0 + r dnu_ch exactly, equal spacing/width in every group
    float dnu_ch;          // output channel spacing when chan_affine
    const float4 *bin_ubar;   // [nbin] bin-mean uvw [m] (x,y,z), Delta t_k [s] (w)
    const float4 *bin_edge;   // [nbin] uvw(t_e) - uvw(t_s) [m] (Eq. 33 edges)
    const int2 *bin_samp;     // [nbin] first raw-sample record, sample count
    const float4 *samp;       // [nsamp] uvw_s - ubar [m] per raw sample of each bin
    const float4 *chan;       // [nout] nu_r, Dnu_r, channel spacing, channel width
    const float4 *rawchan;    // [nout*favg] nu_c - nu_r, dnu_c, dnu_c / Dnu_r, 0
    const float *W;           // [nvis] visibility weights
    const float2 *uv;         // [nvis] bin-centre (u, v) in wavelengths, rounded to float32
    const float2 *uv_lo;      // [nvis] (u, v) - uv: the float64 bin centre is uv + uv_lo
    // windowed average (Eqs. 15-16); win = 0: the boxcar; bit 0: a time window was given,
    // bit 1: a channel window (the exact method reads both tables whenever win != 0, the
    // approximations take the transform of the given window in each direction)
    int32_t win;
    const float *samp_w;      // [nsamp] normalised time weight of each raw-sample record
    const float *chan_win;    // [nbl][nchan] normalised channel weight (window x width)
    const int32_t *bin_bl;    // [nbin] baseline of each bin
};

// One cutout tile of a contraction launch.
struct Tile {
    int32_t slot;     // position index within the current position chunk
    int32_t N;        // cutout size
    int32_t i0, j0;   // first column (l offset index) / row (m offset index)
    int64_t out_off;  // float offset of the cutout in the output
};

// Method selector (matches PSF_METHOD_*).
enum Method { kExact = 0, kUV = 1, kImg = 2 };

// ---- launchers (k_weights.cu) -------------------------------------------
// w[s * ldw + (k - k0)] = W_k * D_k(pos[s]) for s < npos, k0 <= k < k0 + kn.
// fast != 0: MUFU sine/cosine forms (for weights rounded to 16 bits afterwards).
// launch_weights16: complex methods write (Re w, -Im w) pairs, kpitch pairs per row;
// real methods write one value per visibility, kpitch pairs = 2 kpitch visibilities.
cudaError_t launch_weights(const DevObs &o, int method, uint32_t flags, const float4 *pos,
                           int npos, int32_t k0, int32_t kn, float2 *w, int64_t ldw, int fast,
                           cudaStream_t st);
// FP32 CUDA-core contraction; partial[split * split_stride + out_off + j*N + i].
cudaError_t launch_psf_fp32(const DevObs &o, const float2 *w, int64_t ldw, const Tile *tiles,
                            int ntiles, int nsplit, int32_t kper, double cell, float *partial,
                            int64_t split_stride, cudaStream_t st);
// out[out_off_p + q] = sum_s partial[s * stride + loc_off_p + q'] (float64 sum), where
// q' = q for row-major partials and q' = i N + j for q = j N + i when `transposed`.
cudaError_t launch_reduce(const float *partial, int nsplit, int64_t stride, const int64_t *loc_offs,
                          const int64_t *out_offs, const int32_t *npix, int npos, int transposed, float *out,
                          cudaStream_t st);
// Plan-time per-visibility tables: uv[k] + uv_lo[k] (from the float64 bin means and
// channel frequencies) and, if natural, W[k] = tavg * favg.
// Averaging bins of the plan from the raw uvw on the device (k_weights.cu, k_bin).
cudaError_t launch_bin(const double *uvw, int ntime, int nbl, const int32_t *tavg, const int32_t *bin_first,
                       const int64_t *samp_first, int64_t nbin, double dt_raw, float4 *bin_ubar, double2 *bin_uv64,
                       float4 *bin_edge, int2 *bin_samp, float4 *samp, cudaStream_t st);
cudaError_t launch_fill_vis(const DevObs &o, const double2 *bin_uv64, const double2 *chan64, float2 *uv,
                            float2 *uv_lo, float *W, int natural, cudaStream_t st);
// Adjoint (vector-Jacobian product) in FP32, see psf_adjoint (k_adjoint.cu).
// pos: [npos] {L, dL/dl0, dL/dm0} float4 triples; partial: [ctas][npos][2] doubles.
int adjoint_max_n();
int64_t adjoint_ctas(int64_t nvis);
cudaError_t launch_adjoint_chunk(const DevObs &o, int method, uint32_t flags, const void *pos, const int32_t *npix,
                                 const int64_t *offs, int npos, int nmax, double cell, const float *R, float *gW,
                                 int accumulate_gW, double *partial, double *g_lm, cudaStream_t st);

// ---- tensor-core adjoint (k_adj_tc.cu) ------------------------------------
// R of a size group (packed cutouts at offs[row], rows < npos) -> FP16/BF16 [rows][n2].
cudaError_t launch_adj_r16(const float *R, const int64_t *offs, int npos, int rows, int n2, int bf16, void *r16,
                           cudaStream_t st);
// H[row][k - kc0] = sum_q R[row][q] exp(2 pi i (u_k dl_i + v_k dm_j)) for the visibility
// chunk [kc0, kc0 + kcn) (float2 rows of ldh >= 128 ceil(kcn / 128)); rmap: the 2-D tensor
// map of the R rows (make_weight_map with pitch n2 = N^2); N a multiple of 32.
cudaError_t launch_adj_tc(const void *rmap, int ntile_pos, int ntile_vis, int N, const float2 *uv, int32_t kc0,
                          int32_t kcn, float cell, float2 *H, int64_t ldh, int bf16, int nsm, int *err,
                          cudaStream_t st);
int adj_fold_max_pos();
int adj_fold_blocks(int nsm);
// From H of the chunk: gW[k] (+)= sum_p Re(D H) and g_lm[2 idx[p] + d] (+)= sum_k W Re(dD H);
// pos: [npos] {L, dL/dl0, dL/dm0} float4 triples; partial: [adj_fold_blocks(nsm)][npos][2].
cudaError_t launch_adj_fold(const DevObs &o, int method, uint32_t flags, const void *pos, int npos, const float2 *H,
                            int64_t ldh, int32_t kc0, int32_t kcn, float *gW, int accumulate_gW, double *partial,
                            const int32_t *idx, double *g_lm, int accumulate_lm, int fast, int nsm, cudaStream_t st);

// ---- tcgen05 contraction (k_tc.cu) ----------------------------------------
struct TcItem {
    int32_t slot, N;
    int32_t j0, i0;       // first row (M) / first column (N) of the tile
    int32_t ncols;        // tile width (multiple of 32, <= 256)
    int32_t k0, k1;       // visibility range of this split
    int32_t split;
    int64_t out_off;
};
// partial[split * split_stride + out_off + i*N + j] (transposed within each cutout).
// wreal: 0 = complex weights; 1 = the weights of this launch are real (imaginary parts
// zero), which allows the conjugate-symmetric generation of the column twiddles; 2 =
// real weights and every item spans a whole cutout of 64 or 128 pixels (i0 = j0 = 0,
// ncols = N), so every tile is generated conjugate-symmetrically.
// split != 0: split precision (hi + lo operands, three MMA passes; ncols_max <= 128).
cudaError_t launch_psf_tc(const DevObs &o, const float2 *w, int64_t ldw, const TcItem *items,
                          int nitems, int ncols_max, int bf16, float cell, int wreal, float *partial,
                          int64_t split_stride, int *err_flag, cudaStream_t st, int split = 0);
// Fused Methods 1 + 2 on whole cutouts of 64 or 128 pixels (every item: i0 = j0 = 0,
// ncols = N; ncols_max 64 or 128): partial sums of the uv cutouts at `partial` and of
// the image-plane cutouts at partial + part2, both laid out like launch_psf_tc's.
cudaError_t launch_psf_tc_uvimg(const DevObs &o, const float2 *w_uv, const float2 *w_img, int64_t ldw,
                                const TcItem *items, int nitems, int ncols_max, int bf16, float cell, float *partial,
                                int64_t split_stride, int64_t part2, int *err, cudaStream_t st);
// Complex output (every item: one row tile, ncols <= 128): partial sums of the real
// parts at `partial`, of the imaginary parts at partial + part2.
cudaError_t launch_psf_tc_cplx(const DevObs &o, const float2 *w, int64_t ldw, const TcItem *items, int nitems,
                               int ncols_max, int bf16, float cell, float *partial, int64_t split_stride,
                               int64_t part2, int *err, cudaStream_t st);
int selftest_umma(const void *a, const void *b, float *d, int n);
int selftest_timeout(int limit_ms);
int selftest_fma_rate(int packed, double *flops_per_s);   // k_weights.cu

// ---- batched tcgen05 contraction (k_kr.cu) ---------------------------------
struct KrItem {
    int32_t wrow;     // first row of the 128-position tile in the weight buffer
    int32_t npos;     // valid positions of the tile (<= 128)
    int32_t slot0;    // batch index of the tile's first position
    int32_t N;        // cutout size (multiple of 32, <= 256)
    int32_t q0;       // first pixel (row-major) of the 256-pixel tile
    int32_t npx;      // pixels of the tile (256)
    int32_t kb, ke;   // visibility range, kb - chunk start a multiple of the stage size (32 or 64)
};
// real != 0: real weights (Methods 1, 2), one K' column per visibility.
// Persistent: nctas CTAs (one per SM) pull items from the work queue (a device int,
// zeroed by the launch) in array order (largest first).
cudaError_t launch_psf_kr(const void *wmap, const KrItem *items, int nitems, int *queue, int nctas, const float2 *uv,
                          int32_t kchunk0, float cell, const int64_t *out_off, float *out, int bf16, int real, int *err,
                          cudaStream_t st);
int make_weight_map(void *map_out, void *w16, int bf16, int64_t pitch_elems, int64_t rows);
int kr_smem_bytes();
cudaError_t launch_weights16(const DevObs &o, int method, uint32_t flags, const float4 *pos,
                             const int32_t *slot_of_row, int rows, int32_t kc0, int32_t kcn, int64_t kpitch,
                             int bf16, void *w16, cudaStream_t st);
cudaError_t launch_zero_cutouts(float *out, const int64_t *offs, const int32_t *npix, int npos, cudaStream_t st);

// Read-only views of a plan (plan.cu).
const DevObs *plan_devobs(psf_plan_t p);
uint32_t plan_flags(psf_plan_t p);
int plan_device(psf_plan_t p);   // device the plan's arrays live on (-1 for NULL)

// ---- gridded image-plane approximation (k_grid.cu) -------------------------
// One position of the gridded transform: c = (coefficient of a', coefficient of b',
// rho, 0) of Algorithm 1's half phase changes A = alpha (c.x a' + c.y b') and
// B = beta rho; off = float offset of the cutout in the output.
struct GridPos {
    float4 c;
    long long off;
    long long pad;
};

bool img_grid_supported(int N);
cudaError_t launch_grid_cells(const double2 *bin_uv, const int2 *bin_samp, const int32_t *bin_first,
                              const double2 *chan, const float *W, int nbl, int nout, double dt_raw, int N,
                              double ncell, double *acc, double *glob, cudaStream_t st);
cudaError_t launch_grid_dft(const float *P, double2 *Y, double2 *S, int N, cudaStream_t st);
cudaError_t launch_grid_table(const double2 *S, const double *acc, const double *glob, int N, double du,
                              float4 *G, cudaStream_t st);
cudaError_t launch_img_grid(const float4 *G, const GridPos *pos, int npos, int N, float *out, int nsm,
                            cudaStream_t st);

// ---- Hogbom CLEAN (k_clean.cu) ------------------------------------------------
// Device record of the CLEAN loop (one per call).
struct CleanState {
    GridPos gpos;     // position record of the gridded PSF at the current peak (offset 0)
    int32_t done;     // 1 once the loop has stopped
    int32_t iter;     // iterations performed
    int32_t active;   // the current iteration subtracts
    int32_t pix;      // peak pixel y * nl + x
    float peak;       // I_D at the peak
    int32_t pad[3];
};

cudaError_t launch_clean_argmax(const float *res, int64_t n, const CleanState *st, unsigned long long *key, int nsm,
                                cudaStream_t s);
cudaError_t launch_clean_prep(const unsigned long long *key, unsigned long long *key_next, CleanState *st, int nl,
                              int nm, double cell, double lc, double mc, float threshold, int max_iter, int literal,
                              cudaStream_t s);
cudaError_t launch_clean_sub(float *res, float *model, const float *P, CleanState *st, int nl, int nm, int N,
                             float gain, int32_t *comp_pix, float *comp_flux, cudaStream_t s);

// ---- FWHM along radial / tangential directions (k_fwhm.cu) --------------------
struct FwhmItem {
    float er_x, er_y;   // radial unit vector in pixel axes (l, m); the l axis at l0 = 0
    int32_t N;          // cutout size
    int32_t pad;
    long long off;      // float offset of the cutout
};
cudaError_t launch_fwhm(const float *cut, const FwhmItem *items, int npos, double cell, double *out, cudaStream_t s);

}  // namespace psf
