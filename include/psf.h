/*
 * psf.h - C ABI of the GB300 (sm_103a) smeared-PSF library.
 *
 * The library evaluates the averaging-distorted ("smeared") point spread function
 * of a radio interferometer at many sky positions (l0, m0), and the two fast
 * approximations to it, as defined in Atemkeng, Smirnov, Tasse, Foster &
 * Makhathini (2020), arXiv:2009.07010:
 *
 *   P_d(l0, l0 + dl) = sum_k W_k Re( D_k(l0) exp(2 pi i u_k . dl) )     (Eqs. 21-22)
 *
 * where k runs over averaged visibilities (baseline p<q, time bin, output
 * channel), u_k is the bin-centre baseline in wavelengths (Sect. 2.1, Eq. 12),
 * W_k the visibility weight (Eq. 6) and D_k the decorrelation of the bin:
 *   exact      D_k = mean over the bin of the source fringe, with the
 *                    centre-visibility phase removed (Eq. 13, boxcar Eq. 14)
 *   approx_uv  D_k = sinc(dPsi/2) sinc(dPhi/2) from the baseline's uvw change
 *                    across the bin and the channel width (Method 1, Eqs. 31-35)
 *   approx_img D_k = the same sinc product from the circular-track model of
 *                    Eqs. 38-44 / Algorithm 1 (Method 2), taken at the
 *                    visibility's own uv point.
 * Each cutout is the separable complex contraction A diag(w) B^T of per-visibility
 * row twiddles exp(2 pi i u_k dl_i) and column twiddles exp(2 pi i v_k dm_j).
 *
 * Conventions: a source at l0 has visibility exp(-2 pi i u.l0) and imaging uses
 * exp(+2 pi i u.l) (Eq. 1).  sinc(x) = sin(x)/x of the half phase change.  The sum
 * runs over the supplied baselines only (p<q, no Hermitian conjugates), so at zero
 * smearing the cutout peak equals sum_k W_k.  Cutout pixel (i, j) of an N x N
 * cutout (N even) sits at (l0 + (i - N/2) cell, m0 + (j - N/2) cell) and is stored
 * at out[offset + j*N + i] (row j = m offset, column i = l offset).
 *
 * Threading / streams: every compute call is asynchronous on the CUDA stream
 * passed as `cuda_stream` (a cudaStream_t, NULL = legacy default stream).  Host
 * inputs are consumed before the call returns.  A plan holds per-call scratch and
 * must be used from one stream at a time.  Device pointers are plain device
 * addresses on the current device.  No call throws; all return a status code.
 */
#ifndef PSF_GB300_PSF_H
#define PSF_GB300_PSF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define PSF_OK            0
#define PSF_EINVAL       -1   /* bad argument: NULL, size, layout, odd N ... */
#define PSF_ENOMEM       -2   /* host or device allocation failed            */
#define PSF_ECUDA        -3   /* a CUDA runtime call failed (no device, ...) */
#define PSF_EUNSUPPORTED -4   /* valid request outside what a path supports  */
#define PSF_ETIMEOUT     -5   /* a bounded device-side wait gave up          */

/* ---- precision of the contraction -------------------------------------- */
#define PSF_FP32     0   /* FP32 CUDA-core form: weights, twiddles, sums in FP32   */
#define PSF_TC_FP16  1   /* tcgen05 tensor cores, FP16 operands, FP32 accumulate  */
#define PSF_TC_BF16  3   /* tcgen05 tensor cores, BF16 operands, FP32 accumulate  */
/* Split precision on the tensor cores: every operand value x is held as hi = rnd16(x)
 * and lo = rnd16(x - hi) and each product is A_hi B_hi + A_hi B_lo + A_lo B_hi (three
 * MMA passes into one FP32 accumulator), which removes the 16-bit rounding of both
 * operands to second order (BF16: 2^-8 -> ~2^-16 per value; FP16: 2^-11 -> ~2^-22, the
 * low parts of small values being FP16 subnormals).  Weights are evaluated with the
 * accurate FP32 sine/cosine.  Per-cutout form only (the batched form is not used),
 * tiles of at most 128 columns; not with PSF_COMPLEX_OUT (PSF_EUNSUPPORTED).  Executed
 * tensor flops are three times the algorithmic ones. */
#define PSF_TC_FP16X3 2
#define PSF_TC_BF16X3 4

/* ---- option flags ------------------------------------------------------ */
#define PSF_WTERM             1u  /* use L0 = (l0, m0, n0-1): w enters the smearing */
#define PSF_IMG_LITERAL_THETA 2u  /* Method 2 with theta = arctan(u/v) as printed   */
/* Bitwise reproducible results run to run on the same device and library build: the
 * batched form (whose output adds the visibility splits with atomics, in arrival
 * order) is not used; every cutout takes the per-cutout form, whose split partials
 * are summed in float64 in a fixed order.  The adjoint is deterministic anyway. */
#define PSF_DETERMINISTIC     4u
/* Complex cutouts: each cutout takes 2 N^2 floats, the N^2 real parts (the default
 * output) followed by the N^2 imaginary parts of sum_k W_k D_k exp(2 pi i (u_k dl +
 * v_k dm)) (Eqs. 21-22 before taking the real part; the imaginary part is what the
 * Hermitian conjugate baselines would cancel).  Packed default offsets advance by
 * 2 N^2; caller-given offsets must leave 2 N^2 floats per cutout.  Tensor-core
 * precisions and N <= 128 only (PSF_EUNSUPPORTED otherwise); computed by the
 * per-cutout form.  psf_adjoint and psf_exact_noalloc ignore the flag (real parts). */
#define PSF_COMPLEX_OUT       8u

/* ---- contraction algorithm (psf_opts_t.algo) ---------------------------- */
/* PSF_ALGO_AUTO: positions of one cutout size (a multiple of 32 up to 256) take the
 * batched form when their group is large enough, the rest the per-cutout form.  The
 * batched form runs every such group of a call in one persistent launch per visibility
 * chunk (one CTA per SM pulling items from a work queue).  An autotuner, run on the first
 * batched call of a plan for each weight class (real / complex weights, FP16 / BF16) and
 * for each cutout size first met, times probes over the first 2^19 visibilities (the
 * call then synchronizes its stream): the items per SM of the persistent launch, and per
 * cutout size the group size from which the batched form beats the per-cutout form.  The
 * results are kept by the plan. */
#define PSF_ALGO_AUTO 0   /* per-cutout form for small batches, batched otherwise */
#define PSF_ALGO_CUTOUT 1 /* per-cutout separable form, split over visibilities  */

/* ---- methods (psf_adjoint) ---------------------------------------------- */
#define PSF_METHOD_EXACT 0
#define PSF_METHOD_UV    1
#define PSF_METHOD_IMG   2
#define PSF_METHOD_IMG_GRID 3   /* Method 2 in the gridded form of psf_approx_img_grid; psf_clean only */

typedef struct psf_plan_s *psf_plan_t;

/* Raw observation (Sect. 2.1 and Eq. 12).  All arrays are host memory, owned by
 * the caller, read during psf_plan only.
 *   uvw_m          [nbl][ntime][3] float64, baseline q-p in metres, row-major
 *   time_s         [ntime] raw sample centres, uniformly spaced (dt = spacing)
 *   freq_hz        [nchan] raw channel centres
 *   chan_width_hz  [nchan] raw channel widths
 *   tavg           [nbl] raw samples averaged per time bin of each baseline
 *                  (baseline-dependent averaging); a trailing partial bin is dropped
 *   favg           raw channels per output channel; nchan % favg == 0
 *   weights        [nvis] float32 visibility weights W_k in plan order, or NULL
 *                  for natural weights W_k = tavg[b] * favg
 * Plan order of averaged visibilities: baseline, then time bin, then output
 * channel (innermost): k = (bin_index(b, tau)) * (nchan / favg) + r. */
typedef struct {
    int32_t nbl, ntime, nchan;
    const double *uvw_m;
    const double *time_s;
    const double *freq_hz;
    const double *chan_width_hz;
    const int32_t *tavg;
    int32_t favg;
    const float *weights;
} psf_obs_t;

/* prec: PSF_FP32 / PSF_TC_FP16 / PSF_TC_BF16 / PSF_TC_FP16X3 / PSF_TC_BF16X3.  flags: PSF_WTERM |
 * PSF_IMG_LITERAL_THETA | PSF_DETERMINISTIC | PSF_COMPLEX_OUT.  algo: PSF_ALGO_*. */
typedef struct {
    int32_t prec;
    uint32_t flags;
    int32_t algo;
    int32_t reserved;
} psf_opts_t;

/* A batch of cutout requests (positions l0 of Eq. 4, geometry of Algorithm 1).
 *   npos        number of positions (0 is valid and does nothing)
 *   lm          [npos][2] float64 direction cosines (l0, m0), host, l0^2+m0^2 < 1
 *   npix        [npos] even cutout sizes N (2 <= N <= 4096), host, or NULL
 *   npix0       size used for every position when npix is NULL
 *   cell_rad    pixel size dl = dm (direction-cosine units), > 0
 *   out_offset  [npos] float offsets of each cutout in the output, host, or NULL
 *               for packed prefix sums of N^2; cutouts must not overlap */
typedef struct {
    int32_t npos;
    const double *lm;
    const int32_t *npix;
    int32_t npix0;
    double cell_rad;
    const int64_t *out_offset;
} psf_batch_t;

/* Build a plan: copies the raw uvw (host memory, float64) to the current device, bins
 * the raw samples there (Eq. 12), forms bin centres and bin-edge deltas (Eqs. 31-33) in
 * float64 and keeps them as float32 records, with the per-visibility tables, on the
 * device.  Position independent; done once per observation.  Synchronous; the temporary
 * device copy of the uvw (nbl x ntime x 24 bytes) is freed before the call returns.
 * Returns PSF_EINVAL for inconsistent sizes/NULL arrays/non-uniform time steps,
 * PSF_ENOMEM / PSF_ECUDA on allocation or copy failure.  *out is set on success
 * and must be released with psf_plan_destroy. */
int psf_plan(const psf_obs_t *obs, const psf_opts_t *opts, psf_plan_t *out);

/* Windowed averaging (Sect. 2.3, Eqs. 15-16): the normalised boxcar over a bin's raw
 * samples and an output channel's raw channels replaced by a window X_pqkr.  The exact
 * method averages the fringe with the window's weights; Methods 1 and 2 replace their two
 * sincs (the transforms of the boxcar) by the window's transforms under their linear-phase
 * models: with A = dPsi / 2 pi and B = dPhi / 2 pi the phase changes across the bin and the
 * band,
 *   T(A) = sum_s x_s exp(-2 pi i A tau_s) sinc_pi(A / n),  tau_s = (s - (n - 1)/2) / n
 *   F(B) = sum_c y_c exp(-2 pi i B (nu_c - nu_r) / Dnu_r) sinc_pi(B dnu_c / Dnu_r)
 * (raw sample s carrying its weight x_s over its own 1/n of the bin, raw channel c its
 * weight y_c over its width), D = T F, complex for asymmetric windows; a direction
 * without a window keeps its sinc.  Applies to psf_exact, psf_approx_uv, psf_approx_img,
 * psf_approx_uv_img, psf_clean and psf_adjoint (not to the gridded form of
 * psf_approx_img_grid, whose cells mix baselines).  Host float32 arrays, read during the
 * call, either may be NULL (boxcar in that direction; both NULL restores the boxcar):
 *   time_window  per baseline b the tavg[b] weights of a bin's raw samples, in bin order,
 *                concatenated over the baselines (sum of tavg entries)
 *   chan_window  [nbl][favg]: per baseline the weights of an output channel's favg raw
 *                channels
 * Each baseline's windows are normalised by the library: the time weights to sum 1, and
 * per output channel the products weight x raw-channel width to sum 1 (so a constant
 * window is the boxcar).  The windows cover each bin's own samples (bins stay disjoint).
 * PSF_EINVAL for a negative or non-finite weight or a window that sums to 0;
 * PSF_ENOMEM / PSF_ECUDA on allocation or copy failure. */
int psf_plan_set_windows(psf_plan_t plan, const float *time_window, const float *chan_window);

/* Replace the visibility weights W_k (Eq. 6) used by later calls on this plan:
 * weights_dev is a device float32 [nvis] array in plan order, copied on cuda_stream
 * (stream-ordered: the array may be released once the stream has passed the call), or
 * NULL for the natural weights W_k = tavg[b] * favg.  Errors: PSF_EINVAL (NULL plan),
 * PSF_ECUDA (copy failure). */
int psf_plan_set_weights(psf_plan_t plan, const float *weights_dev, void *cuda_stream);

/* Replace the precision / flags / algorithm used by later calls on this plan. */
int psf_plan_set_opts(psf_plan_t plan, const psf_opts_t *opts);

/* Number of averaged visibilities K of the plan (-1 for a NULL plan). */
int64_t psf_plan_nvis(psf_plan_t plan);

/* Exact smeared PSF cutouts (Eqs. 13, 21-22).  out_dev: device float32 buffer
 * of at least max(offset_p + N_p^2) floats (2 N_p^2 with PSF_COMPLEX_OUT), fully
 * overwritten on the cutouts' pixels.  PSF_EUNSUPPORTED if a tensor-core precision
 * is requested for N > 256 (N > 128 with PSF_COMPLEX_OUT). */
int psf_exact(psf_plan_t plan, const psf_batch_t *batch, float *out_dev, void *cuda_stream);

/* Method 1, uv-plane approximation (Eqs. 31-35); same arguments as psf_exact. */
int psf_approx_uv(psf_plan_t plan, const psf_batch_t *batch, float *out_dev, void *cuda_stream);

/* Method 2, image-plane approximation (Eqs. 38-44, Algorithm 1 at each
 * visibility's uv point); same arguments as psf_exact. */
int psf_approx_img(psf_plan_t plan, const psf_batch_t *batch, float *out_dev, void *cuda_stream);

/* Methods 1 and 2 of the same batch in one call (the comparison of both
 * approximations of Sect. 4): out_uv_dev receives what psf_approx_uv writes and
 * out_img_dev what psf_approx_img writes (same layout, out_offset and gaps rules,
 * distinct device float32 buffers).  With a tensor-core precision and cutouts of 64
 * or 128 pixels that the per-cutout form handles, both outputs come from one pass
 * that shares the twiddles of the two methods; otherwise the two calls are made in
 * turn.  Errors as psf_exact; out_uv_dev or out_img_dev NULL -> PSF_EINVAL. */
int psf_approx_uv_img(psf_plan_t plan, const psf_batch_t *batch, float *out_uv_dev, float *out_img_dev,
                      void *cuda_stream);

/* Method 2 in the gridded form of Eq. 45, F^-1{F{P} D} with D of Algorithm 1 evaluated
 * on uv cells; same arguments and output layout as psf_approx_img.  The grid of an
 * N x N cutout of pixel size cell is its N x N Fourier grid: cells du = dv = 1/(N cell),
 * cell (a, b) at ((a - N/2) du, (b - N/2) dv).  Position independent and built on the
 * first call for each (N, cell_rad, precision), then kept by the plan (that first call
 * synchronizes the stream): the effective PSF P (the cutout at the phase centre,
 * evaluated like psf_approx_img in the plan's precision), S = F{P}, and per cell the
 * W-weighted means of dt_k and Dnu_r / nu_r of the visibilities whose nearest cell,
 * modulo N, is the cell or its mirror (the means over all visibilities where none is).
 * Per position: D on every cell (the literal theta with PSF_IMG_LITERAL_THETA), one
 * inverse N x N FFT, FP32.  It differs from psf_approx_img by the gridding: D is taken at
 * cell centres and visibilities beyond the grid (|u| > 1/(2 cell)) alias.
 * N must be 16, 32, 64 or 128 (PSF_EUNSUPPORTED otherwise, and with PSF_COMPLEX_OUT);
 * PSF_WTERM has no effect (Method 2 ignores w).  Other errors as psf_exact. */
int psf_approx_img_grid(psf_plan_t plan, const psf_batch_t *batch, float *out_dev, void *cuda_stream);

/* Diagnostic: the position-independent table psf_approx_img_grid uses for (npix,
 * cell_rad) in the plan's precision (built if needed), copied to table_dev (device
 * float32 [npix][npix][4]).  Entry [b][a] belongs to the cell at ((a - N/2) du,
 * (b - N/2) du), du = 1/(N cell_rad): (Re S, Im S) with S = F{P} / N^2, then
 * omega_E dt_c du and (Dnu/nu)_c |u_c| (dt_c, (Dnu/nu)_c the cell's mean interval and
 * fractional bandwidth).  Errors as psf_approx_img_grid. */
int psf_img_grid_table(psf_plan_t plan, int npix, double cell_rad, float *table_dev, void *cuda_stream);

/* Hogbom CLEAN with position-dependent PSFs (Algorithm 2).  The image has nl columns
 * (l) and nm rows (m), both even; pixel (x, y) is the direction (l_c + (x - nl/2)
 * cell_rad, m_c + (y - nm/2) cell_rad): pixel (nl/2, nm/2) looks at (l_c, m_c), the phase
 * centre for l_c = m_c = 0 or a facet's centre otherwise.  Each iteration
 * takes the peak pixel l0 = argmax I_D (signed maximum; the first in row-major order
 * among equal values), evaluates the psf_npix x psf_npix cutout of `method`
 * (PSF_METHOD_EXACT, _UV, _IMG or _IMG_GRID, in the plan's precision and flags) at l0,
 * normalises it to 1 at its centre pixel, subtracts gain * I_D(l0) times it from I_D on
 * the window around l0 (clipped to the image) and adds gain * I_D(l0) to the model at
 * l0.  As the algorithm's do-while: the first iteration always runs (max_iter >= 1),
 * each later one only while the peak exceeds threshold, at most max_iter in all. */
typedef struct {
    int32_t nl, nm;        /* image size in pixels (columns, rows), even */
    double cell_rad;       /* pixel size (direction-cosine units), > 0 */
    double l_c, m_c;       /* direction of pixel (nl/2, nm/2) */
    int32_t psf_npix;      /* PSF cutout size N: even, 2..4096 (16, 32, 64, 128 for IMG_GRID) */
    int32_t method;        /* PSF_METHOD_* */
    float gain;            /* CLEAN gain gamma, 0 < gain <= 1 */
    float threshold;       /* stop once the peak residual is <= threshold */
    int32_t max_iter;      /* >= 0 */
    int32_t options;       /* PSF_CLEAN_* bits */
} psf_clean_t;

/* One PSF for the whole image: the cutout at the image centre (l_c, m_c), computed once
 * and used for every component -- the faceting approach the paper's cost comparison
 * considers (Sect. 3.3, Eqs. 57-58: the PSF at each facet's centre), instead of the PSF
 * at each peak. */
#define PSF_CLEAN_FACET_PSF 1u

/* Runs the loop of psf_clean_t on the device and returns when it has stopped (the
 * stream is synchronized).  residual_dev: device float32 [nm][nl], in: the dirty image,
 * out: the residual.  model_dev: device float32 [nm][nl] or NULL; components are added
 * to it (it is not cleared).  comp_pix_dev / comp_flux_dev: device int32 / float32
 * [max_iter] or NULL: per iteration the peak pixel index y * nl + x and the subtracted
 * flux gain * I_D(l0).  *niter_out (host, may be NULL): iterations performed.  With
 * PSF_METHOD_IMG_GRID every step stays on the device and the host reads the loop
 * record once per 64 queued iterations (after the first 64, replayed as one CUDA graph
 * on a private stream); the other methods read the peak record back
 * each iteration to place the cutout (with PSF_CLEAN_FACET_PSF every method stays on
 * the device after the one PSF evaluation).  Errors: PSF_EINVAL (sizes, gain, method, NULL
 * residual), PSF_EUNSUPPORTED (a cutout size the method does not support,
 * PSF_COMPLEX_OUT), and those of the PSF calls. */
int psf_clean(psf_plan_t plan, const psf_clean_t *cfg, float *residual_dev, float *model_dev,
              int32_t *comp_pix_dev, float *comp_flux_dev, int32_t *niter_out, void *cuda_stream);
/* (every pixel's direction must satisfy l^2 + m^2 < 1 where the loop places a cutout:
 * PSF_EINVAL from the PSF call otherwise) */

/* Size of PSF cutouts as in Fig. 3: the full width at half maximum along the radial
 * direction (l0, m0)/|l0| of each position and the tangential one perpendicular to it
 * (the l and m axes at l0 = 0).  cutouts_dev: device float32 cutouts laid out as the
 * batch describes (as written by psf_exact etc.); fwhm_dev: device float64 [npos][2]
 * (radial, tangential) in direction-cosine units, overwritten.  Half maximum is half
 * the centre pixel (the PSF at l0); on each side of the centre the profile is sampled by
 * bilinear interpolation every quarter pixel up to the first sample at or below it, and
 * the crossing is interpolated linearly from the previous sample; the width is the sum
 * of both sides.  NaN where a profile leaves the cutout first.  Cutouts need N >= 4;
 * errors as psf_exact's batch checks. */
int psf_fwhm(psf_plan_t plan, const psf_batch_t *batch, const float *cutouts_dev, double *fwhm_dev,
             void *cuda_stream);

/* Vector-Jacobian product of the cutout map of `method` (PSF_METHOD_*), i.e. the
 * adjoint: given dL/dP (device float32, same layout as the forward output) it
 * writes dL/d(l0,m0) to dL_dlm_dev (device float64 [npos][2], overwritten) and,
 * if dL_dW_dev is not NULL, dL/dW_k summed over positions (device float32 [nvis],
 * overwritten).  The position enters only through D_k (the twiddles depend on the
 * pixel offsets only):
 *   H_pk = sum_ij dL/dP_p[j][i] exp(2 pi i (u_k dl_i + v_k dm_j)),
 *   dL/dW_k = sum_p Re(D_k(l0_p) H_pk),  dL/dl0_p = sum_k W_k Re(dD_k/dl0 H_pk).
 * Precision: plans in PSF_TC_FP16 / PSF_TC_BF16 whose cutouts are all multiples of 32
 * pixels (up to 1024) form H on the tensor cores (dL/dP and the twiddles rounded to the
 * plan's 16-bit type, FP32 accumulation; about 3e-4 (FP16) / 3e-3 (BF16) of the largest
 * gradient component) and D with its gradient in FP32 with the MUFU sine/cosine; every
 * other plan (PSF_FP32, the split modes, other sizes, N <= 512) runs the FP32 CUDA-core
 * adjoint (about 1e-6). */
int psf_adjoint(psf_plan_t plan, int method, const psf_batch_t *batch, const float *dL_dP_dev,
                double *dL_dlm_dev, float *dL_dW_dev, void *cuda_stream);

/* Wait for the stream and report device-side failures of earlier calls on this
 * plan: PSF_ETIMEOUT if a bounded wait inside a kernel gave up (the output of
 * that call is then invalid), PSF_ECUDA if the stream reported an error. */
int psf_sync_status(psf_plan_t plan, void *cuda_stream);

/* Diagnostic timing.  With enable != 0, later compute calls on this plan record
 * CUDA events on the caller's stream around every contraction-kernel launch (the
 * dominant kernel of each call) and count the library's kernel launches.
 * psf_profile_read waits for the recorded events and returns, since the previous
 * read: the summed contraction time in milliseconds, the number of contraction
 * launches and the number of kernel launches of any kind; then it resets.  Any
 * output pointer may be NULL. */
int psf_profile_enable(psf_plan_t plan, int enable);
int psf_profile_read(psf_plan_t plan, double *contraction_ms, int64_t *contraction_launches,
                     int64_t *kernel_launches);

/* Exact smeared PSF of ONE cutout without allocating device memory during the call.
 * No counterpart in the paper: it exists for callers that cannot allocate while they
 * compute -- real-time or embedded pipelines that forbid allocation once they have
 * started, and plug-ins whose host application's allocator owns the device memory.
 * It reads the plan's arrays (allocated earlier by psf_plan) and writes npix*npix
 * floats to out_dev (device, row j = m offset, column i = l offset, as psf_exact); the
 * computation is the FP32 path with the weights evaluated inline.
 * Scratch: a fixed 16 MiB array inside the library's device image (every GPU that
 * loads the library holds it until the process exits); it keeps the last call's
 * contents, nothing in it needs to start at zero, and calls that overlap on the GPU
 * (e.g. on two streams) race on it.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress); make that first call before any
 * stream capture.  The current device must be the plan's (PSF_EINVAL otherwise).
 * Limits: npix even, 2 <= npix <= 256 (PSF_EUNSUPPORTED beyond); l0^2 + m0^2 < 1,
 * cell_rad > 0 (PSF_EINVAL otherwise).  Calls no allocating routine. */
int psf_exact_noalloc(psf_plan_t plan, double l0, double m0, int npix, double cell_rad, float *out_dev,
                      void *cuda_stream);

/* Release the plan and its device memory (NULL is ignored). */
void psf_plan_destroy(psf_plan_t plan);

/* Static text for a status code. */
const char *psf_strerror(int status);

/* Diagnostic: one 128 x n x 64 tcgen05 GEMM through the library's shared-memory
 * operand layout and descriptors, D[m][j] = sum_k A[m][k] B[j][k] with FP16
 * operands (a_dev [128][64], b_dev [n][64], row-major, device) and FP32 result
 * d_dev [128][n] (device).  n in {16, 32, ..., 256}.  Synchronous. */
int psf_selftest_umma(const void *a_dev, const void *b_dev, float *d_dev, int n);

/* Diagnostic of the bounded device-side waits every tensor-core kernel uses: one CTA
 * waits on a barrier that nothing completes, with a wall-clock limit of limit_ms
 * milliseconds (1..10000); the wait gives up, the kernel raises its error flag and
 * returns.  Returns PSF_ETIMEOUT when the wait ran out (the expected outcome), PSF_OK
 * if it completed, PSF_EINVAL for a bad limit, PSF_ECUDA on a CUDA error.  The
 * device context stays usable.  Synchronous. */
int psf_selftest_timeout(int limit_ms);

/* Diagnostic: the FP32 FMA throughput of the current device, the denominator of the
 * FP32 path's roofline.  A grid of 8 CTAs of 256 threads per SM runs 16 independent
 * FMA chains per thread, as scalar FMAs (packed = 0) or as packed FP32 pairs
 * (packed = 1, fma.rn.f32x2); *flops_per_s receives the best of three timed launches
 * after one warm-up (2 flops per FMA).  Allocates a small device buffer and a stream
 * of its own.  PSF_EINVAL for a NULL pointer or packed not 0/1, PSF_ENOMEM,
 * PSF_ECUDA.  Synchronous. */
int psf_selftest_fma_rate(int packed, double *flops_per_s);

#ifdef __cplusplus
}
#endif
#endif
