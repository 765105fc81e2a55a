// Host side of the C ABI: plan construction (float64 binning on the host), per-call
// batch preparation, workspace management and dispatch to the kernels.
//
// Plan (Sect. 2.3, Eq. 12): every baseline's raw samples are grouped into bins of
// tavg[b] consecutive samples (a trailing partial bin is dropped) and raw channels
// into groups of favg.  Per bin the host forms, in float64, the mean uvw (bin
// centre), the bin-edge delta uvw(t_e) - uvw(t_s) (Eq. 33; the edges are not
// sampled, so (last - first) n/(n-1) for n >= 2 samples and the central
// difference of the neighbouring samples for n = 1) and each raw sample's offset
// from the mean.  These are rounded to float32 once and kept on the device; the
// per-visibility tables (bin-centre uv in wavelengths, default weights) are then
// filled by a device kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <vector>

#include "psf_internal.cuh"

using namespace psf;

namespace {

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    // Grow-only; contents are not preserved.
    cudaError_t reserve(size_t n) {
        if (n <= bytes) return cudaSuccess;
        release();
        cudaError_t e = cudaMalloc(&p, n);
        if (e != cudaSuccess) { p = nullptr; return e; }
        bytes = n;
        return cudaSuccess;
    }
};

struct HostPinned {
    void *p = nullptr;
    size_t bytes = 0;
    ~HostPinned() { if (p) cudaFreeHost(p); }
    cudaError_t reserve(size_t n) {
        if (n <= bytes) return cudaSuccess;
        if (p) cudaFreeHost(p);
        p = nullptr;
        bytes = 0;
        cudaError_t e = cudaMallocHost(&p, n);
        if (e != cudaSuccess) { p = nullptr; return e; }
        bytes = n;
        return cudaSuccess;
    }
};

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return PSF_OK;
    if (e == cudaErrorMemoryAllocation) return PSF_ENOMEM;
    return PSF_ECUDA;
}

#define PSF_TRY(x)                         \
    do {                                   \
        cudaError_t e_ = (x);              \
        if (e_ != cudaSuccess) {           \
            cudaGetLastError();            \
            return cuda_status(e_);        \
        }                                  \
    } while (0)

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Tensor-core operand type and the split (hi + lo, three MMA passes) precision modes.
bool prec_bf16(int prec) { return prec == PSF_TC_BF16 || prec == PSF_TC_BF16X3; }
bool prec_split(int prec) { return prec == PSF_TC_FP16X3 || prec == PSF_TC_BF16X3; }

// Storage for a CUtensorMap (128 bytes, 64-byte aligned) without including cuda.h here.
struct alignas(64) CUtensorMapStub {
    unsigned char bytes[128];
};

}  // namespace

struct psf_plan_s {
    psf_opts_t opts{};
    int device = 0;
    int nsm = 148;
    int nbl = 0, ntime = 0, nchan = 0, favg = 1, nout = 0;
    int64_t nbin = 0, nsamp = 0, nvis = 0;
    DevObs d{};
    // position-independent device arrays
    DevBuf bin_ubar, bin_edge, bin_samp, samp, chan, rawchan, W, uv, uv_lo;
    // float64 bin-mean (u, v) [m], output channels (nu_r, Dnu_r) and each baseline's
    // first bin: the nearest-cell decisions of the gridded image-plane form
    DevBuf bin_uv64, chan64, bin_first;
    double dt_raw = 0;
    // windowed average (Eqs. 15-16): host copies of the binning, device tables
    std::vector<int32_t> h_tavg;
    std::vector<double> h_width;
    std::vector<int64_t> h_bin_first, h_samp_first;
    int affine0 = 0;
    DevBuf samp_w, chan_win, bin_bl;
    // gridded image-plane tables, one per (cutout size, pixel size, precision)
    struct Grid {
        int N = 0;
        double cell = 0;
        int prec = 0;
        DevBuf G;   // float4 [N][N]
    };
    std::vector<std::unique_ptr<Grid>> grids;
    DevBuf gpairs;   // per-call pair records of the gridded form
    DevBuf err;          // int: device-side wait timeouts
    DevBuf queue;        // int: work queue of the persistent batched kernel
    // autotuner of the batched form, per weight class (bit 0 real weights, bit 1 BF16):
    // items per SM and, per cutout size, the smallest group the batched form takes
    struct KrTune {
        bool done = false;
        int items_per_cta = 4;
        std::map<int, int> min_group;
    };
    KrTune tune[4];
    // per-call workspace
    DevBuf meta;         // positions, sizes, offsets, tiles
    DevBuf wbuf;         // weights of a chunk of positions
    DevBuf partial;      // split-K partial cutouts
    DevBuf w16;          // FP16/BF16 weights of the batched path
    HostPinned hmeta;
    cudaEvent_t meta_done = nullptr;   // staging buffer reusable once this fires
    // diagnostic timing (psf_profile_*)
    bool prof = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_ev;
    size_t prof_used = 0;
    int64_t n_contract = 0, n_kernels = 0;
    ~psf_plan_s() {
        for (auto &e : prof_ev) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
    }
};

namespace {

// Host mirror of the per-call metadata layout.
struct Meta {
    size_t off_pos, off_npix, off_loc, off_out, off_tiles, bytes;
};

int validate_obs(const psf_obs_t *o) {
    if (!o || o->nbl <= 0 || o->ntime <= 0 || o->nchan <= 0 || o->favg <= 0) return PSF_EINVAL;
    if (!o->uvw_m || !o->time_s || !o->freq_hz || !o->chan_width_hz || !o->tavg) return PSF_EINVAL;
    if (o->nchan % o->favg) return PSF_EINVAL;
    for (int b = 0; b < o->nbl; ++b)
        if (o->tavg[b] <= 0) return PSF_EINVAL;
    for (int c = 0; c < o->nchan; ++c)
        if (!(o->freq_hz[c] > 0.0) || !(o->chan_width_hz[c] > 0.0)) return PSF_EINVAL;
    if (o->ntime >= 2) {
        const double dt = (o->time_s[o->ntime - 1] - o->time_s[0]) / (o->ntime - 1);
        if (!(dt > 0.0)) return PSF_EINVAL;
        for (int t = 1; t < o->ntime; ++t)
            if (std::fabs(o->time_s[t] - o->time_s[t - 1] - dt) > 1e-6 * dt) return PSF_EINVAL;
    }
    return PSF_OK;
}

int validate_opts(const psf_opts_t *op) {
    if (!op) return PSF_OK;
    if (op->prec != PSF_FP32 && op->prec != PSF_TC_FP16 && op->prec != PSF_TC_BF16 && op->prec != PSF_TC_FP16X3 &&
        op->prec != PSF_TC_BF16X3)
        return PSF_EINVAL;
    if (op->flags & ~(PSF_WTERM | PSF_IMG_LITERAL_THETA | PSF_DETERMINISTIC | PSF_COMPLEX_OUT)) return PSF_EINVAL;
    if (op->algo != PSF_ALGO_AUTO && op->algo != PSF_ALGO_CUTOUT) return PSF_EINVAL;
    return PSF_OK;
}

}  // namespace

extern "C" {

const char *psf_strerror(int s) {
    switch (s) {
        case PSF_OK: return "ok";
        case PSF_EINVAL: return "invalid argument";
        case PSF_ENOMEM: return "out of memory";
        case PSF_ECUDA: return "CUDA runtime error";
        case PSF_EUNSUPPORTED: return "unsupported request for this path";
        case PSF_ETIMEOUT: return "device-side wait timed out";
        default: return "unknown status";
    }
}

int psf_plan(const psf_obs_t *o, const psf_opts_t *opts, psf_plan_t *out) {
    if (!out) return PSF_EINVAL;
    *out = nullptr;
    int st = validate_obs(o);
    if (st) return st;
    if ((st = validate_opts(opts))) return st;

    const int nout = o->nchan / o->favg;
    std::vector<int64_t> bin_first(o->nbl + 1, 0), samp_first(o->nbl + 1, 0);
    for (int b = 0; b < o->nbl; ++b) {
        const int64_t nb = o->ntime / o->tavg[b];
        bin_first[b + 1] = bin_first[b] + nb;
        samp_first[b + 1] = samp_first[b] + nb * o->tavg[b];
    }
    const int64_t nbin = bin_first[o->nbl], nsamp = samp_first[o->nbl];
    const int64_t nvis = nbin * nout;
    if (nvis <= 0) return PSF_EINVAL;
    if (nvis >= (int64_t(1) << 31)) return PSF_EUNSUPPORTED;

    psf_plan_s *p = new (std::nothrow) psf_plan_s();
    if (!p) return PSF_ENOMEM;
    if (opts) p->opts = *opts;
    p->nbl = o->nbl; p->ntime = o->ntime; p->nchan = o->nchan; p->favg = o->favg; p->nout = nout;
    p->nbin = nbin; p->nsamp = nsamp; p->nvis = nvis;

    auto fail = [&](int s) { delete p; return s; };
    if (cudaGetDevice(&p->device) != cudaSuccess) { cudaGetLastError(); return fail(PSF_ECUDA); }
    if (cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) {
        cudaGetLastError();
        return fail(PSF_ECUDA);
    }

    // ---- channel records on the host (a few per output channel); the averaging bins are
    // formed on the device from the raw uvw (k_bin), float64 in, float32 records out
    const double dt = o->ntime >= 2 ? (o->time_s[o->ntime - 1] - o->time_s[0]) / (o->ntime - 1) : 0.0;
    std::vector<float4> h_chan, h_raw;
    std::vector<double2> h_chan64;
    std::vector<int32_t> h_bf;
    try {
        h_chan.resize(nout); h_raw.resize((size_t)o->nchan);
        h_chan64.resize(nout); h_bf.resize(o->nbl + 1);
    } catch (...) {
        return fail(PSF_ENOMEM);
    }
    if (nsamp >= (int64_t(1) << 31)) return fail(PSF_EUNSUPPORTED);
    int uniform = 1;
    for (int r = 0; r < nout; ++r) {
        double nu = 0, dnu = 0;
        const int c0 = r * o->favg;
        for (int c = c0; c < c0 + o->favg; ++c) { nu += o->freq_hz[c]; dnu += o->chan_width_hz[c]; }
        nu /= o->favg;
        const double wd = o->chan_width_hz[c0];
        const double sp = o->favg > 1 ? o->freq_hz[c0 + 1] - o->freq_hz[c0] : 0.0;
        for (int c = c0; c < c0 + o->favg; ++c) {
            if (std::fabs(o->chan_width_hz[c] - wd) > 1e-9 * wd) uniform = 0;
            if (c > c0 && std::fabs(o->freq_hz[c] - o->freq_hz[c - 1] - sp) > 1e-9 * o->freq_hz[c]) uniform = 0;
            h_raw[c] = make_float4((float)(o->freq_hz[c] - nu), (float)o->chan_width_hz[c],
                                   (float)(o->chan_width_hz[c] / dnu), 0.f);
        }
        h_chan[r] = make_float4((float)nu, (float)dnu, (float)sp, (float)wd);
        h_chan64[r] = make_double2(nu, dnu);
    }

    // ---- device copies and the binning
    cudaError_t e = cudaSuccess;
#define UP(buf, vec)                                                                               \
    if (e == cudaSuccess) e = p->buf.reserve(std::max<size_t>(16, vec.size() * sizeof(vec[0])));   \
    if (e == cudaSuccess && !vec.empty())                                                          \
        e = cudaMemcpy(p->buf.p, vec.data(), vec.size() * sizeof(vec[0]), cudaMemcpyHostToDevice);
    UP(chan, h_chan)
    UP(rawchan, h_raw)
    for (int b = 0; b <= o->nbl; ++b) h_bf[b] = (int32_t)bin_first[b];
    UP(chan64, h_chan64)
    UP(bin_first, h_bf)
#undef UP
    if (e == cudaSuccess) e = p->bin_ubar.reserve((size_t)nbin * sizeof(float4));
    if (e == cudaSuccess) e = p->bin_edge.reserve((size_t)nbin * sizeof(float4));
    if (e == cudaSuccess) e = p->bin_samp.reserve((size_t)nbin * sizeof(int2));
    if (e == cudaSuccess) e = p->bin_uv64.reserve((size_t)nbin * sizeof(double2));
    if (e == cudaSuccess) e = p->samp.reserve((size_t)nsamp * sizeof(float4));
    {
        // the raw uvw, tavg and sample offsets live on the device for the binning only
        DevBuf d_uvw, d_tavg, d_sfirst;
        const size_t uvw_bytes = (size_t)o->nbl * o->ntime * 3 * sizeof(double);
        if (e == cudaSuccess) e = d_uvw.reserve(uvw_bytes);
        if (e == cudaSuccess) e = d_tavg.reserve((size_t)o->nbl * sizeof(int32_t));
        if (e == cudaSuccess) e = d_sfirst.reserve((size_t)(o->nbl + 1) * sizeof(int64_t));
        if (e == cudaSuccess) e = cudaMemcpy(d_uvw.p, o->uvw_m, uvw_bytes, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(d_tavg.p, o->tavg, (size_t)o->nbl * sizeof(int32_t), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(d_sfirst.p, samp_first.data(), (size_t)(o->nbl + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = launch_bin((const double *)d_uvw.p, o->ntime, o->nbl, (const int32_t *)d_tavg.p,
                           (const int32_t *)p->bin_first.p, (const int64_t *)d_sfirst.p, nbin, dt,
                           (float4 *)p->bin_ubar.p, (double2 *)p->bin_uv64.p, (float4 *)p->bin_edge.p,
                           (int2 *)p->bin_samp.p, (float4 *)p->samp.p, 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();   // before the temporaries are freed
    }
    p->dt_raw = dt;
    try {
        p->h_tavg.assign(o->tavg, o->tavg + o->nbl);
        p->h_width.assign(o->chan_width_hz, o->chan_width_hz + o->nchan);
        p->h_bin_first = bin_first;
        p->h_samp_first = samp_first;
    } catch (...) {
        return fail(PSF_ENOMEM);
    }
    if (e == cudaSuccess) e = p->W.reserve(nvis * sizeof(float));
    // uv is padded with zeros to a whole number of 32-visibility stages plus one
    // stage, so bulk copies of full stages never leave the buffer
    if (e == cudaSuccess) e = p->uv.reserve((size_t)(nvis + 64) * sizeof(float2));
    if (e == cudaSuccess) e = cudaMemset(p->uv.p, 0, (size_t)(nvis + 64) * sizeof(float2));
    if (e == cudaSuccess) e = p->uv_lo.reserve((size_t)(nvis + 64) * sizeof(float2));
    if (e == cudaSuccess) e = cudaMemset(p->uv_lo.p, 0, (size_t)(nvis + 64) * sizeof(float2));
    if (e == cudaSuccess) e = p->err.reserve(sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(p->err.p, 0, sizeof(int));
    if (e == cudaSuccess && o->weights)
        e = cudaMemcpy(p->W.p, o->weights, nvis * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->meta_done, cudaEventDisableTiming);
    if (e != cudaSuccess) { cudaGetLastError(); return fail(cuda_status(e)); }

    // affine output channels (nu_r = nu_0 + r dnu, same spacing and width in every
    // group): enables the per-bin channel recurrence of the exact weights
    int affine = uniform && nout >= 2;
    const double dnu_ch = nout >= 2 ? (h_chan[nout - 1].x - (double)h_chan[0].x) / (nout - 1) : 0.0;
    if (affine) {
        double nu0 = 0, nulast = 0;
        for (int c = 0; c < o->favg; ++c) { nu0 += o->freq_hz[c]; nulast += o->freq_hz[(nout - 1) * o->favg + c]; }
        nu0 /= o->favg;
        nulast /= o->favg;
        const double dd = (nulast - nu0) / (nout - 1);
        for (int r = 0; r < nout && affine; ++r) {
            double nur = 0;
            for (int c = 0; c < o->favg; ++c) nur += o->freq_hz[r * o->favg + c];
            nur /= o->favg;
            if (std::fabs(nur - nu0 - r * dd) > 1e-9 * nur) affine = 0;
            if (std::fabs(h_chan[r].z - h_chan[0].z) > 1e-6f * std::fabs(h_chan[0].z) + 1e-3f) affine = 0;
            if (std::fabs(h_chan[r].w - h_chan[0].w) > 1e-6f * h_chan[0].w) affine = 0;
        }
    }
    DevObs &d = p->d;
    d.chan_affine = affine;
    p->affine0 = affine;
    d.dnu_ch = (float)dnu_ch;
    d.nvis = (int32_t)nvis; d.nbin = (int32_t)nbin; d.nout = nout; d.favg = o->favg; d.uniform = uniform;
    d.dt = (float)dt;
    d.bin_ubar = (const float4 *)p->bin_ubar.p;
    d.bin_edge = (const float4 *)p->bin_edge.p;
    d.bin_samp = (const int2 *)p->bin_samp.p;
    d.samp = (const float4 *)p->samp.p;
    d.chan = (const float4 *)p->chan.p;
    d.rawchan = (const float4 *)p->rawchan.p;
    d.W = (const float *)p->W.p;
    d.uv = (const float2 *)p->uv.p;
    d.uv_lo = (const float2 *)p->uv_lo.p;
    e = launch_fill_vis(d, (const double2 *)p->bin_uv64.p, (const double2 *)p->chan64.p, (float2 *)p->uv.p,
                        (float2 *)p->uv_lo.p, (float *)p->W.p, o->weights ? 0 : 1, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) { cudaGetLastError(); return fail(cuda_status(e)); }
    *out = p;
    return PSF_OK;
}

int psf_plan_set_windows(psf_plan_t p, const float *tw, const float *cw) {
    if (!p) return PSF_EINVAL;
    DevObs &d = p->d;
    if (!tw && !cw) {   // back to the boxcar
        d.win = 0;
        d.chan_affine = p->affine0;
        return PSF_OK;
    }
    const int nbl = p->nbl, favg = p->favg, nout = p->nout, nchan = p->nchan;
    std::vector<float> h_sw, h_cw;
    std::vector<int32_t> h_bl;
    try {
        h_sw.resize((size_t)p->nsamp);
        h_cw.resize((size_t)nbl * nchan);
        h_bl.resize((size_t)p->nbin);
    } catch (...) {
        return PSF_ENOMEM;
    }
    int64_t toff = 0;
    for (int b = 0; b < nbl; ++b) {
        const int n = p->h_tavg[b];
        double sum = 0;
        for (int s = 0; s < n; ++s) {
            const double v = tw ? (double)tw[toff + s] : 1.0;
            if (!std::isfinite(v) || v < 0) return PSF_EINVAL;
            sum += v;
        }
        if (!(sum > 0)) return PSF_EINVAL;
        const int64_t nb = p->h_bin_first[b + 1] - p->h_bin_first[b];
        for (int64_t tau = 0; tau < nb; ++tau) {
            const int64_t rec = p->h_samp_first[b] + tau * n;
            for (int s = 0; s < n; ++s) h_sw[rec + s] = (float)((tw ? (double)tw[toff + s] : 1.0) / sum);
            h_bl[p->h_bin_first[b] + tau] = b;
        }
        toff += n;
        for (int r = 0; r < nout; ++r) {
            double cs = 0;
            for (int j = 0; j < favg; ++j) {
                const double v = cw ? (double)cw[(int64_t)b * favg + j] : 1.0;
                if (!std::isfinite(v) || v < 0) return PSF_EINVAL;
                cs += v * p->h_width[r * favg + j];
            }
            if (!(cs > 0)) return PSF_EINVAL;
            for (int j = 0; j < favg; ++j) {
                const double v = cw ? (double)cw[(int64_t)b * favg + j] : 1.0;
                h_cw[(int64_t)b * nchan + r * favg + j] = (float)(v * p->h_width[r * favg + j] / cs);
            }
        }
    }
    PSF_TRY(p->samp_w.reserve(std::max<size_t>(16, h_sw.size() * sizeof(float))));
    PSF_TRY(p->chan_win.reserve(std::max<size_t>(16, h_cw.size() * sizeof(float))));
    PSF_TRY(p->bin_bl.reserve(std::max<size_t>(16, h_bl.size() * sizeof(int32_t))));
    PSF_TRY(cudaMemcpy(p->samp_w.p, h_sw.data(), h_sw.size() * sizeof(float), cudaMemcpyHostToDevice));
    PSF_TRY(cudaMemcpy(p->chan_win.p, h_cw.data(), h_cw.size() * sizeof(float), cudaMemcpyHostToDevice));
    PSF_TRY(cudaMemcpy(p->bin_bl.p, h_bl.data(), h_bl.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    d.samp_w = (const float *)p->samp_w.p;
    d.chan_win = (const float *)p->chan_win.p;
    d.bin_bl = (const int32_t *)p->bin_bl.p;
    d.win = (tw ? 1 : 0) | (cw ? 2 : 0);
    d.chan_affine = 0;   // the channel recurrence of the exact weights assumes the boxcar
    return PSF_OK;
}

int psf_plan_set_weights(psf_plan_t p, const float *w, void *stream) {
    if (!p) return PSF_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (w) {
        PSF_TRY(cudaMemcpyAsync(p->W.p, w, (size_t)p->nvis * sizeof(float), cudaMemcpyDeviceToDevice, st));
        return PSF_OK;
    }
    PSF_TRY(launch_fill_vis(p->d, (const double2 *)p->bin_uv64.p, (const double2 *)p->chan64.p, (float2 *)p->uv.p,
                            (float2 *)p->uv_lo.p, (float *)p->W.p, 1, st));
    return PSF_OK;
}

int psf_plan_set_opts(psf_plan_t p, const psf_opts_t *opts) {
    if (!p || !opts) return PSF_EINVAL;
    int st = validate_opts(opts);
    if (st) return st;
    p->opts = *opts;
    return PSF_OK;
}

int64_t psf_plan_nvis(psf_plan_t p) { return p ? p->nvis : -1; }

void psf_plan_destroy(psf_plan_t p) {
    if (!p) return;
    if (p->meta_done) {
        cudaEventSynchronize(p->meta_done);
        cudaEventDestroy(p->meta_done);
    }
    cudaDeviceSynchronize();
    delete p;
}

int psf_sync_status(psf_plan_t p, void *stream) {
    if (!p) return PSF_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaStreamSynchronize(st) != cudaSuccess) { cudaGetLastError(); return PSF_ECUDA; }
    int flag = 0;
    if (cudaMemcpy(&flag, p->err.p, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return PSF_ECUDA;
    }
    if (flag) {
        cudaMemset(p->err.p, 0, sizeof(int));
        return PSF_ETIMEOUT;
    }
    return PSF_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ per-call path
namespace {

struct BatchHost {
    int npos = 0;
    std::vector<float4> pos;      // l0, m0, n0-1, 0
    std::vector<int32_t> npix;
    std::vector<int64_t> out_off;
    double cell = 0;
};

// per_px: floats per output pixel (2 with complex output: N^2 real parts, then N^2
// imaginary parts per cutout).
int prepare_batch(const psf_plan_s *p, const psf_batch_t *b, BatchHost &h, int max_n, int per_px = 1) {
    if (!b || b->npos < 0) return PSF_EINVAL;
    h.npos = b->npos;
    if (b->npos == 0) return PSF_OK;
    if (!b->lm || !(b->cell_rad > 0.0)) return PSF_EINVAL;
    if (!b->npix && b->npix0 <= 0) return PSF_EINVAL;
    h.cell = b->cell_rad;
    h.pos.resize(b->npos); h.npix.resize(b->npos); h.out_off.resize(b->npos);
    int64_t run = 0;
    for (int i = 0; i < b->npos; ++i) {
        const int N = b->npix ? b->npix[i] : b->npix0;
        if (N < 2 || N > 4096 || (N & 1)) return PSF_EINVAL;
        if (N > max_n) return PSF_EUNSUPPORTED;
        const double l0 = b->lm[2 * i], m0 = b->lm[2 * i + 1];
        const double r2 = l0 * l0 + m0 * m0;
        if (!(r2 < 1.0)) return PSF_EINVAL;
        // n0 - 1 without cancellation: -(l^2+m^2) / (1 + sqrt(1 - l^2 - m^2))
        const double n0m1 = (p->opts.flags & PSF_WTERM) ? -r2 / (1.0 + std::sqrt(1.0 - r2)) : 0.0;
        h.pos[i] = make_float4((float)l0, (float)m0, (float)n0m1, 0.f);
        h.npix[i] = N;
        if (b->out_offset) {
            if (b->out_offset[i] < 0) return PSF_EINVAL;
            h.out_off[i] = b->out_offset[i];
        } else {
            h.out_off[i] = run;
            run += (int64_t)per_px * N * N;
        }
    }
    if (b->out_offset) {   // cutouts must not overlap
        std::vector<int> idx(b->npos);
        for (int i = 0; i < b->npos; ++i) idx[i] = i;
        std::sort(idx.begin(), idx.end(), [&](int a, int c) { return h.out_off[a] < h.out_off[c]; });
        for (int i = 1; i < b->npos; ++i) {
            const int a = idx[i - 1];
            if (h.out_off[a] + (int64_t)per_px * h.npix[a] * h.npix[a] > h.out_off[idx[i]]) return PSF_EINVAL;
        }
    }
    return PSF_OK;
}

// Upload per-call metadata through a pinned staging buffer; the staging buffer is
// reused only after the previous upload has completed.
int upload_meta(psf_plan_s *p, const void *src, size_t bytes, cudaStream_t st) {
    PSF_TRY(cudaEventSynchronize(p->meta_done));
    PSF_TRY(p->hmeta.reserve(bytes));
    PSF_TRY(p->meta.reserve(bytes));
    std::memcpy(p->hmeta.p, src, bytes);
    PSF_TRY(cudaMemcpyAsync(p->meta.p, p->hmeta.p, bytes, cudaMemcpyHostToDevice, st));
    PSF_TRY(cudaEventRecord(p->meta_done, st));
    return PSF_OK;
}

constexpr size_t kWeightBudget = size_t(4) << 30;   // weights of one position chunk (bytes)
constexpr size_t kW16Budget = size_t(4) << 30;      // FP16 weights of one batched chunk (bytes)
constexpr int kKrMinGroup = 32;                     // positions of one size for the batched form

// One size group of the batched form: positions idx (batch indices) of cutout size N.
struct KrGroup {
    int N;
    std::vector<int> idx;
};

// Batched tensor-core path for groups of positions with cutout sizes N (multiples of 32,
// <= 256).  Per chunk of visibilities the weights of every group are written as FP16/BF16
// rows into one buffer (each group padded to whole 128-position tiles), then one
// persistent launch of the Khatri-Rao kernel (one CTA per SM) pulls (128-position tile,
// 256-pixel tile, visibility range) items from an atomic queue and accumulates them into
// the zeroed output.  Every item is 128 positions x 256 pixels, so its cost is its
// visibility range: the ranges are equal, items_per_cta x SMs of them at least (fewer
// when a range would drop below one 64-stage accumulation run).  kmax < nvis restricts
// the call to the first kmax visibilities (the autotuner's probes); ms_out (optional)
// receives the summed time of the contraction launches (the stream is synchronized).
int run_kr(psf_plan_s *p, int method, const BatchHost &h, const std::vector<KrGroup> &groups, float *out,
           cudaStream_t st, int items_per_cta, int64_t kmax = -1, double *ms_out = nullptr) {
    const int64_t K = kmax > 0 ? std::min<int64_t>(kmax, p->nvis) : p->nvis;
    const int bf16 = prec_bf16(p->opts.prec);
    // Methods 1 and 2 have real weights (unless windowed): one K' column per visibility,
    // 64-visibility stages; complex weights: two columns, 32-visibility stages.
    const int real = method != kExact && p->d.win == 0;
    const int64_t ks = real ? 64 : 32;
    const size_t bytes_per = real ? 2 : 4;
    // combined rows: group g occupies rows [row0_g, row0_g + 128 ntile_g)
    std::vector<float4> pos;
    std::vector<int32_t> slot_of_row, npix;
    std::vector<int64_t> outo;
    std::vector<int> row0(groups.size()), slot0(groups.size());
    int rows = 0;
    for (size_t g = 0; g < groups.size(); ++g) {
        const int np = (int)groups[g].idx.size();
        row0[g] = rows;
        slot0[g] = (int)pos.size();
        for (int i = 0; i < np; ++i) {
            pos.push_back(h.pos[groups[g].idx[i]]);
            outo.push_back(h.out_off[groups[g].idx[i]]);
            npix.push_back(groups[g].N);
        }
        const int ntile = (np + 127) / 128;
        for (int r = 0; r < ntile * 128; ++r) slot_of_row.push_back(r < np ? slot0[g] + r : -1);
        rows += ntile * 128;
    }
    const int npos = (int)pos.size();
    if (npos == 0) return PSF_OK;
    int64_t KC = (int64_t)(kW16Budget / ((size_t)rows * bytes_per)) / 64 * 64;
    KC = std::max<int64_t>(64, std::min<int64_t>(KC, (K + 63) / 64 * 64));
    const int64_t nchunk = (K + KC - 1) / KC;
    int64_t nbase = 0;   // (position tile, pixel tile) pairs
    for (const auto &g : groups) nbase += (int64_t)((g.idx.size() + 127) / 128) * (g.N * g.N / 256);
    PSF_TRY(p->w16.reserve((size_t)rows * KC * bytes_per));
    PSF_TRY(p->queue.reserve(sizeof(int)));
    CUtensorMapStub wmap;
    int s = make_weight_map(&wmap, p->w16.p, bf16, real ? KC : 2 * KC, rows);
    if (s) return s;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    double ms_total = 0.0;
    if (ms_out) {
        PSF_TRY(cudaEventCreate(&t0));
        PSF_TRY(cudaEventCreate(&t1));
    }
    for (int64_t c = 0; c < nchunk; ++c) {
        const int64_t kc0 = c * KC, kcn = std::min<int64_t>(KC, K - kc0);
        const int64_t nst = (kcn + ks - 1) / ks;
        // equal visibility ranges: enough items for items_per_cta per CTA, ranges of at
        // least one accumulation run (64 stages)
        const int64_t target = (int64_t)std::max(1, items_per_cta) * p->nsm;
        int64_t nsplit = std::max<int64_t>(1, std::min<int64_t>((target + nbase - 1) / nbase, nst / 64));
        const int64_t sper = (nst + nsplit - 1) / nsplit;
        nsplit = (nst + sper - 1) / sper;
        std::vector<KrItem> items;
        items.reserve(nbase * nsplit);
        // the full ranges first, the shorter last range after them (largest first)
        for (int64_t sp = 0; sp < nsplit; ++sp)
            for (size_t g = 0; g < groups.size(); ++g) {
                const int np = (int)groups[g].idx.size(), N = groups[g].N;
                for (int t = 0; t < (np + 127) / 128; ++t)
                    for (int q = 0; q < N * N / 256; ++q) {
                        KrItem it;
                        it.wrow = row0[g] + t * 128;
                        it.npos = std::min(128, np - t * 128);
                        it.slot0 = slot0[g] + t * 128;
                        it.N = N;
                        it.q0 = q * 256;
                        it.npx = 256;
                        it.kb = (int32_t)(kc0 + sp * sper * ks);
                        it.ke = (int32_t)std::min<int64_t>(kc0 + kcn, kc0 + (sp + 1) * sper * ks);
                        items.push_back(it);
                    }
            }
        const size_t off_pos = 0;
        const size_t off_slot = align_up(off_pos + npos * sizeof(float4), 16);
        const size_t off_outo = align_up(off_slot + rows * sizeof(int32_t), 16);
        const size_t off_npix = align_up(off_outo + npos * sizeof(int64_t), 16);
        const size_t off_items = align_up(off_npix + npos * sizeof(int32_t), 16);
        const size_t bytes = align_up(off_items + items.size() * sizeof(KrItem), 16);
        std::vector<char> blob(bytes, 0);
        std::memcpy(blob.data() + off_pos, pos.data(), npos * sizeof(float4));
        std::memcpy(blob.data() + off_slot, slot_of_row.data(), rows * sizeof(int32_t));
        std::memcpy(blob.data() + off_outo, outo.data(), npos * sizeof(int64_t));
        std::memcpy(blob.data() + off_npix, npix.data(), npos * sizeof(int32_t));
        std::memcpy(blob.data() + off_items, items.data(), items.size() * sizeof(KrItem));
        if ((s = upload_meta(p, blob.data(), bytes, st))) return s;
        char *dm = (char *)p->meta.p;
        if (c == 0) {
            PSF_TRY(launch_zero_cutouts(out, (const int64_t *)(dm + off_outo), (const int32_t *)(dm + off_npix), npos,
                                        st));
            p->n_kernels++;
        }
        PSF_TRY(launch_weights16(p->d, method, p->opts.flags, (const float4 *)(dm + off_pos),
                                 (const int32_t *)(dm + off_slot), rows, (int32_t)kc0, (int32_t)kcn, KC, bf16,
                                 p->w16.p, st));
        p->n_kernels++;
        cudaEvent_t ev1 = nullptr, ev2 = nullptr;
        if (p->prof) {
            if (p->prof_used == p->prof_ev.size()) {
                cudaEvent_t a, e2;
                PSF_TRY(cudaEventCreate(&a));
                PSF_TRY(cudaEventCreate(&e2));
                p->prof_ev.emplace_back(a, e2);
            }
            ev1 = p->prof_ev[p->prof_used].first;
            ev2 = p->prof_ev[p->prof_used].second;
            p->prof_used++;
            PSF_TRY(cudaEventRecord(ev1, st));
        }
        if (ms_out) PSF_TRY(cudaEventRecord(t0, st));
        PSF_TRY(launch_psf_kr(&wmap, (const KrItem *)(dm + off_items), (int)items.size(), (int *)p->queue.p, p->nsm,
                              p->d.uv, (int32_t)kc0, (float)h.cell, (const int64_t *)(dm + off_outo), out, bf16, real,
                              (int *)p->err.p, st));
        if (ms_out) {
            PSF_TRY(cudaEventRecord(t1, st));
            PSF_TRY(cudaEventSynchronize(t1));
            float ms = 0.f;
            PSF_TRY(cudaEventElapsedTime(&ms, t0, t1));
            ms_total += ms;
        }
        if (p->prof) PSF_TRY(cudaEventRecord(ev2, st));
        p->n_contract++;
        p->n_kernels += 2;   // the queue reset and the contraction
    }
    if (ms_out) {
        *ms_out = ms_total;
        cudaEventDestroy(t0);
        cudaEventDestroy(t1);
    }
    return PSF_OK;
}

// Autotuner of the batched form, run on the first batched call of a plan for each weight
// class (real / complex weights, operand type) and cached in the plan.  (1) Items per CTA:
// the batched call of this batch's groups over a probe of the first kProbeVis
// visibilities, timed for each candidate (2, 4, 8, 16 items per SM), into scratch output;
// the fastest is kept.  (2) Per cutout size N present, the crossover between the forms:
// the per-cutout form's time for one position and the batched form's time for one
// 128-position tile over the same probe; the batched form takes a group of n positions
// when ceil(n / 128) t_tile < n t_cutout.
constexpr int64_t kProbeVis = int64_t(1) << 19;

int run_forward(psf_plan_s *p, int method, const psf_batch_t *b, float *out, cudaStream_t st, int64_t kmax = -1);

int kr_tune(psf_plan_s *p, int method, const BatchHost &hall, const std::vector<KrGroup> &cand, cudaStream_t st,
            psf_plan_s::KrTune &t) {
    PSF_TRY(cudaStreamSynchronize(st));
    const int64_t probe = std::min<int64_t>(kProbeVis, p->nvis);
    // scratch output: packed offsets of the candidate groups' cutouts
    BatchHost hs = hall;
    int64_t run = 0;
    for (const auto &g : cand)
        for (int i : g.idx) {
            hs.out_off[i] = run;
            run += (int64_t)g.N * g.N;
        }
    DevBuf scratch;
    PSF_TRY(scratch.reserve((size_t)std::max<int64_t>(run, 1) * sizeof(float)));
    const bool prof = p->prof;
    p->prof = false;
    double best = 1e300;
    int s = PSF_OK;
    std::vector<KrGroup> big;
    for (const auto &g : cand)
        if ((int)g.idx.size() >= kKrMinGroup) big.push_back(g);
    if (!t.done && !big.empty()) {
        for (int ipc : {2, 4, 8, 16}) {
            double ms = 0.0;
            if ((s = run_kr(p, method, hs, big, (float *)scratch.p, st, ipc, probe, &ms))) break;
            if (ms < best) { best = ms; t.items_per_cta = ipc; }
        }
        t.done = s == PSF_OK;
    }
    // crossover per size: one position per-cutout against one 128-position tile batched
    for (const auto &g : cand) {
        if (s) break;
        if (t.min_group.count(g.N) || (int)g.idx.size() < 8) continue;
        std::vector<KrGroup> one(1);
        one[0].N = g.N;
        one[0].idx.assign(g.idx.begin(), g.idx.begin() + std::min<size_t>(g.idx.size(), 128));
        double t_tile = 0.0;
        if ((s = run_kr(p, method, hs, one, (float *)scratch.p, st, t.items_per_cta, probe, &t_tile))) break;
        const double lm[2] = {0.0, 0.0};   // cost does not depend on the position
        psf_batch_t b1{};
        b1.npos = 1;
        b1.lm = lm;
        b1.npix0 = g.N;
        b1.cell_rad = hall.cell;
        const psf_opts_t saved = p->opts;
        p->opts.algo = PSF_ALGO_CUTOUT;
        cudaEvent_t a, z;
        PSF_TRY(cudaEventCreate(&a));
        PSF_TRY(cudaEventCreate(&z));
        PSF_TRY(cudaEventRecord(a, st));
        s = run_forward(p, method, &b1, (float *)scratch.p, st, probe);
        PSF_TRY(cudaEventRecord(z, st));
        PSF_TRY(cudaEventSynchronize(z));
        float t_cut = 0.f;
        PSF_TRY(cudaEventElapsedTime(&t_cut, a, z));
        cudaEventDestroy(a);
        cudaEventDestroy(z);
        p->opts = saved;
        const double thr = t_cut > 0.f ? t_tile / (double)t_cut : 1e9;
        t.min_group[g.N] = (int)std::max(1.0, std::min(128.0, std::ceil(thr)));
    }
    p->prof = prof;
    PSF_TRY(cudaStreamSynchronize(st));
    return s;
}

int run_forward_cplx(psf_plan_s *p, int method, const BatchHost &h, float *out, cudaStream_t st);

int run_forward(psf_plan_s *p, int method, const psf_batch_t *b, float *out, cudaStream_t st, int64_t kmax) {
    if (!p || !out) return PSF_EINVAL;
    const bool tc = p->opts.prec != PSF_FP32;
    const bool split = prec_split(p->opts.prec);
    const bool cplx = (p->opts.flags & PSF_COMPLEX_OUT) != 0;
    BatchHost hall;
    int s = prepare_batch(p, b, hall, cplx ? 128 : (tc ? 256 : 4096), cplx ? 2 : 1);
    if (s || hall.npos == 0) return s;
    if (cplx) return (tc && !split) ? run_forward_cplx(p, method, hall, out, st) : PSF_EUNSUPPORTED;
    if (kmax > 0 && !tc) return PSF_EINVAL;   // visibility probes (the autotuner) are tensor-core only
    const int64_t K = kmax > 0 ? std::min<int64_t>(kmax, p->nvis) : p->nvis;
    // Batched tensor-core form for groups of one eligible size that are large enough (the
    // autotuner's crossover, else kKrMinGroup positions); the rest goes through the
    // per-cutout form below.
    BatchHost h;
    h.cell = hall.cell;
    if (tc && !split && p->opts.algo == PSF_ALGO_AUTO && !(p->opts.flags & PSF_DETERMINISTIC) && kmax < 0) {
        std::vector<KrGroup> present;
        {
            std::vector<std::vector<int>> by(257);
            for (int i = 0; i < hall.npos; ++i) {
                const int N = hall.npix[i];
                if (N % 32 == 0 && N >= 32 && N <= 256) by[N].push_back(i);
            }
            for (int N = 32; N <= 256; N += 32)
                if (!by[N].empty()) present.push_back(KrGroup{N, by[N]});
        }
        const int real = method != kExact && p->d.win == 0;
        psf_plan_s::KrTune &t = p->tune[(real ? 1 : 0) | (prec_bf16(p->opts.prec) ? 2 : 0)];
        bool need = false;
        for (const auto &g : present) need = need || (!t.min_group.count(g.N) && (int)g.idx.size() >= 8);
        if (need && (s = kr_tune(p, method, hall, present, st, t))) return s;
        std::vector<KrGroup> batched;
        std::vector<char> done(hall.npos, 0);
        for (const auto &g : present) {
            const auto f = t.min_group.find(g.N);
            const int thr = f != t.min_group.end() ? f->second : kKrMinGroup;
            if ((int)g.idx.size() < thr) continue;
            batched.push_back(g);
            for (int i : g.idx) done[i] = 1;
        }
        if (!batched.empty() && (s = run_kr(p, method, hall, batched, out, st, t.items_per_cta))) return s;
        for (int i = 0; i < hall.npos; ++i)
            if (!done[i]) {
                h.pos.push_back(hall.pos[i]);
                h.npix.push_back(hall.npix[i]);
                h.out_off.push_back(hall.out_off[i]);
            }
        h.npos = (int)h.pos.size();
        if (h.npos == 0) return PSF_OK;
    } else {
        h = hall;
    }
    const int chunk = (int)std::max<int64_t>(
        1, std::min<int64_t>(std::min<int64_t>(h.npos, 32768), kWeightBudget / (K * 8)));

    for (int c0 = 0; c0 < h.npos; c0 += chunk) {
        const int cn = std::min(chunk, h.npos - c0);
        // chunk-local packed layout for the partial sums
        std::vector<int64_t> loc(cn);
        int64_t chunk_px = 0;
        for (int i = 0; i < cn; ++i) { loc[i] = chunk_px; chunk_px += (int64_t)h.npix[c0 + i] * h.npix[c0 + i]; }

        std::vector<Tile> tiles;
        std::vector<TcItem> items;
        int nsplit = 1, ncols_max = 16;
        int32_t kper = (int32_t)K;
        if (!tc) {
            for (int i = 0; i < cn; ++i) {
                const int N = h.npix[c0 + i];
                for (int j0 = 0; j0 < N; j0 += 64)
                    for (int i0 = 0; i0 < N; i0 += 64) tiles.push_back(Tile{i, N, i0, j0, loc[i]});
            }
            const int64_t target = 4LL * p->nsm;
            nsplit = (int)std::max<int64_t>(1, std::min<int64_t>((target + tiles.size() - 1) / tiles.size(),
                                                                  (K + 4095) / 4096));
            kper = (int32_t)(((K + nsplit - 1) / nsplit + 31) / 32 * 32);
            nsplit = (int)((K + kper - 1) / kper);
        } else {
            std::vector<TcItem> base;
            const int tw = split ? 128 : 256;   // tile width (split precision: <= 128 columns)
            for (int i = 0; i < cn; ++i) {
                const int N = h.npix[c0 + i];
                for (int j0 = 0; j0 < N; j0 += 128)
                    for (int i0 = 0; i0 < N; i0 += tw) {
                        const int w = std::min(tw, N - i0);
                        const int nc = (w + 31) / 32 * 32;   // whole 32-row twiddle chains
                        ncols_max = std::max(ncols_max, nc);
                        base.push_back(TcItem{i, N, j0, i0, nc, 0, 0, 0, loc[i]});
                    }
            }
            const int64_t target = p->nsm;
            nsplit = (int)std::max<int64_t>(1, std::min<int64_t>((target + base.size() - 1) / base.size(),
                                                                  (K + 8191) / 8192));
            kper = (int32_t)(((K + nsplit - 1) / nsplit + 31) / 32 * 32);
            nsplit = (int)((K + kper - 1) / kper);
            for (int sp = 0; sp < nsplit; ++sp)
                for (auto it : base) {
                    it.k0 = (int32_t)(sp * (int64_t)kper);
                    it.k1 = (int32_t)std::min<int64_t>(K, (int64_t)(sp + 1) * kper);
                    it.split = sp;
                    items.push_back(it);
                }
        }
        const bool direct = (nsplit == 1) && !tc;
        if (direct)
            for (auto &t : tiles) t.out_off = h.out_off[c0 + t.slot];

        // metadata block: pos | npix | loc offs | out offs | tiles/items
        Meta m;
        m.off_pos = 0;
        m.off_npix = align_up(m.off_pos + cn * sizeof(float4), 16);
        m.off_loc = align_up(m.off_npix + cn * sizeof(int32_t), 16);
        m.off_out = align_up(m.off_loc + cn * sizeof(int64_t), 16);
        m.off_tiles = align_up(m.off_out + cn * sizeof(int64_t), 16);
        const size_t tbytes = tc ? items.size() * sizeof(TcItem) : tiles.size() * sizeof(Tile);
        m.bytes = align_up(m.off_tiles + tbytes, 16);
        std::vector<char> blob(m.bytes, 0);
        std::memcpy(blob.data() + m.off_pos, &h.pos[c0], cn * sizeof(float4));
        std::memcpy(blob.data() + m.off_npix, &h.npix[c0], cn * sizeof(int32_t));
        std::memcpy(blob.data() + m.off_loc, loc.data(), cn * sizeof(int64_t));
        std::memcpy(blob.data() + m.off_out, &h.out_off[c0], cn * sizeof(int64_t));
        if (tc) std::memcpy(blob.data() + m.off_tiles, items.data(), tbytes);
        else std::memcpy(blob.data() + m.off_tiles, tiles.data(), tbytes);
        if ((s = upload_meta(p, blob.data(), m.bytes, st))) return s;
        char *dm = (char *)p->meta.p;
        const float4 *d_pos = (const float4 *)(dm + m.off_pos);
        const int32_t *d_npix = (const int32_t *)(dm + m.off_npix);
        const int64_t *d_loc = (const int64_t *)(dm + m.off_loc);
        const int64_t *d_out = (const int64_t *)(dm + m.off_out);

        // weight rows padded to 32 visibilities (16-byte aligned stage copies), plus
        // one stage of slack after the last row
        const int64_t ldw = (K + 31) / 32 * 32;
        PSF_TRY(p->wbuf.reserve((size_t)(cn * ldw + 64) * sizeof(float2)));
        float2 *w = (float2 *)p->wbuf.p;
        // weights in FP32 with the accurate sine/cosine for the FP32 path and the split
        // precision modes, the MUFU forms where they are rounded to 16 bits
        PSF_TRY(launch_weights(p->d, method, p->opts.flags, d_pos, cn, 0, (int32_t)K, w, ldw, (tc && !split) ? 1 : 0,
                               st));

        p->n_kernels++;
        float *part = out;
        int64_t stride = 0;
        if (!direct) {
            PSF_TRY(p->partial.reserve((size_t)nsplit * chunk_px * sizeof(float)));
            part = (float *)p->partial.p;
            stride = chunk_px;
        }
        cudaEvent_t ev1 = nullptr, ev2 = nullptr;
        if (p->prof) {
            if (p->prof_used == p->prof_ev.size()) {
                cudaEvent_t a, c;
                PSF_TRY(cudaEventCreate(&a));
                PSF_TRY(cudaEventCreate(&c));
                p->prof_ev.emplace_back(a, c);
            }
            ev1 = p->prof_ev[p->prof_used].first;
            ev2 = p->prof_ev[p->prof_used].second;
            p->prof_used++;
            PSF_TRY(cudaEventRecord(ev1, st));
        }
        if (!tc) {
            PSF_TRY(launch_psf_fp32(p->d, w, ldw, (const Tile *)(dm + m.off_tiles), (int)tiles.size(), nsplit,
                                    kper, h.cell, part, stride, st));
        } else {
            // the approximations' weights are real unless windowed (Eqs. 15-16: a window's
            // transform is complex in general)
            int wreal = (method != PSF_METHOD_EXACT && p->d.win == 0) ? 1 : 0;
            if (wreal) {
                bool whole = true;
                for (const auto &t : items)
                    whole = whole && t.j0 == 0 && t.i0 == 0 && t.ncols == t.N && t.N <= 128 && (t.N % 64) == 0;
                if (whole) wreal = 2;
            }
            PSF_TRY(launch_psf_tc(p->d, w, ldw, (const TcItem *)(dm + m.off_tiles), (int)items.size(), ncols_max,
                                  prec_bf16(p->opts.prec), (float)h.cell, wreal, part, stride, (int *)p->err.p, st,
                                  split ? 1 : 0));
        }
        if (p->prof) PSF_TRY(cudaEventRecord(ev2, st));
        p->n_contract++;
        p->n_kernels++;
        if (!direct) {
            PSF_TRY(launch_reduce(part, nsplit, stride, d_loc, d_out, d_npix, cn, tc ? 1 : 0, out, st));
            p->n_kernels++;
        }
    }
    return PSF_OK;
}

// Methods 1 and 2 of one batch in one pass (tensor-core precisions, cutouts of 64 or
// 128 pixels that the per-cutout form computes): the fused kernel shares the twiddles
// of both methods and writes both cutouts.  Any other batch (the FP32 precision,
// other sizes, groups large enough for the batched form, PSF_ALGO_CUTOUT off) takes
// the two separate calls.
int run_forward_uvimg(psf_plan_s *p, const psf_batch_t *b, float *out_uv, float *out_img, cudaStream_t st) {
    if (!p || !out_uv || !out_img) return PSF_EINVAL;
    const bool tc = p->opts.prec != PSF_FP32 && !prec_split(p->opts.prec);   // fused pass: single-pass operands
    if (p->opts.flags & PSF_COMPLEX_OUT) {   // the fused pass writes real parts only
        const int s2 = run_forward(p, kUV, b, out_uv, st);
        return s2 ? s2 : run_forward(p, kImg, b, out_img, st);
    }
    BatchHost h;
    int s = prepare_batch(p, b, h, tc ? 256 : 4096);
    if (s || h.npos == 0) return s;
    bool fused = tc && p->d.win == 0;   // the fused pass needs real weights
    int n64 = 0, n128 = 0;
    for (int i = 0; i < h.npos && fused; ++i) {
        if (h.npix[i] == 64) ++n64;
        else if (h.npix[i] == 128) ++n128;
        else fused = false;
    }
    if (fused && p->opts.algo == PSF_ALGO_AUTO && !(p->opts.flags & PSF_DETERMINISTIC) &&
        (n64 >= kKrMinGroup || n128 >= kKrMinGroup))
        fused = false;
    if (!fused) {
        s = run_forward(p, kUV, b, out_uv, st);
        return s ? s : run_forward(p, kImg, b, out_img, st);
    }
    const int64_t K = p->nvis;
    const int chunk = (int)std::max<int64_t>(
        1, std::min<int64_t>(std::min<int64_t>(h.npos, 32768), kWeightBudget / (K * 16)));
    for (int c0 = 0; c0 < h.npos; c0 += chunk) {
        const int cn = std::min(chunk, h.npos - c0);
        std::vector<int64_t> loc(cn);
        int64_t chunk_px = 0;
        int ncols_max = 64;
        for (int i = 0; i < cn; ++i) {
            loc[i] = chunk_px;
            chunk_px += (int64_t)h.npix[c0 + i] * h.npix[c0 + i];
            ncols_max = std::max(ncols_max, (int)h.npix[c0 + i]);
        }
        // one whole-cutout item per position, visibility splits to fill the SMs
        std::vector<TcItem> base, items;
        for (int i = 0; i < cn; ++i) {
            const int N = h.npix[c0 + i];
            base.push_back(TcItem{i, N, 0, 0, N, 0, 0, 0, loc[i]});
        }
        int nsplit = (int)std::max<int64_t>(1, std::min<int64_t>((p->nsm + cn - 1) / cn, (K + 8191) / 8192));
        const int32_t kper = (int32_t)(((K + nsplit - 1) / nsplit + 31) / 32 * 32);
        nsplit = (int)((K + kper - 1) / kper);
        for (int sp = 0; sp < nsplit; ++sp)
            for (auto it : base) {
                it.k0 = (int32_t)(sp * (int64_t)kper);
                it.k1 = (int32_t)std::min<int64_t>(K, (int64_t)(sp + 1) * kper);
                it.split = sp;
                items.push_back(it);
            }
        Meta m;
        m.off_pos = 0;
        m.off_npix = align_up(m.off_pos + cn * sizeof(float4), 16);
        m.off_loc = align_up(m.off_npix + cn * sizeof(int32_t), 16);
        m.off_out = align_up(m.off_loc + cn * sizeof(int64_t), 16);
        m.off_tiles = align_up(m.off_out + cn * sizeof(int64_t), 16);
        const size_t tbytes = items.size() * sizeof(TcItem);
        m.bytes = align_up(m.off_tiles + tbytes, 16);
        std::vector<char> blob(m.bytes, 0);
        std::memcpy(blob.data() + m.off_pos, &h.pos[c0], cn * sizeof(float4));
        std::memcpy(blob.data() + m.off_npix, &h.npix[c0], cn * sizeof(int32_t));
        std::memcpy(blob.data() + m.off_loc, loc.data(), cn * sizeof(int64_t));
        std::memcpy(blob.data() + m.off_out, &h.out_off[c0], cn * sizeof(int64_t));
        std::memcpy(blob.data() + m.off_tiles, items.data(), tbytes);
        if ((s = upload_meta(p, blob.data(), m.bytes, st))) return s;
        char *dm = (char *)p->meta.p;
        const float4 *d_pos = (const float4 *)(dm + m.off_pos);
        const int32_t *d_npix = (const int32_t *)(dm + m.off_npix);
        const int64_t *d_loc = (const int64_t *)(dm + m.off_loc);
        const int64_t *d_out = (const int64_t *)(dm + m.off_out);
        // two weight blocks (Method 1, Method 2), rows padded as in run_forward
        const int64_t ldw = (K + 31) / 32 * 32;
        const int64_t wblock = cn * ldw + 64;
        PSF_TRY(p->wbuf.reserve((size_t)(2 * wblock) * sizeof(float2)));
        float2 *w_uv = (float2 *)p->wbuf.p, *w_img = w_uv + wblock;
        PSF_TRY(launch_weights(p->d, kUV, p->opts.flags, d_pos, cn, 0, (int32_t)K, w_uv, ldw, 1, st));
        PSF_TRY(launch_weights(p->d, kImg, p->opts.flags, d_pos, cn, 0, (int32_t)K, w_img, ldw, 1, st));
        p->n_kernels += 2;
        const int64_t part2 = (int64_t)nsplit * chunk_px;
        PSF_TRY(p->partial.reserve((size_t)(2 * part2) * sizeof(float)));
        float *part = (float *)p->partial.p;
        cudaEvent_t ev1 = nullptr, ev2 = nullptr;
        if (p->prof) {
            if (p->prof_used == p->prof_ev.size()) {
                cudaEvent_t a, c;
                PSF_TRY(cudaEventCreate(&a));
                PSF_TRY(cudaEventCreate(&c));
                p->prof_ev.emplace_back(a, c);
            }
            ev1 = p->prof_ev[p->prof_used].first;
            ev2 = p->prof_ev[p->prof_used].second;
            p->prof_used++;
            PSF_TRY(cudaEventRecord(ev1, st));
        }
        PSF_TRY(launch_psf_tc_uvimg(p->d, w_uv, w_img, ldw, (const TcItem *)(dm + m.off_tiles), (int)items.size(),
                                    ncols_max, prec_bf16(p->opts.prec), (float)h.cell, part, chunk_px, part2,
                                    (int *)p->err.p, st));
        if (p->prof) PSF_TRY(cudaEventRecord(ev2, st));
        p->n_contract++;
        p->n_kernels++;
        PSF_TRY(launch_reduce(part, nsplit, chunk_px, d_loc, d_out, d_npix, cn, 1, out_uv, st));
        PSF_TRY(launch_reduce(part + part2, nsplit, chunk_px, d_loc, d_out, d_npix, cn, 1, out_img, st));
        p->n_kernels += 2;
    }
    return PSF_OK;
}

// Complex output: one per-cutout item per position (N <= 128, one row tile), B
// doubled into real and imaginary halves, split partials of both halves reduced in
// float64 into the cutout's N^2 real parts and the N^2 imaginary parts after them.
int run_forward_cplx(psf_plan_s *p, int method, const BatchHost &h, float *out, cudaStream_t st) {
    const int64_t K = p->nvis;
    const int chunk = (int)std::max<int64_t>(
        1, std::min<int64_t>(std::min<int64_t>(h.npos, 32768), kWeightBudget / (K * 8)));
    for (int c0 = 0; c0 < h.npos; c0 += chunk) {
        const int cn = std::min(chunk, h.npos - c0);
        std::vector<int64_t> loc(cn), out_im(cn);
        int64_t chunk_px = 0;
        int ncols_max = 32;
        std::vector<TcItem> base, items;
        for (int i = 0; i < cn; ++i) {
            const int N = h.npix[c0 + i];
            loc[i] = chunk_px;
            chunk_px += (int64_t)N * N;
            out_im[i] = h.out_off[c0 + i] + (int64_t)N * N;
            const int nc = (N + 31) / 32 * 32;
            ncols_max = std::max(ncols_max, nc);
            base.push_back(TcItem{i, N, 0, 0, nc, 0, 0, 0, loc[i]});
        }
        int nsplit = (int)std::max<int64_t>(1, std::min<int64_t>((p->nsm + cn - 1) / cn, (K + 8191) / 8192));
        const int32_t kper = (int32_t)(((K + nsplit - 1) / nsplit + 31) / 32 * 32);
        nsplit = (int)((K + kper - 1) / kper);
        for (int sp = 0; sp < nsplit; ++sp)
            for (auto it : base) {
                it.k0 = (int32_t)(sp * (int64_t)kper);
                it.k1 = (int32_t)std::min<int64_t>(K, (int64_t)(sp + 1) * kper);
                it.split = sp;
                items.push_back(it);
            }
        // metadata block: pos | npix | loc offs | out offs (real) | out offs (imaginary) | items
        const size_t off_pos = 0;
        const size_t off_npix = align_up(off_pos + cn * sizeof(float4), 16);
        const size_t off_loc = align_up(off_npix + cn * sizeof(int32_t), 16);
        const size_t off_out = align_up(off_loc + cn * sizeof(int64_t), 16);
        const size_t off_outi = align_up(off_out + cn * sizeof(int64_t), 16);
        const size_t off_items = align_up(off_outi + cn * sizeof(int64_t), 16);
        const size_t bytes = align_up(off_items + items.size() * sizeof(TcItem), 16);
        std::vector<char> blob(bytes, 0);
        std::memcpy(blob.data() + off_pos, &h.pos[c0], cn * sizeof(float4));
        std::memcpy(blob.data() + off_npix, &h.npix[c0], cn * sizeof(int32_t));
        std::memcpy(blob.data() + off_loc, loc.data(), cn * sizeof(int64_t));
        std::memcpy(blob.data() + off_out, &h.out_off[c0], cn * sizeof(int64_t));
        std::memcpy(blob.data() + off_outi, out_im.data(), cn * sizeof(int64_t));
        std::memcpy(blob.data() + off_items, items.data(), items.size() * sizeof(TcItem));
        int s = upload_meta(p, blob.data(), bytes, st);
        if (s) return s;
        char *dm = (char *)p->meta.p;
        const float4 *d_pos = (const float4 *)(dm + off_pos);
        const int32_t *d_npix = (const int32_t *)(dm + off_npix);
        const int64_t *d_loc = (const int64_t *)(dm + off_loc);
        const int64_t ldw = (K + 31) / 32 * 32;
        PSF_TRY(p->wbuf.reserve((size_t)(cn * ldw + 64) * sizeof(float2)));
        float2 *w = (float2 *)p->wbuf.p;
        PSF_TRY(launch_weights(p->d, method, p->opts.flags, d_pos, cn, 0, (int32_t)K, w, ldw, 1, st));
        p->n_kernels++;
        const int64_t part2 = (int64_t)nsplit * chunk_px;
        PSF_TRY(p->partial.reserve((size_t)(2 * part2) * sizeof(float)));
        float *part = (float *)p->partial.p;
        cudaEvent_t ev1 = nullptr, ev2 = nullptr;
        if (p->prof) {
            if (p->prof_used == p->prof_ev.size()) {
                cudaEvent_t a, c;
                PSF_TRY(cudaEventCreate(&a));
                PSF_TRY(cudaEventCreate(&c));
                p->prof_ev.emplace_back(a, c);
            }
            ev1 = p->prof_ev[p->prof_used].first;
            ev2 = p->prof_ev[p->prof_used].second;
            p->prof_used++;
            PSF_TRY(cudaEventRecord(ev1, st));
        }
        PSF_TRY(launch_psf_tc_cplx(p->d, w, ldw, (const TcItem *)(dm + off_items), (int)items.size(), ncols_max,
                                   prec_bf16(p->opts.prec), (float)h.cell, part, chunk_px, part2,
                                   (int *)p->err.p, st));
        if (p->prof) PSF_TRY(cudaEventRecord(ev2, st));
        p->n_contract++;
        p->n_kernels++;
        PSF_TRY(launch_reduce(part, nsplit, chunk_px, d_loc, (const int64_t *)(dm + off_out), d_npix, cn, 1, out, st));
        PSF_TRY(launch_reduce(part + part2, nsplit, chunk_px, d_loc, (const int64_t *)(dm + off_outi), d_npix, cn, 1,
                              out, st));
        p->n_kernels += 2;
    }
    return PSF_OK;
}

// Tables of the gridded image-plane form (Eq. 45, Algorithm 1) for one (N, cell,
// precision), built on first use and kept by the plan: the effective PSF through the
// visibility-level path (Method 2 at the phase centre, where every decorrelation is 1),
// its FP64 DFT, the per-cell mean intervals and fractional bandwidths, and the table.
// The build synchronizes the stream (its temporaries are released on return).
int grid_tables(psf_plan_s *p, int N, double cell, cudaStream_t st, const float4 **G) {
    for (auto &g : p->grids)
        if (g->N == N && g->cell == cell && g->prec == p->opts.prec) {
            *G = (const float4 *)g->G.p;
            return PSF_OK;
        }
    std::unique_ptr<psf_plan_s::Grid> g(new (std::nothrow) psf_plan_s::Grid());
    if (!g) return PSF_ENOMEM;
    g->N = N;
    g->cell = cell;
    g->prec = p->opts.prec;
    const int64_t NN = (int64_t)N * N;
    DevBuf P, Y, S, acc;
    PSF_TRY(P.reserve(NN * sizeof(float)));
    PSF_TRY(Y.reserve(NN * sizeof(double2)));
    PSF_TRY(S.reserve(NN * sizeof(double2)));
    PSF_TRY(acc.reserve((3 * NN + 3) * sizeof(double)));
    PSF_TRY(g->G.reserve(NN * sizeof(float4)));
    const double lm0[2] = {0.0, 0.0};
    psf_batch_t b0{};
    b0.npos = 1;
    b0.lm = lm0;
    b0.npix0 = N;
    b0.cell_rad = cell;
    int s = run_forward(p, kImg, &b0, (float *)P.p, st);
    if (s) return s;
    double *accp = (double *)acc.p;
    PSF_TRY(launch_grid_dft((const float *)P.p, (double2 *)Y.p, (double2 *)S.p, N, st));
    PSF_TRY(cudaMemsetAsync(accp, 0, (3 * NN + 3) * sizeof(double), st));
    PSF_TRY(launch_grid_cells((const double2 *)p->bin_uv64.p, (const int2 *)p->bin_samp.p,
                              (const int32_t *)p->bin_first.p, (const double2 *)p->chan64.p, p->d.W, p->nbl, p->nout,
                              p->dt_raw, N, (double)N * cell, accp, accp + 3 * NN, st));
    PSF_TRY(launch_grid_table((const double2 *)S.p, accp, accp + 3 * NN, N, 1.0 / ((double)N * cell),
                              (float4 *)g->G.p, st));
    if (p->prof) p->n_kernels += 4;
    PSF_TRY(cudaStreamSynchronize(st));
    *G = (const float4 *)g->G.p;
    p->grids.push_back(std::move(g));
    return PSF_OK;
}

int run_img_grid(psf_plan_s *p, const psf_batch_t *b, float *out, cudaStream_t st) {
    if (p->opts.flags & PSF_COMPLEX_OUT) return PSF_EUNSUPPORTED;
    BatchHost h;
    int s = prepare_batch(p, b, h, 4096);
    if (s) return s;
    if (h.npos == 0) return PSF_OK;
    for (int i = 0; i < h.npos; ++i)
        if (!img_grid_supported(h.npix[i])) return PSF_EUNSUPPORTED;
    const bool literal = (p->opts.flags & PSF_IMG_LITERAL_THETA) != 0;
    // Algorithm 1's A = alpha (c.x a' + c.y b'): (m0, -l0) with theta = atan2(v, u), (-l0, m0)
    // with the literal arctan(u/v) (the sign of A does not matter to the sinc)
    auto coef = [&](int i) {
        const double l0 = b->lm[2 * i], m0 = b->lm[2 * i + 1];
        const float rho = (float)std::sqrt(l0 * l0 + m0 * m0);
        return literal ? make_float4((float)-l0, (float)m0, rho, 0.f) : make_float4((float)m0, (float)-l0, rho, 0.f);
    };
    static const int kSizes[] = {16, 32, 64, 128};
    std::vector<GridPos> gpos;
    int start[4] = {0, 0, 0, 0}, count[4] = {0, 0, 0, 0};
    const float4 *G[4] = {nullptr, nullptr, nullptr, nullptr};
    for (int t = 0; t < 4; ++t) {
        start[t] = (int)gpos.size();
        for (int i = 0; i < h.npos; ++i)
            if (h.npix[i] == kSizes[t]) {
                GridPos g{};
                g.c = coef(i);
                g.off = h.out_off[i];
                gpos.push_back(g);
            }
        count[t] = (int)gpos.size() - start[t];
        if (count[t] && (s = grid_tables(p, kSizes[t], h.cell, st, &G[t]))) return s;
    }
    if ((s = upload_meta(p, gpos.data(), gpos.size() * sizeof(GridPos), st))) return s;
    for (int t = 0; t < 4; ++t) {
        if (!count[t]) continue;
        cudaEvent_t ev1 = nullptr, ev2 = nullptr;
        if (p->prof) {
            if (p->prof_used == p->prof_ev.size()) {
                cudaEvent_t a, e2;
                PSF_TRY(cudaEventCreate(&a));
                PSF_TRY(cudaEventCreate(&e2));
                p->prof_ev.emplace_back(a, e2);
            }
            ev1 = p->prof_ev[p->prof_used].first;
            ev2 = p->prof_ev[p->prof_used].second;
            p->prof_used++;
            PSF_TRY(cudaEventRecord(ev1, st));
        }
        PSF_TRY(launch_img_grid(G[t], (const GridPos *)p->meta.p + start[t], count[t], kSizes[t], out, p->nsm, st));
        if (p->prof) PSF_TRY(cudaEventRecord(ev2, st));
        p->n_contract++;
        p->n_kernels++;
    }
    return PSF_OK;
}

// Hogbom CLEAN with position-dependent PSFs (Algorithm 2).  With the gridded PSF every
// step of an iteration is a kernel reading the device loop record (k_clean.cu), queued in
// chunks; the other methods read the peak record back to place the cutout.
int run_clean(psf_plan_s *p, const psf_clean_t *c, float *res, float *model, int32_t *cpix, float *cflux,
              int32_t *niter_out, cudaStream_t st) {
    if (!c || !res) return PSF_EINVAL;
    if (c->nl < 2 || c->nm < 2 || (c->nl & 1) || (c->nm & 1) || !(c->cell_rad > 0.0) || !(c->gain > 0.f) ||
        !(c->gain <= 1.f) || c->max_iter < 0)
        return PSF_EINVAL;
    const int N = c->psf_npix;
    if (N < 2 || N > 4096 || (N & 1)) return PSF_EINVAL;
    if (c->method < kExact || c->method > PSF_METHOD_IMG_GRID) return PSF_EINVAL;
    if (!std::isfinite(c->l_c) || !std::isfinite(c->m_c)) return PSF_EINVAL;
    if ((int64_t)c->nl * c->nm >= (int64_t(1) << 31)) return PSF_EUNSUPPORTED;
    if (p->opts.flags & PSF_COMPLEX_OUT) return PSF_EUNSUPPORTED;
    if (c->method == PSF_METHOD_IMG_GRID && !img_grid_supported(N)) return PSF_EUNSUPPORTED;
    if (c->options & ~PSF_CLEAN_FACET_PSF) return PSF_EINVAL;
    const bool facet = (c->options & PSF_CLEAN_FACET_PSF) != 0;
    if (niter_out) *niter_out = 0;
    if (c->max_iter == 0) return PSF_OK;
    const size_t ws_bytes = sizeof(CleanState) + 2 * sizeof(unsigned long long);
    DevBuf ws, P;
    PSF_TRY(ws.reserve(ws_bytes));
    PSF_TRY(P.reserve((size_t)N * N * sizeof(float)));
    PSF_TRY(cudaMemsetAsync(ws.p, 0, ws_bytes, st));
    CleanState *sd = (CleanState *)ws.p;
    unsigned long long *key = (unsigned long long *)((char *)ws.p + sizeof(CleanState));
    const int literal = (p->opts.flags & PSF_IMG_LITERAL_THETA) ? 1 : 0;
    const int64_t npx = (int64_t)c->nl * c->nm;
    CleanState h{};
    int64_t t = 0;
    if (facet || c->method == PSF_METHOD_IMG_GRID) {
        // every step of an iteration on the device: the PSF at the image centre once
        // (facet), or the gridded PSF at each peak from the kept table
        const float4 *G = nullptr;
        if (facet) {
            double lm[2] = {c->l_c, c->m_c};
            psf_batch_t b{};
            b.npos = 1;
            b.lm = lm;
            b.npix0 = N;
            b.cell_rad = c->cell_rad;
            int s = c->method == PSF_METHOD_IMG_GRID ? run_img_grid(p, &b, (float *)P.p, st)
                                                     : run_forward(p, c->method, &b, (float *)P.p, st);
            if (s) return s;
        } else {
            int s = grid_tables(p, N, c->cell_rad, st, &G);
            if (s) return s;
        }
        // one chunk of kChunk iterations; kChunk is even, so the alternating argmax keys
        // repeat identically in every chunk
        constexpr int kChunk = 64;
        const int per_iter = facet ? 3 : 4;
        auto chunk = [&](cudaStream_t cs) -> cudaError_t {
            for (int q = 0; q < kChunk; ++q) {
                cudaError_t e = launch_clean_argmax(res, npx, sd, key + (q & 1), p->nsm, cs);
                if (e == cudaSuccess)
                    e = launch_clean_prep(key + (q & 1), key + ((q + 1) & 1), sd, c->nl, c->nm, c->cell_rad, c->l_c,
                                          c->m_c, c->threshold, c->max_iter, literal, cs);
                if (e == cudaSuccess && !facet) e = launch_img_grid(G, &sd->gpos, 1, N, (float *)P.p, p->nsm, cs);
                if (e == cudaSuccess)
                    e = launch_clean_sub(res, model, (const float *)P.p, sd, c->nl, c->nm, N, c->gain, cpix, cflux,
                                         cs);
                if (e != cudaSuccess) return e;
            }
            return cudaSuccess;
        };
        // the first chunk on the caller's stream (it also sets the kernels' one-time
        // attributes); the loop record is read once per chunk
        PSF_TRY(chunk(st));
        if (p->prof) p->n_kernels += per_iter * kChunk;
        PSF_TRY(cudaMemcpyAsync(&h, sd, sizeof(h), cudaMemcpyDeviceToHost, st));
        PSF_TRY(cudaStreamSynchronize(st));
        if (!h.done) {
            // later chunks: the same launches captured once into a CUDA graph and replayed on
            // a private stream (the caller's stream has drained; the call returns after the
            // private stream does)
            cudaStream_t cs = nullptr;
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ge = nullptr;
            cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
            if (e == cudaSuccess) {
                const cudaError_t ec = chunk(cs);
                e = cudaStreamEndCapture(cs, &g);
                if (ec != cudaSuccess) e = ec;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
            while (e == cudaSuccess) {
                e = cudaGraphLaunch(ge, cs);
                if (e == cudaSuccess) e = cudaMemcpyAsync(&h, sd, sizeof(h), cudaMemcpyDeviceToHost, cs);
                if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
                if (p->prof) p->n_kernels += per_iter * kChunk;
                if (e == cudaSuccess && h.done) break;
            }
            if (ge) cudaGraphExecDestroy(ge);
            if (g) cudaGraphDestroy(g);
            if (cs) cudaStreamDestroy(cs);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return cuda_status(e);
            }
        }
    } else {
        double lm[2] = {0.0, 0.0};
        psf_batch_t b{};
        b.npos = 1;
        b.lm = lm;
        b.npix0 = N;
        b.cell_rad = c->cell_rad;
        for (;; ++t) {
            PSF_TRY(launch_clean_argmax(res, npx, sd, key + (t & 1), p->nsm, st));
            PSF_TRY(launch_clean_prep(key + (t & 1), key + ((t + 1) & 1), sd, c->nl, c->nm, c->cell_rad,
                                      c->l_c, c->m_c, c->threshold, c->max_iter, literal, st));
            if (p->prof) p->n_kernels += 2;
            PSF_TRY(cudaMemcpyAsync(&h, sd, sizeof(h), cudaMemcpyDeviceToHost, st));
            PSF_TRY(cudaStreamSynchronize(st));
            if (!h.active) break;
            const int x = h.pix % c->nl, y = h.pix / c->nl;
            lm[0] = c->l_c + (x - c->nl / 2) * c->cell_rad;
            lm[1] = c->m_c + (y - c->nm / 2) * c->cell_rad;
            int s = run_forward(p, c->method, &b, (float *)P.p, st);
            if (s) return s;
            PSF_TRY(launch_clean_sub(res, model, (const float *)P.p, sd, c->nl, c->nm, N, c->gain, cpix, cflux, st));
            if (p->prof) p->n_kernels += 1;
        }
    }
    if (niter_out) *niter_out = h.iter;
    return PSF_OK;
}

}  // namespace

namespace {

struct AdjPosHost {
    float4 L, dLl, dLm;
};

AdjPosHost adj_pos(const psf_plan_s *p, const BatchHost &h, const psf_batch_t *b, int i) {
    const double l0 = b->lm[2 * i], m0 = b->lm[2 * i + 1];
    float dzl = 0.f, dzm = 0.f;
    if (p->opts.flags & PSF_WTERM) {   // d(n0 - 1)/dl0 = -l0 / n0
        const double n0 = std::sqrt(1.0 - l0 * l0 - m0 * m0);
        dzl = (float)(-l0 / n0);
        dzm = (float)(-m0 / n0);
    }
    AdjPosHost a;
    a.L = h.pos[i];
    a.dLl = make_float4(1.f, 0.f, dzl, 0.f);
    a.dLm = make_float4(0.f, 1.f, dzm, 0.f);
    return a;
}

constexpr size_t kAdjHBudget = size_t(4) << 30;   // H of one visibility chunk (bytes)

// Tensor-core adjoint (single-pass FP16/BF16 plans, cutouts of a multiple of 32 pixels):
// per size group and chunk of at most adj_fold_max_pos() positions, R as 16-bit rows, H by
// tcgen05 per visibility chunk, then the decorrelation gradients and the reductions.
int run_adjoint_tc(psf_plan_s *p, int method, const psf_batch_t *b, const BatchHost &h, const float *dLdP,
                   double *dLdlm, float *dLdW, cudaStream_t st) {
    const int64_t K = p->nvis;
    const int bf16 = prec_bf16(p->opts.prec);
    std::vector<std::vector<int>> groups(1025);
    for (int i = 0; i < h.npos; ++i) groups[h.npix[i]].push_back(i);
    bool wrote_W = false;
    for (int N = 32; N <= 1024; N += 32) {
        const std::vector<int> &g = groups[N];
        for (size_t c0 = 0; c0 < g.size(); c0 += (size_t)adj_fold_max_pos()) {
            const int np = (int)std::min<size_t>(g.size() - c0, (size_t)adj_fold_max_pos());
            const int rows = (np + 127) / 128 * 128;
            const int64_t n2 = (int64_t)N * N;
            std::vector<AdjPosHost> ap(np);
            std::vector<int64_t> offs(np);
            std::vector<int32_t> idx(np);
            for (int q = 0; q < np; ++q) {
                const int i = g[c0 + q];
                ap[q] = adj_pos(p, h, b, i);
                offs[q] = h.out_off[i];
                idx[q] = i;
            }
            const size_t off_pos = 0;
            const size_t off_offs = align_up(off_pos + np * sizeof(AdjPosHost), 16);
            const size_t off_idx = align_up(off_offs + np * sizeof(int64_t), 16);
            const size_t bytes = align_up(off_idx + np * sizeof(int32_t), 16);
            std::vector<char> blob(bytes, 0);
            std::memcpy(blob.data() + off_pos, ap.data(), np * sizeof(AdjPosHost));
            std::memcpy(blob.data() + off_offs, offs.data(), np * sizeof(int64_t));
            std::memcpy(blob.data() + off_idx, idx.data(), np * sizeof(int32_t));
            int s = upload_meta(p, blob.data(), bytes, st);
            if (s) return s;
            char *dm = (char *)p->meta.p;
            PSF_TRY(p->w16.reserve((size_t)rows * n2 * 2));
            PSF_TRY(launch_adj_r16(dLdP, (const int64_t *)(dm + off_offs), np, rows, (int)n2, bf16, p->w16.p, st));
            CUtensorMapStub rmap;
            if ((s = make_weight_map(&rmap, p->w16.p, bf16, n2, rows))) return s;
            int64_t Kc = (int64_t)(kAdjHBudget / ((size_t)rows * sizeof(float2))) / 128 * 128;
            Kc = std::max<int64_t>(128, std::min<int64_t>(Kc, (K + 127) / 128 * 128));
            const int64_t ldh = Kc;
            PSF_TRY(p->wbuf.reserve((size_t)rows * ldh * sizeof(float2)));
            PSF_TRY(p->partial.reserve((size_t)adj_fold_blocks(p->nsm) * np * 2 * sizeof(double)));
            for (int64_t kc0 = 0; kc0 < K; kc0 += Kc) {
                const int64_t kcn = std::min<int64_t>(Kc, K - kc0);
                cudaEvent_t ev1 = nullptr, ev2 = nullptr;
                if (p->prof) {
                    if (p->prof_used == p->prof_ev.size()) {
                        cudaEvent_t a, e2;
                        PSF_TRY(cudaEventCreate(&a));
                        PSF_TRY(cudaEventCreate(&e2));
                        p->prof_ev.emplace_back(a, e2);
                    }
                    ev1 = p->prof_ev[p->prof_used].first;
                    ev2 = p->prof_ev[p->prof_used].second;
                    p->prof_used++;
                    PSF_TRY(cudaEventRecord(ev1, st));
                }
                PSF_TRY(launch_adj_tc(&rmap, rows / 128, (int)((kcn + 127) / 128), N, p->d.uv, (int32_t)kc0,
                                      (int32_t)kcn, (float)h.cell, (float2 *)p->wbuf.p, ldh, bf16, p->nsm,
                                      (int *)p->err.p, st));
                if (p->prof) PSF_TRY(cudaEventRecord(ev2, st));
                p->n_contract++;
                PSF_TRY(launch_adj_fold(p->d, method, p->opts.flags, dm + off_pos, np, (const float2 *)p->wbuf.p, ldh,
                                        (int32_t)kc0, (int32_t)kcn, dLdW, wrote_W ? 1 : 0, (double *)p->partial.p,
                                        (const int32_t *)(dm + off_idx), dLdlm, kc0 > 0 ? 1 : 0, 1, p->nsm, st));
                p->n_kernels += 4;
            }
            wrote_W = dLdW != nullptr;
        }
    }
    return PSF_OK;
}

}  // namespace

extern "C" {

int psf_approx_img_grid(psf_plan_t p, const psf_batch_t *b, float *out, void *stream) {
    if (!p || !out) return PSF_EINVAL;
    return run_img_grid(p, b, out, (cudaStream_t)stream);
}

int psf_clean(psf_plan_t p, const psf_clean_t *cfg, float *residual, float *model, int32_t *comp_pix,
              float *comp_flux, int32_t *niter_out, void *stream) {
    if (!p) return PSF_EINVAL;
    return run_clean(p, cfg, residual, model, comp_pix, comp_flux, niter_out, (cudaStream_t)stream);
}

int psf_fwhm(psf_plan_t p, const psf_batch_t *b, const float *cutouts_dev, double *fwhm_dev, void *stream) {
    if (!p || !cutouts_dev || !fwhm_dev) return PSF_EINVAL;
    BatchHost h;
    int s = prepare_batch(p, b, h, 4096);
    if (s) return s;
    if (h.npos == 0) return PSF_OK;
    std::vector<FwhmItem> items((size_t)h.npos);
    for (int i = 0; i < h.npos; ++i) {
        const double l0 = b->lm[2 * i], m0 = b->lm[2 * i + 1], rho = std::sqrt(l0 * l0 + m0 * m0);
        if (h.npix[i] < 4) return PSF_EINVAL;
        items[i].er_x = rho > 0 ? (float)(l0 / rho) : 1.f;
        items[i].er_y = rho > 0 ? (float)(m0 / rho) : 0.f;
        items[i].N = h.npix[i];
        items[i].pad = 0;
        items[i].off = h.out_off[i];
    }
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = upload_meta(p, items.data(), items.size() * sizeof(FwhmItem), st))) return s;
    PSF_TRY(launch_fwhm(cutouts_dev, (const FwhmItem *)p->meta.p, h.npos, h.cell, fwhm_dev, st));
    if (p->prof) p->n_kernels++;
    return PSF_OK;
}

int psf_img_grid_table(psf_plan_t p, int npix, double cell_rad, float *table_dev, void *stream) {
    if (!p || !table_dev || !(cell_rad > 0.0)) return PSF_EINVAL;
    if (!img_grid_supported(npix)) return PSF_EUNSUPPORTED;
    cudaStream_t st = (cudaStream_t)stream;
    const float4 *G = nullptr;
    int s = grid_tables(p, npix, cell_rad, st, &G);
    if (s) return s;
    PSF_TRY(cudaMemcpyAsync(table_dev, G, (size_t)npix * npix * sizeof(float4), cudaMemcpyDeviceToDevice, st));
    return PSF_OK;
}

int psf_exact(psf_plan_t p, const psf_batch_t *b, float *out, void *stream) {
    return run_forward(p, kExact, b, out, (cudaStream_t)stream);
}
int psf_approx_uv(psf_plan_t p, const psf_batch_t *b, float *out, void *stream) {
    return run_forward(p, kUV, b, out, (cudaStream_t)stream);
}
int psf_approx_img(psf_plan_t p, const psf_batch_t *b, float *out, void *stream) {
    return run_forward(p, kImg, b, out, (cudaStream_t)stream);
}
int psf_approx_uv_img(psf_plan_t p, const psf_batch_t *b, float *out_uv, float *out_img, void *stream) {
    return run_forward_uvimg(p, b, out_uv, out_img, (cudaStream_t)stream);
}

int psf_adjoint(psf_plan_t p, int method, const psf_batch_t *b, const float *dLdP, double *dLdlm, float *dLdW,
                void *stream) {
    if (!p || !dLdP || !dLdlm) return PSF_EINVAL;
    if (method < 0 || method > 2) return PSF_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    // the tensor-core adjoint takes single-pass FP16/BF16 plans whose cutouts are all
    // multiples of 32 pixels (up to 1024); the FP32 CUDA-core adjoint everything else
    const bool tc1 = p->opts.prec == PSF_TC_FP16 || p->opts.prec == PSF_TC_BF16;
    BatchHost h;
    int s = prepare_batch(p, b, h, tc1 ? 1024 : adjoint_max_n());
    if (s) return s;
    if (h.npos == 0) {
        if (dLdW) PSF_TRY(cudaMemsetAsync(dLdW, 0, p->nvis * sizeof(float), st));
        return PSF_OK;
    }
    bool use_tc = tc1;
    int nmax_all = 0;
    for (int i = 0; i < h.npos; ++i) {
        use_tc = use_tc && h.npix[i] % 32 == 0;
        nmax_all = std::max(nmax_all, (int)h.npix[i]);
    }
    if (use_tc) return run_adjoint_tc(p, method, b, h, dLdP, dLdlm, dLdW, st);
    if (nmax_all > adjoint_max_n()) return PSF_EUNSUPPORTED;
    const int64_t ncta = adjoint_ctas(p->nvis);
    const int64_t budget = int64_t(512) << 20;
    const int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(h.npos, budget / (ncta * 16)));
    for (int c0 = 0; c0 < h.npos; c0 += chunk) {
        const int cn = std::min(chunk, h.npos - c0);
        int nmax = 2;
        std::vector<AdjPosHost> ap(cn);
        for (int i = 0; i < cn; ++i) {
            ap[i] = adj_pos(p, h, b, c0 + i);
            nmax = std::max(nmax, (int)h.npix[c0 + i]);
        }
        const size_t off_pos = 0;
        const size_t off_npix = align_up(off_pos + cn * sizeof(AdjPosHost), 16);
        const size_t off_offs = align_up(off_npix + cn * sizeof(int32_t), 16);
        const size_t bytes = align_up(off_offs + cn * sizeof(int64_t), 16);
        std::vector<char> blob(bytes, 0);
        std::memcpy(blob.data() + off_pos, ap.data(), cn * sizeof(AdjPosHost));
        std::memcpy(blob.data() + off_npix, &h.npix[c0], cn * sizeof(int32_t));
        std::memcpy(blob.data() + off_offs, &h.out_off[c0], cn * sizeof(int64_t));
        if ((s = upload_meta(p, blob.data(), bytes, st))) return s;
        char *dm = (char *)p->meta.p;
        PSF_TRY(p->partial.reserve((size_t)ncta * cn * 2 * sizeof(double)));
        PSF_TRY(launch_adjoint_chunk(p->d, method, p->opts.flags, dm + off_pos, (const int32_t *)(dm + off_npix),
                                     (const int64_t *)(dm + off_offs), cn, nmax, h.cell, dLdP, dLdW,
                                     c0 > 0, (double *)p->partial.p, dLdlm + 2 * c0, st));
        p->n_kernels += 2;
    }
    return PSF_OK;
}

int psf_profile_enable(psf_plan_t p, int enable) {
    if (!p) return PSF_EINVAL;
    p->prof = enable != 0;
    return PSF_OK;
}

int psf_profile_read(psf_plan_t p, double *ms, int64_t *ncontract, int64_t *nkernels) {
    if (!p) return PSF_EINVAL;
    double tot = 0.0;
    for (size_t i = 0; i < p->prof_used; ++i) {
        float t = 0.f;
        PSF_TRY(cudaEventSynchronize(p->prof_ev[i].second));
        PSF_TRY(cudaEventElapsedTime(&t, p->prof_ev[i].first, p->prof_ev[i].second));
        tot += t;
    }
    if (ms) *ms = tot;
    if (ncontract) *ncontract = p->n_contract;
    if (nkernels) *nkernels = p->n_kernels;
    p->prof_used = 0;
    p->n_contract = 0;
    p->n_kernels = 0;
    return PSF_OK;
}

}  // extern "C"

// Read-only views of a plan for other translation units of the library.
namespace psf {
const DevObs *plan_devobs(psf_plan_t p) { return p ? &p->d : nullptr; }
uint32_t plan_flags(psf_plan_t p) { return p ? p->opts.flags : 0u; }
int plan_device(psf_plan_t p) { return p ? p->device : -1; }
}  // namespace psf

extern "C" {

int psf_selftest_timeout(int limit_ms) {
    if (limit_ms < 1 || limit_ms > 10000) return PSF_EINVAL;
    return selftest_timeout(limit_ms);
}

int psf_selftest_fma_rate(int packed, double *flops_per_s) {
    if (!flops_per_s || (packed != 0 && packed != 1)) return PSF_EINVAL;
    return selftest_fma_rate(packed, flops_per_s);
}

int psf_selftest_umma(const void *a, const void *b, float *d, int n) {
    if (!a || !b || !d || n < 16 || n > 256 || (n % 16)) return PSF_EINVAL;
    return selftest_umma(a, b, d, n);
}

}  // extern "C"
