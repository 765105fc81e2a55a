// Per-visibility decorrelation D_k(l0) on the device (float32), and its gradient.
//
// All phases are formed difference-first: the centre-visibility phase u_k . L0
// (thousands of turns) cancels analytically against the cutout centring, so only
// small quantities (sample offsets from the bin mean, channel offsets from the
// bin centre, sinc arguments) are ever evaluated.  sinpif / sincospif are CUDA's
// own functions; sinc, the Dirichlet kernel and their derivatives are written out
// from their definitions here.
#pragma once

#include "psf_internal.cuh"

namespace psf {

constexpr float kInvC = (float)(1.0 / kCLight);
constexpr float kPiF = 3.14159265358979f;

// sinc_pi(y) = sin(pi y) / (pi y), 1 at y = 0.
__device__ __forceinline__ float sincpi(float y) {
    return y == 0.0f ? 1.0f : sinpif(y) / (kPiF * y);
}

// d/dy sinc_pi(y) = (cos(pi y) - sinc_pi(y)) / y.  Below |pi y| = 1/2 the two
// terms cancel, so the Taylor series of d/dx (sin x / x) at x = pi y is used.
__device__ __forceinline__ float dsincpi(float y) {
    const float x = kPiF * y;
    if (fabsf(x) < 0.5f) {
        const float x2 = x * x;
        return kPiF * x * (-1.0f / 3.0f + x2 * (1.0f / 30.0f + x2 * (-1.0f / 840.0f + x2 * (1.0f / 45360.0f))));
    }
    float s, c;
    sincospif(y, &s, &c);
    return (c - s / x) / y;
}

// Mean of exp(-2 pi i (c - (F-1)/2) a) over c = 0..F-1, i.e. the Dirichlet kernel
// sin(pi F a) / (F sin(pi a)).  a is split as n + r with |r| <= 1/2 so the ratio
// is taken between two small sines: sin(pi F (n+r)) = (-1)^(F n) sin(pi F r).
__device__ __forceinline__ float dirichlet(int F, float a) {
    if (F == 1) return 1.0f;
    float n = rintf(a);
    float r = a - n;
    float sgn = (((int)n * (F - 1)) & 1) ? -1.0f : 1.0f;
    if (r == 0.0f) return sgn;
    return sgn * sinpif((float)F * r) / ((float)F * sinpif(r));
}

// d/da of the Dirichlet kernel above.  With x = pi r the numerator
// F cos(F x) sin(x) - sin(F x) cos(x) cancels to O((F x)^3) for small F x; there
// the series 1 - (F^2-1) x^2 / 6 + (7/360 - F^2/36 + F^4/120) x^4 is differentiated.
__device__ __forceinline__ float ddirichlet(int F, float a) {
    if (F == 1) return 0.0f;
    float n = rintf(a);
    float r = a - n;
    float sgn = (((int)n * (F - 1)) & 1) ? -1.0f : 1.0f;
    const float Ff = (float)F, F2 = Ff * Ff;
    const float x = kPiF * r;
    if (fabsf(Ff * x) < 0.05f) {
        const float c4 = 7.0f / 360.0f - F2 / 36.0f + F2 * F2 / 120.0f;
        return sgn * kPiF * (x * (1.0f - F2) / 3.0f + 4.0f * c4 * x * x * x);
    }
    float sF, cF, s1, c1;
    sincospif(Ff * r, &sF, &cF);
    sincospif(r, &s1, &c1);
    return sgn * kPiF * (Ff * cF * s1 - sF * c1) / (Ff * s1 * s1);
}

__device__ __forceinline__ float dot3(float4 a, float4 L) { return a.x * L.x + a.y * L.y + a.z * L.z; }

// Fast variants for weights that are rounded to FP16/BF16 afterwards (tensor-core
// paths): the argument is reduced exactly to |r| <= 1/2 turn (x - rint(x)) and the
// MUFU sine/cosine (__sinf, __sincosf) is used.  Its error bound is absolute (~4e-7 on
// [-pi, pi]), so a ratio of two sines of small arguments is not taken from it: below
// |pi y| = 0.1 (sinc) and |pi F r| = 0.1 (Dirichlet) the Taylor series of the ratio is
// evaluated instead (truncation error < 3e-10); without this a sinc of a tiny argument
// came out anywhere between 0 and 1 and the Dirichlet kernel as 0/0.
__device__ __forceinline__ float sinpi_fast(float x) {   // sin(pi x)
    const float n = rintf(x * 0.5f);
    return __sinf(kPiF * (x - 2.0f * n));
}
__device__ __forceinline__ void sincospi2_fast(float x, float *s, float *c) {   // sin, cos of 2 pi x
    const float r = x - rintf(x);
    __sincosf(2.0f * kPiF * r, s, c);
}
__device__ __forceinline__ float sincpi_fast(float y) {
    const float x = kPiF * y;
    if (fabsf(x) < 0.1f) {   // sin x / x = 1 - x^2/6 + x^4/120 - ...
        const float x2 = x * x;
        return 1.0f + x2 * (-1.0f / 6.0f + x2 * (1.0f / 120.0f));
    }
    return __fdividef(sinpi_fast(y), x);   // |x| >= 0.1: the approximate quotient (2 ulp) suffices
}
__device__ __forceinline__ float dirichlet_fast(int F, float a) {
    if (F == 1) return 1.0f;
    const float n = rintf(a);
    const float r = a - n;
    const float sgn = (((int)n * (F - 1)) & 1) ? -1.0f : 1.0f;
    const float Ff = (float)F, x = kPiF * r;
    if (fabsf(Ff * x) < 0.1f) {   // sin(F x) / (F sin x) = 1 - (F^2-1) x^2/6 + (7/360 - F^2/36 + F^4/120) x^4
        const float x2 = x * x, F2 = Ff * Ff;
        return sgn * (1.0f + x2 * ((1.0f - F2) / 6.0f + x2 * (7.0f / 360.0f - F2 / 36.0f + F2 * F2 / 120.0f)));
    }
    return sgn * __fdividef(sinpi_fast(Ff * r), Ff * __sinf(x));
}

// Uniform dispatch between the accurate and the fast forms.
template <bool FAST>
__device__ __forceinline__ float sincpi_t(float y) { return FAST ? sincpi_fast(y) : sincpi(y); }
template <bool FAST>
__device__ __forceinline__ float dirichlet_t(int F, float a) { return FAST ? dirichlet_fast(F, a) : dirichlet(F, a); }
template <bool FAST>
__device__ __forceinline__ void sincospi2_t(float x, float *s, float *c) {   // sin, cos of 2 pi x
    if (FAST) sincospi2_fast(x, s, c);
    else sincospif(2.0f * x, s, c);
}

// Exact bin average (Eq. 13), centre phase removed.  With uniform channels the
// channel sum is the Dirichlet kernel times the per-channel sinc (exact identity
// for equally spaced, equally wide channels); otherwise channels are summed.  With
// windows (Eqs. 15-16) each raw sample carries its normalised time weight and each raw
// channel its normalised channel weight in place of 1/n and dnu_c / Dnu_r.
// grad (optional): d/dl0 (re, im), d/dm0 (re, im) with dL0/dl0 = dLl, dL0/dm0 = dLm.
template <bool GRAD, bool FAST = false>
__device__ __forceinline__ float2 decorr_exact(const DevObs &o, int bin, int r, float4 L, float4 dLl,
                                               float4 dLm, float4 *grad) {
    const float4 ub = o.bin_ubar[bin];
    const int2 sm = o.bin_samp[bin];
    const float4 ch = o.chan[r];
    const float Xbar = dot3(ub, L);
    float re = 0.f, im = 0.f, glr = 0.f, gli = 0.f, gmr = 0.f, gmi = 0.f;
    float Xbl = 0.f, Xbm = 0.f;
    if (GRAD) { Xbl = dot3(ub, dLl); Xbm = dot3(ub, dLm); }
    const bool win = o.win != 0;
    const float *cw = win ? o.chan_win + (int64_t)o.bin_bl[bin] * (o.nout * o.favg) + (int64_t)r * o.favg : nullptr;
    for (int s = 0; s < sm.y; ++s) {
        const float4 d = o.samp[sm.x + s];
        const float wt = win ? o.samp_w[sm.x + s] : 1.0f;
        const float ds = dot3(d, L);
        const float Xs = Xbar + ds;
        // exp(-2 pi i nu_r ds / c): the sample's offset from the bin centre
        float sn, cs;
        sincospi2_t<FAST>(-ch.x * ds * kInvC, &sn, &cs);
        float dsl = 0.f, dsm = 0.f;
        if (GRAD) { dsl = dot3(d, dLl); dsm = dot3(d, dLm); }
        if (o.uniform && !win) {
            const float a = ch.z * Xs * kInvC;
            const float y = ch.w * Xs * kInvC;
            const float dir = dirichlet_t<FAST>(o.favg, a);
            const float sc = sincpi_t<FAST>(y);
            const float f = dir * sc;
            re += cs * f;
            im += sn * f;
            if (GRAD) {
                const float df = (ddirichlet(o.favg, a) * ch.z * sc + dir * dsincpi(y) * ch.w) * kInvC;
                const float Xl = Xbl + dsl, Xm = Xbm + dsm;
                const float pl = -2.0f * kPiF * ch.x * dsl * kInvC;   // d(phase)/dl0 [rad]
                const float pm = -2.0f * kPiF * ch.x * dsm * kInvC;
                // d[(cs + i sn) f] = (cs + i sn)(i dphase f + df dX)
                glr += cs * df * Xl - sn * pl * f;
                gli += sn * df * Xl + cs * pl * f;
                gmr += cs * df * Xm - sn * pm * f;
                gmi += sn * df * Xm + cs * pm * f;
            }
        } else {
            for (int c = 0; c < o.favg; ++c) {
                const float4 rc = o.rawchan[r * o.favg + c];
                float s2, c2;
                sincospi2_t<FAST>(-rc.x * Xs * kInvC, &s2, &c2);
                const float y = rc.y * Xs * kInvC;
                const float cwt = win ? wt * cw[c] : rc.z;
                const float S = sincpi_t<FAST>(y) * cwt;
                const float er = cs * c2 - sn * s2, ei = cs * s2 + sn * c2;
                re += er * S;
                im += ei * S;
                if (GRAD) {
                    const float dS = dsincpi(y) * rc.y * kInvC * cwt;
                    const float Xl = Xbl + dsl, Xm = Xbm + dsm;
                    const float pl = -2.0f * kPiF * (ch.x * dsl + rc.x * Xl) * kInvC;
                    const float pm = -2.0f * kPiF * (ch.x * dsm + rc.x * Xm) * kInvC;
                    glr += er * dS * Xl - ei * pl * S;
                    gli += ei * dS * Xl + er * pl * S;
                    gmr += er * dS * Xm - ei * pm * S;
                    gmi += ei * dS * Xm + er * pm * S;
                }
            }
        }
    }
    const float inv = win ? 1.0f : 1.0f / (float)sm.y;
    if (GRAD) *grad = make_float4(glr * inv, gli * inv, gmr * inv, gmi * inv);
    return make_float2(re * inv, im * inv);
}

// Windowed time factor of Methods 1 and 2 (Eqs. 15-16 with the linear phase of the
// approximations): with A the phase change across the bin in turns, the bin average of
// exp(-2 pi i A tau), tau in [-1/2, 1/2] the time from the bin centre in bin lengths, when
// raw sample s of the n carries its normalised weight x_s over its own 1/n of the bin:
//   T(A) = sum_s x_s exp(-2 pi i A tau_s) sinc_pi(A / n),  tau_s = (s - (n - 1)/2) / n
// (sinc_pi(A) for x_s = 1/n).  dT: dT/dA.
template <bool GRAD, bool FAST>
__device__ __forceinline__ float2 win_time(const DevObs &o, int2 sm, float A, float2 *dT) {
    const float n = (float)sm.y;
    float sr = 0.f, si = 0.f, dr = 0.f, di = 0.f;
    for (int s = 0; s < sm.y; ++s) {
        const float xs = o.samp_w[sm.x + s];
        const float tau = ((float)s - 0.5f * (n - 1.0f)) / n;
        float sn, cs;
        sincospi2_t<FAST>(-A * tau, &sn, &cs);   // exp(-2 pi i A tau)
        sr += xs * cs;
        si += xs * sn;
        if (GRAD) {   // d/dA exp(-2 pi i A tau) = -2 pi i tau exp(...), the 2 pi applied below
            dr += xs * tau * sn;
            di -= xs * tau * cs;
        }
    }
    const float sc = sincpi_t<FAST>(A / n);
    if (GRAD) {
        const float dsc = dsincpi(A / n) / n;
        *dT = make_float2(dsc * sr + 2.0f * kPiF * sc * dr, dsc * si + 2.0f * kPiF * sc * di);
    }
    return make_float2(sc * sr, sc * si);
}

// Windowed frequency factor: with B the phase change across the output channel's band
// Dnu_r in turns, raw channel c (offset nu_c - nu_r, width dnu_c) carrying its normalised
// weight y_c (window x width) with its phase integrated over its width:
//   F(B) = sum_c y_c exp(-2 pi i B (nu_c - nu_r) / Dnu_r) sinc_pi(B dnu_c / Dnu_r).
template <bool GRAD, bool FAST>
__device__ __forceinline__ float2 win_freq(const DevObs &o, int bin, int r, float B, float2 *dF) {
    const float Dnu = o.chan[r].y;
    const float *cw = o.chan_win + (int64_t)o.bin_bl[bin] * (o.nout * o.favg) + (int64_t)r * o.favg;
    float fr = 0.f, fi = 0.f, dr = 0.f, di = 0.f;
    for (int c = 0; c < o.favg; ++c) {
        const float4 rc = o.rawchan[r * o.favg + c];
        const float yc = cw[c];
        const float nt = rc.x / Dnu, om = rc.z;
        float sn, cs;
        sincospi2_t<FAST>(-B * nt, &sn, &cs);
        const float sc = sincpi_t<FAST>(B * om);
        fr += yc * cs * sc;
        fi += yc * sn * sc;
        if (GRAD) {   // d/dB [exp(-2 pi i B nt) sc] = exp(...) (dsc - 2 pi i nt sc)
            const float dsc = dsincpi(B * om) * om;
            dr += yc * (cs * dsc + 2.0f * kPiF * nt * sn * sc);
            di += yc * (sn * dsc - 2.0f * kPiF * nt * cs * sc);
        }
    }
    if (GRAD) *dF = make_float2(dr, di);
    return make_float2(fr, fi);
}

// D = T(A) F(B) of a windowed approximation (win: bit 0 a time window, bit 1 a channel
// window; the direction without a window keeps the boxcar's sinc_pi), with the gradient
// from dA/dl0, dA/dm0, dB/dl0, dB/dm0.
template <bool GRAD, bool FAST>
__device__ __forceinline__ float2 decorr_windowed(const DevObs &o, int bin, int r, float A, float B, float Al,
                                                  float Am, float Bl, float Bm, float4 *grad) {
    float2 dT = make_float2(0.f, 0.f), dF = make_float2(0.f, 0.f);
    const float2 T = (o.win & 1) ? win_time<GRAD, FAST>(o, o.bin_samp[bin], A, &dT)
                                 : make_float2(sincpi_t<FAST>(A), 0.f);
    const float2 F = (o.win & 2) ? win_freq<GRAD, FAST>(o, bin, r, B, &dF) : make_float2(sincpi_t<FAST>(B), 0.f);
    if (GRAD) {
        if (!(o.win & 1)) dT = make_float2(dsincpi(A), 0.f);
        if (!(o.win & 2)) dF = make_float2(dsincpi(B), 0.f);
        const float2 tF = make_float2(dT.x * F.x - dT.y * F.y, dT.x * F.y + dT.y * F.x);   // dT F
        const float2 Tf = make_float2(T.x * dF.x - T.y * dF.y, T.x * dF.y + T.y * dF.x);   // T dF
        *grad = make_float4(Al * tF.x + Bl * Tf.x, Al * tF.y + Bl * Tf.y, Am * tF.x + Bm * Tf.x, Am * tF.y + Bm * Tf.y);
    }
    return make_float2(T.x * F.x - T.y * F.y, T.x * F.y + T.y * F.x);
}

// Method 1 (Eqs. 31-35): sinc_pi(dedge.L0 nu_r / c) * sinc_pi(ubar.L0 Dnu_r / c); with
// windows the window transforms T, F above in place of the two sincs.
template <bool GRAD, bool FAST = false>
__device__ __forceinline__ float2 decorr_uv(const DevObs &o, int bin, int r, float4 L, float4 dLl,
                                            float4 dLm, float4 *grad) {
    const float4 ub = o.bin_ubar[bin];
    const float4 ed = o.bin_edge[bin];
    const float4 ch = o.chan[r];
    const float A = dot3(ed, L) * ch.x * kInvC;
    const float B = dot3(ub, L) * ch.y * kInvC;
    if (o.win) {
        float Al = 0.f, Am = 0.f, Bl = 0.f, Bm = 0.f;
        if (GRAD) {
            Al = dot3(ed, dLl) * ch.x * kInvC; Am = dot3(ed, dLm) * ch.x * kInvC;
            Bl = dot3(ub, dLl) * ch.y * kInvC; Bm = dot3(ub, dLm) * ch.y * kInvC;
        }
        return decorr_windowed<GRAD, FAST>(o, bin, r, A, B, Al, Am, Bl, Bm, grad);
    }
    const float sA = sincpi_t<FAST>(A), sB = sincpi_t<FAST>(B);
    if (GRAD) {
        const float dA = dsincpi(A), dB = dsincpi(B);
        const float Al = dot3(ed, dLl) * ch.x * kInvC, Am = dot3(ed, dLm) * ch.x * kInvC;
        const float Bl = dot3(ub, dLl) * ch.y * kInvC, Bm = dot3(ub, dLm) * ch.y * kInvC;
        *grad = make_float4(dA * Al * sB + sA * dB * Bl, 0.f, dA * Am * sB + sA * dB * Bm, 0.f);
    }
    return make_float2(sA * sB, 0.0f);
}

// Method 2 (Eqs. 38-44, Algorithm 1 at the visibility's own uv point; with windows the
// window transforms in place of the two sincs):
//   (du/dt, dv/dt) = omega_E (-v, u) for theta = atan2(v, u), or the literal
//   arctan(u/v) reading when PSF_IMG_LITERAL_THETA is set;
//   D = sinc_pi(omega_E Dt (udot l0 + vdot m0)) sinc_pi((Dnu/nu) |u| |l0|).
template <bool GRAD, bool FAST = false>
__device__ __forceinline__ float2 decorr_img(const DevObs &o, int bin, int r, float4 L,
                                             uint32_t flags, float4 *grad) {
    const float4 ub = o.bin_ubar[bin];
    const float4 ch = o.chan[r];
    const float s = ch.x * kInvC;
    const float u = ub.x * s, v = ub.y * s;
    const float uvlen = sqrtf(u * u + v * v);
    float udot = -v, vdot = u;
    if (flags & PSF_IMG_LITERAL_THETA) {
        const float th = (v != 0.0f) ? atanf(u / v) : (u >= 0.0f ? 0.5f * kPiF : -0.5f * kPiF);
        float st, ct;
        sincosf(th, &st, &ct);
        udot = -uvlen * st;
        vdot = uvlen * ct;
    }
    const float wdt = (float)kOmegaE * ub.w;
    const float rho = sqrtf(L.x * L.x + L.y * L.y);
    const float fb = ch.y / ch.x * uvlen;
    const float A = wdt * (udot * L.x + vdot * L.y);
    const float B = fb * rho;
    if (o.win) {
        const float Bl = rho > 0.f ? fb * L.x / rho : 0.f, Bm = rho > 0.f ? fb * L.y / rho : 0.f;
        return decorr_windowed<GRAD, FAST>(o, bin, r, A, B, wdt * udot, wdt * vdot, Bl, Bm, grad);
    }
    const float sA = sincpi_t<FAST>(A), sB = sincpi_t<FAST>(B);
    if (GRAD) {
        const float dA = dsincpi(A), dB = dsincpi(B);
        const float Bl = rho > 0.f ? fb * L.x / rho : 0.f, Bm = rho > 0.f ? fb * L.y / rho : 0.f;
        *grad = make_float4(dA * wdt * udot * sB + sA * dB * Bl, 0.f, dA * wdt * vdot * sB + sA * dB * Bm, 0.f);
    }
    return make_float2(sA * sB, 0.0f);
}

template <bool GRAD, bool FAST = false>
__device__ __forceinline__ float2 decorr(const DevObs &o, int method, uint32_t flags, int bin, int r,
                                         float4 L, float4 dLl, float4 dLm, float4 *grad) {
    if (method == kExact) return decorr_exact<GRAD, FAST>(o, bin, r, L, dLl, dLm, grad);
    if (method == kUV) return decorr_uv<GRAD, FAST>(o, bin, r, L, dLl, dLm, grad);
    return decorr_img<GRAD, FAST>(o, bin, r, L, flags, grad);
}

}  // namespace psf
