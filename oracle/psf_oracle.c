/*
 * FP64 CPU oracle for the averaging-distorted ("smeared") PSF of Atemkeng et al.
 * (2020), "Fast algorithms to approximate the position-dependent point spread
 * function responses in radio interferometric wide-field imaging".
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the benchmark's CPU-baseline leg load this file.  It shares no code, header or
 * table with the CUDA library; the two meet only in the seeded input generator.
 *
 * Everything here is the plain definition, evaluated term by term in double
 * precision, in the paper's order:
 *   - sampling bins and bin centres .................. Sect. 2.3, Eq. 12
 *   - exact bin average of the source fringe .......... Eq. 13 (boxcar, Eq. 14)
 *   - distorted PSF as a weighted sum over averaged
 *     visibilities ................................... Eqs. 21-23
 *   - Method 1 (uv-plane) sinc x sinc decorrelation ... Eqs. 31-35
 *   - Method 2 (image-plane) circular-track model ..... Eqs. 38-44, Algorithm 1
 *   - windowed averages (exact, Methods 1 and 2) ...... Eqs. 15-16
 *   - Method 2 gridded on the cutout's uv grid ........ Eq. 45, Algorithm 1
 *   - vector-Jacobian product of the PSF sum (adjoint)  chain rule on Eqs. 21-22
 *
 * Conventions (readings of the paper, one line each):
 *   - a source at l0 has visibility exp(-2 pi i u.l0); imaging uses exp(+2 pi i u.l) (Eq. 1)
 *   - sinc is sin(x)/x of the half phase change, i.e. sinc_pi(y) = sin(pi y)/(pi y) (Eq. 35)
 *   - raw time samples are instantaneous and averaged discretely; each raw channel
 *     is integrated continuously over its width (Eq. 13 with a discrete time axis)
 *   - the cutout pixel (N/2, N/2) is (l0, m0); pixel offsets are (i - N/2) * cell
 *   - the sum runs over the supplied baselines p<q only (no Hermitian conjugates)
 *   - with the w-term flag the direction is L0 = (l0, m0, n0 - 1), otherwise (l0, m0, 0)
 *   - Method 1 bin-edge delta: (last - first) * n / (n - 1) for n >= 2 samples,
 *     central difference of neighbouring samples for n = 1 (the paper is silent)
 *   - Method 2 uses theta = atan2(v, u) so that (du/dt, dv/dt) = omega_E (-v, u);
 *     flag bit 1 selects the literal arctan(u/v) of Algorithm 1 instead
 *   - Method 2 ignores w; its uv cell is the visibility's own (u, v) in wavelengths
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_C_LIGHT 299792458.0
#define OR_OMEGA_E 7.2921150e-5
#define OR_PI 3.14159265358979323846

#define OR_WTERM 1
#define OR_LITERAL_THETA 2

typedef struct {
    int nbl, ntime, nchan, favg;
    const double *uvw;     /* [nbl][ntime][3] metres */
    const double *time_s;  /* [ntime] */
    const double *freq;    /* [nchan] */
    const double *width;   /* [nchan] */
    const int *tavg;       /* [nbl] */
    const float *weights;  /* [nvis] or NULL */
    const float *twin;     /* time windows: per baseline tavg[b] values, concatenated, or NULL */
    const float *cwin;     /* channel windows: [nbl][favg], or NULL */
} or_obs;

/* Per averaged visibility k, everything the definitions need. */
typedef struct {
    int b, s0, n, r;       /* baseline, first raw sample, sample count, out channel */
    int64_t toff;          /* offset of the baseline's time window in or_obs.twin */
    double ubar[3];        /* bin-mean uvw [m] (Eq. 12 bin centre) */
    double dedge[3];       /* uvw(t_e) - uvw(t_s) [m] (Eq. 33 edges) */
    double nu, dnu, dt;    /* nu_r, Delta nu_r, Delta t_k */
    double W;              /* visibility weight W_pqkr (Eq. 6) */
} or_vis;

static double or_sincpi(double y) {
    if (y == 0.0) return 1.0;
    return sin(OR_PI * y) / (OR_PI * y);
}

/* d/dy sinc_pi(y) = (cos(pi y) - sinc_pi(y)) / y.  For |pi y| < 0.05 the two terms
 * cancel; there the Taylor series of d/dx (sin x / x), x = pi y, is used. */
static double or_dsincpi(double y) {
    double x = OR_PI * y;
    if (fabs(x) < 0.05) {
        double x2 = x * x;
        return OR_PI * x * (-1.0 / 3.0 + x2 * (1.0 / 30.0 + x2 * (-1.0 / 840.0 + x2 * (1.0 / 45360.0))));
    }
    return (cos(x) - sin(x) / x) / y;
}

static double or_dt(const or_obs *o) {
    if (o->ntime < 2) return 0.0;
    return (o->time_s[o->ntime - 1] - o->time_s[0]) / (double)(o->ntime - 1);
}

int64_t or_nvis(int nbl, int ntime, int nchan, int favg, const int *tavg) {
    if (favg <= 0 || nchan % favg) return -1;
    int64_t nb = 0;
    for (int b = 0; b < nbl; ++b) {
        if (tavg[b] <= 0) return -1;
        nb += ntime / tavg[b];
    }
    return nb * (nchan / favg);
}

/* Enumerate averaged visibilities in the interface order: baseline, time bin,
 * output channel (innermost).  Sect. 2.3 / Eq. 12: bin k covers tavg[b]
 * consecutive raw samples and favg consecutive raw channels. */
static or_vis *or_make_vis(const or_obs *o, int64_t *nvis_out) {
    int nout = o->nchan / o->favg;
    int64_t nvis = or_nvis(o->nbl, o->ntime, o->nchan, o->favg, o->tavg);
    *nvis_out = nvis;
    if (nvis <= 0) return NULL;
    or_vis *v = (or_vis *)calloc((size_t)nvis, sizeof(or_vis));
    double dt = or_dt(o);
    int64_t k = 0;
    int64_t toff = 0;
    for (int b = 0; b < o->nbl; toff += o->tavg[b], ++b) {
        int n = o->tavg[b];
        int nbins = o->ntime / n;
        const double *ub = o->uvw + (size_t)b * o->ntime * 3;
        for (int tau = 0; tau < nbins; ++tau) {
            int s0 = tau * n;
            double mean[3] = {0, 0, 0}, edge[3] = {0, 0, 0};
            for (int s = s0; s < s0 + n; ++s)
                for (int d = 0; d < 3; ++d) mean[d] += ub[s * 3 + d];
            for (int d = 0; d < 3; ++d) mean[d] /= n;
            if (n >= 2) {
                for (int d = 0; d < 3; ++d)
                    edge[d] = (ub[(s0 + n - 1) * 3 + d] - ub[s0 * 3 + d]) * n / (double)(n - 1);
            } else if (o->ntime >= 2) {
                int sa = s0 > 0 ? s0 - 1 : s0;
                int sb = s0 < o->ntime - 1 ? s0 + 1 : s0;
                for (int d = 0; d < 3; ++d)
                    edge[d] = (ub[sb * 3 + d] - ub[sa * 3 + d]) / (double)(sb - sa);
            }
            for (int r = 0; r < nout; ++r, ++k) {
                or_vis *x = &v[k];
                x->b = b; x->s0 = s0; x->n = n; x->r = r; x->toff = toff;
                double nu = 0, dnu = 0;
                for (int c = r * o->favg; c < (r + 1) * o->favg; ++c) {
                    nu += o->freq[c];
                    dnu += o->width[c];
                }
                x->nu = nu / o->favg;
                x->dnu = dnu;
                x->dt = n * dt;
                for (int d = 0; d < 3; ++d) { x->ubar[d] = mean[d]; x->dedge[d] = edge[d]; }
                x->W = o->weights ? (double)o->weights[k] : (double)(n * o->favg);
            }
        }
    }
    return v;
}

/* Direction vector L0 and its derivatives with respect to l0 and m0. */
static void or_direction(double l0, double m0, int flags, double L[3], double dLl[3], double dLm[3]) {
    L[0] = l0; L[1] = m0; L[2] = 0.0;
    dLl[0] = 1; dLl[1] = 0; dLl[2] = 0;
    dLm[0] = 0; dLm[1] = 1; dLm[2] = 0;
    if (flags & OR_WTERM) {
        double n0 = sqrt(1.0 - l0 * l0 - m0 * m0);
        L[2] = n0 - 1.0;
        dLl[2] = -l0 / n0;
        dLm[2] = -m0 / n0;
    }
}

static double or_dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* Method 2 (Eqs. 38-44, Algorithm 1) at one uv point (u, v) [lambda] with time interval
 * dt and fractional bandwidth r = dnu / nu: the half phase changes over the bin,
 * A = dPsi / (2 pi) from the circular-track rates (Eqs. 40-41) and B = dPhi / (2 pi)
 * (Eqs. 42-43), and their derivatives with respect to l0 and m0.  w is ignored. */
static void or_img_args(double u, double v, double dt, double r, double l0, double m0, int flags,
                        double AB[6] /* A, dA/dl0, dA/dm0, B, dB/dl0, dB/dm0 */) {
    double uvlen = sqrt(u * u + v * v);
    double udot, vdot;   /* Eqs. 40-41 divided by omega_E */
    if (flags & OR_LITERAL_THETA) {
        double th = (v != 0.0) ? atan(u / v) : (u >= 0 ? OR_PI / 2 : -OR_PI / 2);
        udot = -uvlen * sin(th);
        vdot = uvlen * cos(th);
    } else {
        double th = atan2(v, u);
        udot = -uvlen * sin(th);
        vdot = uvlen * cos(th);
    }
    double rho = sqrt(l0 * l0 + m0 * m0);
    AB[0] = OR_OMEGA_E * dt * (udot * l0 + vdot * m0);        /* dPsi / (2 pi) */
    AB[1] = OR_OMEGA_E * dt * udot;
    AB[2] = OR_OMEGA_E * dt * vdot;
    AB[3] = r * uvlen * rho;                                  /* dPhi / (2 pi) */
    AB[4] = rho > 0 ? r * uvlen * l0 / rho : 0.0;
    AB[5] = rho > 0 ? r * uvlen * m0 / rho : 0.0;
}

/* Method 2 with the boxcar: D = sinc(dPsi/2) sinc(dPhi/2) and its derivatives. */
static void or_img_decorr(double u, double v, double dt, double r, double l0, double m0, int flags,
                          double *D, double *Dl, double *Dm) {
    double AB[6];
    or_img_args(u, v, dt, r, l0, m0, flags, AB);
    double sA = or_sincpi(AB[0]), sB = or_sincpi(AB[3]), dA = or_dsincpi(AB[0]), dB = or_dsincpi(AB[3]);
    *D = sA * sB;
    *Dl = dA * AB[1] * sB + sA * dB * AB[4];
    *Dm = dA * AB[2] * sB + sA * dB * AB[5];
}

/* Time factor of Methods 1 and 2 with A = dPsi / (2 pi), the phase change across the bin
 * in turns: the bin average of exp(-2 pi i A tau), tau in [-1/2, 1/2] the time from the bin
 * centre in bin lengths (Eq. 35's sinc(dPsi/2) for the boxcar).  With a time window
 * (Eqs. 15-16) raw sample s of the n carries its normalised weight x_s over its own 1/n of
 * the bin, centred at tau_s = (s - (n - 1)/2) / n, so the average is
 *   T(A) = sum_s x_s exp(-2 pi i A tau_s) sinc_pi(A / n),
 * which for x_s = 1/n is sinc_pi(A) again.  T and dT/dA as (re, im). */
static void or_time_factor(const or_obs *o, const or_vis *x, double A, double T[2], double dT[2]) {
    if (!o->twin) {
        T[0] = or_sincpi(A); T[1] = 0;
        dT[0] = or_dsincpi(A); dT[1] = 0;
        return;
    }
    double tnorm = 0;
    for (int s = 0; s < x->n; ++s) tnorm += o->twin[x->toff + s];
    double Sr = 0, Si = 0, dSr = 0, dSi = 0;
    for (int s = 0; s < x->n; ++s) {
        double xs = o->twin[x->toff + s] / tnorm;
        double tau = (s - 0.5 * (x->n - 1)) / x->n;
        double ph = -2 * OR_PI * A * tau;                 /* exp(i ph) */
        Sr += xs * cos(ph);
        Si += xs * sin(ph);
        /* d/dA exp(i ph) = -2 pi i tau exp(i ph) */
        dSr += xs * 2 * OR_PI * tau * sin(ph);
        dSi += -xs * 2 * OR_PI * tau * cos(ph);
    }
    double sc = or_sincpi(A / x->n), dsc = or_dsincpi(A / x->n) / x->n;
    T[0] = sc * Sr; T[1] = sc * Si;
    dT[0] = dsc * Sr + sc * dSr; dT[1] = dsc * Si + sc * dSi;
}

/* Frequency factor of Methods 1 and 2 with B = dPhi / (2 pi) over the output channel's band
 * Dnu_r (Eq. 35's sinc(dPhi/2) for the boxcar).  With a channel window raw channel c (centre
 * nu_c, width dnu_c) carries its normalised weight y_c (window x width) and its phase is
 * integrated over its width, the phase across the band being linear in frequency:
 *   F(B) = sum_c y_c exp(-2 pi i B (nu_c - nu_r) / Dnu_r) sinc_pi(B dnu_c / Dnu_r). */
static void or_freq_factor(const or_obs *o, const or_vis *x, double B, double F[2], double dF[2]) {
    if (!o->cwin) {
        F[0] = or_sincpi(B); F[1] = 0;
        dF[0] = or_dsincpi(B); dF[1] = 0;
        return;
    }
    const int c0 = x->r * o->favg;
    double cnorm = 0;
    for (int c = c0; c < c0 + o->favg; ++c) cnorm += (double)o->cwin[(int64_t)x->b * o->favg + (c - c0)] * o->width[c];
    F[0] = F[1] = dF[0] = dF[1] = 0;
    for (int c = c0; c < c0 + o->favg; ++c) {
        double yc = o->cwin[(int64_t)x->b * o->favg + (c - c0)] * o->width[c] / cnorm;
        double nt = (o->freq[c] - x->nu) / x->dnu, om = o->width[c] / x->dnu;
        double ph = -2 * OR_PI * B * nt;
        double cs = cos(ph), sn = sin(ph), sc = or_sincpi(B * om), dsc = or_dsincpi(B * om) * om;
        F[0] += yc * cs * sc;
        F[1] += yc * sn * sc;
        /* d/dB [exp(i ph) sc] = exp(i ph) (-2 pi i nt sc + dsc) */
        dF[0] += yc * (cs * dsc + 2 * OR_PI * nt * sn * sc);
        dF[1] += yc * (sn * dsc - 2 * OR_PI * nt * cs * sc);
    }
}

/* Decorrelation D_k(l0) and its gradient, for one averaged visibility.
 *   exact (method 0): Eq. 13 with the centre-visibility phase removed, i.e.
 *     D = (1/n) sum_s sum_c (dnu_c / Dnu_r) exp(-2 pi i (nu_c X_s - nu_r Xbar) / c)
 *                                     * sinc_pi(X_s dnu_c / c),   X = uvw . L0
 *   uv (method 1): Eq. 35, sinc(dPsi/2) sinc(dPhi/2) with dPsi from the bin-edge
 *     delta (Eq. 31) and dPhi = 2 pi ubar.L0 Dnu/c (Eq. 32)
 *   img (method 2): Eqs. 42-44 with the circular-track rates of Eqs. 40-41. */
static void or_decorr_one(const or_obs *o, const or_vis *x, int method, double l0, double m0,
                          int flags, double *Dre, double *Dim, double g[4]) {
    double L[3], dLl[3], dLm[3];
    or_direction(l0, m0, flags, L, dLl, dLm);
    double re = 0, im = 0, gl_re = 0, gl_im = 0, gm_re = 0, gm_im = 0;
    if (method == 0) {
        const double *ub = o->uvw + (size_t)x->b * o->ntime * 3;
        double Xbar = or_dot3(x->ubar, L);
        double Xbar_l = or_dot3(x->ubar, dLl), Xbar_m = or_dot3(x->ubar, dLm);
        /* windowed average (Eqs. 15-16): time weight per raw sample of the bin and
         * channel weight per raw channel, each normalised to sum 1 (a channel's weight
         * is its window value times its width); the boxcar is 1/n and dnu_c / Dnu_r */
        double tnorm = 0, cnorm = 0;
        if (o->twin)
            for (int s = 0; s < x->n; ++s) tnorm += o->twin[x->toff + s];
        if (o->cwin)
            for (int c = x->r * o->favg; c < (x->r + 1) * o->favg; ++c)
                cnorm += (double)o->cwin[(int64_t)x->b * o->favg + (c - x->r * o->favg)] * o->width[c];
        for (int s = x->s0; s < x->s0 + x->n; ++s) {
            const double *us = ub + s * 3;
            double Xs = or_dot3(us, L), Xs_l = or_dot3(us, dLl), Xs_m = or_dot3(us, dLm);
            const double ft = o->twin ? o->twin[x->toff + (s - x->s0)] / tnorm : 1.0 / x->n;
            for (int c = x->r * o->favg; c < (x->r + 1) * o->favg; ++c) {
                const double fc = o->cwin ? o->cwin[(int64_t)x->b * o->favg + (c - x->r * o->favg)] * o->width[c] / cnorm
                                          : o->width[c] / x->dnu;
                double f = ft * fc;
                double phi = (o->freq[c] * Xs - x->nu * Xbar) / OR_C_LIGHT;
                double y = Xs * o->width[c] / OR_C_LIGHT;
                double S = or_sincpi(y), dS = or_dsincpi(y) * o->width[c] / OR_C_LIGHT;
                double cp = cos(2 * OR_PI * phi), sp = -sin(2 * OR_PI * phi);  /* exp(-2 pi i phi) */
                re += f * cp * S;
                im += f * sp * S;
                /* d/dtheta [e S] = e * (-2 pi i dphi S + dS dX) */
                double phl = (o->freq[c] * Xs_l - x->nu * Xbar_l) / OR_C_LIGHT;
                double phm = (o->freq[c] * Xs_m - x->nu * Xbar_m) / OR_C_LIGHT;
                /* (-2 pi i a) * (cp + i sp) = 2 pi a sp - i 2 pi a cp */
                gl_re += f * (2 * OR_PI * phl * sp * S + cp * dS * Xs_l);
                gl_im += f * (-2 * OR_PI * phl * cp * S + sp * dS * Xs_l);
                gm_re += f * (2 * OR_PI * phm * sp * S + cp * dS * Xs_m);
                gm_im += f * (-2 * OR_PI * phm * cp * S + sp * dS * Xs_m);
            }
        }
    } else {
        /* Methods 1 and 2: D = T(A) F(B), the time and frequency factors of the bin with the
         * half phase changes A = dPsi / (2 pi) and B = dPhi / (2 pi):
         *   Method 1 (Eqs. 31-35): A from the bin-edge uvw delta at nu_r, B from the bin
         *   centre across the band Dnu_r;
         *   Method 2 (Eqs. 38-44): A, B of the circular-track model at the visibility's uv. */
        double AB[6];
        if (method == 1) {
            AB[0] = or_dot3(x->dedge, L) * x->nu / OR_C_LIGHT;
            AB[1] = or_dot3(x->dedge, dLl) * x->nu / OR_C_LIGHT;
            AB[2] = or_dot3(x->dedge, dLm) * x->nu / OR_C_LIGHT;
            AB[3] = or_dot3(x->ubar, L) * x->dnu / OR_C_LIGHT;
            AB[4] = or_dot3(x->ubar, dLl) * x->dnu / OR_C_LIGHT;
            AB[5] = or_dot3(x->ubar, dLm) * x->dnu / OR_C_LIGHT;
        } else {
            double u = x->ubar[0] * x->nu / OR_C_LIGHT, v = x->ubar[1] * x->nu / OR_C_LIGHT;
            or_img_args(u, v, x->dt, x->dnu / x->nu, l0, m0, flags, AB);
        }
        double T[2], dT[2], F[2], dF[2];
        or_time_factor(o, x, AB[0], T, dT);
        or_freq_factor(o, x, AB[3], F, dF);
        re = T[0] * F[0] - T[1] * F[1];
        im = T[0] * F[1] + T[1] * F[0];
        /* dD = dT/dA dA F + T dF/dB dB */
        for (int q = 0; q < 2; ++q) {
            const double a = AB[1 + q], b = AB[4 + q];
            const double gr = a * (dT[0] * F[0] - dT[1] * F[1]) + b * (T[0] * dF[0] - T[1] * dF[1]);
            const double gi = a * (dT[0] * F[1] + dT[1] * F[0]) + b * (T[0] * dF[1] + T[1] * dF[0]);
            if (q == 0) { gl_re = gr; gl_im = gi; } else { gm_re = gr; gm_im = gi; }
        }
    }
    *Dre = re; *Dim = im;
    if (g) { g[0] = gl_re; g[1] = gl_im; g[2] = gm_re; g[3] = gm_im; }
}

#define OR_OBS_ARGS int nbl, int ntime, int nchan, int favg, const double *uvw, const double *time_s, \
    const double *freq, const double *width, const int *tavg, const float *weights, const float *twin, \
    const float *cwin
#define OR_OBS_INIT {nbl, ntime, nchan, favg, uvw, time_s, freq, width, tavg, weights, twin, cwin}

/* Per-visibility table: u,v,w [lambda] at nu_r, nu_r, Dnu_r, Dt_k, W_k, bin-mean uvw [m],
 * bin-edge delta [m].  Row layout: 13 doubles. */
int or_vis_table(OR_OBS_ARGS, double *out) {
    or_obs o = OR_OBS_INIT;
    int64_t nvis;
    or_vis *v = or_make_vis(&o, &nvis);
    if (!v) return -1;
    for (int64_t k = 0; k < nvis; ++k) {
        double *row = out + k * 13;
        for (int d = 0; d < 3; ++d) row[d] = v[k].ubar[d] * v[k].nu / OR_C_LIGHT;
        row[3] = v[k].nu; row[4] = v[k].dnu; row[5] = v[k].dt; row[6] = v[k].W;
        for (int d = 0; d < 3; ++d) { row[7 + d] = v[k].ubar[d]; row[10 + d] = v[k].dedge[d]; }
    }
    free(v);
    return 0;
}

/* D_k(l0, m0) for every averaged visibility (and optionally dD/dl0, dD/dm0). */
int or_decorr(OR_OBS_ARGS, int method, double l0, double m0, int flags,
              double *D_re, double *D_im, double *dD /* [nvis][4] or NULL */) {
    or_obs o = OR_OBS_INIT;
    int64_t nvis;
    or_vis *v = or_make_vis(&o, &nvis);
    if (!v) return -1;
    #pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nvis; ++k)
        or_decorr_one(&o, &v[k], method, l0, m0, flags, &D_re[k], &D_im[k], dD ? dD + 4 * k : NULL);
    free(v);
    return 0;
}

/* Smeared PSF cutouts (Eqs. 21-22 with the averaged fringe of Eq. 13 and the
 * decorrelation models of Eqs. 35 / 44):
 *   out[off_p + j N + i] = sum_k W_k Re( D_k(l0_p) exp(2 pi i (u_k dl_i + v_k dm_j)) ),
 *   dl_i = (i - N/2) cell,  dm_j = (j - N/2) cell.
 * If pix_sel is given, only the listed packed pixel indices are computed (the
 * others are left untouched); otherwise every pixel of every cutout. */
int or_psf(OR_OBS_ARGS, int method, int npos, const double *lm, const int *npix, double cell,
           int flags, const int64_t *offsets, double *out,
           int64_t nsel, const int64_t *pix_sel) {
    or_obs o = OR_OBS_INIT;
    int64_t nvis;
    /* flag bit 8: the imaginary part of the (complex) sum of Eqs. 21-22 instead of
     * the real part; the other bits go to the decorrelation */
    const int imag = (flags & 8) != 0;
    flags &= ~8;
    or_vis *v = or_make_vis(&o, &nvis);
    if (!v) return -1;
    double *Dre = (double *)malloc(sizeof(double) * nvis), *Dim = (double *)malloc(sizeof(double) * nvis);
    double *uu = (double *)malloc(sizeof(double) * nvis), *vv = (double *)malloc(sizeof(double) * nvis);
    for (int64_t k = 0; k < nvis; ++k) {
        uu[k] = v[k].ubar[0] * v[k].nu / OR_C_LIGHT;
        vv[k] = v[k].ubar[1] * v[k].nu / OR_C_LIGHT;
    }
    for (int p = 0; p < npos; ++p) {
        double l0 = lm[2 * p], m0 = lm[2 * p + 1];
        #pragma omp parallel for schedule(static)
        for (int64_t k = 0; k < nvis; ++k)
            or_decorr_one(&o, &v[k], method, l0, m0, flags, &Dre[k], &Dim[k], NULL);
        int N = npix[p];
        int64_t off = offsets[p], npx = (int64_t)N * N;
        if (pix_sel) {
            #pragma omp parallel for schedule(dynamic, 1)
            for (int64_t q = 0; q < nsel; ++q) {
                int64_t g = pix_sel[q];
                if (g < off || g >= off + npx) continue;
                int64_t loc = g - off;
                int i = (int)(loc % N), j = (int)(loc / N);
                double dl = (i - N / 2) * cell, dm = (j - N / 2) * cell, acc = 0;
                for (int64_t k = 0; k < nvis; ++k) {
                    double ph = 2 * OR_PI * (uu[k] * dl + vv[k] * dm);
                    acc += imag ? v[k].W * (Dre[k] * sin(ph) + Dim[k] * cos(ph))
                                : v[k].W * (Dre[k] * cos(ph) - Dim[k] * sin(ph));
                }
                out[g] = acc;
            }
        } else {
            #pragma omp parallel for schedule(dynamic, 1)
            for (int64_t loc = 0; loc < npx; ++loc) {
                int i = (int)(loc % N), j = (int)(loc / N);
                double dl = (i - N / 2) * cell, dm = (j - N / 2) * cell, acc = 0;
                for (int64_t k = 0; k < nvis; ++k) {
                    double ph = 2 * OR_PI * (uu[k] * dl + vv[k] * dm);
                    acc += imag ? v[k].W * (Dre[k] * sin(ph) + Dim[k] * cos(ph))
                                : v[k].W * (Dre[k] * cos(ph) - Dim[k] * sin(ph));
                }
                out[off + loc] = acc;
            }
        }
    }
    free(Dre); free(Dim); free(uu); free(vv); free(v);
    return 0;
}

/* Vector-Jacobian product of the PSF map above with a cotangent R (same packed
 * layout as the output):
 *   g_W[k]    += sum_p Re( D_k(l0_p) H_pk ),
 *   g_lm[p,0]  = sum_k W_k Re( dD_k/dl0 H_pk ),  g_lm[p,1] likewise for m0,
 *   H_pk       = sum_ij R_p[j,i] exp(2 pi i (u_k dl_i + v_k dm_j)).
 * The twiddles depend on the offsets only, so l0 enters through D alone. */
int or_vjp(OR_OBS_ARGS, int method, int npos, const double *lm, const int *npix, double cell,
           int flags, const int64_t *offsets, const double *R, double *g_lm, double *g_W) {
    or_obs o = OR_OBS_INIT;
    int64_t nvis;
    or_vis *v = or_make_vis(&o, &nvis);
    if (!v) return -1;
    if (g_W) memset(g_W, 0, sizeof(double) * nvis);
    for (int p = 0; p < npos; ++p) {
        double l0 = lm[2 * p], m0 = lm[2 * p + 1];
        int N = npix[p];
        const double *Rp = R + offsets[p];
        double gl = 0, gm = 0;
        #pragma omp parallel for schedule(static) reduction(+ : gl, gm)
        for (int64_t k = 0; k < nvis; ++k) {
            double Dre, Dim, g[4];
            or_decorr_one(&o, &v[k], method, l0, m0, flags, &Dre, &Dim, g);
            double u = v[k].ubar[0] * v[k].nu / OR_C_LIGHT, w = v[k].ubar[1] * v[k].nu / OR_C_LIGHT;
            double Hre = 0, Him = 0;
            for (int j = 0; j < N; ++j) {
                double dm = (j - N / 2) * cell;
                for (int i = 0; i < N; ++i) {
                    double dl = (i - N / 2) * cell;
                    double ph = 2 * OR_PI * (u * dl + w * dm), r = Rp[(int64_t)j * N + i];
                    Hre += r * cos(ph);
                    Him += r * sin(ph);
                }
            }
            if (g_W) g_W[k] += Dre * Hre - Dim * Him;
            gl += v[k].W * (g[0] * Hre - g[1] * Him);
            gm += v[k].W * (g[2] * Hre - g[3] * Him);
        }
        g_lm[2 * p] = gl;
        g_lm[2 * p + 1] = gm;
    }
    free(v);
    return 0;
}

/* ---------------------------------------------------------------------------------
 * Gridded image-plane approximation: Eq. 45 with Algorithm 1 evaluated on uv cells.
 *
 * Readings (the paper leaves these open):
 *   - the grid is the N x N Fourier grid of the N x N cutout: cell spacing
 *     du = dv = 1 / (N cell), cell (a, b) at u = (a - N/2) du, v = (b - N/2) dv, so that
 *     the pixel phase 2 pi u dl is 2 pi (a - N/2)(i - N/2) / N and the transform pair is
 *     the N x N DFT; the cell steps of Algorithm 1 are read as exactly du, dv, and its
 *     half-cell start offset as this DFT-conjugate origin
 *   - F{P} is the DFT of the effective PSF P, the cutout at the phase centre with no
 *     distortion: P[j][i] = sum_k W_k cos(2 pi (u_k dl_i + v_k dm_j))
 *   - Algorithm 1 holds one dt, dnu and nu; with several channels and baseline-dependent
 *     averaging each cell takes the W-weighted means of dt_k and dnu_r / nu_r over the
 *     visibilities nearest to it and over the conjugates of those nearest to its mirror
 *     cell (a visibility at c also samples -c), cells taken modulo N (the DFT cannot tell
 *     u from u + N du); cells that receive none take the means over all visibilities
 *   - nearest cell: a' = floor(u_k N cell + 0.5) with u_k = ubar nu_r / c, evaluated in
 *     double precision in that order (the library decides the same way)
 *   - the cutout is Re F^-1{F{P} D}, F^-1 with the 1/N^2 of the inverse DFT
 * --------------------------------------------------------------------------------- */

/* Twiddle table tw[x][y] = exp(+2 pi i (x - N/2)(y - N/2) / N), angle reduced exactly. */
static void or_grid_twiddles(int N, double *twr, double *twi) {
    for (int x = 0; x < N; ++x)
        for (int y = 0; y < N; ++y) {
            int64_t m = ((int64_t)(x - N / 2) * (int64_t)(y - N / 2)) % N;
            if (m < 0) m += N;
            twr[x * N + y] = cos(2 * OR_PI * (double)m / N);
            twi[x * N + y] = sin(2 * OR_PI * (double)m / N);
        }
}

static int or_mod(int64_t x, int N) {
    int64_t r = x % N;
    return (int)(r < 0 ? r + N : r);
}

/* Position-independent tables of the gridded form:
 *   S    [N][N][2] F{P} (row b = v cell, column a = u cell; re, im)
 *   dtc  [N][N]    per-cell mean dt, rc [N][N] per-cell mean dnu/nu
 *   wsum [N][N]    per-cell sum of W over the visibilities and conjugates it received
 *   P    [N][N]    the effective PSF (any of the outputs may be NULL). */
int or_grid_tables(OR_OBS_ARGS, int N, double cell, double *S, double *dtc, double *rc, double *wsum,
                   double *Pout) {
    or_obs o = OR_OBS_INIT;
    int64_t nvis;
    if (N < 2 || N % 2 || !(cell > 0)) return -1;
    or_vis *v = or_make_vis(&o, &nvis);
    if (!v) return -1;
    const int64_t NN = (int64_t)N * N;
    double *P = (double *)calloc((size_t)NN, sizeof(double));
    double *twr = (double *)malloc(sizeof(double) * NN), *twi = (double *)malloc(sizeof(double) * NN);
    double *sw = (double *)calloc((size_t)NN, sizeof(double));
    double *sdt = (double *)calloc((size_t)NN, sizeof(double));
    double *sr = (double *)calloc((size_t)NN, sizeof(double));
    or_grid_twiddles(N, twr, twi);

    /* effective PSF (Eqs. 21-22 with D = 1), when S or P is asked for */
    #pragma omp parallel for schedule(dynamic, 1)
    for (int64_t q = 0; q < ((S || Pout) ? NN : 0); ++q) {
        int i = (int)(q % N), j = (int)(q / N);
        double dl = (i - N / 2) * cell, dm = (j - N / 2) * cell, acc = 0;
        for (int64_t k = 0; k < nvis; ++k) {
            double u = v[k].ubar[0] * v[k].nu / OR_C_LIGHT, w = v[k].ubar[1] * v[k].nu / OR_C_LIGHT;
            acc += v[k].W * cos(2 * OR_PI * (u * dl + w * dm));
        }
        P[q] = acc;
    }

    /* F{P}: S[b][a] = sum_j sum_i P[j][i] exp(-2 pi i ((a-N/2)(i-N/2) + (b-N/2)(j-N/2)) / N) */
    if (S) {
        #pragma omp parallel for schedule(dynamic, 1)
        for (int64_t q = 0; q < NN; ++q) {
            int a = (int)(q % N), b = (int)(q / N);
            double re = 0, im = 0;
            for (int j = 0; j < N; ++j)
                for (int i = 0; i < N; ++i) {
                    /* exp(-i x) exp(-i y) = conj(tw[a][i] tw[b][j]) */
                    double cr = twr[a * N + i] * twr[b * N + j] - twi[a * N + i] * twi[b * N + j];
                    double ci = twr[a * N + i] * twi[b * N + j] + twi[a * N + i] * twr[b * N + j];
                    re += P[(int64_t)j * N + i] * cr;
                    im -= P[(int64_t)j * N + i] * ci;
                }
            S[2 * q] = re;
            S[2 * q + 1] = im;
        }
    }

    /* per-cell means of dt and dnu/nu, nearest cell and its mirror, modulo N */
    double gw = 0, gdt = 0, gr = 0;
    const double s = (double)N * cell;
    for (int64_t k = 0; k < nvis; ++k) {
        double u = v[k].ubar[0] * v[k].nu / OR_C_LIGHT, w = v[k].ubar[1] * v[k].nu / OR_C_LIGHT;
        double qa = u * s, qb = w * s;
        int64_t ia = (int64_t)floor(qa + 0.5), ib = (int64_t)floor(qb + 0.5);
        double r = v[k].dnu / v[k].nu, W = v[k].W;
        int c1 = or_mod(ib + N / 2, N) * N + or_mod(ia + N / 2, N);
        int c2 = or_mod(-ib + N / 2, N) * N + or_mod(-ia + N / 2, N);
        sw[c1] += W; sdt[c1] += W * v[k].dt; sr[c1] += W * r;
        sw[c2] += W; sdt[c2] += W * v[k].dt; sr[c2] += W * r;
        gw += W; gdt += W * v[k].dt; gr += W * r;
    }
    for (int64_t q = 0; q < NN; ++q) {
        if (dtc) dtc[q] = sw[q] > 0 ? sdt[q] / sw[q] : (gw > 0 ? gdt / gw : 0.0);
        if (rc) rc[q] = sw[q] > 0 ? sr[q] / sw[q] : (gw > 0 ? gr / gw : 0.0);
        if (wsum) wsum[q] = sw[q];
        if (Pout) Pout[q] = P[q];
    }
    free(P); free(twr); free(twi); free(sw); free(sdt); free(sr); free(v);
    return 0;
}

/* Gridded cutouts from the tables of or_grid_tables:
 *   out[p][j N + i] = (1/N^2) Re sum_b sum_a S[b][a] D_ab(l0_p)
 *                              exp(2 pi i ((a-N/2)(i-N/2) + (b-N/2)(j-N/2)) / N),
 * D_ab = Algorithm 1 at the cell centre with the cell's mean dt and dnu/nu. */
int or_psf_img_grid_tables(int N, double cell, const double *S, const double *dtc, const double *rc, int npos,
                           const double *lm, int flags, double *out) {
    if (N < 2 || N % 2 || !(cell > 0)) return -1;
    const int64_t NN = (int64_t)N * N;
    double *twr = (double *)malloc(sizeof(double) * NN), *twi = (double *)malloc(sizeof(double) * NN);
    double *Tr = (double *)malloc(sizeof(double) * NN), *Ti = (double *)malloc(sizeof(double) * NN);
    or_grid_twiddles(N, twr, twi);
    const double du = 1.0 / ((double)N * cell);
    for (int p = 0; p < npos; ++p) {
        double l0 = lm[2 * p], m0 = lm[2 * p + 1];
        for (int64_t q = 0; q < NN; ++q) {
            int a = (int)(q % N), b = (int)(q / N);
            double D, Dl, Dm;
            or_img_decorr((a - N / 2) * du, (b - N / 2) * du, dtc[q], rc[q], l0, m0, flags & OR_LITERAL_THETA,
                          &D, &Dl, &Dm);
            Tr[q] = S[2 * q] * D;
            Ti[q] = S[2 * q + 1] * D;
        }
        double *op = out + (int64_t)p * NN;
        #pragma omp parallel for schedule(dynamic, 1)
        for (int64_t q = 0; q < NN; ++q) {
            int i = (int)(q % N), j = (int)(q / N);
            double acc = 0;
            for (int b = 0; b < N; ++b)
                for (int a = 0; a < N; ++a) {
                    double cr = twr[a * N + i] * twr[b * N + j] - twi[a * N + i] * twi[b * N + j];
                    double ci = twr[a * N + i] * twi[b * N + j] + twi[a * N + i] * twr[b * N + j];
                    acc += Tr[(int64_t)b * N + a] * cr - Ti[(int64_t)b * N + a] * ci;
                }
            op[q] = acc / (double)NN;
        }
    }
    free(twr); free(twi); free(Tr); free(Ti);
    return 0;
}

/* Gridded cutouts (Eq. 45 with Algorithm 1): the tables, then or_psf_img_grid_tables. */
int or_psf_img_grid(OR_OBS_ARGS, int npos, const double *lm, int N, double cell, int flags, double *out) {
    if (N < 2 || N % 2 || !(cell > 0)) return -1;
    const int64_t NN = (int64_t)N * N;
    double *S = (double *)malloc(sizeof(double) * 2 * NN);
    double *dtc = (double *)malloc(sizeof(double) * NN), *rc = (double *)malloc(sizeof(double) * NN);
    int rc0 = or_grid_tables(nbl, ntime, nchan, favg, uvw, time_s, freq, width, tavg, weights, twin, cwin, N,
                             cell, S, dtc, rc, NULL, NULL);
    if (rc0 == 0) rc0 = or_psf_img_grid_tables(N, cell, S, dtc, rc, npos, lm, flags, out);
    free(S); free(dtc); free(rc);
    return rc0;
}
