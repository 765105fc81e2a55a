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
} or_obs;

/* Per averaged visibility k, everything the definitions need. */
typedef struct {
    int b, s0, n, r;       /* baseline, first raw sample, sample count, out channel */
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
    for (int b = 0; b < o->nbl; ++b) {
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
                x->b = b; x->s0 = s0; x->n = n; x->r = r;
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
        for (int s = x->s0; s < x->s0 + x->n; ++s) {
            const double *us = ub + s * 3;
            double Xs = or_dot3(us, L), Xs_l = or_dot3(us, dLl), Xs_m = or_dot3(us, dLm);
            for (int c = x->r * o->favg; c < (x->r + 1) * o->favg; ++c) {
                double f = o->width[c] / (x->dnu * x->n);
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
    } else if (method == 1) {
        double A = or_dot3(x->dedge, L) * x->nu / OR_C_LIGHT;
        double B = or_dot3(x->ubar, L) * x->dnu / OR_C_LIGHT;
        double Al = or_dot3(x->dedge, dLl) * x->nu / OR_C_LIGHT, Am = or_dot3(x->dedge, dLm) * x->nu / OR_C_LIGHT;
        double Bl = or_dot3(x->ubar, dLl) * x->dnu / OR_C_LIGHT, Bm = or_dot3(x->ubar, dLm) * x->dnu / OR_C_LIGHT;
        double sA = or_sincpi(A), sB = or_sincpi(B), dA = or_dsincpi(A), dB = or_dsincpi(B);
        re = sA * sB;
        gl_re = dA * Al * sB + sA * dB * Bl;
        gm_re = dA * Am * sB + sA * dB * Bm;
    } else {
        double u = x->ubar[0] * x->nu / OR_C_LIGHT, v = x->ubar[1] * x->nu / OR_C_LIGHT;
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
        double A = OR_OMEGA_E * x->dt * (udot * l0 + vdot * m0);        /* dPsi / (2 pi) */
        double B = (x->dnu / x->nu) * uvlen * rho;                      /* dPhi / (2 pi) */
        double Al = OR_OMEGA_E * x->dt * udot, Am = OR_OMEGA_E * x->dt * vdot;
        double Bl = rho > 0 ? (x->dnu / x->nu) * uvlen * l0 / rho : 0.0;
        double Bm = rho > 0 ? (x->dnu / x->nu) * uvlen * m0 / rho : 0.0;
        double sA = or_sincpi(A), sB = or_sincpi(B), dA = or_dsincpi(A), dB = or_dsincpi(B);
        re = sA * sB;
        gl_re = dA * Al * sB + sA * dB * Bl;
        gm_re = dA * Am * sB + sA * dB * Bm;
    }
    *Dre = re; *Dim = im;
    if (g) { g[0] = gl_re; g[1] = gl_im; g[2] = gm_re; g[3] = gm_im; }
}

#define OR_OBS_ARGS int nbl, int ntime, int nchan, int favg, const double *uvw, const double *time_s, \
    const double *freq, const double *width, const int *tavg, const float *weights
#define OR_OBS_INIT {nbl, ntime, nchan, favg, uvw, time_s, freq, width, tavg, weights}

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
