/*
 * Plain FP64 CPU oracle for the inverse spherical harmonic transform (alm2map)
 * and its real-linear transpose (map2alm_adjoint).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is used by the test-suite, by the
 * smoke check and by the benchmark's CPU-baseline leg.  It shares no code,
 * header, table or constant with the CUDA library and must never be linked
 * into, or called from, the product path.
 *
 * Everything here is written to be read against the paper (Hupca, Falcou,
 * Grigori, Stompor, "Spherical harmonic transform with GPUs", INRIA RR-7409),
 * section 2.1, not to be fast:
 *
 *   alm2map            s(theta,phi) = sum_{l<=lmax} sum_{|m|<=l} a_lm Y_lm    (Eq. alm2mapDef)
 *   Y_lm               = lambda_lm(cos theta) e^{i m phi}                    (sec. 2.1)
 *   Delta_m(theta)     = sum_{l>=m} a_lm lambda_lm(cos theta)                 (Eq. DeltaDef)
 *   s(theta,phi)       = sum_{m=-M..M} e^{i m phi} Delta_m(theta)             (Eq. Delta2map)
 *   recurrence         lambda_lm = beta_lm (x lambda_{l-1,m} - lambda_{l-2,m}/beta_{l-1,m})
 *                                                                            (Eq. assLegRec, sign read as "-")
 *   beta_lm            = sqrt((4 l^2 - 1)/(l^2 - m^2))                        (Eq. betaDef)
 *   lambda_mm          = mu_m (1-x^2)^{m/2}, mu_m = (-1)^m sqrt((2m+1)!/(4 pi))/(2^m m!)
 *                                                                            (Eq. pmm, power read as m/2,
 *                                                                             Condon-Shortley sign included)
 *   lambda_{m+1,m}     = beta_{m+1,m} x lambda_mm = sqrt(2m+3) x lambda_mm     (Eq. pm1m)
 *   rescaling          values carried as (v, k) meaning v * 2^(ORC_S k); the pair
 *                      (lambda_l, lambda_{l-1}) is rescaled together whenever the newest
 *                      value leaves [2^-ORC_S, 2^ORC_S]                        (sec. 2.2.2, Algorithm 2)
 *
 * The ring synthesis is a literal O(n_phi * M) sum per ring (no FFT, no fold):
 *   s_r(j) = Delta_0(r) + 2 Re sum_{m=1..M} Delta_m(r) e^{i m (phi0_r + 2 pi j / n_phi_r)}.
 * Im(a_l0) is ignored because the field is real (sec. 2.1).
 *
 * Geometry: Gauss-Legendre nodes by Newton iteration on the Legendre
 * three-term recurrence; HEALPix RING geometry from Gorski et al. 2005 (the
 * paper's reference for the pixelisation).  Rings are ordered north to south.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ORC_S 400 /* rescaling unit: one step of k is a factor 2^400 */

static const double ORC_PI = 3.14159265358979323846264338327950288;

/* ------------------------------------------------------------------------ */
/* Geometry                                                                  */
/* ------------------------------------------------------------------------ */

/* Gauss-Legendre nodes x (descending: north to south) and weights w for n
 * points.  P_n and P_{n-1} come from (j+1) P_{j+1} = (2j+1) x P_j - j P_{j-1};
 * P_n'(x) = n (x P_n - P_{n-1}) / (x^2 - 1).  Returns 0 on success. */
int orc_gl_nodes(int n, double *x, double *w)
{
    if (n < 1) return -1;
    for (int k = 1; k <= n; k++) {
        double xk = cos(ORC_PI * (k - 0.25) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = xk;
            for (int j = 1; j < n; j++) {
                double p2 = ((2.0 * j + 1.0) * xk * p1 - j * p0) / (j + 1.0);
                p0 = p1;
                p1 = p2;
            }
            double pn = (n == 1) ? xk : p1;
            double pnm1 = (n == 1) ? 1.0 : p0;
            dp = n * (xk * pn - pnm1) / (xk * xk - 1.0);
            double dx = pn / dp;
            xk -= dx;
            if (fabs(dx) < 1e-16) break;
        }
        /* recompute the derivative at the converged node for the weight */
        {
            double p0 = 1.0, p1 = xk;
            for (int j = 1; j < n; j++) {
                double p2 = ((2.0 * j + 1.0) * xk * p1 - j * p0) / (j + 1.0);
                p0 = p1;
                p1 = p2;
            }
            double pn = (n == 1) ? xk : p1;
            double pnm1 = (n == 1) ? 1.0 : p0;
            dp = n * (xk * pn - pnm1) / (xk * xk - 1.0);
        }
        x[k - 1] = xk;
        w[k - 1] = 2.0 / ((1.0 - xk * xk) * dp * dp);
    }
    return 0;
}

/* HEALPix RING geometry for nside >= 1: 4 nside - 1 rings, north to south.
 * Outputs cos(theta), sin(theta), n_phi and phi0 (azimuth of the ring's first
 * pixel).  sin(theta) is formed from the exact 1-z of the cap formula (or
 * (1-z)(1+z) in the belt) to avoid cancellation near the poles. */
int orc_healpix_rings(int nside, double *z, double *st, int *nphi, double *phi0)
{
    if (nside < 1) return -1;
    const int nr = 4 * nside - 1;
    const double n = (double)nside;
    for (int i = 1; i <= nr; i++) {
        double zi, si, p0;
        int np;
        if (i < nside || i > 3 * nside) {
            int ic = (i < nside) ? i : 4 * nside - i; /* cap ring index */
            double omz = (double)ic * (double)ic / (3.0 * n * n); /* 1 - |z| */
            zi = 1.0 - omz;
            si = sqrt(omz * (2.0 - omz));
            np = 4 * ic;
            p0 = ORC_PI / (4.0 * ic); /* (pi / (2 ic)) * (0 + 1/2) */
            if (i > 3 * nside) zi = -zi;
        } else {
            zi = 4.0 / 3.0 - 2.0 * i / (3.0 * n);
            si = sqrt((1.0 - zi) * (1.0 + zi));
            np = 4 * nside;
            int sft = (i - nside + 1) % 2;
            p0 = (ORC_PI / (2.0 * n)) * (0.5 * sft);
        }
        z[i - 1] = zi;
        st[i - 1] = si;
        nphi[i - 1] = np;
        phi0[i - 1] = p0;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Normalised associated Legendre functions                                  */
/* ------------------------------------------------------------------------ */

static inline long orc_nalm(int lmax, int mmax)
{
    return (long)(mmax + 1) * (2L * lmax + 2 - mmax) / 2;
}

/* offset of column m in the m-major packed (l, m) layout */
static inline long orc_mofs(int lmax, int m)
{
    return (long)m * (2L * lmax + 3 - m) / 2;
}

/* beta_lm of Eq. betaDef */
static double orc_beta(int l, int m)
{
    double dl = l, dm = m;
    return sqrt((4.0 * dl * dl - 1.0) / (dl * dl - dm * dm));
}

/* mu_m of Eq. pmm with the Condon-Shortley sign, by the product
 * mu_0 = 1/sqrt(4 pi), mu_m = -mu_{m-1} sqrt((2m+1)/(2m)). */
static void orc_mu(int mmax, double *mu)
{
    mu[0] = 1.0 / sqrt(4.0 * ORC_PI);
    for (int m = 1; m <= mmax; m++) mu[m] = -mu[m - 1] * sqrt((2.0 * m + 1.0) / (2.0 * m));
}

/* value carried with a power-of-two exponent: true value = v * 2^(ORC_S k) */
typedef struct {
    double v;
    int k;
} orc_scaled;

static double orc_unscale(double v, int k)
{
    double t = ldexp(v, ORC_S * k);
    /* contributions below the FP64 normal range are flushed to zero */
    if (fabs(t) < 2.2250738585072014e-308) return 0.0;
    return t;
}

/* lambda_lm(x) for every (l, m), 0<=m<=mmax, m<=l<=lmax, written m-major
 * packed into out.  s = sin(theta) >= 0.  If track == 0 the recurrence runs
 * without rescaling (used only to pin the exactness of the rescaling). */
static void orc_lambda_impl(int lmax, int mmax, double x, double s, int track,
                            const double *mu, double *out)
{
    /* s^m with exponent tracking, built one factor at a time */
    orc_scaled pw = {1.0, 0};
    for (int m = 0; m <= mmax; m++) {
        if (m > 0) {
            pw.v *= s;
            if (track && pw.v != 0.0 && fabs(pw.v) < ldexp(1.0, -ORC_S)) {
                pw.v = ldexp(pw.v, ORC_S);
                pw.k -= 1;
            }
        }
        double *col = out + orc_mofs(lmax, m);
        /* lambda_mm = mu_m s^m */
        double l0 = mu[m] * pw.v; /* lambda_{l-2} */
        int k = pw.k;
        col[0] = track ? orc_unscale(l0, k) : l0;
        if (m == lmax) continue;
        /* lambda_{m+1,m} = sqrt(2m+3) x lambda_mm */
        double l1 = sqrt(2.0 * m + 3.0) * x * l0; /* lambda_{l-1} */
        col[1] = track ? orc_unscale(l1, k) : l1;
        double bprev = orc_beta(m + 1, m);
        for (int l = m + 2; l <= lmax; l++) {
            double b = orc_beta(l, m);
            double l2 = b * (x * l1 - l0 / bprev);
            l0 = l1;
            l1 = l2;
            bprev = b;
            if (track) {
                if (fabs(l1) > ldexp(1.0, ORC_S)) {
                    l1 = ldexp(l1, -ORC_S);
                    l0 = ldexp(l0, -ORC_S);
                    k += 1;
                } else if (l1 != 0.0 && fabs(l1) < ldexp(1.0, -ORC_S) &&
                           fabs(l0) < ldexp(1.0, -ORC_S)) {
                    l1 = ldexp(l1, ORC_S);
                    l0 = ldexp(l0, ORC_S);
                    k -= 1;
                }
                col[l - m] = orc_unscale(l1, k);
            } else {
                col[l - m] = l1;
            }
        }
    }
}

/* Public: lambda_lm at one ring.  Returns 0 on success. */
int orc_lambda(int lmax, int mmax, double x, double s, int track, double *out)
{
    if (lmax < 0 || mmax < 0 || mmax > lmax) return -1;
    double *mu = (double *)malloc(sizeof(double) * (mmax + 1));
    if (!mu) return -2;
    orc_mu(mmax, mu);
    orc_lambda_impl(lmax, mmax, x, s, track, mu, out);
    free(mu);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* alm2map (Algorithm 1 order: for each ring, Delta_m for all m, then ring sum) */
/* ------------------------------------------------------------------------ */

typedef struct {
    int lmax, mmax, nmaps;
    const double *x, *st, *phi0;
    const int *nphi;
    const long *ofs;     /* first pixel of each ring */
    const double *alm;   /* [nmaps][nalm][2] */
    double *map;         /* [nmaps][npix] */
    long npix;
    const int *rings;    /* rings to compute */
    int nsel;
    const double *mu;
    int tid, nthreads;
    int status;
} orc_fwd_job;

static void *orc_fwd_worker(void *arg)
{
    orc_fwd_job *J = (orc_fwd_job *)arg;
    const int L = J->lmax, M = J->mmax;
    const long nalm = orc_nalm(L, M);
    double *lam = (double *)malloc(sizeof(double) * nalm);
    double *dre = (double *)malloc(sizeof(double) * (M + 1));
    double *dim = (double *)malloc(sizeof(double) * (M + 1));
    if (!lam || !dre || !dim) {
        J->status = -2;
        free(lam); free(dre); free(dim);
        return NULL;
    }
    for (int q = J->tid; q < J->nsel; q += J->nthreads) {
        const int r = J->rings[q];
        const int np = J->nphi[r];
        orc_lambda_impl(L, M, J->x[r], J->st[r], 1, J->mu, lam);
        /* cs[t] = e^{2 pi i t / np}; ph[m] = e^{i m phi0} */
        double *cs = (double *)malloc(sizeof(double) * 2 * np);
        double *ph = (double *)malloc(sizeof(double) * 2 * (M + 1));
        if (!cs || !ph) { free(cs); free(ph); J->status = -2; break; }
        for (int t = 0; t < np; t++) {
            double ang = 2.0 * ORC_PI * t / np;
            cs[2 * t] = cos(ang);
            cs[2 * t + 1] = sin(ang);
        }
        for (int m = 0; m <= M; m++) {
            ph[2 * m] = cos(m * J->phi0[r]);
            ph[2 * m + 1] = sin(m * J->phi0[r]);
        }
        for (int b = 0; b < J->nmaps; b++) {
            const double *a = J->alm + (long)b * nalm * 2;
            /* step 1: Delta_m(r) = sum_{l>=m} a_lm lambda_lm(x_r) (Eq. DeltaDef) */
            for (int m = 0; m <= M; m++) {
                const long c = orc_mofs(L, m);
                double sr = 0.0, si = 0.0;
                for (int l = m; l <= L; l++) {
                    sr += a[2 * (c + l - m)] * lam[c + l - m];
                    si += a[2 * (c + l - m) + 1] * lam[c + l - m];
                }
                dre[m] = sr;
                dim[m] = (m == 0) ? 0.0 : si; /* Im(a_l0) ignored: real field */
            }
            /* step 2: s_r(j) = Delta_0 + 2 Re sum_{m>=1} Delta_m e^{i m phi_j} (Eq. Delta2map) */
            double *out = J->map + (long)b * J->npix + J->ofs[r];
            for (int j = 0; j < np; j++) {
                double acc = dre[0];
                for (int m = 1; m <= M; m++) {
                    /* e^{i m phi_j} = e^{i m phi0} e^{2 pi i (m j mod np)/np} */
                    double pr = ph[2 * m], pi_ = ph[2 * m + 1];
                    long qq = ((long)m * j) % np;
                    double er = pr * cs[2 * qq] - pi_ * cs[2 * qq + 1];
                    double ei = pr * cs[2 * qq + 1] + pi_ * cs[2 * qq];
                    acc += 2.0 * (dre[m] * er - dim[m] * ei);
                }
                out[j] = acc;
            }
        }
        free(cs);
        free(ph);
    }
    free(lam); free(dre); free(dim);
    return NULL;
}

static int orc_nthreads(int req)
{
    if (req > 0) return req;
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int)n : 1;
}

/* alm2map on the selected rings of a ring grid.
 *   x, st, phi0, nphi, ofs : per-ring cos(theta), sin(theta), phi0, n_phi, first pixel
 *   alm  : [nmaps][nalm] complex (interleaved re, im), m-major packed
 *   map  : [nmaps][npix] real; only the pixels of the selected rings are written
 *   rings: indices of the rings to compute (nsel of them)
 * Returns the number of threads used (> 0) or a negative error. */
int orc_alm2map(int lmax, int mmax, int nrings, const double *x, const double *st,
                const double *phi0, const int *nphi, const long *ofs, long npix,
                int nmaps, const double *alm, double *map, int nsel, const int *rings,
                int nthreads)
{
    if (lmax < 0 || mmax < 0 || mmax > lmax || nmaps < 0 || nsel < 0) return -1;
    for (int q = 0; q < nsel; q++)
        if (rings[q] < 0 || rings[q] >= nrings) return -1;
    const int nt = orc_nthreads(nthreads);
    double *mu = (double *)malloc(sizeof(double) * (mmax + 1));
    orc_fwd_job *jobs = (orc_fwd_job *)calloc(nt, sizeof(orc_fwd_job));
    pthread_t *th = (pthread_t *)calloc(nt, sizeof(pthread_t));
    if (!mu || !jobs || !th) { free(mu); free(jobs); free(th); return -2; }
    orc_mu(mmax, mu);
    for (int t = 0; t < nt; t++) {
        orc_fwd_job j = {lmax, mmax, nmaps, x, st, phi0, nphi, ofs, alm, map, npix,
                         rings, nsel, mu, t, nt, 0};
        jobs[t] = j;
        pthread_create(&th[t], NULL, orc_fwd_worker, &jobs[t]);
    }
    int st_ = nt;
    for (int t = 0; t < nt; t++) {
        pthread_join(th[t], NULL);
        if (jobs[t].status) st_ = jobs[t].status;
    }
    free(mu); free(jobs); free(th);
    return st_;
}

/* ------------------------------------------------------------------------ */
/* map2alm_adjoint: the literal real-linear transpose of alm2map             */
/*   g_lm = c_m sum_r lambda_lm(x_r) sum_j y_rj e^{-i m (phi0_r + 2 pi j/n_phi_r)}
 *   c_0 = 1 (and Im g_l0 = 0), c_m = 2 for m > 0.                             */
/* ------------------------------------------------------------------------ */

typedef struct {
    int lmax, mmax, nmaps, nrings;
    const double *x, *st, *phi0;
    const int *nphi;
    const long *ofs;
    const double *map; /* [nmaps][npix] */
    long npix;
    int nm;            /* number of selected m */
    const int *msel;
    const double *mu;
    double *part;      /* per-thread partial g: [nmaps][nm][lmax+1][2] */
    int tid, nthreads;
    int status;
} orc_adj_job;

static void *orc_adj_worker(void *arg)
{
    orc_adj_job *J = (orc_adj_job *)arg;
    const int L = J->lmax, M = J->mmax;
    const long nalm = orc_nalm(L, M);
    double *lam = (double *)malloc(sizeof(double) * nalm);
    if (!lam) { J->status = -2; return NULL; }
    for (int r = J->tid; r < J->nrings; r += J->nthreads) {
        const int np = J->nphi[r];
        orc_lambda_impl(L, M, J->x[r], J->st[r], 1, J->mu, lam);
        /* cs[t] = e^{2 pi i t / np} */
        double *cs = (double *)malloc(sizeof(double) * 2 * np);
        if (!cs) { J->status = -2; break; }
        for (int t = 0; t < np; t++) {
            double ang = 2.0 * ORC_PI * t / np;
            cs[2 * t] = cos(ang);
            cs[2 * t + 1] = sin(ang);
        }
        for (int b = 0; b < J->nmaps; b++) {
            const double *y = J->map + (long)b * J->npix + J->ofs[r];
            for (int q = 0; q < J->nm; q++) {
                const int m = J->msel[q];
                /* ring projection sum_j y_j e^{-i m phi_j}, with
                 * e^{i m phi_j} = e^{i m phi0} e^{2 pi i (m j mod np)/np} */
                const double c0 = cos(m * J->phi0[r]), s0 = sin(m * J->phi0[r]);
                double pr = 0.0, pim = 0.0;
                for (int j = 0; j < np; j++) {
                    long qq = ((long)m * j) % np;
                    double er = c0 * cs[2 * qq] - s0 * cs[2 * qq + 1];
                    double ei = c0 * cs[2 * qq + 1] + s0 * cs[2 * qq];
                    pr += y[j] * er;
                    pim -= y[j] * ei;
                }
                const double cm = (m == 0) ? 1.0 : 2.0;
                const long c = orc_mofs(L, m);
                double *g = J->part + (((long)b * J->nm + q) * (L + 1)) * 2;
                for (int l = m; l <= L; l++) {
                    g[2 * l] += cm * lam[c + l - m] * pr;
                    if (m > 0) g[2 * l + 1] += cm * lam[c + l - m] * pim;
                }
            }
        }
        free(cs);
    }
    free(lam);
    return NULL;
}

/* map2alm_adjoint for the selected m values (all l of each); alm entries of
 * unselected m are left untouched.  Returns threads used or a negative error. */
int orc_map2alm_adjoint(int lmax, int mmax, int nrings, const double *x, const double *st,
                        const double *phi0, const int *nphi, const long *ofs, long npix,
                        int nmaps, const double *map, double *alm, int nm, const int *msel,
                        int nthreads)
{
    if (lmax < 0 || mmax < 0 || mmax > lmax || nmaps < 0 || nm < 0) return -1;
    for (int q = 0; q < nm; q++)
        if (msel[q] < 0 || msel[q] > mmax) return -1;
    int nt = orc_nthreads(nthreads);
    if (nt > nrings && nrings > 0) nt = nrings;
    const long psz = (long)nmaps * nm * (lmax + 1) * 2;
    double *mu = (double *)malloc(sizeof(double) * (mmax + 1));
    orc_adj_job *jobs = (orc_adj_job *)calloc(nt, sizeof(orc_adj_job));
    pthread_t *th = (pthread_t *)calloc(nt, sizeof(pthread_t));
    double *part = (double *)calloc((size_t)nt * (psz > 0 ? psz : 1), sizeof(double));
    if (!mu || !jobs || !th || !part) { free(mu); free(jobs); free(th); free(part); return -2; }
    orc_mu(mmax, mu);
    for (int t = 0; t < nt; t++) {
        orc_adj_job j = {lmax, mmax, nmaps, nrings, x, st, phi0, nphi, ofs, map, npix,
                         nm, msel, mu, part + (long)t * psz, t, nt, 0};
        jobs[t] = j;
        pthread_create(&th[t], NULL, orc_adj_worker, &jobs[t]);
    }
    int st_ = nt;
    for (int t = 0; t < nt; t++) {
        pthread_join(th[t], NULL);
        if (jobs[t].status) st_ = jobs[t].status;
    }
    /* reduce the per-thread partial sums in a fixed order */
    const long nalm = orc_nalm(lmax, mmax);
    for (int b = 0; b < nmaps; b++)
        for (int q = 0; q < nm; q++) {
            const int m = msel[q];
            const long c = orc_mofs(lmax, m);
            for (int l = m; l <= lmax; l++) {
                double gr = 0.0, gi = 0.0;
                for (int t = 0; t < nt; t++) {
                    const double *g = part + (long)t * psz + (((long)b * nm + q) * (lmax + 1)) * 2;
                    gr += g[2 * l];
                    gi += g[2 * l + 1];
                }
                double *o = alm + ((long)b * nalm + c + (l - m)) * 2;
                o[0] = gr;
                o[1] = gi;
            }
        }
    free(mu); free(jobs); free(th); free(part);
    return st_;
}

/* ------------------------------------------------------------------------ */
/* Spin-2 (polarisation) synthesis: the Q/U maps of E/B coefficients.        */
/*                                                                            */
/* Not in the paper (an extension of its transform to the CMB's polarisation  */
/* field).  Definitions, written out here and pinned by the tests:            */
/*   spin-raising  ð f = -(sin t)^s (d/dt + (i / sin t) d/dphi) ((sin t)^-s f) */
/*   lowering      ð̄ f = -(sin t)^-s (d/dt - (i / sin t) d/dphi) ((sin t)^s f) */
/*   2Y_lm = ð ð Y_lm / K_l,  -2Y_lm = ð̄ ð̄ Y_lm / K_l,                        */
/*   K_l = sqrt((l-1) l (l+1) (l+2)), l >= 2, Y_lm = lambda_lm e^{i m phi}     */
/*   (Y_{l,-m} = (-1)^m conj(Y_lm), Condon-Shortley as the scalar part),     */
/*   Q + i U = - sum_{l>=2} sum_{|m|<=l} (E_lm + i B_lm) 2Y_lm,               */
/*   E_{l,-m} = (-1)^m conj(E_lm), B likewise (Q, U real).                    */
/* With L = lambda_lm, D = d lambda_lm / d theta, c = cos t, s = sin t, the  */
/* two raisings give (m of either sign)                                       */
/*   K_l 2lambda_lm = D'' - D (c + 2m)/s + L (2 m c + m^2)/s^2                 */
/* and the Legendre equation D'' = -(c/s) D + (m^2/s^2 - l(l+1)) L with       */
/* s D = l c L - c_lm lambda_{l-1,m}, c_lm = sqrt((2l+1)(l^2-m^2)/(2l-1)),   */
/* turn it into values of lambda_lm and lambda_{l-1,m} only:                  */
/*   K_l 2lambda_lm = -2 (c + m) (l c L - c_lm L1)/s^2                        */
/*                    + L ((2 m^2 + 2 m c)/s^2 - l (l+1)).                    */
/* The oracle evaluates this for every m in [-M, M] (lambda_{l,-m} =          */
/* (-1)^m lambda_lm) and sums the definition literally, pixel by pixel of    */
/* each ring, over all m of both signs.  sin t must be > 0.                   */
/* ------------------------------------------------------------------------ */

/* 2lambda_lm(t) for m >= 0 (plus) and for -m (minus), m-major packed like the
 * scalar table (entries with l < 2 are 0).  lam: the scalar table at this
 * ring (true values, from orc_lambda_impl). */
static void orc_spin2_from_scalar(int lmax, int mmax, double x, double s, const double *lam,
                                  double *plus, double *minus)
{
    const double u = 1.0 / (s * s);
    for (int m = 0; m <= mmax; m++) {
        const long c = orc_mofs(lmax, m);
        for (int l = m; l <= lmax; l++) {
            if (l < 2) {
                plus[c + l - m] = 0.0;
                minus[c + l - m] = 0.0;
                continue;
            }
            const double L = lam[c + l - m];
            const double L1 = (l - 1 >= m) ? lam[c + l - 1 - m] : 0.0;
            const double clm = sqrt((2.0 * l + 1.0) * ((double)l * l - (double)m * m) / (2.0 * l - 1.0));
            const double K = sqrt((l - 1.0) * l * (l + 1.0) * (l + 2.0));
            const double sD = l * x * L - clm * L1; /* s dlambda/dtheta */
            for (int sg = 0; sg < 2; sg++) {
                /* order mm = +m or -m: lambda_{l,-m} = (-1)^m lambda_lm (and likewise L1) */
                const double mm = sg ? -(double)m : (double)m;
                const double f = (sg && (m & 1)) ? -1.0 : 1.0;
                const double Lm = f * L, sDm = f * sD;
                const double v = (-2.0 * (x + mm) * sDm * u + Lm * ((2.0 * mm * mm + 2.0 * mm * x) * u - l * (l + 1.0))) / K;
                if (sg)
                    minus[c + l - m] = v;
                else
                    plus[c + l - m] = v;
            }
        }
    }
}

int orc_lambda_spin2(int lmax, int mmax, double x, double s, double *plus, double *minus)
{
    if (lmax < 0 || mmax < 0 || mmax > lmax || !(s > 0.0)) return -1;
    double *mu = (double *)malloc(sizeof(double) * (mmax + 1));
    double *lam = (double *)malloc(sizeof(double) * orc_nalm(lmax, mmax));
    if (!mu || !lam) { free(mu); free(lam); return -2; }
    orc_mu(mmax, mu);
    orc_lambda_impl(lmax, mmax, x, s, 1, mu, lam);
    orc_spin2_from_scalar(lmax, mmax, x, s, lam, plus, minus);
    free(mu); free(lam);
    return 0;
}

typedef struct {
    int lmax, mmax, nmaps;
    const double *x, *st, *phi0;
    const int *nphi;
    const long *ofs;
    const double *elm, *blm; /* [nmaps][nalm][2] */
    double *qmap, *umap;     /* [nmaps][npix] */
    long npix;
    const int *rings;
    int nsel;
    const double *mu;
    int tid, nthreads;
    int status;
} orc_spin_job;

static void *orc_spin_worker(void *arg)
{
    orc_spin_job *J = (orc_spin_job *)arg;
    const int L = J->lmax, M = J->mmax;
    const long nalm = orc_nalm(L, M);
    double *lam = (double *)malloc(sizeof(double) * nalm);
    double *lp = (double *)malloc(sizeof(double) * nalm);
    double *lmn = (double *)malloc(sizeof(double) * nalm);
    double *cr = (double *)malloc(sizeof(double) * (2 * M + 1)); /* C_m, m = -M..M */
    double *ci = (double *)malloc(sizeof(double) * (2 * M + 1));
    if (!lam || !lp || !lmn || !cr || !ci) {
        J->status = -2;
        free(lam); free(lp); free(lmn); free(cr); free(ci);
        return NULL;
    }
    for (int q = J->tid; q < J->nsel; q += J->nthreads) {
        const int r = J->rings[q];
        const int np = J->nphi[r];
        orc_lambda_impl(L, M, J->x[r], J->st[r], 1, J->mu, lam);
        orc_spin2_from_scalar(L, M, J->x[r], J->st[r], lam, lp, lmn);
        /* tab[q] = e^{2 pi i q / np}; ph[m + M] = e^{i m phi0} */
        double *tab = (double *)malloc(sizeof(double) * 2 * np);
        double *ph = (double *)malloc(sizeof(double) * 2 * (2 * M + 1));
        if (!tab || !ph) { free(tab); free(ph); J->status = -2; break; }
        for (int t = 0; t < np; t++) {
            tab[2 * t] = cos(2.0 * ORC_PI * t / np);
            tab[2 * t + 1] = sin(2.0 * ORC_PI * t / np);
        }
        for (int m = -M; m <= M; m++) {
            ph[2 * (m + M)] = cos(m * J->phi0[r]);
            ph[2 * (m + M) + 1] = sin(m * J->phi0[r]);
        }
        for (int b = 0; b < J->nmaps; b++) {
            const double *E = J->elm + (long)b * nalm * 2, *B = J->blm + (long)b * nalm * 2;
            /* C_m = - sum_l (E_lm + i B_lm) 2lambda_lm for m = -M..M, with
             * E_{l,-m} = (-1)^m conj(E_lm) and B likewise */
            for (int m = -M; m <= M; m++) {
                const int am = m < 0 ? -m : m;
                const long c = orc_mofs(L, am);
                const double f = (m < 0 && (am & 1)) ? -1.0 : 1.0;
                double sr = 0.0, si = 0.0;
                for (int l = am; l <= L; l++) {
                    double er = E[2 * (c + l - am)], ei = E[2 * (c + l - am) + 1];
                    double br = B[2 * (c + l - am)], bi = B[2 * (c + l - am) + 1];
                    if (am == 0) { ei = 0.0; bi = 0.0; } /* real fields: E_l0, B_l0 real */
                    if (m < 0) { er *= f; ei *= -f; br *= f; bi *= -f; }
                    const double y = (m < 0) ? lmn[c + l - am] : lp[c + l - am];
                    /* (E + i B) y = (er - bi) y + i (ei + br) y */
                    sr -= (er - bi) * y;
                    si -= (ei + br) * y;
                }
                cr[m + M] = sr;
                ci[m + M] = si;
            }
            /* Q + i U at phi_j = phi0 + 2 pi j / np: sum_m C_m e^{i m phi_j}, with
             * e^{i m phi_j} = e^{i m phi0} e^{2 pi i ((m j) mod np) / np} */
            double *qo = J->qmap + (long)b * J->npix + J->ofs[r];
            double *uo = J->umap + (long)b * J->npix + J->ofs[r];
            for (int j = 0; j < np; j++) {
                double ar = 0.0, ai = 0.0;
                for (int m = -M; m <= M; m++) {
                    long qq = ((long)m * j) % np;
                    if (qq < 0) qq += np;
                    const double pr = ph[2 * (m + M)], pi_ = ph[2 * (m + M) + 1];
                    const double tr = tab[2 * qq], ti = tab[2 * qq + 1];
                    const double er = pr * tr - pi_ * ti, ei = pr * ti + pi_ * tr;
                    ar += cr[m + M] * er - ci[m + M] * ei;
                    ai += cr[m + M] * ei + ci[m + M] * er;
                }
                qo[j] = ar;
                uo[j] = ai;
            }
        }
        free(tab);
        free(ph);
    }
    free(lam); free(lp); free(lmn); free(cr); free(ci);
    return NULL;
}

/* Spin-2 synthesis on the selected rings: elm, blm [nmaps][nalm] complex
 * (m-major packed, entries with l < 2 ignored), qmap, umap [nmaps][npix].
 * Returns the number of threads used or a negative error (-1 also when a
 * selected ring has sin(theta) = 0). */
int orc_alm2map_spin2(int lmax, int mmax, int nrings, const double *x, const double *st,
                      const double *phi0, const int *nphi, const long *ofs, long npix, int nmaps,
                      const double *elm, const double *blm, double *qmap, double *umap, int nsel,
                      const int *rings, int nthreads)
{
    if (lmax < 0 || mmax < 0 || mmax > lmax || nmaps < 0 || nsel < 0) return -1;
    for (int q = 0; q < nsel; q++)
        if (rings[q] < 0 || rings[q] >= nrings || !(st[rings[q]] > 0.0)) return -1;
    const int nt = orc_nthreads(nthreads);
    double *mu = (double *)malloc(sizeof(double) * (mmax + 1));
    orc_spin_job *jobs = (orc_spin_job *)calloc(nt, sizeof(orc_spin_job));
    pthread_t *th = (pthread_t *)calloc(nt, sizeof(pthread_t));
    if (!mu || !jobs || !th) { free(mu); free(jobs); free(th); return -2; }
    orc_mu(mmax, mu);
    for (int t = 0; t < nt; t++) {
        orc_spin_job j = {lmax, mmax, nmaps, x, st, phi0, nphi, ofs, elm, blm, qmap, umap, npix,
                          rings, nsel, mu, t, nt, 0};
        jobs[t] = j;
        pthread_create(&th[t], NULL, orc_spin_worker, &jobs[t]);
    }
    int st_ = nt;
    for (int t = 0; t < nt; t++) {
        pthread_join(th[t], NULL);
        if (jobs[t].status) st_ = jobs[t].status;
    }
    free(mu); free(jobs); free(th);
    return st_;
}
