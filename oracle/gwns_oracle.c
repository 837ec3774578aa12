/*
 * gwns_oracle.c -- plain, slow, FP64 CPU oracle for the nested-slice-sampling
 * hot path (TEST INFRASTRUCTURE ONLY).
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may call
 * this code; the library never links it. It shares no code, header, table or
 * constant generator with the CUDA path.
 *
 * What it computes, and where each piece comes from:
 *   - prior transform u -> theta (uniform boxes; distance uniform in volume);
 *   - the frequency-domain TaylorF2 (stationary-phase) inspiral, evaluated
 *     directly on every bin: 3.5PN non-spinning phasing (Buonanno, Iyer,
 *     Ochsner, Pan, Sathyaprakash 2009) plus aligned-spin terms beta, sigma,
 *     gamma (Arun, Buonanno, Faye, Ochsner 2009), cut off above f_ISCO;
 *   - antenna patterns F+, Fx and geocentre time delays of each detector
 *     (Anderson et al. 2001 wave-frame convention);
 *   - the Whittle log-likelihood ratio written as its plain definition:
 *     log L = sum_d [<d_d|h_d> - 1/2 <h_d|h_d>], <a|b> = 4 df Re sum_j a_j b_j^* / S_j;
 *   - a correlated-Gaussian toy likelihood;
 *   - Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), the counter-based
 *     generator both sides implement from its published definition;
 *   - the slice-sampling update of one nested-sampling iteration (paper Sec. 2:
 *     slice sampling with covariance-tuned directions, vectorised across the
 *     k deleted points), with stepping out and shrinkage as in Neal (2003),
 *     Sec. 4, applied along a hit-and-run direction.
 *
 *   - relative binning (Zackay, Dai & Venumadhav 2018; the paper's heterodyned,
 *     coarse-grid likelihood, Sec. 2-3): summary data of a fiducial waveform
 *     over geometric coarse bins, and the ratio r = h/h0 interpolated linearly
 *     inside each bin from its values at the bin edges.
 *
 * Parity status: the non-spinning phasing is pinned by re-deriving it from the
 * PN energy and flux, and so are the spin-orbit terms beta (1.5PN) and gamma
 * (2.5PN), from the spin-orbit parts of the energy and flux; beta and sigma
 * also against the Cutler-Flanagan mass-weighted form. Everything is FP64 with
 * the C library's cbrt/pow/log/sincos.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_NPARAM 11
#define OR_MAXD 16
#define OR_MAXDET 8

/* physical constants (SI) */
static const double OR_TSUN = 4.925490947641267e-6;    /* G Msun / c^3 [s] */
static const double OR_C = 299792458.0;                /* m/s */
static const double OR_MPC = 3.085677581491367e22;     /* m */
static const double OR_GAMMA_E = 0.5772156649015329;   /* Euler's constant */
static const double OR_PI = 3.14159265358979323846;

enum { P_MC, P_Q, P_CHI1, P_CHI2, P_DL, P_COSI, P_PSI, P_PHIC, P_TC, P_RA, P_SINDEC };
enum { PRIOR_FIXED = 0, PRIOR_UNIFORM = 1, PRIOR_VOLUME = 2 };
enum { MODEL_GW = 0, MODEL_TOY = 1 };

typedef struct {
    int model;               /* MODEL_GW or MODEL_TOY */
    /* GW problem */
    int n_det, N;
    double f0, df;           /* f_j = f0 + j df */
    const double *psd;       /* [n_det][N] */
    const double *d_re, *d_im; /* [n_det][N] */
    const double *pos;       /* [n_det][3] metres */
    const double *xarm, *yarm; /* [n_det][3] unit vectors */
    int ideal;               /* 1: F+ = 1, Fx = 0, no delay */
    int cutoff;              /* 1: h = 0 above f_ISCO */
    const int *kind;         /* [11] prior kind */
    const double *lo, *hi;   /* [11] */
    /* toy problem: x = toy_lo + (toy_hi - toy_lo) u, log L = -x^T P x / 2 + lognorm */
    int toy_d;
    const double *toy_prec;  /* [d][d] precision matrix */
    double toy_lognorm, toy_lo, toy_hi;
    /* relative binning (rb_nedge > 0): edges, summary data, fiducial point */
    int rb_nedge;
    const int *rb_J;
    const double *rb_sum[6];  /* A0re, A0im, A1re, A1im, B0, B1: [n_det][nedge-1] */
    const double *rb_theta_fid;
    /* bit i set: unit-cube coordinate i is periodic (uniform prior on a
     * periodic parameter): slice positions wrap mod 1 instead of leaving the box */
    unsigned periodic;
} or_problem;

/* ------------------------------------------------------------------ prior */

int or_dim(const or_problem *pb)
{
    if (pb->model == MODEL_TOY) return pb->toy_d;
    int d = 0;
    for (int p = 0; p < OR_NPARAM; p++) d += (pb->kind[p] != PRIOR_FIXED);
    return d;
}

/* Map a unit-cube point to the 11 physical parameters, in parameter order. */
void or_theta_from_u(const or_problem *pb, const double *u, double *theta)
{
    int i = 0;
    for (int p = 0; p < OR_NPARAM; p++) {
        double lo = pb->lo[p], hi = pb->hi[p];
        if (pb->kind[p] == PRIOR_FIXED) {
            theta[p] = lo;
        } else if (pb->kind[p] == PRIOR_UNIFORM) {
            theta[p] = lo + (hi - lo) * u[i++];
        } else { /* uniform in volume: p(x) ~ x^2 on [lo, hi] */
            double lo3 = lo * lo * lo, hi3 = hi * hi * hi;
            theta[p] = cbrt(lo3 + u[i++] * (hi3 - lo3));
        }
    }
}

/* ------------------------------------------------------------ waveform */

/* TaylorF2 phasing coefficients phi_k(v), k = 0..7, such that
 *   Psi(f) = 2 pi f t_c - phi_c - pi/4 + 3/(128 eta v^5) sum_k phi_k v^k,
 * with v = (pi M f)^(1/3) and delta = (m1 - m2)/M. The log(v) dependence of the 2.5PN and 3PN terms is
 * folded into phi_5 and phi_6. Spin terms: beta (1.5PN spin-orbit), sigma
 * (2PN spin-spin, aligned), gamma (2.5PN spin-orbit). */
void or_pn_phi(double eta, double delta, double chi1, double chi2, double v, double phi[8])
{
    double pi = OR_PI;
    double chis = 0.5 * (chi1 + chi2), chia = 0.5 * (chi1 - chi2);
    double beta = (113.0 / 12.0) * (chis + delta * chia - (76.0 / 113.0) * eta * chis);
    double sigma = (79.0 / 8.0) * eta * chi1 * chi2;
    double gamma = (732985.0 / 2268.0 - 24260.0 / 81.0 * eta - 340.0 / 9.0 * eta * eta) * chis
                 + (732985.0 / 2268.0 + 140.0 / 9.0 * eta) * delta * chia;
    phi[0] = 1.0;
    phi[1] = 0.0;
    phi[2] = 3715.0 / 756.0 + 55.0 / 9.0 * eta;
    phi[3] = -16.0 * pi + 4.0 * beta;
    phi[4] = 15293365.0 / 508032.0 + 27145.0 / 504.0 * eta + 3085.0 / 72.0 * eta * eta - 10.0 * sigma;
    phi[5] = (pi * (38645.0 / 756.0 - 65.0 / 9.0 * eta) - gamma) * (1.0 + 3.0 * log(v * sqrt(6.0)));
    phi[6] = 11583231236531.0 / 4694215680.0 - 640.0 / 3.0 * pi * pi - 6848.0 / 21.0 * OR_GAMMA_E
           + eta * (-15737765635.0 / 3048192.0 + 2255.0 / 12.0 * pi * pi)
           + 76055.0 / 1728.0 * eta * eta - 127825.0 / 1296.0 * eta * eta * eta
           - 6848.0 / 21.0 * log(4.0 * v);
    phi[7] = pi * (77096675.0 / 254016.0 + 378515.0 / 1512.0 * eta - 74045.0 / 756.0 * eta * eta);
}

/* Source-frame derived quantities used below. */
static void source_masses(const double *th, double *eta, double *mtot_s, double *mc_s)
{
    double q = th[P_Q];
    *eta = q / ((1.0 + q) * (1.0 + q));     /* m1 m2 / M^2 with q = m2/m1 */
    *mc_s = th[P_MC] * OR_TSUN;
    *mtot_s = *mc_s * pow(*eta, -0.6);        /* M = Mc eta^(-3/5) */
}

double or_fisco(const double *th)
{
    double eta, mt, mc;
    source_masses(th, &eta, &mt, &mc);
    return 1.0 / (pow(6.0, 1.5) * OR_PI * mt);
}

/* TaylorF2 phase Psi(f) (radians). */
double or_phase(const double *th, double f)
{
    double eta, mt, mc;
    source_masses(th, &eta, &mt, &mc);
    double v = cbrt(OR_PI * mt * f);
    double q = th[P_Q];
    double delta = (1.0 - q) / (1.0 + q);    /* (m1 - m2)/M, exact in q */
    double phi[8];
    or_pn_phi(eta, delta, th[P_CHI1], th[P_CHI2], v, phi);
    double sum = 0.0, vk = 1.0;
    for (int k = 0; k < 8; k++) { sum += phi[k] * vk; vk *= v; }
    double v5 = v * v * v * v * v;
    return 2.0 * OR_PI * f * th[P_TC] - th[P_PHIC] - OR_PI / 4.0 + 3.0 / (128.0 * eta * v5) * sum;
}

/* Stationary-phase amplitude A f^(-7/6) of a face-on source,
 * A = sqrt(5/24) pi^(-2/3) c T_Mc^(5/6) / D_L. */
double or_amplitude(const double *th, double f)
{
    double tmc = th[P_MC] * OR_TSUN;
    double dl = th[P_DL] * OR_MPC;
    return sqrt(5.0 / 24.0) * pow(OR_PI, -2.0 / 3.0) * OR_C * pow(tmc, 5.0 / 6.0) / dl * pow(f, -7.0 / 6.0);
}

/* h_+ and h_x at frequency f (complex, returned as re/im pairs):
 *   h_+ = A f^(-7/6) (1 + cos^2 i)/2 exp(-i Psi),  h_x = -i A f^(-7/6) cos i exp(-i Psi). */
void or_polarizations(const double *th, double f, double hp[2], double hc[2])
{
    double a = or_amplitude(th, f);
    double psi = or_phase(th, f);
    double c = cos(psi), s = sin(psi);      /* exp(-i Psi) = c - i s */
    double ci = th[P_COSI];
    double ap = a * 0.5 * (1.0 + ci * ci);
    double ac = a * ci;
    hp[0] = ap * c;
    hp[1] = -ap * s;
    /* -i (c - i s) = -s - i c */
    hc[0] = -ac * s;
    hc[1] = -ac * c;
}

/* Antenna patterns of a detector with arm unit vectors x, y (detector tensor
 * D = (x x^T - y y^T)/2) for a source at right ascension ra (Greenwich sidereal
 * time taken as 0) and declination asin(sindec), polarisation angle psi. */
void or_antenna(const double *x, const double *y, double ra, double sindec, double psi,
                double *fp, double *fc)
{
    double cosdec = sqrt(1.0 - sindec * sindec);
    double sa = sin(ra), ca = cos(ra), sp = sin(psi), cp = cos(psi);
    double X[3] = { sa * cp - sp * ca * sindec, -ca * cp - sp * sa * sindec, sp * cosdec };
    double Y[3] = { -sa * sp - cp * ca * sindec, ca * sp - cp * sa * sindec, cp * cosdec };
    double D[3][3];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) D[i][j] = 0.5 * (x[i] * x[j] - y[i] * y[j]);
    double xdx = 0, ydy = 0, xdy = 0, ydx = 0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            xdx += X[i] * D[i][j] * X[j];
            ydy += Y[i] * D[i][j] * Y[j];
            xdy += X[i] * D[i][j] * Y[j];
            ydx += Y[i] * D[i][j] * X[j];
        }
    *fp = xdx - ydy;
    *fc = xdy + ydx;
}

/* Arrival-time offset of a detector at position r relative to the geocentre,
 * dt = -(r . n)/c with n the unit vector towards the source. */
double or_delay(const double *r, double ra, double sindec)
{
    double cosdec = sqrt(1.0 - sindec * sindec);
    double n[3] = { cosdec * cos(ra), cosdec * sin(ra), sindec };
    return -(r[0] * n[0] + r[1] * n[1] + r[2] * n[2]) / OR_C;
}

static void det_response(const or_problem *pb, const double *th, int det,
                         double *fp, double *fc, double *dt)
{
    if (pb->ideal) { *fp = 1.0; *fc = 0.0; *dt = 0.0; return; }
    or_antenna(pb->xarm + 3 * det, pb->yarm + 3 * det, th[P_RA], th[P_SINDEC], th[P_PSI], fp, fc);
    *dt = or_delay(pb->pos + 3 * det, th[P_RA], th[P_SINDEC]);
}

/* Detector strain h_d(f_j) = (F+ h_+ + Fx h_x) exp(-2 pi i f dt), zero above
 * f_ISCO when the cutoff is on. Writes N complex values. */
void or_strain(const or_problem *pb, const double *th, int det, double *h_re, double *h_im)
{
    double fp, fc, dt;
    det_response(pb, th, det, &fp, &fc, &dt);
    double fisco = or_fisco(th);
    for (int j = 0; j < pb->N; j++) {
        double f = pb->f0 + j * pb->df;
        if (pb->cutoff && f > fisco) { h_re[j] = 0.0; h_im[j] = 0.0; continue; }
        double hp[2], hc[2];
        or_polarizations(th, f, hp, hc);
        double re = fp * hp[0] + fc * hc[0];
        double im = fp * hp[1] + fc * hc[1];
        double ph = -2.0 * OR_PI * f * dt;
        double c = cos(ph), s = sin(ph);
        h_re[j] = re * c - im * s;
        h_im[j] = re * s + im * c;
    }
}

/* Noise-weighted inner product <a|b> = 4 df Re sum_j a_j conj(b_j) / S_j on
 * detector det's PSD. */
double or_inner(const or_problem *pb, int det, const double *a_re, const double *a_im,
                const double *b_re, const double *b_im)
{
    const double *S = pb->psd + (size_t)det * pb->N;
    double acc = 0.0;
    for (int j = 0; j < pb->N; j++) acc += (a_re[j] * b_re[j] + a_im[j] * b_im[j]) / S[j];
    return 4.0 * pb->df * acc;
}

/* log-likelihood ratio against the noise-only model, plain definition:
 * sum over detectors and bins of 4 df [Re(d h^*) - |h|^2/2] / S. */
double or_loglike_theta(const or_problem *pb, const double *th)
{
    double fisco = or_fisco(th);
    double total = 0.0;
    for (int det = 0; det < pb->n_det; det++) {
        double fp, fc, dt;
        det_response(pb, th, det, &fp, &fc, &dt);
        const double *S = pb->psd + (size_t)det * pb->N;
        const double *dre = pb->d_re + (size_t)det * pb->N;
        const double *dim = pb->d_im + (size_t)det * pb->N;
        double acc = 0.0;
        for (int j = 0; j < pb->N; j++) {
            double f = pb->f0 + j * pb->df;
            if (pb->cutoff && f > fisco) continue;       /* h = 0 there */
            double hp[2], hc[2];
            or_polarizations(th, f, hp, hc);
            double re = fp * hp[0] + fc * hc[0];
            double im = fp * hp[1] + fc * hc[1];
            double ph = -2.0 * OR_PI * f * dt;
            double c = cos(ph), s = sin(ph);
            double hr = re * c - im * s, hi = re * s + im * c;
            double dh = dre[j] * hr + dim[j] * hi;        /* Re(d h^*) */
            double hh = hr * hr + hi * hi;
            acc += (dh - 0.5 * hh) / S[j];
        }
        total += 4.0 * pb->df * acc;
    }
    return total;
}

double or_toy_loglike(const or_problem *pb, const double *u)
{
    int d = pb->toy_d;
    double x[OR_MAXD];
    for (int i = 0; i < d; i++) x[i] = pb->toy_lo + (pb->toy_hi - pb->toy_lo) * u[i];
    double q = 0.0;
    for (int i = 0; i < d; i++)
        for (int j = 0; j < d; j++) q += x[i] * pb->toy_prec[i * d + j] * x[j];
    return -0.5 * q + pb->toy_lognorm;
}

double or_loglike_rb(const or_problem *pb, const double *theta_fid, const int *J, int nedge,
                     const double *A0re, const double *A0im, const double *A1re, const double *A1im,
                     const double *B0, const double *B1, const double *theta);

double or_loglike_u(const or_problem *pb, const double *u)
{
    if (pb->model == MODEL_TOY) return or_toy_loglike(pb, u);
    double th[OR_NPARAM];
    or_theta_from_u(pb, u, th);
    if (pb->rb_nedge > 0)
        return or_loglike_rb(pb, pb->rb_theta_fid, pb->rb_J, pb->rb_nedge, pb->rb_sum[0], pb->rb_sum[1],
                             pb->rb_sum[2], pb->rb_sum[3], pb->rb_sum[4], pb->rb_sum[5], th);
    return or_loglike_theta(pb, th);
}

void or_loglike_batch(const or_problem *pb, const double *u, int m, double *out, int nthreads)
{
    int d = or_dim(pb);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int i = 0; i < m; i++) out[i] = or_loglike_u(pb, u + (size_t)i * d);
}

void or_loglike_theta_batch(const or_problem *pb, const double *th, int m, double *out, int nthreads)
{
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int i = 0; i < m; i++) out[i] = or_loglike_theta(pb, th + (size_t)i * OR_NPARAM);
}

/* ---------------------------------------------------------- Philox4x32-10 */

/* One Philox4x32-10 block: 10 rounds of the multiply-xor bijection with the
 * Weyl key schedule (Salmon et al. 2011, Sec. 4). */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Draw stream layout shared with the library (key = 64-bit seed):
 *   counter = (slot, step, chain_or_point, iteration).
 * A uniform in (0,1) is built from two words: 26 + 26 bits, (x + 1/2) 2^-52. */
static void draw(uint64_t seed, uint32_t slot, uint32_t step, uint32_t idx, uint32_t iter, uint32_t w[4])
{
    uint32_t ctr[4] = { slot, step, idx, iter };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    or_philox4x32_10(ctr, key, w);
}

double or_u01(uint32_t a, uint32_t b)
{
    uint64_t x = ((uint64_t)(a >> 6) << 26) | (uint64_t)(b >> 6);
    return ((double)x + 0.5) * (1.0 / 4503599627370496.0);   /* 2^-52 */
}

#define SLOT_OFFSET 16u
#define SLOT_SHRINK0 17u
#define STEP_START 0xFFFFFFFFu
#define ITER_INIT 0xFFFFFFFFu
#define ITER_REPLICATE 0xFFFFFFFEu

/* Initial live points: point i, dimensions 2p and 2p+1 from slot p. */
void or_initial_points(uint64_t seed, int n, int d, double *u)
{
    for (int i = 0; i < n; i++)
        for (int p = 0; 2 * p < d; p++) {
            uint32_t w[4];
            draw(seed, (uint32_t)p, 0u, (uint32_t)i, ITER_INIT, w);
            u[(size_t)i * d + 2 * p] = or_u01(w[0], w[1]);
            if (2 * p + 1 < d) u[(size_t)i * d + 2 * p + 1] = or_u01(w[2], w[3]);
        }
}

/* Replicate shrinkage draws for the evidence error: log t = log(U)/n_j. */
double or_replicate_uniform(uint64_t seed, int replicate, long long dead_index)
{
    uint32_t w[4];
    draw(seed, 0u, (uint32_t)dead_index, (uint32_t)replicate, ITER_REPLICATE, w);
    return or_u01(w[0], w[1]);
}

void or_replicate_uniforms(uint64_t seed, int replicate, long long m, double *out)
{
    for (long long i = 0; i < m; i++) out[i] = or_replicate_uniform(seed, replicate, i);
}

/* -------------------------------------------------------- slice sampling */

/* Candidate on the line x + t e; periodic coordinates wrapped into [0, 1). */
static void line_point(const or_problem *pb, int d, const double *x, double t, const double *e, double *y)
{
    for (int i = 0; i < d; i++) {
        y[i] = x[i] + t * e[i];
        if ((pb->periodic >> i) & 1u) y[i] -= floor(y[i]);
    }
}

static int in_slice(const or_problem *pb, int d, const double *y, double lstar, double *ly, long long *evals)
{
    for (int i = 0; i < d; i++)
        if (!(y[i] >= 0.0 && y[i] <= 1.0)) return 0;      /* prior-bound rejection, no evaluation */
    *ly = or_loglike_u(pb, y);
    (*evals)++;
    return *ly > lstar;
}

/* Evolve one chain of the iteration: start from a uniformly chosen survivor,
 * then `steps` slice-sampling updates along hit-and-run directions
 * e = L z / |z| (z ~ N(0, I), L the Cholesky factor of the survivors'
 * covariance, so e has unit Mahalanobis length and the initial bracket width
 * is 1), with stepping out on both sides (at most max_stepout steps per side)
 * and shrinkage (at most max_shrink draws) as in Neal (2003), Sec. 4. */
static void evolve_chain(const or_problem *pb, uint64_t seed, uint32_t iter, int chain, int d,
                         const double *surv_u, const double *surv_logl, int m,
                         const double *chol, double lstar, int steps, int max_stepout,
                         int max_shrink, double *out_u, double *out_logl,
                         long long *evals, int *caps)
{
    double x[OR_MAXD], y[OR_MAXD], e[OR_MAXD], z[OR_MAXD];
    uint32_t w[4];
    draw(seed, 0u, STEP_START, (uint32_t)chain, iter, w);
    int idx = (int)(or_u01(w[0], w[1]) * m);
    if (idx >= m) idx = m - 1;
    for (int i = 0; i < d; i++) x[i] = surv_u[(size_t)idx * d + i];
    double lx = surv_logl[idx];

    for (int s = 0; s < steps; s++) {
        /* direction: Box-Muller normals, two per draw */
        for (int p = 0; 2 * p < d; p++) {
            draw(seed, (uint32_t)p, (uint32_t)s, (uint32_t)chain, iter, w);
            double u1 = or_u01(w[0], w[1]), u2 = or_u01(w[2], w[3]);
            double r = sqrt(-2.0 * log(u1));
            z[2 * p] = r * cos(2.0 * OR_PI * u2);
            if (2 * p + 1 < d) z[2 * p + 1] = r * sin(2.0 * OR_PI * u2);
        }
        double nz = 0.0;
        for (int i = 0; i < d; i++) nz += z[i] * z[i];
        nz = sqrt(nz);
        for (int i = 0; i < d; i++) {
            double acc = 0.0;
            for (int j = 0; j <= i; j++) acc += chol[i * d + j] * z[j];
            e[i] = acc / nz;
        }
        /* bracket of width 1 placed at a random offset around 0 */
        draw(seed, SLOT_OFFSET, (uint32_t)s, (uint32_t)chain, iter, w);
        double r = or_u01(w[0], w[1]);
        double a = -r, b = 1.0 - r, ly;
        for (int n = 0; n < max_stepout; n++) {
            line_point(pb, d, x, a, e, y);
            if (!in_slice(pb, d, y, lstar, &ly, evals)) break;
            a -= 1.0;
        }
        for (int n = 0; n < max_stepout; n++) {
            line_point(pb, d, x, b, e, y);
            if (!in_slice(pb, d, y, lstar, &ly, evals)) break;
            b += 1.0;
        }
        /* shrinkage */
        int accepted = 0;
        for (int n = 0; n < max_shrink; n++) {
            draw(seed, SLOT_SHRINK0 + (uint32_t)n, (uint32_t)s, (uint32_t)chain, iter, w);
            double t = a + (b - a) * or_u01(w[0], w[1]);
            line_point(pb, d, x, t, e, y);
            if (in_slice(pb, d, y, lstar, &ly, evals)) {
                for (int i = 0; i < d; i++) x[i] = y[i];
                lx = ly;
                accepted = 1;
                break;
            }
            if (t < 0.0) a = t; else b = t;
        }
        if (!accepted) (*caps)++;
    }
    for (int i = 0; i < d; i++) out_u[(size_t)chain * d + i] = x[i];
    out_logl[chain] = lx;
}

/* Constrained random walk (the acceptance-walk alternative to slice sampling
 * as an inner kernel): from a uniformly chosen survivor, `walk` proposals
 * y = x + scale L z (z ~ N(0, I) from the draws of proposal p, L the
 * Cholesky factor of the survivors' covariance) are accepted when inside the
 * prior box (periodic coordinates wrapped) and above L*, otherwise the walk
 * stays. A uniform prior restricted to L > L* is the walk's stationary law
 * (symmetric proposal, rejection outside the constraint) for any fixed walk
 * length; the length adapts between iterations only (or_walk_next). Adds the
 * accepted moves to *accepted. */
static void evolve_walk(const or_problem *pb, uint64_t seed, uint32_t iter, int chain, int d,
                        const double *surv_u, const double *surv_logl, int m, const double *chol,
                        double lstar, int walk, double scale, double *out_u,
                        double *out_logl, long long *evals, long long *accepted)
{
    double x[OR_MAXD], y[OR_MAXD], z[OR_MAXD];
    uint32_t w[4];
    draw(seed, 0u, STEP_START, (uint32_t)chain, iter, w);
    int idx = (int)(or_u01(w[0], w[1]) * m);
    if (idx >= m) idx = m - 1;
    for (int i = 0; i < d; i++) x[i] = surv_u[(size_t)idx * d + i];
    double lx = surv_logl[idx], ly;
    long long acc_moves = 0;
    for (int p = 0; p < walk; p++) {
        for (int q = 0; 2 * q < d; q++) {
            draw(seed, (uint32_t)q, (uint32_t)p, (uint32_t)chain, iter, w);
            double u1 = or_u01(w[0], w[1]), u2 = or_u01(w[2], w[3]);
            double r = sqrt(-2.0 * log(u1));
            z[2 * q] = r * cos(2.0 * OR_PI * u2);
            if (2 * q + 1 < d) z[2 * q + 1] = r * sin(2.0 * OR_PI * u2);
        }
        for (int i = 0; i < d; i++) {
            double acc = 0.0;
            for (int j = 0; j <= i; j++) acc += chol[i * d + j] * z[j];
            y[i] = x[i] + acc * scale;
            if ((pb->periodic >> i) & 1u) y[i] -= floor(y[i]);
        }
        if (in_slice(pb, d, y, lstar, &ly, evals)) {
            for (int i = 0; i < d; i++) x[i] = y[i];
            lx = ly;
            acc_moves++;
        }
    }
    *accepted += acc_moves;
    for (int i = 0; i < d; i++) out_u[(size_t)chain * d + i] = x[i];
    out_logl[chain] = lx;
}

/* The k walks of one iteration; *accepted receives their accepted moves. */
long long or_evolve_walk(const or_problem *pb, int nthreads, uint64_t seed, uint32_t iter, int k,
                         const double *surv_u, const double *surv_logl, int m, const double *chol,
                         double lstar, int walk, double scale, double *out_u, double *out_logl,
                         long long *accepted)
{
    int d = or_dim(pb);
    long long total = 0, acc = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total, acc) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int c = 0; c < k; c++) {
        long long ev = 0, a = 0;
        evolve_walk(pb, seed, iter, c, d, surv_u, surv_logl, m, chol, lstar, walk, scale, out_u,
                    out_logl, &ev, &a);
        total += ev;
        acc += a;
    }
    *accepted = acc;
    return total;
}

/* Walk length of the next iteration, as in bilby's acceptance walk: scaled so
 * that a walk would make `target` accepted moves at this iteration's
 * acceptance (accepted moves over k walks of length walk), kept within
 * [target, 64 target]. */
int or_walk_next(int walk, int target, int k, long long accepted)
{
    if (accepted <= 0) return 64 * target;
    double t = ceil(((double)walk * (double)target) * (double)k / (double)accepted);
    if (t < (double)target) t = (double)target;
    if (t > 64.0 * (double)target) t = 64.0 * (double)target;
    return (int)t;
}

/* Evolve chains first .. first + count - 1 of one iteration (chains are
 * independent: a chain's draws are keyed by its own index, so a subset of the
 * chains follows exactly the trajectories those chains have in the whole
 * iteration; OpenMP over chains does not change any result). out_u and
 * out_logl are indexed by the chain (first + count entries). Returns the total
 * number of likelihood evaluations; caps receives the number of steps that hit
 * the shrink cap. */
long long or_evolve_chains(const or_problem *pb, int nthreads, uint64_t seed, uint32_t iter, int first,
                           int count, const double *surv_u, const double *surv_logl, int m,
                           const double *chol, double lstar, int steps, int max_stepout,
                           int max_shrink, double *out_u, double *out_logl, int *caps)
{
    int d = or_dim(pb);
    long long total = 0;
    int capsum = 0;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total, capsum) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (int c = first; c < first + count; c++) {
        long long ev = 0;
        int cp = 0;
        evolve_chain(pb, seed, iter, c, d, surv_u, surv_logl, m, chol, lstar, steps,
                     max_stepout, max_shrink, out_u, out_logl, &ev, &cp);
        total += ev;
        capsum += cp;
    }
    *caps = capsum;
    return total;
}

/* All k chains of one iteration (or_evolve_chains over 0 .. k-1). */
long long or_evolve(const or_problem *pb, int nthreads, uint64_t seed, uint32_t iter, int k,
                    const double *surv_u, const double *surv_logl, int m, const double *chol,
                    double lstar, int steps, int max_stepout, int max_shrink,
                    double *out_u, double *out_logl, int *caps)
{
    return or_evolve_chains(pb, nthreads, seed, iter, 0, k, surv_u, surv_logl, m, chol, lstar, steps,
                            max_stepout, max_shrink, out_u, out_logl, caps);
}

/* ------------------------------------------------------ relative binning */

/* Coarse-bin edges: B+1 geometric frequencies f0 (f_last/f0)^(b/B), each moved
 * to the nearest grid index; repeated indices are dropped. Writes the edge
 * indices to J and returns their count (= number of bins + 1). */
int or_rb_edges(const or_problem *pb, int B, int *J)
{
    double flo = pb->f0, fhi = pb->f0 + (pb->N - 1) * pb->df;
    int n = 0;
    for (int b = 0; b <= B; b++) {
        double target = flo * pow(fhi / flo, (double)b / B);
        int j = (int)floor((target - pb->f0) / pb->df + 0.5);
        if (j < 0) j = 0;
        if (j > pb->N - 1) j = pb->N - 1;
        if (b == B) j = pb->N - 1;
        if (n == 0 || j > J[n - 1]) J[n++] = j;
    }
    return n;
}

/* Fine bins of coarse bin b: J[b] <= j < J[b+1], the last bin also holding
 * J[nb]. Centre frequency: midpoint of the edge frequencies. */
static int rb_hi(const int *J, int nb, int b) { return (b == nb - 1) ? J[b + 1] + 1 : J[b + 1]; }

/* Summary data of detector det against the fiducial strain h0 (no cutoff):
 * A0 = 4 df sum d h0^* / S, A1 = 4 df sum d h0^* / S (f - fm),
 * B0 = 4 df sum |h0|^2 / S,  B1 = 4 df sum |h0|^2 / S (f - fm), per coarse bin. */
void or_rb_summary(const or_problem *pb, const double *theta_fid, const int *J, int nedge,
                   double *A0re, double *A0im, double *A1re, double *A1im, double *B0, double *B1)
{
    int nb = nedge - 1;
    or_problem nc = *pb;
    nc.cutoff = 0;
    double *hr = (double *)malloc(sizeof(double) * pb->N), *hi = (double *)malloc(sizeof(double) * pb->N);
    for (int det = 0; det < pb->n_det; det++) {
        or_strain(&nc, theta_fid, det, hr, hi);
        const double *S = pb->psd + (size_t)det * pb->N;
        const double *dre = pb->d_re + (size_t)det * pb->N, *dim = pb->d_im + (size_t)det * pb->N;
        for (int b = 0; b < nb; b++) {
            double fm = 0.5 * ((pb->f0 + J[b] * pb->df) + (pb->f0 + J[b + 1] * pb->df));
            double a0r = 0, a0i = 0, a1r = 0, a1i = 0, b0 = 0, b1 = 0;
            for (int j = J[b]; j < rb_hi(J, nb, b); j++) {
                double f = pb->f0 + j * pb->df;
                double w = 4.0 * pb->df / S[j];
                /* d h0^* */
                double xr = dre[j] * hr[j] + dim[j] * hi[j];
                double xi = dim[j] * hr[j] - dre[j] * hi[j];
                double hh = hr[j] * hr[j] + hi[j] * hi[j];
                a0r += w * xr; a0i += w * xi;
                a1r += w * xr * (f - fm); a1i += w * xi * (f - fm);
                b0 += w * hh; b1 += w * hh * (f - fm);
            }
            size_t o = (size_t)det * nb + b;
            A0re[o] = a0r; A0im[o] = a0i; A1re[o] = a1r; A1im[o] = a1i; B0[o] = b0; B1[o] = b1;
        }
    }
    free(hr);
    free(hi);
}

/* Relative-binning log-likelihood: r = h/h0 at the bin edges (both without
 * cutoff), r0 = (r(e_b) + r(e_b+1))/2, r1 = (r(e_b+1) - r(e_b))/(e_b+1 - e_b),
 * <d|h> = Re sum_b [A0 r0^* + A1 r1^*], <h|h> = sum_b [B0 |r0|^2 + 2 B1 Re(r0 r1^*)],
 * with bins whose centre lies above f_ISCO(theta) dropped when the cutoff is on. */
double or_loglike_rb(const or_problem *pb, const double *theta_fid, const int *J, int nedge,
                     const double *A0re, const double *A0im, const double *A1re, const double *A1im,
                     const double *B0, const double *B1, const double *theta)
{
    int nb = nedge - 1;
    double fisco = or_fisco(theta);
    double total = 0.0;
    for (int det = 0; det < pb->n_det; det++) {
        double fp, fc, dt, fp0, fc0, dt0;
        det_response(pb, theta, det, &fp, &fc, &dt);
        det_response(pb, theta_fid, det, &fp0, &fc0, &dt0);
        double prev_r = 0, prev_i = 0;
        double dh = 0.0, hh = 0.0;
        for (int e = 0; e < nedge; e++) {
            double f = pb->f0 + J[e] * pb->df;
            double hp[2], hc[2], gp[2], gc[2];
            or_polarizations(theta, f, hp, hc);
            or_polarizations(theta_fid, f, gp, gc);
            double ph = -2.0 * OR_PI * f * dt, ph0 = -2.0 * OR_PI * f * dt0;
            double hr = fp * hp[0] + fc * hc[0], hi = fp * hp[1] + fc * hc[1];
            double h0r = fp0 * gp[0] + fc0 * gc[0], h0i = fp0 * gp[1] + fc0 * gc[1];
            double c = cos(ph), s_ = sin(ph), c0 = cos(ph0), s0 = sin(ph0);
            double Hr = hr * c - hi * s_, Hi = hr * s_ + hi * c;
            double H0r = h0r * c0 - h0i * s0, H0i = h0r * s0 + h0i * c0;
            double den = H0r * H0r + H0i * H0i;
            double rr = (Hr * H0r + Hi * H0i) / den, ri = (Hi * H0r - Hr * H0i) / den;
            if (e > 0) {
                int b = e - 1;
                double fm = 0.5 * ((pb->f0 + J[b] * pb->df) + f);
                if (!(pb->cutoff && fm > fisco)) {
                    double r0r = 0.5 * (prev_r + rr), r0i = 0.5 * (prev_i + ri);
                    double de = f - (pb->f0 + J[b] * pb->df);
                    double r1r = (rr - prev_r) / de, r1i = (ri - prev_i) / de;
                    size_t o = (size_t)det * nb + b;
                    /* Re(A0 r0^* + A1 r1^*) */
                    dh += A0re[o] * r0r + A0im[o] * r0i + A1re[o] * r1r + A1im[o] * r1i;
                    hh += B0[o] * (r0r * r0r + r0i * r0i) + 2.0 * B1[o] * (r0r * r1r + r0i * r1i);
                }
            }
            prev_r = rr;
            prev_i = ri;
        }
        total += dh - 0.5 * hh;
    }
    return total;
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
