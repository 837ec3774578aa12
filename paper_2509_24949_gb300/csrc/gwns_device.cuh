// gwns_device.cuh -- device-side building blocks of the nested-slice-sampling
// hot path on sm_103a: problem description, Philox4x32-10, prior transform,
// per-point waveform coefficients, and the per-bin likelihood loops in FP64 and
// in mixed precision (double-float phase, FP32 sincos and products).
//
// The likelihood is the Whittle log-likelihood ratio of a TaylorF2 signal
// (paper Sec. 3 uses the same likelihood with an IMRPhenomD waveform):
//   log L = sum_d [ Re(G_d Z_d) - <h_d|h_d>/2 ],
//   Z_d   = sum_{j <= jcut} w_dj exp(i Psi_dj),  w_dj = 4 df f_j^(-7/6) d_dj / S_dj,
//   G_d   = A conj(Q_d),  Q_d = F+ (1 + cos^2 i)/2 - i Fx cos i,
//   Psi_dj = sum_m a_m B_m(f_j) + c0 + 2 pi f_j (t_c + dt_d),
//   <h_d|h_d> = A^2 |Q_d|^2 P_d(jcut),  P_d(j) = sum_{i <= j} 4 df f_i^(-7/3) / S_di,
// with the TaylorF2 phase written as a dot product of per-point coefficients
// a_m with the per-grid basis B = {f^-5/3, f^-1, f^-2/3, f^-1/3, ln f, f^1/3,
// f^1/3 ln f, f^2/3}, so that no transcendental of f is evaluated per bin.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "gwns_df.cuh"
#include "gwns_tables.cuh"

namespace gwns {

constexpr int NPARAM = 11;
constexpr int MAXD = 16;
constexpr int MAXDET = 4;
constexpr int NB = 8;

enum { P_MC = 0, P_Q, P_CHI1, P_CHI2, P_DL, P_COSI, P_PSI, P_PHIC, P_TC, P_RA, P_SINDEC };
enum { K_FIXED = 0, K_UNIFORM = 1, K_VOLUME = 2 };
enum { M_GW = 0, M_TOY = 1 };

constexpr double TSUN = 4.925490947641267e-6;   // G Msun / c^3 [s]
constexpr double C_SI = 299792458.0;
constexpr double MPC_SI = 3.085677581491367e22;
constexpr double GAMMA_E = 0.5772156649015329;
constexpr double PI_D = 3.141592653589793;
constexpr double TWO_PI_D = 6.283185307179586;
constexpr double INV_TWO_PI_D = 0.15915494309189535;

// Problem description passed by value to every kernel.
struct Model {
    int model;        // M_GW or M_TOY
    int n_det, N, ideal, cutoff, dim;
    int rb;           // 1: relative-binning likelihood on the coarse bins
    int coop;         // 1: mixed slice update spreads each candidate's tile groups over all warps
    unsigned periodic;   // bit i: unit-cube coordinate i wraps mod 1 on the slice line
    int tlg;          // mixed form: 0 per bin, else log2 of the bins per lane tile (tiled form)
    int np;           // tiled form: N padded to whole groups of 32 tiles
    double f0, df;
    double inv_df;    // 1 / df
    int kind[NPARAM];
    double lo[NPARAM], hi[NPARAM];
    double pbase[NPARAM], pspan[NPARAM];   // uniform: lo, hi - lo; volume: lo^3, hi^3 - lo^3
    double pos[MAXDET][3], xarm[MAXDET][3], yarm[MAXDET][3];
    // toy: x = toy_lo + (toy_hi - toy_lo) u, Sigma_ij = rho^|i-j|
    double toy_lo, toy_hi, toy_rho, toy_lognorm;
    // mixed form's coefficient stage in double-float (cdf = 1): parameter p is
    // pbase_x[p] + pspan_x[p] u[uidx[p]] (a fixed parameter: its value and a
    // zero span), df_x the bin spacing
    int cdf;
    int uidx[NPARAM];
    dfl pbase_x[NPARAM], pspan_x[NPARAM];
    dfl df_x;
};

// Relative-binning (heterodyned) tables: coarse bins between grid indices
// J[b] .. J[b+1], summary data of the fiducial waveform h0 per detector and
// bin, and the phase basis at the edge frequencies.
struct Coef;
struct RBTables {
    int nedge, nb;
    const double *fe;          // [nedge] edge frequencies
    const double *basis64;     // [NB][nedge]
    const float2 *basis32;     // [NB][nedge] (hi, lo)
    const float2 *fe32;        // [nedge] (hi, lo)
    const double *fm;          // [nb] bin centres (cutoff test)
    const double *inv_de;      // [nb] 1/(e_{b+1} - e_b)
    const double2 *A0, *A1;    // [n_det][nb] sum d h0^* w, sum d h0^* w (f - fm)
    const double *B0, *B1;     // [n_det][nb] sum |h0|^2 w, sum |h0|^2 w (f - fm)
    const float2 *A0f, *A1f;   // FP32 copies for the mixed form
    const float *B0f, *B1f, *inv_de_f;
    const Coef *fid;           // fiducial point's coefficients
};

// Device tables of one grid.
struct Tables {
    const double *basis64;   // [NB][N]   B_m(f_j)
    const double *f64;       // [N]       f_j
    const double2 *w64;      // [n_det][N] weighted data
    const double *prefix;    // [n_det][N] P_d(j)
    // mixed form, per bin (Model::tlg == 0)
    const float2 *basis32;   // [NB][N]   B_m(f_j) as (hi, lo) floats
    const float2 *f32;       // [N]       f_j as (hi, lo)
    const float2 *w32;       // [n_det][N]
    // mixed form, tiled (Model::tlg > 0): tile t = bins tL .. tL + L - 1 about
    // its centre c = tL + L/2, L = 1 << tlg, nt = np / L tiles
    const float2 *tb0;       // [NB][nt]  B_m(f_c) as (hi, lo)
    const float2 *tb1;       // [NB][nt]  B_m'(f_c) df as (hi, lo)
    const float *tbk;        // [TK-1][NB][nt] B_m^(k)(f_c) df^k / k!, k = 2..TK
    const float2 *fc;        // [nt]      f_c as (hi, lo)
    const float2 *wt;        // [n_det][np] weighted data, pair-tile order (zero beyond N)
    int g_lo;                // tile groups g >= g_lo take the Taylor degree TK_LO, the rest TK
    RBTables rb;             // used when Model::rb is set
};

// Per-point likelihood coefficients.
struct Coef {
    double a[NB];          // phase coefficients [rad per basis unit]
    double c0;             // constant phase [rad]
    double tau[MAXDET];    // t_c + dt_d [s]
    double gre[MAXDET], gim[MAXDET];   // G_d = A conj(Q_d)
    double hh;             // sum_d <h_d|h_d>
    double toy;            // toy model log L
    double rot_re[MAXDET], rot_im[MAXDET];   // exp(2 pi i rot_stride df tau_d) (FP64 loop)
    double fisco;          // f_ISCO [Hz]
    double amp;            // Newtonian amplitude factor A
    int jcut;              // last bin with f_j <= f_ISCO (-1: none)
    int pad;
};

// Mixed-precision view of the coefficients: phase in turns as (hi, lo) floats.
struct CoefMixed {
    float ah[NB], al[NB];
    float c0h, c0l;
    float tauh[MAXDET], taul[MAXDET];
    float dtau[MAXDET];     // df tau_d: phase advance per bin [turns]
    // tiled form, detectors d >= 1 against detector 0: beta_d = 2 pi df (tau_d - tau_0)
    // [rad per bin], rho_d = exp(-i beta_d), eps8_d = exp(-8 i beta_d) - 1 (its real part
    // -2 sin^2(4 beta_d) kept to full relative precision); rho2_d = rho_d^2, the
    // step between the even (odd) bins of a tile
    float beta[MAXDET];
    float rho[MAXDET][2];
    float rho2[MAXDET][2];
    float eps8[MAXDET][2];
};

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon et al. 2011): 10 rounds of the multiply-xor bijection
// with the Weyl key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; r++) {
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Draw-stream layout (key = 64-bit seed): counter = (slot, step, index, iteration).
constexpr uint32_t SLOT_OFFSET = 16u;
constexpr uint32_t SLOT_SHRINK0 = 17u;
constexpr uint32_t STEP_START = 0xFFFFFFFFu;
constexpr uint32_t ITER_INIT = 0xFFFFFFFFu;
constexpr uint32_t ITER_REPLICATE = 0xFFFFFFFEu;

__device__ __forceinline__ uint4 draw(uint64_t seed, uint32_t slot, uint32_t step, uint32_t idx,
                                      uint32_t iter) {
    return philox4x32_10(make_uint4(slot, step, idx, iter), (uint32_t)seed, (uint32_t)(seed >> 32));
}

// Uniform in (0,1): 26 + 26 bits of two words, (x + 1/2) 2^-52 (exact in FP64).
__device__ __forceinline__ double u01(uint32_t a, uint32_t b) {
    uint64_t x = ((uint64_t)(a >> 6) << 26) | (uint64_t)(b >> 6);
    return ((double)x + 0.5) * 2.220446049250313e-16;
}

// ------------------------------------------- FP64 exp and log (table-driven)
// The per-point coefficient stage is FP64 and, on grids of a few thousand bins
// per evaluation, its instruction count binds; these two functions follow
// Tang's table-driven method (ACM TOMS 15 (1989) 144; 16 (1990) 378): reduce
// against a table point, then a short polynomial. Tables: gwns_tables.cuh.

// exp(x) = 2^m 2^(j/64) (1 + p(r)) with x = (64 m + j) ln2/64 + r, |r| <= ln2/128,
// p the degree-5 Taylor polynomial of e^r - 1 (truncation below 4e-17) and
// 2^(j/64) as hi + lo; within 1 ulp for |x| < 700 with a normal result (the
// coefficient stage's arguments lie in [-60, 10]).
__device__ __forceinline__ double exp_tab(double x) {
    const double shift = 6755399441055744.0;                     // 1.5 2^52
    const double kk = fma(x, 0x1.71547652b82fep+6, shift);       // 64 / ln 2
    const int ki = __double2loint(kk);
    const double k = kk - shift;
    double r = fma(-k, 0x1.62e42fef00000p-7, x);                 // ln2/64, 33-bit head
    r = fma(-k, 0x1.473de6af278edp-40, r);                       // and its tail
    const int j = ki & 63, m = ki >> 6;
    double q = fma(r, 1.0 / 120.0, 1.0 / 24.0);
    q = fma(q, r, 1.0 / 6.0);
    q = fma(q, r, 0.5);
    const double p = fma(r * r, q, r);
    const double th = __ldg(EXP_T_HI + j), tl = __ldg(EXP_T_LO + j);
    const double res = th + fma(th, p, tl);
    return __hiloint2double(__double2hiint(res) + (m << 20), __double2loint(res));
}

// ln x = e ln 2 - ln c + ln(1 + r) with x = 2^e m, m in [1, 2), c the table's
// double nearest 1/(1 + (j + 1/2)/128) for the top 7 fraction bits j of m,
// r = m c - 1 (|r| < 0.004, one rounding) and ln(1 + r) by its degree-6 Taylor
// polynomial (truncation below 1e-17); -ln c and ln 2 as hi + lo. Within 1 ulp
// of max(1, |ln x|) for positive normal x.
__device__ __forceinline__ double log_tab(double x) {
    const int hi = __double2hiint(x), lo = __double2loint(x);
    const int e = ((hi >> 20) & 0x7ff) - 1023;
    const int j = (hi >> 13) & 127;
    const double m = __hiloint2double((hi & 0x000fffff) | 0x3ff00000, lo);
    const double r = fma(m, __ldg(LOG_INV_C + j), -1.0);
    double q = fma(r, -1.0 / 6.0, 0.2);
    q = fma(q, r, -0.25);
    q = fma(q, r, 1.0 / 3.0);
    q = fma(q, r, -0.5);
    const double p = fma(r * r, q, r);
    const double ed = (double)e;
    const double h = fma(ed, 0x1.62e42fef00000p-1, __ldg(LOG_NLN_HI + j));   // ln 2, 33-bit head
    const double l = fma(ed, 0x1.473de6af278edp-34, __ldg(LOG_NLN_LO + j)) + p;
    return h + l;
}

// 1 / x for 1 <= x <= 2 (the mass-ratio factor 1 / (1 + q)): an FP32 reciprocal
// refined by two Newton steps y <- y + y (1 - x y) (error 2^-23 -> 2^-92, then
// the final rounding).
__device__ __forceinline__ double recip_12(double x) {
    double y = (double)__frcp_rn((float)x);
    y = fma(y, fma(-x, y, 1.0), y);
    return fma(y, fma(-x, y, 1.0), y);
}

__device__ __forceinline__ void sincos_bf(double x, double &s, double &c);

// ------------------------------------------------------------ prior transform
__device__ __forceinline__ double prior_one(const Model &M, int p, double u) {
    double lo = M.lo[p], hi = M.hi[p];
    if (M.kind[p] == K_UNIFORM) return __dadd_rn(lo, __dmul_rn(__dsub_rn(hi, lo), u));
    double lo3 = lo * lo * lo, hi3 = hi * hi * hi;
    return cbrt(__dadd_rn(lo3, __dmul_rn(u, __dsub_rn(hi3, lo3))));
}

// u[dim] -> theta[11], in parameter order (fixed parameters take lo).
__device__ __forceinline__ void prior_transform(const Model &M, const double *u, double *th) {
    int i = 0;
#pragma unroll
    for (int p = 0; p < NPARAM; p++) {
        if (M.kind[p] == K_FIXED) th[p] = M.lo[p];
        else th[p] = prior_one(M, p, u[i++]);
    }
}

// --------------------------------------------------------- point coefficients
// Last grid index with f_j <= fisco, in [-1, N-1], from the grid's frequency
// table (f64[j] holds the rounded f0 + j*df the tables use): a first guess by
// one multiplication, then at most a few steps either way against the table.
__device__ __forceinline__ int cutoff_index_tab(const Model &M, const double *f64, double fisco) {
    if (!M.cutoff) return M.N - 1;
    const double jf = floor((fisco - M.f0) * M.inv_df);
    if (!(jf >= -1.0)) return -1;
    int j = jf > (double)(M.N - 1) ? M.N - 1 : (int)jf;
    for (int it = 0; it < 4 && j + 1 <= M.N - 1 && __ldg(f64 + j + 1) <= fisco; it++) j++;
    for (int it = 0; it < 4 && j >= 0 && __ldg(f64 + j) > fisco; it++) j--;
    return j;
}

// eta-polynomial part of each phase coefficient, c0 + c1 eta + c2 eta^2 + c3 eta^3,
// in basis order (f^-5/3, f^-1, f^-2/3, f^-1/3, ln f, f^1/3, f^1/3 ln f, f^2/3):
// 1; phi_2; phi_3 without spin; phi_4 without spin; phi_5 without spin (the
// ln v part of the 2.5PN term, 3 ln v = 3 ln a + ln f); phi_6 without its log
// term; the f^1/3 ln f part -6848/63 of the 3PN log; phi_7.
#define GWNS_PN_POLY(F)                                                                          \
    F(1.0), F(0.0), F(0.0), F(0.0),                                                              \
    F(3715.0 / 756.0), F(55.0 / 9.0), F(0.0), F(0.0),                                            \
    F(-16.0 * PI_D), F(0.0), F(0.0), F(0.0),                                                     \
    F(15293365.0 / 508032.0), F(27145.0 / 504.0), F(3085.0 / 72.0), F(0.0),                      \
    F(PI_D * 38645.0 / 756.0), F(-PI_D * 65.0 / 9.0), F(0.0), F(0.0),                            \
    F(11583231236531.0 / 4694215680.0 - 640.0 / 3.0 * PI_D * PI_D - 6848.0 / 21.0 * GAMMA_E),    \
    F(-15737765635.0 / 3048192.0 + 2255.0 / 12.0 * PI_D * PI_D), F(76055.0 / 1728.0),            \
    F(-127825.0 / 1296.0),                                                                       \
    F(-6848.0 / 63.0), F(0.0), F(0.0), F(0.0),                                                   \
    F(PI_D * 77096675.0 / 254016.0), F(PI_D * 378515.0 / 1512.0), F(-PI_D * 74045.0 / 756.0), F(0.0)
#define GWNS_AS_DOUBLE(x) (x)
__device__ const double PN_POLY[NB * 4] = {GWNS_PN_POLY(GWNS_AS_DOUBLE)};
// the same as double-floats, for the mixed form's coefficient stage
__device__ const dfl PN_POLY_X[NB * 4] = {GWNS_PN_POLY(DFC)};

// Per-point coefficients, computed by lane groups of 8: group g of the calling
// warp handles point g (g < count), so one warp computes up to four points at
// the cost of one (FP64 costs one warp instruction whatever the number of
// active lanes). Inside a group, parameter-only quantities are computed
// redundantly by all 8 lanes (uniform control flow), transcendentals of
// independent arguments are packed into different lanes of a single call (one
// log, one exp, one sincos), and the detector terms run on sub-lanes
// 0 .. n_det-1. The distance enters only through ln D_L, so a uniform-in-volume
// distance needs no cube root. u0 + g*ustride: point g's unit-cube coordinates;
// out0[g]: its coefficients. rot_stride > 0 also stores, per detector,
// exp(2 pi i rot_stride df tau_d), the rotation between bins rot_stride apart
// used by the FP64 bin loop. GW model only; all 32 lanes must call.
__device__ inline void point_coef_group(const Model &M, const Tables &T, const double *u0, int ustride,
                                        Coef *out0, int count, int rot_stride, int half = 0) {
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31, g = lane >> 3, sl = lane & 7;
    const bool writer = g < count;
    const double *u = u0 + (writer ? g : 0) * ustride;
    Coef *out = out0 + (writer ? g : 0);
    // prior transform; a uniform-in-volume distance keeps its volume argument
    double th[NPARAM];
    double dl_arg = 0.0;
    bool dl_vol = false;
    {
        int i = 0;
#pragma unroll
        for (int p = 0; p < NPARAM; p++) {
            // each half transforms only the parameters it uses (mass and phase:
            // chirp mass, q, spins, distance, phi_c; sky and detectors: cos i,
            // psi, t_c, RA, sin dec)
            const bool mass_p = p == P_MC || p == P_Q || p == P_CHI1 || p == P_CHI2 || p == P_DL || p == P_PHIC;
            if (M.kind[p] == K_FIXED) {
                th[p] = M.lo[p];
            } else if ((half == 1 && !mass_p) || (half == 2 && mass_p)) {
                th[p] = 0.0;
                i++;
            } else if (M.kind[p] == K_UNIFORM) {
                th[p] = fma(M.pspan[p], u[i++], M.pbase[p]);
            } else {
                const double v = fma(M.pspan[p], u[i++], M.pbase[p]);
                if (p == P_DL) { dl_vol = true; dl_arg = v; th[p] = 0.0; }
                else th[p] = cbrt(v);
            }
        }
        if (!dl_vol) dl_arg = th[P_DL];
    }
    // mass and phase part (half 0 or 1)
    double amp = 0.0;
    int jcut = -1;
    if (half != 2) {
        const double q = th[P_Q];
        const double r1q = recip_12(1.0 + q);
        const double eta = q * r1q * r1q;               // m1 m2 / M^2
        const double delta = (1.0 - q) * r1q;           // (m1 - m2)/M, m1 >= m2
        const double chis = 0.5 * (th[P_CHI1] + th[P_CHI2]);
        const double chia = 0.5 * (th[P_CHI1] - th[P_CHI2]);
        const double tmc = th[P_MC] * TSUN;
        // packed log: sub-lane 0 ln(eta), 1 ln(T_Mc), others ln(D_L) (or of D_L^3)
        const double lg = log_tab(sl == 0 ? eta : (sl == 1 ? tmc : dl_arg));
        const double ln_eta = __shfl_sync(FULL, lg, 0, 8);
        const double ln_tmc = __shfl_sync(FULL, lg, 1, 8);
        const double ln_dlx = __shfl_sync(FULL, lg, 2, 8);
        const double ln_dl = dl_vol ? ln_dlx * (1.0 / 3.0) : ln_dlx;
        // ln(pi T_M) with T_M = T_Mc eta^(-3/5); a = (pi T_M)^(1/3), v = a f^(1/3)
        const double ln_x = 1.1447298858494002 + ln_tmc - 0.6 * ln_eta;
        const double ln_a = ln_x * (1.0 / 3.0);
        // packed exp: 0 a, 1 1/a, 2 1/(pi T_M), 3 K = 3/(128 eta),
        // others A = sqrt(5/24) pi^(-2/3) c T_Mc^(5/6) / D_L (D_L in Mpc)
        const double ex_arg = sl == 0 ? ln_a
                            : sl == 1 ? -ln_a
                            : sl == 2 ? -ln_x
                            : sl == 3 ? -3.7534179752515073 - ln_eta
                            : -33.81250354619071 + (5.0 / 6.0) * ln_tmc - ln_dl;
        const double ex = exp_tab(ex_arg);
        const double a = __shfl_sync(FULL, ex, 0, 8);
        const double ia = __shfl_sync(FULL, ex, 1, 8);
        const double inv_pitm = __shfl_sync(FULL, ex, 2, 8);
        const double K = __shfl_sync(FULL, ex, 3, 8);
        amp = __shfl_sync(FULL, ex, 4, 8);
        // f_ISCO = 1/(6^(3/2) pi T_M)
        jcut = cutoff_index_tab(M, T.f64, inv_pitm * 0.06804138174397717);

        // TaylorF2 phasing (3.5PN non-spinning + aligned-spin beta, sigma, gamma):
        // sub-lane m computes basis coefficient m = K a^e_m (P_m(eta) + s_m), with
        // K v^(k-5) = K a^(k-5) f^((k-5)/3), P_m the eta polynomial of its PN order
        // and s_m its spin (or log) term.
        const double pi = PI_D;
        const double beta = (113.0 / 12.0) * (chis + delta * chia - (76.0 / 113.0) * eta * chis);
        const double sigma = (79.0 / 8.0) * eta * th[P_CHI1] * th[P_CHI2];
        const double gamma = (732985.0 / 2268.0 - 24260.0 / 81.0 * eta - 340.0 / 9.0 * eta * eta) * chis
                           + (732985.0 / 2268.0 + 140.0 / 9.0 * eta) * delta * chia;
        {
            const int m = sl;
            // |e_m| for e = (-5, -3, -2, -1, 0, 1, 1, 2); negative powers from 1/a
            const int e = m == 0 ? 5 : m == 1 ? 3 : (m == 2 || m == 7) ? 2 : m == 4 ? 0 : 1;
            const double base = m < 4 ? ia : a;
            const double b2 = base * base;
            double pw = (e & 1) ? base : 1.0;
            pw *= (e & 2) ? b2 : 1.0;
            pw *= (e & 4) ? b2 * b2 : 1.0;
            const double *pc = PN_POLY + 4 * m;
            const double poly = fma(fma(fma(__ldg(pc + 3), eta, __ldg(pc + 2)), eta, __ldg(pc + 1)), eta, __ldg(pc));
            const double sp = m == 2 ? 4.0 * beta
                            : m == 3 ? -10.0 * sigma
                            : m == 4 ? -gamma
                            : m == 5 ? -6848.0 / 21.0 * (1.3862943611198906 + ln_a) : 0.0;
            if (writer) out->a[m] = K * pw * (poly + sp);
        }
        if (sl == 0 && writer) {
            // constant: -phi_c - pi/4 + K phi5 (1 + 3 ln sqrt 6 + 3 ln a), reduced mod 2 pi
            const double phi5 = pi * (38645.0 / 756.0 - 65.0 / 9.0 * eta) - gamma;
            const double c0 = -th[P_PHIC] - 0.25 * pi + K * phi5 * (1.0 + 3.0 * 0.8958797346140275 + 3.0 * ln_a);
            out->c0 = c0 - TWO_PI_D * rint(c0 * INV_TWO_PI_D);
            out->jcut = jcut;
            out->fisco = inv_pitm * 0.06804138174397717;
            out->amp = amp;
        }
    }
    // sky and detector part (half 0 or 2)
    if (half == 1) return;
    const double ci = th[P_COSI];
    // packed sincos: sub-lane 0 ra, others psi
    double sn, cs;
    sincos_bf(sl == 0 ? th[P_RA] : th[P_PSI], sn, cs);
    const double sa = __shfl_sync(FULL, sn, 0, 8), ca = __shfl_sync(FULL, cs, 0, 8);
    const double sp = __shfl_sync(FULL, sn, 1, 8), cp = __shfl_sync(FULL, cs, 1, 8);
    double hh_part = 0.0, tau = 0.0;
    if (sl < M.n_det) {
        const int dd = sl;
        double fp, fc, dt;
        if (M.ideal) {
            fp = 1.0; fc = 0.0; dt = 0.0;
        } else {
            const double sd = th[P_SINDEC];
            const double cd = sqrt(1.0 - sd * sd);
            // wave-frame basis X, Y (Anderson et al. 2001) and source direction n
            const double X0 = sa * cp - sp * ca * sd, X1 = -ca * cp - sp * sa * sd, X2 = sp * cd;
            const double Y0 = -sa * sp - cp * ca * sd, Y1 = ca * sp - cp * sa * sd, Y2 = cp * cd;
            const double *x = M.xarm[dd], *y = M.yarm[dd];
            // D = (x x^T - y y^T)/2: X^T D Y = ((x.X)(x.Y) - (y.X)(y.Y))/2
            const double xX = x[0] * X0 + x[1] * X1 + x[2] * X2;
            const double xY = x[0] * Y0 + x[1] * Y1 + x[2] * Y2;
            const double yX = y[0] * X0 + y[1] * X1 + y[2] * X2;
            const double yY = y[0] * Y0 + y[1] * Y1 + y[2] * Y2;
            fp = 0.5 * ((xX * xX - yX * yX) - (xY * xY - yY * yY));
            fc = (xX * xY - yX * yY);
            const double *r = M.pos[dd];
            dt = -(r[0] * cd * ca + r[1] * cd * sa + r[2] * sd) * (1.0 / C_SI);
        }
        const double qre = fp * 0.5 * (1.0 + ci * ci);
        const double qim = -fc * ci;
        tau = th[P_TC] + dt;
        if (writer) {
            out->tau[dd] = tau;
            // half 2 leaves the amplitude to point_coef_join
            out->gre[dd] = half == 2 ? qre : amp * qre;
            out->gim[dd] = half == 2 ? -qim : -amp * qim;
        }
        if (half == 0 && jcut >= 0)
            hh_part = amp * amp * (qre * qre + qim * qim) * T.prefix[(size_t)dd * M.N + jcut];
    }
    if (rot_stride > 0) {
        double rs, rc;
        sincos(TWO_PI_D * ((double)rot_stride * M.df) * tau, &rs, &rc);
        if (sl < M.n_det && writer) { out->rot_re[sl] = rc; out->rot_im[sl] = rs; }
    }
    if (half == 2) return;
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) hh_part += __shfl_xor_sync(FULL, hh_part, o, 8);
    if (sl == 0 && writer) out->hh = hh_part;
}

// After the two halves of point_coef_group ran on ns points (different warps,
// then a barrier): one warp applies the amplitude to G_d and forms <h|h>.
// Lane = (point, detector).
__device__ __forceinline__ void point_coef_join(const Model &M, const Tables &T, Coef *c, int ns) {
    const int lane = threadIdx.x & 31, nd = M.n_det;
    const int pnt = lane / nd, dd = lane - pnt * nd;
    double hh = 0.0;
    if (pnt < ns && lane < 32 / nd * nd) {
        const double amp = c[pnt].amp, qre = c[pnt].gre[dd], nqim = c[pnt].gim[dd];
        c[pnt].gre[dd] = amp * qre;
        c[pnt].gim[dd] = amp * nqim;
        const int jcut = c[pnt].jcut;
        if (jcut >= 0) hh = amp * amp * (qre * qre + nqim * nqim) * T.prefix[(size_t)dd * M.N + jcut];
    }
    // sum over the point's detectors (lanes pnt*nd .. pnt*nd + nd - 1)
    double t = hh;
    for (int k = 1; k < nd; k++) t += __shfl_down_sync(0xffffffffu, hh, k);
    if (dd == 0 && pnt < ns && lane < 32 / nd * nd) c[pnt].hh = t;
}

// Coefficients of one point by one warp (toy model, or GW via lane group 0).
__device__ inline void point_coef_warp(const Model &M, const Tables &T, const double *u, Coef *out,
                                       int rot_stride = 0) {
    const int lane = threadIdx.x & 31;
    if (M.model == M_TOY) {
        // log N(x; 0, Sigma) with Sigma_ij = rho^|i-j|: the inverse is tridiagonal,
        // (1/(1-rho^2)) [diag(1, 1+rho^2, ..., 1+rho^2, 1), off-diagonal -rho].
        int d = M.dim;
        double rho = M.toy_rho;
        double xi = 0.0, xn = 0.0;
        if (lane < d) xi = M.toy_lo + (M.toy_hi - M.toy_lo) * u[lane];
        if (lane + 1 < d) xn = M.toy_lo + (M.toy_hi - M.toy_lo) * u[lane + 1];
        double diag = (lane == 0 || lane == d - 1) ? 1.0 : 1.0 + rho * rho;
        double term = 0.0;
        if (lane < d) term = diag * xi * xi - ((lane + 1 < d) ? 2.0 * rho * xi * xn : 0.0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) term += __shfl_xor_sync(0xffffffffu, term, o);
        if (lane == 0) {
            out->toy = -0.5 * term / (1.0 - rho * rho) + M.toy_lognorm;
            out->jcut = -1;
            out->hh = 0.0;
        }
        return;
    }
    point_coef_group(M, T, u, 0, out, 1, rot_stride);
}

// Split a double into (hi, lo) floats.
__device__ __forceinline__ void split_df(double x, float &h, float &l) {
    h = __double2float_rn(x);
    l = __double2float_rn(x - (double)h);
}

// Mixed-precision coefficients (phase in turns), from lane-parallel
// conversions; with fid, the differences from the fiducial point's; with rot,
// the rotation constants of the tiled form's long tiles too.
__device__ __forceinline__ void coef_to_mixed_warp(const Coef &c, int n_det, double df, CoefMixed *m,
                                                   const Coef *fid = nullptr, bool rot = false) {
    const int lane = threadIdx.x & 31;
    // phase coefficients (lanes 0..7, in turns), constant phase (lane 8, turns)
    // and delays (lanes 16..): one common path, so each FP64 step is one warp
    // instruction for all three
    const bool isa = lane < NB, isc = lane == NB, ist = lane >= 16 && lane < 16 + n_det;
    const int ia = isa ? lane : 0, it = ist ? lane - 16 : 0;
    double v = isa ? c.a[ia] : (isc ? c.c0 : c.tau[it]);
    if (fid) v -= isa ? fid->a[ia] : (isc ? fid->c0 : fid->tau[it]);
    const double y = ist ? v : v * INV_TWO_PI_D;
    float yh, yl;
    split_df(y, yh, yl);
    if (isa) { m->ah[ia] = yh; m->al[ia] = yl; }
    else if (isc) { m->c0h = yh; m->c0l = yl; }
    else if (ist) { m->tauh[it] = yh; m->taul[it] = yl; }
    if (lane >= 24 && lane < 24 + n_det) {
        const int d = lane - 24;
        const double td = c.tau[d] - (fid ? fid->tau[d] : 0.0), t0 = c.tau[0] - (fid ? fid->tau[0] : 0.0);
        m->dtau[d] = __double2float_rn(df * td);
        if (!rot) return;
        // the rotation of detector d's phase against detector 0's per bin, its
        // unit, two-bin and eight-bin steps (FP32 libm sine: within 2 ulp)
        const float b = __double2float_rn(TWO_PI_D * df * (td - t0));
        const float h1 = sinf(0.5f * b), h2 = sinf(b), h4 = sinf(4.0f * b);
        m->beta[d] = b;
        m->rho[d][0] = 1.0f - 2.0f * h1 * h1;
        m->rho[d][1] = -h2;
        m->rho2[d][0] = 1.0f - 2.0f * h2 * h2;
        m->rho2[d][1] = -sinf(2.0f * b);
        m->eps8[d][0] = -2.0f * h4 * h4;
        m->eps8[d][1] = -sinf(8.0f * b);
    }
}

// Mixed form: the coefficients of up to four unit-cube points (lane groups of
// 8, as point_coef_group) in double-float on the FP32 pipe, written straight
// into the mixed view (phase coefficients and constant in turns, delays in
// seconds, as (hi, lo) floats; the per-bin delay phase; with rot, the tiled
// form's rotation constants) and into the FP64 fields the log L combine reads
// (G_d, <h|h>, jcut, amp, fisco). The steps and the lane packing are those of
// point_coef_group: the prior transform (here lane-parallel, one parameter per
// sub-lane), one packed log (ln eta, ln T_Mc, ln D_L), one packed exp (a, 1/a,
// 1/(pi T_M), 3/(128 eta), the amplitude), one basis coefficient per sub-lane,
// one packed sine/cosine (RA, psi) and the detector terms on sub-lanes
// 0 .. n_det-1. Same halves: 1 mass and phase, 2 sky and detectors (G_d without
// the amplitude, joined by point_coef_join), 0 both. GW model, uniform priors
// and a uniform-in-volume distance (Model::cdf); all 32 lanes must call.
__device__ __forceinline__ dfl shfl_df(dfl v, int src) {
    return dfl{__shfl_sync(0xffffffffu, v.h, src, 8), __shfl_sync(0xffffffffu, v.l, src, 8)};
}

__device__ inline void point_coef_group_mx(const Model &M, const Tables &T, const double *u0, int ustride,
                                           Coef *out0, CoefMixed *cm0, int count, bool rot, int half = 0) {
    const int lane = threadIdx.x & 31, g = lane >> 3, sl = lane & 7;
    const bool writer = g < count;
    const double *u = u0 + (writer ? g : 0) * ustride;
    Coef *out = out0 + (writer ? g : 0);
    CoefMixed *cm = cm0 + (writer ? g : 0);
    // prior transform: sub-lane s forms parameters s and s + 8
    dfl thp[2];
#pragma unroll
    for (int r = 0; r < 2; r++) {
        const int p = sl + 8 * r < NPARAM ? sl + 8 * r : 0;
        const dfl ux = df_from_double(u[M.uidx[p]]);
        thp[r] = df_add(df_mul(M.pspan_x[p], ux), M.pbase_x[p]);
    }
    auto TH = [&](int p) { return shfl_df(p < 8 ? thp[0] : thp[1], p & 7); };
    const dfl one = dfl{1.0f, 0.0f};
    dfl amp = dfl{0.0f, 0.0f};
    int jcut = -1;
    // mass and phase part (half 0 or 1)
    if (half != 2) {
        const dfl q = TH(P_Q), c1 = TH(P_CHI1), c2 = TH(P_CHI2);
        const dfl mc = TH(P_MC), dlx = TH(P_DL), phic = TH(P_PHIC);
        const dfl r1q = df_rcp(df_add_f(q, 1.0f));
        const dfl eta = df_mul(q, df_sqr(r1q));                     // m1 m2 / M^2
        const dfl delta = df_mul(df_sub(one, q), r1q);              // (m1 - m2)/M
        const dfl chis = df_scale(df_add(c1, c2), 0.5f);
        const dfl chia = df_scale(df_sub(c1, c2), 0.5f);
        const dfl tmc = df_mul(mc, DFC(TSUN));
        // packed log: sub-lane 0 ln(eta), 1 ln(T_Mc), others ln(D_L) (or of D_L^3)
        const dfl lg = df_log(sl == 0 ? eta : (sl == 1 ? tmc : dlx));
        const dfl ln_eta = shfl_df(lg, 0), ln_tmc = shfl_df(lg, 1), ln_dlx = shfl_df(lg, 2);
        const dfl ln_dl = M.kind[P_DL] == K_VOLUME ? df_mul(ln_dlx, DFC(1.0 / 3.0)) : ln_dlx;
        // ln(pi T_M) with T_M = T_Mc eta^(-3/5); a = (pi T_M)^(1/3), v = a f^(1/3)
        const dfl ln_x = df_add(df_add(DFC(1.1447298858494002), ln_tmc), df_mul(ln_eta, DFC(-0.6)));
        const dfl ln_a = df_mul(ln_x, DFC(1.0 / 3.0));
        // packed exp: 0 a, 1 1/a, 2 1/(pi T_M), 3 K = 3/(128 eta),
        // others A = sqrt(5/24) pi^(-2/3) c T_Mc^(5/6) / D_L (D_L in Mpc)
        const dfl ex_arg = sl == 0 ? ln_a
                         : sl == 1 ? df_neg(ln_a)
                         : sl == 2 ? df_neg(ln_x)
                         : sl == 3 ? df_sub(DFC(-3.7534179752515073), ln_eta)
                         : df_sub(df_add(DFC(-33.81250354619071), df_mul(ln_tmc, DFC(5.0 / 6.0))), ln_dl);
        const dfl ex = df_exp(ex_arg);
        const dfl a = shfl_df(ex, 0), ia = shfl_df(ex, 1), inv_pitm = shfl_df(ex, 2), K = shfl_df(ex, 3);
        amp = shfl_df(ex, 4);
        // f_ISCO = 1/(6^(3/2) pi T_M); the cutoff index against the FP64 frequency table
        const double fisco = df_to_double(df_mul(inv_pitm, DFC(0.06804138174397717)));
        jcut = cutoff_index_tab(M, T.f64, fisco);
        // TaylorF2 phasing: sub-lane m computes basis coefficient m = K a^e_m (P_m(eta) + s_m)
        const dfl beta = df_mul(df_add(df_add(chis, df_mul(delta, chia)), df_mul(df_mul(eta, chis), DFC(-76.0 / 113.0))),
                                DFC(113.0 / 12.0));
        const dfl sigma = df_mul(df_mul(df_mul(eta, c1), c2), DFC(79.0 / 8.0));
        const dfl gamma = df_add(
            df_mul(df_add(df_add(DFC(732985.0 / 2268.0), df_mul(eta, DFC(-24260.0 / 81.0))),
                          df_mul(df_sqr(eta), DFC(-340.0 / 9.0))), chis),
            df_mul(df_mul(df_add(DFC(732985.0 / 2268.0), df_mul(eta, DFC(140.0 / 9.0))), delta), chia));
        {
            const int m = sl;
            // |e_m| for e = (-5, -3, -2, -1, 0, 1, 1, 2); negative powers from 1/a
            const int e = m == 0 ? 5 : m == 1 ? 3 : (m == 2 || m == 7) ? 2 : m == 4 ? 0 : 1;
            const dfl base = m < 4 ? ia : a;
            const dfl b2 = df_sqr(base);
            dfl pw = (e & 1) ? base : one;
            if (e & 2) pw = df_mul(pw, b2);
            if (e & 4) pw = df_mul(pw, df_sqr(b2));
            const float2 *pc = reinterpret_cast<const float2 *>(PN_POLY_X + 4 * m);
            const float2 p0 = __ldg(pc), p1 = __ldg(pc + 1), p2 = __ldg(pc + 2), p3 = __ldg(pc + 3);
            dfl poly = df_add(df_mul(dfl{p3.x, p3.y}, eta), dfl{p2.x, p2.y});
            poly = df_add(df_mul(poly, eta), dfl{p1.x, p1.y});
            poly = df_add(df_mul(poly, eta), dfl{p0.x, p0.y});
            const dfl sp = m == 2 ? df_scale(beta, 4.0f)
                         : m == 3 ? df_mul(sigma, DFC(-10.0))
                         : m == 4 ? df_neg(gamma)
                         : m == 5 ? df_mul(df_add(DFC(1.3862943611198906), ln_a), DFC(-6848.0 / 21.0))
                                  : dfl{0.0f, 0.0f};
            // in turns
            const dfl am = df_mul(df_mul(df_mul(K, pw), df_add(poly, sp)), DFC(INV_TWO_PI_D));
            if (writer) { cm->ah[m] = am.h; cm->al[m] = am.l; }
        }
        if (sl == 0 && writer) {
            // constant: -phi_c - pi/4 + K phi5 (1 + 3 ln sqrt 6 + 3 ln a), in turns, reduced mod 1
            const dfl phi5 = df_sub(df_add(DFC(PI_D * 38645.0 / 756.0), df_mul(eta, DFC(-PI_D * 65.0 / 9.0))), gamma);
            const dfl lnf = df_add(DFC(1.0 + 3.0 * 0.8958797346140275), df_mul(ln_a, DFC(3.0)));
            dfl c0 = df_sub(df_mul(df_mul(K, phi5), lnf), df_add(phic, DFC(0.25 * PI_D)));
            c0 = df_mul(c0, DFC(INV_TWO_PI_D));
            c0 = df_add_f(c0, -rintf(c0.h));
            cm->c0h = c0.h;
            cm->c0l = c0.l;
            out->jcut = jcut;
            out->fisco = fisco;
            out->amp = df_to_double(amp);
        }
    }
    // sky and detector part (half 0 or 2)
    if (half == 1) return;
    const dfl ci = TH(P_COSI), tc = TH(P_TC), sd = TH(P_SINDEC);
    // packed sine and cosine: sub-lane 0 RA, others psi (both shuffled by every lane)
    const dfl ra = TH(P_RA), psi = TH(P_PSI);
    dfl sn, cs;
    df_sincos(sl == 0 ? ra : psi, sn, cs);
    const dfl sa = shfl_df(sn, 0), ca = shfl_df(cs, 0), sp = shfl_df(sn, 1), cp = shfl_df(cs, 1);
    const int dd = sl < M.n_det ? sl : 0;
    dfl qre, qim, dt = dfl{0.0f, 0.0f};
    if (M.ideal) {
        qre = df_scale(df_add_f(df_sqr(ci), 1.0f), 0.5f);
        qim = dfl{0.0f, 0.0f};
    } else {
        const dfl cd = df_sqrt(df_sub(one, df_sqr(sd)));
        // wave-frame basis X, Y (Anderson et al. 2001) and source direction n
        const dfl X0 = df_sub(df_mul(sa, cp), df_mul(df_mul(sp, ca), sd));
        const dfl X1 = df_neg(df_add(df_mul(ca, cp), df_mul(df_mul(sp, sa), sd)));
        const dfl X2 = df_mul(sp, cd);
        const dfl Y0 = df_neg(df_add(df_mul(sa, sp), df_mul(df_mul(cp, ca), sd)));
        const dfl Y1 = df_sub(df_mul(ca, sp), df_mul(df_mul(cp, sa), sd));
        const dfl Y2 = df_mul(cp, cd);
        dfl x[3], y[3], r[3];
#pragma unroll
        for (int i = 0; i < 3; i++) {
            x[i] = df_from_double(M.xarm[dd][i]);
            y[i] = df_from_double(M.yarm[dd][i]);
            r[i] = df_from_double(M.pos[dd][i]);
        }
        // D = (x x^T - y y^T)/2
        const dfl xX = df_add(df_add(df_mul(x[0], X0), df_mul(x[1], X1)), df_mul(x[2], X2));
        const dfl xY = df_add(df_add(df_mul(x[0], Y0), df_mul(x[1], Y1)), df_mul(x[2], Y2));
        const dfl yX = df_add(df_add(df_mul(y[0], X0), df_mul(y[1], X1)), df_mul(y[2], X2));
        const dfl yY = df_add(df_add(df_mul(y[0], Y0), df_mul(y[1], Y1)), df_mul(y[2], Y2));
        const dfl fp = df_scale(df_sub(df_sub(df_sqr(xX), df_sqr(yX)), df_sub(df_sqr(xY), df_sqr(yY))), 0.5f);
        const dfl fc = df_sub(df_mul(xX, xY), df_mul(yX, yY));
        const dfl rn = df_add(df_add(df_mul(df_mul(r[0], cd), ca), df_mul(df_mul(r[1], cd), sa)), df_mul(r[2], sd));
        dt = df_mul(rn, DFC(-1.0 / C_SI));
        qre = df_mul(fp, df_scale(df_add_f(df_sqr(ci), 1.0f), 0.5f));
        qim = df_neg(df_mul(fc, ci));
    }
    const dfl tau = df_add(tc, dt);
    const dfl tau0 = shfl_df(tau, 0);
    if (sl < M.n_det && writer) {
        cm->tauh[dd] = tau.h;
        cm->taul[dd] = tau.l;
        cm->dtau[dd] = df_mul(tau, M.df_x).h;
        if (half == 2) {
            out->gre[dd] = df_to_double(qre);
            out->gim[dd] = -df_to_double(qim);
        } else {
            out->gre[dd] = df_to_double(df_mul(amp, qre));
            out->gim[dd] = -df_to_double(df_mul(amp, qim));
        }
        if (rot) {
            // the rotation of detector d's phase against detector 0's per bin, its
            // unit, two-bin and eight-bin steps (FP32 libm sine: within 2 ulp)
            const float b = df_mul(df_mul(df_sub(tau, tau0), M.df_x), DFC(TWO_PI_D)).h;
            const float h1 = sinf(0.5f * b), h2 = sinf(b), h4 = sinf(4.0f * b);
            cm->beta[dd] = b;
            cm->rho[dd][0] = 1.0f - 2.0f * h1 * h1;
            cm->rho[dd][1] = -h2;
            cm->rho2[dd][0] = 1.0f - 2.0f * h2 * h2;
            cm->rho2[dd][1] = -sinf(2.0f * b);
            cm->eps8[dd][0] = -2.0f * h4 * h4;
            cm->eps8[dd][1] = -sinf(8.0f * b);
        }
    }
    if (half == 2) return;
    double hh_part = 0.0;
    if (sl < M.n_det && jcut >= 0) {
        // A^2 (~1e-42) is below the float range: square the amplitude in FP64
        const double a = df_to_double(amp);
        hh_part = a * a * df_to_double(df_add(df_sqr(qre), df_sqr(qim))) * T.prefix[(size_t)dd * M.N + jcut];
    }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) hh_part += __shfl_xor_sync(0xffffffffu, hh_part, o, 8);
    if (sl == 0 && writer) out->hh = hh_part;
}

// ------------------------------------------------------------ bin loops
// Branch-free FP64 sine and cosine for |x| < 2^16 pi/2 (TaylorF2 phases are
// below 1e5 rad): Cody-Waite reduction r = x - k pi/2 with pi/2 split into
// three parts of which the first two have 36 significant bits (k pi/2_i exact
// for |k| < 2^17), k taken by the 1.5 2^52 rounding shift (its low mantissa
// bits give the quadrant); then the Taylor series of sin and cos about 0 up to
// r^15 and r^16 (truncation below 5e-17 for |r| <= pi/4) and the quadrant's
// swap and signs by selects. Having no branch, two calls interleave.
__device__ __forceinline__ void sincos_bf(double x, double &s, double &c) {
    const double shift = 6755399441055744.0;                  // 1.5 * 2^52
    const double kk = fma(x, 0.6366197723675814, shift);      // 2/pi
    const int q = __double2loint(kk) & 3;
    const double k = kk - shift;
    double r = fma(-k, 1.5707963267923333, x);
    r = fma(-k, 2.5633441515839558e-12, r);
    r = fma(-k, 1.0562999066987428e-23, r);
    const double r2 = r * r;
    // sin r = r + r^3 (-1/3! + r^2 (1/5! - ...)), up to r^15/15!
    double ps = -7.647163731819816e-13;
    ps = fma(ps, r2, 1.6059043836821613e-10);
    ps = fma(ps, r2, -2.505210838544172e-08);
    ps = fma(ps, r2, 2.7557319223985893e-06);
    ps = fma(ps, r2, -0.0001984126984126984);
    ps = fma(ps, r2, 0.008333333333333333);
    ps = fma(ps, r2, -0.16666666666666666);
    const double sn = fma(r * r2, ps, r);
    // cos r = 1 + r^2 (-1/2! + r^2 (1/4! - ...)), up to r^16/16!
    double pc = 4.779477332387385e-14;
    pc = fma(pc, r2, -1.1470745597729725e-11);
    pc = fma(pc, r2, 2.08767569878681e-09);
    pc = fma(pc, r2, -2.755731922398589e-07);
    pc = fma(pc, r2, 2.48015873015873e-05);
    pc = fma(pc, r2, -0.001388888888888889);
    pc = fma(pc, r2, 0.041666666666666664);
    pc = fma(pc, r2, -0.5);
    const double cs = fma(r2, pc, 1.0);
    // quadrant q: (sin, cos) = (sn, cs), (cs, -sn), (-sn, -cs), (-cs, sn)
    const double a = (q & 1) ? cs : sn;
    const double b = (q & 1) ? sn : cs;
    s = (q & 2) ? -a : a;
    c = ((q + 1) & 2) ? -b : b;
}

// FP64: Psi_j from the basis (FP64 FMAs), exp(i Psi_j) by sincos, the detector
// factor exp(2 pi i f_j tau_d) by a rotation recurrence along the thread's bins
// (f advances by stride*df per step).
// With PRE_ROT the coefficients carry the rotation for a stride of 32 bins;
// the stride here is 32 << rot_sq (the rotation squared rot_sq times).
template <int NDET, bool PRE_ROT = false>
__device__ __forceinline__ void bins_fp64(const Tables &T, int N, double f0, double df, const Coef &c,
                                          int tid, int stride, double zr[NDET], double zi[NDET],
                                          int rot_sq = 0) {
    double a[NB];
#pragma unroll
    for (int m = 0; m < NB; m++) a[m] = c.a[m];
    const double c0 = c.c0;
    // the thread's bins j_n = tid + n stride, n = 0 .. nb-1; the detector factor
    // exp(2 pi i f_j tau_d) = R_d rho_d^n with R_d at j_0 and rho_d the rotation
    // over one stride, so Z_d = R_d sum_n (w_dj exp(i Psi_j)) rho_d^n, evaluated
    // by Horner's rule from the last bin down: per bin and detector a complex
    // product and a Horner step (8 FP64) instead of advancing, applying and
    // accumulating a running phasor (12)
    const int nb = tid <= c.jcut ? (c.jcut - tid) / stride + 1 : 0;
    double pr[NDET], pi_[NDET], hr[NDET], hi[NDET];
#pragma unroll
    for (int d = 0; d < NDET; d++) {
        hr[d] = 0.0; hi[d] = 0.0;
        if (PRE_ROT) {
            pr[d] = c.rot_re[d];
            pi_[d] = c.rot_im[d];
            for (int q = 0; q < rot_sq; q++) {
                const double re = pr[d] * pr[d] - pi_[d] * pi_[d];
                pi_[d] = 2.0 * pr[d] * pi_[d];
                pr[d] = re;
            }
        } else if (nb > 0) {
            sincos_bf(TWO_PI_D * (stride * df) * c.tau[d], pi_[d], pr[d]);
        }
    }
    for (int n = nb - 1; n >= 0; n--) {
        const int j = tid + n * stride;
        double psi = c0;
#pragma unroll
        for (int m = 0; m < NB; m++) psi = fma(a[m], __ldg(T.basis64 + (size_t)m * N + j), psi);
        double s, co;
        sincos_bf(psi, s, co);
#pragma unroll
        for (int d = 0; d < NDET; d++) {
            const double2 w = __ldg(T.w64 + (size_t)d * N + j);
            const double cr = fma(w.x, co, -w.y * s), ci = fma(w.x, s, w.y * co);
            const double h2r = fma(hr[d], pr[d], fma(-hi[d], pi_[d], cr));
            const double h2i = fma(hr[d], pi_[d], fma(hi[d], pr[d], ci));
            hr[d] = h2r;
            hi[d] = h2i;
        }
    }
#pragma unroll
    for (int d = 0; d < NDET; d++) {
        zr[d] = 0.0; zi[d] = 0.0;
        if (nb > 0) {
            double rs, rc;
            sincos_bf(TWO_PI_D * (f0 + tid * df) * c.tau[d], rs, rc);
            zr[d] = rc * hr[d] - rs * hi[d];
            zi[d] = rc * hi[d] + rs * hr[d];
        }
    }
}

// Mixed form, per bin (grids too coarse for the tiled form below): the phase
// in turns accumulated as a double-float dot product (error-free FP32 products
// via FMA, TwoSum accumulation), reduced mod 1, then FP32 __sincosf and FP32
// products. Partial sums are flushed every FLUSH bins into double-float
// accumulators (compensated summation).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void df_acc(float &hi, float &lo, float x) {
    float s, e;
    two_sum(hi, x, s, e);
    hi = s;
    lo += e;
}

// Returns the thread's double-float sums zh/zl[d][re, im], not reduced over
// threads.
template <int NDET>
__device__ __forceinline__ void bins_mixed(const Tables &T, int N, const CoefMixed &c, int jcut,
                                           int tid, int stride, float zh[NDET][2], float zl[NDET][2]) {
    float ah[NB], al[NB];
#pragma unroll
    for (int m = 0; m < NB; m++) { ah[m] = c.ah[m]; al[m] = c.al[m]; }
    float th_[NDET], tl_[NDET];
#pragma unroll
    for (int d = 0; d < NDET; d++) { th_[d] = c.tauh[d]; tl_[d] = c.taul[d]; }
    float zrh[NDET], zrl[NDET], zih[NDET], zil[NDET];
#pragma unroll
    for (int d = 0; d < NDET; d++) { zrh[d] = zrl[d] = zih[d] = zil[d] = 0.f; }
    constexpr int FLUSH = 16;
    int j = tid;
    while (j <= jcut) {
        float pr[NDET], pim[NDET];
#pragma unroll
        for (int d = 0; d < NDET; d++) { pr[d] = 0.f; pim[d] = 0.f; }
        for (int it = 0; it < FLUSH && j <= jcut; it++, j += stride) {
            float sh = c.c0h, sl = c.c0l;
#pragma unroll
            for (int m = 0; m < NB; m++) {
                const float2 b = __ldg(T.basis32 + (size_t)m * N + j);
                const float p = ah[m] * b.x;
                float e = fmaf(ah[m], b.x, -p);
                e = fmaf(ah[m], b.y, e);
                e = fmaf(al[m], b.x, e);
                float s, e2;
                two_sum(sh, p, s, e2);
                sh = s;
                sl += e2 + e;
            }
            const float2 fj = __ldg(T.f32 + j);
#pragma unroll
            for (int d = 0; d < NDET; d++) {
                const float p = th_[d] * fj.x;
                float e = fmaf(th_[d], fj.x, -p);
                e = fmaf(th_[d], fj.y, e);
                e = fmaf(tl_[d], fj.x, e);
                float s, e2;
                two_sum(sh, p, s, e2);
                const float n = rintf(s);
                const float r = (s - n) + (sl + (e2 + e));
                float sv, cv;
                __sincosf(r * 6.283185307179586f, &sv, &cv);
                const float2 w = __ldg(T.w32 + (size_t)d * N + j);
                pr[d] = fmaf(w.x, cv, fmaf(-w.y, sv, pr[d]));
                pim[d] = fmaf(w.x, sv, fmaf(w.y, cv, pim[d]));
            }
        }
#pragma unroll
        for (int d = 0; d < NDET; d++) { df_acc(zrh[d], zrl[d], pr[d]); df_acc(zih[d], zil[d], pim[d]); }
    }
#pragma unroll
    for (int d = 0; d < NDET; d++) {
        zh[d][0] = zrh[d]; zl[d][0] = zrl[d];
        zh[d][1] = zih[d]; zl[d][1] = zil[d];
    }
}

// Sum of v over the NDET consecutive lanes of a group starting at a multiple of
// NDET (NDET * groups <= 32): the group's first lane gets v_0 + v_1 + ... in lane
// order.
template <int NDET>
__device__ __forceinline__ double group_sum_down(double v) {
    double t = v;
#pragma unroll
    for (int k = 1; k < NDET; k++) t += __shfl_down_sync(0xffffffffu, v, k);
    return t;
}

// Mixed, several candidates at once: every thread of the CTA strides over the
// bins and applies each of the ns candidates (coefficients in shared memory) to
// the bin's table values, which are loaded once. Candidate s only takes bins
// j <= jcut[s]. Per (candidate, detector) the thread keeps FP32 partials over
// FLUSH bins and double-float running sums (zh, zl), returned unreduced.
template <int NDET, int S>
__device__ __forceinline__ void bins_mixed_multi(const Tables &T, int N, const CoefMixed *cm, const int *jcut,
                                                 int ns, int tid, int stride, float zrh[S][NDET],
                                                 float zrl[S][NDET], float zih[S][NDET], float zil[S][NDET]) {
    int jmax = -1;
    for (int s = 0; s < ns; s++) jmax = max(jmax, jcut[s]);
#pragma unroll
    for (int s = 0; s < S; s++)
#pragma unroll
        for (int d = 0; d < NDET; d++) zrh[s][d] = zrl[s][d] = zih[s][d] = zil[s][d] = 0.f;
    constexpr int FLUSH = 16;
    int j = tid;
    while (j <= jmax) {
        float pr[S][NDET], pim[S][NDET];
#pragma unroll
        for (int s = 0; s < S; s++)
#pragma unroll
            for (int d = 0; d < NDET; d++) pr[s][d] = pim[s][d] = 0.f;
        for (int it = 0; it < FLUSH && j <= jmax; it++, j += stride) {
            float2 b[NB];
#pragma unroll
            for (int m = 0; m < NB; m++) b[m] = __ldg(T.basis32 + (size_t)m * N + j);
            const float2 fj = __ldg(T.f32 + j);
            float2 w[NDET];
#pragma unroll
            for (int d = 0; d < NDET; d++) w[d] = __ldg(T.w32 + (size_t)d * N + j);
#pragma unroll
            for (int s = 0; s < S; s++) {
                if (s >= ns || j > jcut[s]) continue;
                const CoefMixed &c = cm[s];
                float sh = c.c0h, sl = c.c0l;
#pragma unroll
                for (int m = 0; m < NB; m++) {
                    const float ah = c.ah[m], al = c.al[m];
                    const float p = ah * b[m].x;
                    float e = fmaf(ah, b[m].x, -p);
                    e = fmaf(ah, b[m].y, e);
                    e = fmaf(al, b[m].x, e);
                    float s2, e2;
                    two_sum(sh, p, s2, e2);
                    sh = s2;
                    sl += e2 + e;
                }
#pragma unroll
                for (int d = 0; d < NDET; d++) {
                    const float th = c.tauh[d], tl = c.taul[d];
                    const float p = th * fj.x;
                    float e = fmaf(th, fj.x, -p);
                    e = fmaf(th, fj.y, e);
                    e = fmaf(tl, fj.x, e);
                    float s2, e2;
                    two_sum(sh, p, s2, e2);
                    const float n = rintf(s2);
                    const float r = (s2 - n) + (sl + (e2 + e));
                    float sv, cv;
                    __sincosf(r * 6.283185307179586f, &sv, &cv);
                    pr[s][d] = fmaf(w[d].x, cv, fmaf(-w[d].y, sv, pr[s][d]));
                    pim[s][d] = fmaf(w[d].x, sv, fmaf(w[d].y, cv, pim[s][d]));
                }
            }
        }
#pragma unroll
        for (int s = 0; s < S; s++)
#pragma unroll
            for (int d = 0; d < NDET; d++) {
                df_acc(zrh[s][d], zrl[s][d], pr[s][d]);
                df_acc(zih[s][d], zil[s][d], pim[s][d]);
            }
    }
}

// ------------------------------------------------------------- warp helpers
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Mixed form, tiled (fine grids). Lane l of a warp owns tile t = 32 g + l of
// group g, the L bins j = tL + i about the centre c = tL + L/2 (x = i - L/2).
// The phase of bin j at detector d, in turns, is
//   [c0 + sum_m a_m B_m(f_c) + f_c tau_d] + sum_{k=1..TK} C_k x^k + x df tau_d,
// C_k = sum_m a_m B_m^(k)(f_c) df^k / k!: the Taylor expansion of each basis
// function about the tile centre, its remainder bounded on the host below 1e-8
// rad when the tiled form is chosen: degree TK on the tile groups nearest f0,
// TK_LO on those far enough above it. Per lane and tile, the anchor in brackets
// and C_1 are double-float dot products (error-free FP32 products via FMA,
// TwoSum), C_2..C_TK plain FP32 (below a turn on 128-bin tiles, so their FP32
// rounding stays below 4e-7 rad).
// Detector 0, per bin: C_1 x as an error-free FP32 product reduced mod 1, the
// rest a short Horner sum (the delay term f tau_0 rides in its linear
// coefficient), the phase psi_0 in radians, FP32 __sincosf for
// E = exp(i psi_0) and the complex MAC with the weighted data.
// Detector d >= 1 differs from detector 0 by alpha_d + beta_d x, linear in the
// bin, so its tile sum  sum_x w_dx E_x exp(i (alpha_d + beta_d x))  is
// exp(i (alpha_d + beta_d x_e)) times a Horner sum in rho_d = exp(-i beta_d)
// anchored at the last bin x_e. The long-tile form (tile_pairs) runs that sum
// as two, over the even and the odd bins, each in steps of rho_d^2:
// S <- S rho_d^2 + w_dx E_x within segments of eight bins, T <- T + T eps8_d + S
// across them, eps8_d = exp(-8 i beta_d) - 1 (the magnitude error of a rounded
// step builds up over three steps at most), and at the tile's end
// T_even rho_d + T_odd. These detectors take no sine or cosine per bin. Two
// bins (i, i + 1) travel together in the two halves of the packed FP32 pair
// instructions (FFMA2, FMUL2): the same FP32 arithmetic on half the issue
// slots. Tiles of 16 bins or fewer keep a sine and cosine per detector and bin
// (tile_bins_direct), as does the serving kernel at every tile length. Each
// tile's sums are flushed into double-float accumulators; the only per-bin
// table is the weighted data, stored per detector, tile group and bin pair as
// float4 (Re w_i, Re w_i+1, Im w_i, Im w_i+1).
constexpr int TK = 7;
constexpr int TK_LO = 3;        // the degree of tile groups far enough above f0 (Tables::g_lo)
constexpr float TWO_PI_F = 6.28318530717958648f;

// Position of bin j in the pair-tile order of the weighted data, in float2
// slots: at step i of a tile, lanes read consecutive float4s (bins i, i + 1 of
// their tiles; the float4 holds both real parts, then both imaginary parts).
__device__ __forceinline__ int tile_pos2(int j, int lg) {
    const int t = j >> lg, i = j & ((1 << lg) - 1);
    return ((t >> 5) << (lg + 5)) + ((i >> 1) << 6) + ((t & 31) << 1) + (i & 1);
}

// Packed FP32 pairs: lane x of a float2 carries bin i, lane y bin i + 1.
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b, as one packed FMA with the pair (-1, -1)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, bc2(-1.0f), a); }

// Constants of one candidate over one lane's tile.
template <int NDET>
struct TileCand {
    float c1h, c1l, ck[TK - 1];     // C_1 (double-float; c1l also holds df tau_0), C_2..C_TK [turns]
    float aa0;                      // detector 0: 2 pi anchor [rad]
    float alpha[NDET];              // detectors d >= 1: alpha_d [rad]
};

// Four bins (two pairs) of one candidate over one lane's tile, from bin q:
// detector 0's sums in (pr, pim), detector d's segment sums in (sr, si)[d].
// FIRST: the segment's first bins (its sums start here). MASK: bins >= cnt
// add nothing.
template <int NDET, bool MASK, bool FIRST, int K>
__device__ __forceinline__ void pair_step(const float4 (&w)[NDET][2], int q, int cnt, float2 x0,
                                          const TileCand<NDET> &k, const float2 (&r2)[NDET][3],
                                          float2 &pr, float2 &pim, float2 (&sr)[NDET], float2 (&si)[NDET]) {
    const float2 c1h = bc2(k.c1h), nc1h = bc2(-k.c1h);
#pragma unroll
    for (int h = 0; h < 2; h++) {
        const float2 x = h ? add2(x0, bc2(2.0f)) : x0;
        // p + e = C_1h x exactly (ne = -e); nsm = -(rest of the phase) by Horner's
        // rule on the negated coefficients, down to the C_1 low part
        const float2 p = mul2(c1h, x);
        const float2 ne = fma2(nc1h, x, p);
        float2 nh = bc2(-k.ck[K - 2]);
#pragma unroll
        for (int j = K - 3; j >= 0; j--) nh = fma2(nh, x, bc2(-k.ck[j]));
        nh = fma2(nh, x, bc2(-k.c1l));
        const float2 nsm = fma2(nh, x, ne);
        const float2 u = sub2(sub2(p, make_float2(rintf(p.x), rintf(p.y))), nsm);
        const float2 a = fma2(u, bc2(TWO_PI_F), bc2(k.aa0));
        float2 sv, cv;
        __sincosf(a.x, &sv.x, &cv.x);
        __sincosf(a.y, &sv.y, &cv.y);
        const float2 nsv = mul2(sv, bc2(-1.0f));
        float2 ok;
        if (MASK) {
            const int i = q + 2 * h;
            ok = make_float2(i < cnt ? 1.0f : 0.0f, i + 1 < cnt ? 1.0f : 0.0f);
        }
#pragma unroll
        for (int d = 0; d < NDET; d++) {
            const float4 ww = w[d][h];
            float2 wr = make_float2(ww.x, ww.y), wi = make_float2(ww.z, ww.w);
            if (MASK) {
                wr = mul2(wr, ok);
                wi = mul2(wi, ok);
            }
            if (d == 0) {
                pr = fma2(wi, nsv, fma2(wr, cv, pr));
                pim = fma2(wi, cv, fma2(wr, sv, pim));
            } else if (FIRST && h == 0) {
                sr[d] = fma2(wi, nsv, mul2(wr, cv));
                si[d] = fma2(wi, cv, mul2(wr, sv));
            } else {
                // S <- S rho^2 + w E  (r2[d]: Re rho^2, -Im rho^2, Im rho^2, broadcast); w E
                // first, so the chain through S is two instructions per step
                const float2 cr = fma2(wi, nsv, mul2(wr, cv)), ci = fma2(wi, cv, mul2(wr, sv));
                const float2 nr = fma2(sr[d], r2[d][0], fma2(si[d], r2[d][1], cr));
                si[d] = fma2(sr[d], r2[d][2], fma2(si[d], r2[d][0], ci));
                sr[d] = nr;
            }
        }
    }
}

// One candidate over one lane's tile, bins i < nproc (a multiple of 8); with
// MASK, bins i >= cnt add nothing (tiles at the cutoff). Returns the sums
// sum_i w_di exp(2 pi i phase_di) per detector in zr, zi. With PF the next
// four bins' weighted data are loaded while these four are summed (the
// batched likelihood waits on these loads otherwise; in the slice kernels, at
// their register cap, neither this nor an L1 prefetch hint pays: GB300, c4
// slice update 217.5 ms without, 220 ms with, 250 ms with the hint).
template <int NDET, bool MASK, bool PF, int K>
__device__ __forceinline__ void tile_pairs(const float4 *w4, size_t dstride, int lane, int half, int nproc,
                                           int cnt, const TileCand<NDET> &k, const CoefMixed &cm,
                                           float (&zr)[NDET], float (&zi)[NDET]) {
    float2 pr = bc2(0.0f), pim = bc2(0.0f);
    float2 sr[NDET], si[NDET], tr[NDET], ti[NDET], r2[NDET][3];
#pragma unroll
    for (int d = 1; d < NDET; d++) {
        tr[d] = ti[d] = bc2(0.0f);
        r2[d][0] = bc2(cm.rho2[d][0]);
        r2[d][1] = bc2(-cm.rho2[d][1]);
        r2[d][2] = bc2(cm.rho2[d][1]);
    }
    float4 w[NDET][2];
    const float4 *wp = w4 + lane;
    if (PF) {
#pragma unroll
        for (int d = 0; d < NDET; d++) {
            w[d][0] = __ldg(wp + d * dstride);
            w[d][1] = __ldg(wp + d * dstride + 32);
        }
    }
    float2 x0 = make_float2((float)-half, (float)(1 - half));
    for (int q = 0; q < nproc; q += 8) {
#pragma unroll
        for (int s = 0; s < 2; s++) {
            const int qs = q + 4 * s;
            float4 wn[NDET][2];
            if (PF) {
                const int qn = qs + 4 < nproc ? qs + 4 : qs;     // the last step reloads its own bins
#pragma unroll
                for (int d = 0; d < NDET; d++) {
                    wn[d][0] = __ldg(wp + d * dstride + (qn << 4));
                    wn[d][1] = __ldg(wp + d * dstride + (qn << 4) + 32);
                }
            } else {
#pragma unroll
                for (int d = 0; d < NDET; d++) {
                    w[d][0] = __ldg(wp + d * dstride + (qs << 4));
                    w[d][1] = __ldg(wp + d * dstride + (qs << 4) + 32);
                }
            }
            if (s == 0)
                pair_step<NDET, MASK, true, K>(w, qs, cnt, x0, k, r2, pr, pim, sr, si);
            else
                pair_step<NDET, MASK, false, K>(w, qs, cnt, x0, k, r2, pr, pim, sr, si);
            x0 = add2(x0, bc2(4.0f));
            if (PF) {
#pragma unroll
                for (int d = 0; d < NDET; d++) {
                    w[d][0] = wn[d][0];
                    w[d][1] = wn[d][1];
                }
            }
        }
        // the eight-bin segment ends: T <- T + T eps8 + S
#pragma unroll
        for (int d = 1; d < NDET; d++) {
            const float2 er = bc2(cm.eps8[d][0]), ei = bc2(cm.eps8[d][1]), nei = bc2(-cm.eps8[d][1]);
            const float2 ur = fma2(tr[d], er, fma2(ti[d], nei, sr[d]));
            const float2 ui = fma2(tr[d], ei, fma2(ti[d], er, si[d]));
            tr[d] = add2(tr[d], ur);
            ti[d] = add2(ti[d], ui);
        }
    }
    zr[0] = pr.x + pr.y;
    zi[0] = pim.x + pim.y;
    const float xe = (float)(nproc - 1 - half);
#pragma unroll
    for (int d = 1; d < NDET; d++) {
        // the even bins' sum is anchored one bin before the last: T = T_even rho + T_odd
        const float rr = cm.rho[d][0], ri = cm.rho[d][1];
        const float Tr = fmaf(tr[d].x, rr, fmaf(-ti[d].x, ri, tr[d].y));
        const float Ti = fmaf(tr[d].x, ri, fmaf(ti[d].x, rr, ti[d].y));
        float as, ac;
        __sincosf(fmaf(cm.beta[d], xe, k.alpha[d]), &as, &ac);
        zr[d] = fmaf(ac, Tr, -as * Ti);
        zi[d] = fmaf(ac, Ti, as * Tr);
    }
}

// Short tiles (L <= 16): every detector's phase reduced mod 1 and its own
// FP32 __sincosf per bin, the nc <= NC candidates sharing the table loads (on
// few bins per tile the rotation's per-tile setup and the candidates taken one
// after the other cost more than the sines save). Same sums as tile_bins.
template <int NDET, int NC>
__device__ __forceinline__ void tile_bins_direct(const Tables &T, int lg, int np, const CoefMixed *cm,
                                          const int *jcut, int nc, int g0, int gstride,
                                          float zh[NC][NDET][2], float zl[NC][NDET][2],
                                          int g_end = 0x7fffffff) {
    const int lane = threadIdx.x & 31;
    const int L = 1 << lg, half = L >> 1, nt = np >> lg;
#pragma unroll
    for (int c = 0; c < NC; c++)
#pragma unroll
        for (int d = 0; d < NDET; d++) zh[c][d][0] = zh[c][d][1] = zl[c][d][0] = zl[c][d][1] = 0.f;
    int jmax = -1;
#pragma unroll
    for (int c = 0; c < NC; c++)
        if (c < nc) jmax = max(jmax, jcut[c]);
    const int ngroups = min(jmax < 0 ? 0 : (jmax >> (lg + 5)) + 1, g_end);
    const float4 *wt4 = reinterpret_cast<const float4 *>(T.wt);
    for (int g = g0; g < ngroups; g += gstride) {
        const int t = (g << 5) + lane, s = t << lg;
        int cnt[NC];
        int nmax = 0;
        float c1h[NC], c1l[NC], ck[NC][TK - 1], Ah[NC][NDET], Al[NC][NDET];
        const float2 fc = __ldg(T.fc + t);
#pragma unroll
        for (int c = 0; c < NC; c++) {
            cnt[c] = (c < nc) ? min(max(jcut[c] - s + 1, 0), L) : 0;
            nmax = max(nmax, (c < nc) ? min(max(jcut[c] - (g << (lg + 5)) + 1, 0), L) : 0);
            float sh = cm[c].c0h, sl = cm[c].c0l, h1 = 0.f, l1 = 0.f;
#pragma unroll
            for (int k = 0; k < TK - 1; k++) ck[c][k] = 0.f;
#pragma unroll
            for (int m = 0; m < NB; m++) {
                const float ah = cm[c].ah[m], al = cm[c].al[m];
                // anchor term a_m B_m(f_c)
                const float2 b0 = __ldg(T.tb0 + (size_t)m * nt + t);
                float p = ah * b0.x;
                float e = fmaf(ah, b0.x, -p);
                e = fmaf(ah, b0.y, e);
                e = fmaf(al, b0.x, e);
                float s2, e2;
                two_sum(sh, p, s2, e2);
                sh = s2;
                sl += e2 + e;
                // first-order term a_m B_m'(f_c) df
                const float2 b1 = __ldg(T.tb1 + (size_t)m * nt + t);
                p = ah * b1.x;
                e = fmaf(ah, b1.x, -p);
                e = fmaf(ah, b1.y, e);
                e = fmaf(al, b1.x, e);
                two_sum(h1, p, s2, e2);
                h1 = s2;
                l1 += e2 + e;
#pragma unroll
                for (int k = 0; k < TK - 1; k++)
                    ck[c][k] = fmaf(ah, __ldg(T.tbk + ((size_t)k * NB + m) * nt + t), ck[c][k]);
            }
            c1h[c] = h1 + l1;
            c1l[c] = l1 - (c1h[c] - h1);
            sh -= rintf(sh);
#pragma unroll
            for (int d = 0; d < NDET; d++) {
                const float th = cm[c].tauh[d], tl = cm[c].taul[d];
                const float p = th * fc.x;
                float e = fmaf(th, fc.x, -p);
                e = fmaf(th, fc.y, e);
                e = fmaf(tl, fc.x, e);
                float s2, e2;
                two_sum(sh, p, s2, e2);
                Ah[c][d] = s2 - rintf(s2);
                Al[c][d] = sl + (e2 + e);
            }
        }
        float pr[NC][NDET], pim[NC][NDET];
#pragma unroll
        for (int c = 0; c < NC; c++)
#pragma unroll
            for (int d = 0; d < NDET; d++) pr[c][d] = pim[c][d] = 0.f;
        const size_t gb = (size_t)g << (lg + 5);
        for (int q = 0; q < nmax; q += 4) {
            float4 w[NDET][2];
#pragma unroll
            for (int d = 0; d < NDET; d++) {
                const size_t base = ((size_t)d * np + gb) >> 1;
                w[d][0] = __ldg(wt4 + base + (q << 4) + lane);
                w[d][1] = __ldg(wt4 + base + (q << 4) + 32 + lane);
            }
#pragma unroll
            for (int r = 0; r < 4; r++) {
                const int i = q + r;
                const float x = (float)(i - half);
#pragma unroll
                for (int c = 0; c < NC; c++) {
                    if (i >= cnt[c]) continue;
                    const float p = c1h[c] * x;
                    const float e = fmaf(c1h[c], x, -p);
                    float hq = ck[c][TK - 2];
#pragma unroll
                    for (int k = TK - 3; k >= 0; k--) hq = fmaf(hq, x, ck[c][k]);
                    hq = fmaf(hq, x, c1l[c]);
                    const float sm = fmaf(hq, x, e);
                    const float P = p - rintf(p);
#pragma unroll
                    for (int d = 0; d < NDET; d++) {
                        const float y = (P + Ah[c][d]) + (sm + fmaf(x, cm[c].dtau[d], Al[c][d]));
                        const float red = y - rintf(y);
                        float sv, cv;
                        __sincosf(red * 6.283185307179586f, &sv, &cv);
                        const float4 ww = w[d][r >> 1];
                        const float wr = (r & 1) ? ww.y : ww.x, wi = (r & 1) ? ww.w : ww.z;
                        pr[c][d] = fmaf(wr, cv, fmaf(-wi, sv, pr[c][d]));
                        pim[c][d] = fmaf(wr, sv, fmaf(wi, cv, pim[c][d]));
                    }
                }
            }
        }
#pragma unroll
        for (int c = 0; c < NC; c++)
#pragma unroll
            for (int d = 0; d < NDET; d++) {
                df_acc(zh[c][d][0], zl[c][d][0], pr[c][d]);
                df_acc(zh[c][d][1], zl[c][d][1], pim[c][d]);
            }
    }
}
// One candidate over tile group g (its 32 tiles, one per lane) by rotation,
// with K - 1 Taylor terms C_2..C_K: the tile's constants (anchors, C_1 in
// double-float, C_2..C_K), then its sums zr, zi per detector.
template <int NDET, bool PF, int K>
__device__ __forceinline__ void rot_group(const Tables &T, int lg, int np, const CoefMixed &cm, int jcut, int g,
                                          float (&zr)[NDET], float (&zi)[NDET]) {
    const int lane = threadIdx.x & 31;
    const int L = 1 << lg, half = L >> 1, nt = np >> lg;
    const int t = (g << 5) + lane, s = t << lg, gbin = g << (lg + 5);
    const float2 fc = __ldg(T.fc + t);
    const float4 *w4 = reinterpret_cast<const float4 *>(T.wt) + ((size_t)gbin >> 1);
    const size_t dstride = (size_t)np >> 1;
    const int nmax = min(max(jcut - gbin + 1, 0), L);
    const int cnt = min(max(jcut - s + 1, 0), L);
    TileCand<NDET> k;
    float sh = cm.c0h, sl = cm.c0l, h1 = 0.f, l1 = 0.f;
#pragma unroll
    for (int j = 0; j < TK - 1; j++) k.ck[j] = 0.f;
#pragma unroll
    for (int m = 0; m < NB; m++) {
        const float ah = cm.ah[m], al = cm.al[m];
        // anchor term a_m B_m(f_c)
        const float2 b0 = __ldg(T.tb0 + (size_t)m * nt + t);
        float p = ah * b0.x;
        float e = fmaf(ah, b0.x, -p);
        e = fmaf(ah, b0.y, e);
        e = fmaf(al, b0.x, e);
        float s2, e2;
        two_sum(sh, p, s2, e2);
        sh = s2;
        sl += e2 + e;
        // first-order term a_m B_m'(f_c) df
        const float2 b1 = __ldg(T.tb1 + (size_t)m * nt + t);
        p = ah * b1.x;
        e = fmaf(ah, b1.x, -p);
        e = fmaf(ah, b1.y, e);
        e = fmaf(al, b1.x, e);
        two_sum(h1, p, s2, e2);
        h1 = s2;
        l1 += e2 + e;
#pragma unroll
        for (int j = 0; j < K - 1; j++)
            k.ck[j] = fmaf(ah, __ldg(T.tbk + ((size_t)j * NB + m) * nt + t), k.ck[j]);
    }
    k.c1h = h1 + l1;
    k.c1l = (l1 - (k.c1h - h1)) + cm.dtau[0];
    sh -= rintf(sh);
    // detector anchors A_d = anchor + f_c tau_d (turns, reduced), high and low parts
    float Ah[NDET], Al[NDET];
#pragma unroll
    for (int d = 0; d < NDET; d++) {
        const float th = cm.tauh[d], tl = cm.taul[d];
        const float p = th * fc.x;
        float e = fmaf(th, fc.x, -p);
        e = fmaf(th, fc.y, e);
        e = fmaf(tl, fc.x, e);
        float s2, e2;
        two_sum(sh, p, s2, e2);
        Ah[d] = s2 - rintf(s2);
        Al[d] = sl + (e2 + e);
    }
    k.aa0 = TWO_PI_F * (Ah[0] + Al[0]);
#pragma unroll
    for (int d = 1; d < NDET; d++) {
        float a = (Ah[d] - Ah[0]) + (Al[d] - Al[0]);
        a -= rintf(a);
        k.alpha[d] = TWO_PI_F * a;
    }
    if (jcut >= gbin + (32 << lg) - 1)      // every tile of the group below the cutoff
        tile_pairs<NDET, false, PF, K>(w4, dstride, lane, half, L, L, k, cm, zr, zi);
    else
        tile_pairs<NDET, true, PF, K>(w4, dstride, lane, half, (nmax + 7) & ~7, cnt, k, cm, zr, zi);
}

// One warp's double-float sums over tile groups g0, g0 + gstride, ... for nc <= NC
// candidates (coefficients cm[c], last bins jcut[c]): zh/zl[c][d][0/1] =
// real/imaginary part of sum_j w_dj exp(2 pi i phase_dj), not yet reduced over
// the warp. Detector 0 direct and the others by their rotation, one candidate
// after the other. With LO, groups g >= T.g_lo take the Taylor degree TK_LO and
// the rest TK (GB300, 519,169 bins: slice update 205.8 -> 192.3 ms); without it
// every group takes TK, one copy of the tile code (the c2 slice update, bound by
// latency and instruction fetch, runs 13.5 ms with one copy and 14.5 with two).
template <int NDET, int NC, bool PF, bool LO>
__device__ __forceinline__ void tile_bins_rot(const Tables &T, int lg, int np, const CoefMixed *cm,
                                              const int *jcut, int nc, int g0, int gstride,
                                              float zh[NC][NDET][2], float zl[NC][NDET][2],
                                              int g_end = 0x7fffffff) {
#pragma unroll
    for (int c = 0; c < NC; c++)
#pragma unroll
        for (int d = 0; d < NDET; d++) zh[c][d][0] = zh[c][d][1] = zl[c][d][0] = zl[c][d][1] = 0.f;
    // candidates one after the other (a run-time loop: one copy of the tile
    // code, so the kernels' hot code is smaller; GB300: 64,897 bins, slice
    // update 14.7 -> 13.9 ms; 519,169 bins, 249 -> 244 ms), each over its own
    // groups in order, so each candidate's sums are the same as with the
    // candidates taken in turn over each group
#pragma unroll 1
    for (int c = 0; c < nc; c++) {
        float ah[NDET][2], al[NDET][2];
#pragma unroll
        for (int d = 0; d < NDET; d++) ah[d][0] = ah[d][1] = al[d][0] = al[d][1] = 0.f;
        const int ngroups = min(jcut[c] < 0 ? 0 : (jcut[c] >> (lg + 5)) + 1, g_end);
        for (int g = g0; g < ngroups; g += gstride) {
            if (jcut[c] < (g << (lg + 5))) continue;
            float zr[NDET], zi[NDET];
            if (LO && g >= T.g_lo)
                rot_group<NDET, PF, TK_LO>(T, lg, np, cm[c], jcut[c], g, zr, zi);
            else
                rot_group<NDET, PF, TK>(T, lg, np, cm[c], jcut[c], g, zr, zi);
#pragma unroll
            for (int d = 0; d < NDET; d++) {
                df_acc(ah[d][0], al[d][0], zr[d]);
                df_acc(ah[d][1], al[d][1], zi[d]);
            }
        }
#pragma unroll
        for (int cc = 0; cc < NC; cc++)
            if (cc == c) {
#pragma unroll
                for (int d = 0; d < NDET; d++) {
                    zh[cc][d][0] = ah[d][0]; zh[cc][d][1] = ah[d][1];
                    zl[cc][d][0] = al[d][0]; zl[cc][d][1] = al[d][1];
                }
            }
    }
}
// The tiled form's sums, by rotation (ROT: tiles of 32 bins or more; GB300,
// 519,169 bins in 64-bin tiles: slice update 478 -> 326 ms; 64,897 bins in
// 32-bin tiles: 14.3 -> 13.8 ms) or direct (shorter tiles, where the per-tile
// rotation setup outweighs the saved sines: 64,897 bins in 16-bin tiles, 14.3
// against 15.9 ms by rotation). Callers choose by the tile length.
template <int NDET, int NC, bool ROT, bool PF = false, bool LO = false>
__device__ __forceinline__ void tile_bins(const Tables &T, int lg, int np, const CoefMixed *cm,
                                          const int *jcut, int nc, int g0, int gstride,
                                          float zh[NC][NDET][2], float zl[NC][NDET][2],
                                          int g_end = 0x7fffffff) {
    if constexpr (ROT)
        tile_bins_rot<NDET, NC, PF, LO>(T, lg, np, cm, jcut, nc, g0, gstride, zh, zl, g_end);
    else
        tile_bins_direct<NDET, NC>(T, lg, np, cm, jcut, nc, g0, gstride, zh, zl, g_end);
}

// Double-float warp sum (TwoSum of the high parts, low parts added).
__device__ __forceinline__ void warp_sum_df(float &h, float &l) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
        float s, e;
        two_sum(h, oh, s, e);
        h = s;
        l = l + ol + e;
    }
}

// Warp sums of V <= 16 double-float values at once (a transposing butterfly):
// at each of the first four steps a lane hands half of the values it carries
// to its partner and adds the half it keeps, so that 8 + 4 + 2 + 1 + 1
// double-float adds replace 5 V. On return lanes 2i and 2i + 1 hold the sum of
// value i in (rh, rl).
template <int V>
__device__ __forceinline__ void warp_sum_df_many(float (&h)[16], float (&l)[16], float &rh, float &rl) {
    static_assert(V <= 16, "at most 16 values");
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int i = V; i < 16; i++) { h[i] = 0.f; l[i] = 0.f; }
#pragma unroll
    for (int step = 0; step < 4; step++) {
        const int half = 8 >> step, o = 16 >> step;
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < half; i++) {
            const float kh = upper ? h[i + half] : h[i], kl = upper ? l[i + half] : l[i];
            const float sh = upper ? h[i] : h[i + half], sl = upper ? l[i] : l[i + half];
            const float oh = __shfl_xor_sync(0xffffffffu, sh, o), ol = __shfl_xor_sync(0xffffffffu, sl, o);
            float s, e;
            two_sum(kh, oh, s, e);
            h[i] = s;
            l[i] = kl + ol + e;
        }
    }
    const float oh = __shfl_xor_sync(0xffffffffu, h[0], 1), ol = __shfl_xor_sync(0xffffffffu, l[0], 1);
    float s, e;
    two_sum(h[0], oh, s, e);
    rh = s;
    rl = l[0] + ol + e;
}

// ------------------------------------------------------- relative binning
// One warp, edges striped over lanes in chunks of 31 bins (32 edges): each lane
// computes E_d(e) = exp(-i dPsi_d(e)) at its edge, with dPsi the phase
// difference from the fiducial point, takes E_d(e+1) from the next lane and
// accumulates its bin:
//   Y_d += A0 conj(S)/2 + A1 conj(D),  H_d += B0 |S|^2/4 + B1 Re(S conj(D)),
//   S = E_b + E_b+1,  D = (E_b+1 - E_b)/(e_b+1 - e_b),
// so that with rho_d = conj(G_d)/conj(G0_d) (r = h/h0 = rho_d E_d):
//   <d|h_d> = Re(conj(rho_d) Y_d),  <h_d|h_d> = |rho_d|^2 H_d.
// Bins whose centre lies above f_ISCO are dropped when the cutoff is on.
template <int NDET>
__device__ __forceinline__ void rb_fp64(const Model &M, const RBTables &R, const Coef &c, int lane,
                                        double Yr[NDET], double Yi[NDET], double H[NDET]) {
    const Coef &f = *R.fid;
    double da[NB];
#pragma unroll
    for (int m = 0; m < NB; m++) da[m] = c.a[m] - f.a[m];
    const double dc = c.c0 - f.c0;
    double dtau[NDET];
#pragma unroll
    for (int d = 0; d < NDET; d++) { dtau[d] = c.tau[d] - f.tau[d]; Yr[d] = Yi[d] = H[d] = 0.0; }
    for (int base = 0; base < R.nb; base += 31) {
        const int e = base + lane;
        const bool ok = e < R.nedge;
        double psi = dc;
        if (ok) {
#pragma unroll
            for (int m = 0; m < NB; m++) psi = fma(da[m], __ldg(R.basis64 + (size_t)m * R.nedge + e), psi);
        }
        const double fe = ok ? __ldg(R.fe + e) : 0.0;
        const int b = base + lane;
        const bool use = lane < 31 && b < R.nb && (!M.cutoff || __ldg(R.fm + b) <= c.fisco);
#pragma unroll
        for (int d = 0; d < NDET; d++) {
            double sn, cs;
            sincos(psi + TWO_PI_D * fe * dtau[d], &sn, &cs);
            const double er = cs, ei = -sn;                    // exp(-i dPsi)
            const double nr = __shfl_down_sync(0xffffffffu, er, 1);
            const double ni = __shfl_down_sync(0xffffffffu, ei, 1);
            if (use) {
                const double idl = __ldg(R.inv_de + b);
                const double Sr = er + nr, Si = ei + ni;
                const double Dr = (nr - er) * idl, Di = (ni - ei) * idl;
                const size_t o = (size_t)d * R.nb + b;
                const double2 a0 = __ldg(R.A0 + o), a1 = __ldg(R.A1 + o);
                // A0 conj(S)/2 + A1 conj(D)
                Yr[d] += 0.5 * (a0.x * Sr + a0.y * Si) + (a1.x * Dr + a1.y * Di);
                Yi[d] += 0.5 * (a0.y * Sr - a0.x * Si) + (a1.y * Dr - a1.x * Di);
                H[d] += 0.25 * __ldg(R.B0 + o) * (Sr * Sr + Si * Si) + __ldg(R.B1 + o) * (Sr * Dr + Si * Di);
            }
        }
    }
}

template <int NDET>
__device__ __forceinline__ void rb_mixed(const Model &M, const RBTables &R, const CoefMixed &c, double fisco,
                                         int lane, double Yr[NDET], double Yi[NDET], double H[NDET]) {
    float yr[NDET], yi[NDET], hh[NDET];
#pragma unroll
    for (int d = 0; d < NDET; d++) yr[d] = yi[d] = hh[d] = 0.f;
    for (int base = 0; base < R.nb; base += 31) {
        const int e = base + lane;
        const bool ok = e < R.nedge;
        float sh = c.c0h, sl = c.c0l;
        float2 fe = make_float2(0.f, 0.f);
        if (ok) {
#pragma unroll
            for (int m = 0; m < NB; m++) {
                const float2 bb = __ldg(R.basis32 + (size_t)m * R.nedge + e);
                const float p = c.ah[m] * bb.x;
                float er = fmaf(c.ah[m], bb.x, -p);
                er = fmaf(c.ah[m], bb.y, er);
                er = fmaf(c.al[m], bb.x, er);
                float s2, e2;
                two_sum(sh, p, s2, e2);
                sh = s2;
                sl += e2 + er;
            }
            fe = __ldg(R.fe32 + e);
        }
        const int b = base + lane;
        const bool use = lane < 31 && b < R.nb && (!M.cutoff || __ldg(R.fm + b) <= fisco);
#pragma unroll
        for (int d = 0; d < NDET; d++) {
            const float p = c.tauh[d] * fe.x;
            float er = fmaf(c.tauh[d], fe.x, -p);
            er = fmaf(c.tauh[d], fe.y, er);
            er = fmaf(c.taul[d], fe.x, er);
            float s2, e2;
            two_sum(sh, p, s2, e2);
            const float n = rintf(s2);
            const float r = (s2 - n) + (sl + (e2 + er));
            float sv, cv;
            __sincosf(r * 6.283185307179586f, &sv, &cv);
            const float Er = cv, Ei = -sv;
            const float Nr = __shfl_down_sync(0xffffffffu, Er, 1);
            const float Ni = __shfl_down_sync(0xffffffffu, Ei, 1);
            if (use) {
                const float idl = __ldg(R.inv_de_f + b);
                const float Sr = Er + Nr, Si = Ei + Ni;
                const float Dr = (Nr - Er) * idl, Di = (Ni - Ei) * idl;
                const size_t o = (size_t)d * R.nb + b;
                const float2 a0 = __ldg(R.A0f + o), a1 = __ldg(R.A1f + o);
                yr[d] += 0.5f * (a0.x * Sr + a0.y * Si) + (a1.x * Dr + a1.y * Di);
                yi[d] += 0.5f * (a0.y * Sr - a0.x * Si) + (a1.y * Dr - a1.x * Di);
                hh[d] += 0.25f * __ldg(R.B0f + o) * (Sr * Sr + Si * Si) + __ldg(R.B1f + o) * (Sr * Dr + Si * Di);
            }
        }
    }
#pragma unroll
    for (int d = 0; d < NDET; d++) { Yr[d] = yr[d]; Yi[d] = yi[d]; H[d] = hh[d]; }
}

// log L of one point from the relative-binning sums (lane 0 holds the result).
template <int NDET, int PREC>
__device__ __forceinline__ double rb_loglike_warp(const Model &M, const RBTables &R, const Coef &c,
                                                  const CoefMixed &cm, int lane) {
    double Yr[NDET], Yi[NDET], H[NDET];
    if (PREC == 0) rb_fp64<NDET>(M, R, c, lane, Yr, Yi, H);
    else rb_mixed<NDET>(M, R, cm, c.fisco, lane, Yr, Yi, H);
    double v = 0.0;
#pragma unroll
    for (int d = 0; d < NDET; d++) {
        double yr = Yr[d], yi = Yi[d], h = H[d];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            yr += __shfl_xor_sync(0xffffffffu, yr, o);
            yi += __shfl_xor_sync(0xffffffffu, yi, o);
            h += __shfl_xor_sync(0xffffffffu, h, o);
        }
        // rho = conj(G)/conj(G0)
        const double g0r = R.fid->gre[d], g0i = R.fid->gim[d];
        const double den = g0r * g0r + g0i * g0i;
        const double rr = (c.gre[d] * g0r + c.gim[d] * g0i) / den;
        const double ri = -(c.gim[d] * g0r - c.gre[d] * g0i) / den;
        v += (rr * yr + ri * yi) - 0.5 * (rr * rr + ri * ri) * h;
    }
    return v;
}

}  // namespace gwns
