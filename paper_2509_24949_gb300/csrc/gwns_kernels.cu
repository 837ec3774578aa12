// gwns_kernels.cu -- sm_103a kernels of one nested-slice-sampling iteration
// (paper Sec. 2) and of the batched likelihood.
//
// One iteration = five launches, captured once into a CUDA graph by the host:
//   k_select    sort the n live log L ascending (ties by index): order[]
//   k_evidence  the k lowest die: log w_j, log X, log Z, dead records
//   k_cov_chol  survivors' covariance in unit-cube coordinates + Cholesky
//   k_slice     one CTA per chain: slice-sampling state machine (warp 0) with
//               the likelihood of each candidate evaluated by the whole CTA
//   k_finish    largest live log L, stopping test, iteration counter
#include <float.h>
#include <math.h>

#include <mutex>

#include "gwns_kernels.cuh"

namespace gwns {

// File-scope staging array of the allocation-free host-buffer likelihood
// entry point (ns_eval_lnl_host_noalloc). Every GPU that loads the library
// holds these NOALLOC_DOUBLES doubles (557,056 bytes) until the process exits.
// Host code must not pass the symbol itself to a kernel (on the host it is a
// stand-in, not a device address): noalloc_scratch_address() returns the
// device address obtained with cudaGetSymbolAddress.
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

cudaError_t noalloc_scratch_address(double **ptr) {
    static std::mutex mu;
    static double *addr[64] = {nullptr};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        addr[dev] = (double *)p;
    }
    *ptr = addr[dev];
    return cudaSuccess;
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

// Block-wide sum (all threads get the result). scratch: >= 32 doubles.
__device__ double block_sum(double v, double *scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    double r = (lane < nw) ? scratch[lane] : 0.0;
    r = warp_sum(r);
    return r;
}
__device__ double block_max(double v, double *scratch) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_max(v);
    __syncthreads();
    if (lane == 0) scratch[warp] = v;
    __syncthreads();
    double r = (lane < nw) ? scratch[lane] : -DBL_MAX;
    r = warp_max(r);
    return r;
}

// ----------------------------------------------------------------- tables
// Per bin: f_j, the phase basis B_m(f_j) (FP64 and double-float), the weighted
// data w_dj = 4 df f^(-7/6) d_dj / S_dj and the terms 4 df f^(-7/3) / S_dj of
// the <h|h> prefix sums (scanned by k_prefix_scan).
__global__ void k_build_tables(Model M, const double *dre, const double *dim, const double *psd,
                               double *basis64, double *f64, double2 *w64, double *prefix,
                               float2 *basis32, float2 *f32, float2 *w32) {
    const int N = M.N;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
        const double f = __dadd_rn(M.f0, __dmul_rn((double)j, M.df));
        const double lf = log(f);
        const double c = cbrt(f);          // f^(1/3)
        const double ic = 1.0 / c;
        double B[NB];
        B[0] = ic * ic * ic * ic * ic;      // f^(-5/3)
        B[1] = 1.0 / f;                     // f^(-1)
        B[2] = ic * ic;                     // f^(-2/3)
        B[3] = ic;                          // f^(-1/3)
        B[4] = lf;                          // ln f
        B[5] = c;                           // f^(1/3)
        B[6] = c * lf;                      // f^(1/3) ln f
        B[7] = c * c;                       // f^(2/3)
#pragma unroll
        for (int m = 0; m < NB; m++) {
            basis64[(size_t)m * N + j] = B[m];
            float h = __double2float_rn(B[m]);
            basis32[(size_t)m * N + j] = make_float2(h, __double2float_rn(B[m] - (double)h));
        }
        f64[j] = f;
        {
            float h = __double2float_rn(f);
            f32[j] = make_float2(h, __double2float_rn(f - (double)h));
        }
        const double f76 = pow(f, -7.0 / 6.0);
        for (int d = 0; d < M.n_det; d++) {
            const size_t o = (size_t)d * N + j;
            const double s = psd[o];
            const double wr = 4.0 * M.df * f76 * dre[o] / s;
            const double wi = 4.0 * M.df * f76 * dim[o] / s;
            w64[o] = make_double2(wr, wi);
            w32[o] = make_float2(__double2float_rn(wr), __double2float_rn(wi));
            prefix[o] = 4.0 * M.df * f76 * f76 / s;
        }
    }
}

// Inclusive scan of prefix[d][0..N) in place, one block per detector: each
// thread scans a contiguous chunk, chunk totals are scanned by the block.
__global__ void k_prefix_scan(double *prefix, int N) {
    double *p = prefix + (size_t)blockIdx.x * N;
    __shared__ double tot[1024];
    const int T = blockDim.x, t = threadIdx.x;
    const int chunk = (N + T - 1) / T;
    const int lo = t * chunk, hi = min(N, lo + chunk);
    double s = 0.0;
    for (int j = lo; j < hi; j++) { s += p[j]; p[j] = s; }
    tot[t] = s;
    __syncthreads();
    if (t == 0) {
        double acc = 0.0;
        for (int i = 0; i < T; i++) { double v = tot[i]; tot[i] = acc; acc += v; }
    }
    __syncthreads();
    const double off = tot[t];
    for (int j = lo; j < hi; j++) p[j] += off;
}

cudaError_t launch_build_tables(const Model &M, const double *data_re, const double *data_im,
                                const double *psd, double *basis64, double *f64, double2 *w64,
                                double *prefix, float2 *basis32, float2 *f32, float2 *w32,
                                cudaStream_t s) {
    int blocks = min((M.N + 255) / 256, 152 * 8);
    k_build_tables<<<blocks, 256, 0, s>>>(M, data_re, data_im, psd, basis64, f64, w64, prefix, basis32,
                                          f32, w32);
    k_prefix_scan<<<M.n_det, 1024, 0, s>>>(prefix, M.N);
    return cudaGetLastError();
}

// -------------------------------------------------------------- live init
__global__ void k_init_live(Model M, uint64_t seed, int n, double *live_u) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int d = M.dim;
    for (int p = 0; 2 * p < d; p++) {
        uint4 w = draw(seed, (uint32_t)p, 0u, (uint32_t)i, ITER_INIT);
        live_u[(size_t)i * d + 2 * p] = u01(w.x, w.y);
        if (2 * p + 1 < d) live_u[(size_t)i * d + 2 * p + 1] = u01(w.z, w.w);
    }
}

cudaError_t launch_init_live(const Model &M, uint64_t seed, int n, double *live_u, cudaStream_t s) {
    k_init_live<<<(n + 127) / 128, 128, 0, s>>>(M, seed, n, live_u);
    return cudaGetLastError();
}

// ------------------------------------------------------ likelihood (CTA)
// Coefficients of one point from warp 0 (shared), then all warps run the bin
// loop and the CTA reduces Z_d. Returns log L in *lval (shared) after the
// second barrier; every thread of the CTA must call it.
template <int PREC, int NDET, int W>
__device__ __forceinline__ void cta_loglike_bins(const Model &M, const Tables &T, Coef &coef,
                                                 CoefMixed &cm, double (*red)[2 * MAXDET], double *lval) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double zr[NDET], zi[NDET];
    if (PREC == 0) {
        bins_fp64<NDET>(T, M.N, M.f0, M.df, coef, threadIdx.x, W * 32, zr, zi);
    } else {
        bins_mixed<NDET>(T, M.N, cm, coef.jcut, threadIdx.x, W * 32, zr, zi);
    }
#pragma unroll
    for (int d = 0; d < NDET; d++) {
        zr[d] = warp_sum(zr[d]);
        zi[d] = warp_sum(zi[d]);
    }
    if (lane == 0) {
#pragma unroll
        for (int d = 0; d < NDET; d++) { red[warp][2 * d] = zr[d]; red[warp][2 * d + 1] = zi[d]; }
    }
    __syncthreads();
    if (warp == 0) {
        double v = 0.0;
        if (lane < NDET) {
            double ZR = 0.0, ZI = 0.0;
            for (int w = 0; w < W; w++) { ZR += red[w][2 * lane]; ZI += red[w][2 * lane + 1]; }
            v = coef.gre[lane] * ZR - coef.gim[lane] * ZI;
        }
        v = warp_sum(v);
        if (lane == 0) *lval = (M.model == M_TOY) ? coef.toy : v - 0.5 * coef.hh;
    }
}

// Warp 0 computes the coefficients of the point with unit-cube coordinates u
// (or physical parameters theta when in_is_theta).
__device__ __forceinline__ void warp_point_coef(const Model &M, const Tables &T, const double *in,
                                                int in_is_theta, int precision, Coef *coef,
                                                CoefMixed *cm) {
    const int lane = threadIdx.x & 31;
    if (M.model == M_TOY) {
        point_coef_warp(M, T, in, coef);
        return;
    }
    if (in_is_theta) {
        // a model whose parameters are all FIXED at theta
        Model Mt = M;
#pragma unroll
        for (int p = 0; p < NPARAM; p++) { Mt.kind[p] = K_FIXED; Mt.lo[p] = in[p]; }
        point_coef_warp(Mt, T, in, coef);
    } else {
        point_coef_warp(M, T, in, coef);
    }
    __syncwarp();
    if (precision == 1) coef_to_mixed_warp(*coef, M.n_det, cm, M.rb ? T.rb.fid : nullptr);
    (void)lane;
}

template <int PREC, int NDET, int W>
__global__ void __launch_bounds__(W * 32) k_eval(Model M, Tables T, const double *in, int in_is_theta,
                                                 int m, double *logl) {
    __shared__ Coef coef;
    __shared__ CoefMixed cm;
    __shared__ double red[W][2 * MAXDET];
    __shared__ double lval;
    __shared__ double pt[NPARAM + MAXD];
    const int i = blockIdx.x;
    if (i >= m) return;
    const int stride_in = in_is_theta ? NPARAM : M.dim;
    if (threadIdx.x < stride_in) pt[threadIdx.x] = in[(size_t)i * stride_in + threadIdx.x];
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) warp_point_coef(M, T, pt, in_is_theta, PREC, &coef, &cm);
    __syncthreads();
    if (M.rb) {
        // relative-binning sums: one warp
        if ((threadIdx.x >> 5) == 0) {
            const int lane = threadIdx.x & 31;
            const double v = rb_loglike_warp<NDET, PREC>(M, T.rb, coef, cm, lane);
            if (lane == 0) logl[i] = v;
        }
        return;
    }
    cta_loglike_bins<PREC, NDET, W>(M, T, coef, cm, red, &lval);
    if (threadIdx.x == 0) logl[i] = lval;
}

template <int PREC, int NDET>
static cudaError_t eval_w(const Model &M, const Tables &T, int warps, const double *in, int th, int m,
                          double *logl, cudaStream_t s) {
    switch (warps) {
        case 1: k_eval<PREC, NDET, 1><<<m, 32, 0, s>>>(M, T, in, th, m, logl); break;
        case 2: k_eval<PREC, NDET, 2><<<m, 64, 0, s>>>(M, T, in, th, m, logl); break;
        case 4: k_eval<PREC, NDET, 4><<<m, 128, 0, s>>>(M, T, in, th, m, logl); break;
        default: k_eval<PREC, NDET, 8><<<m, 256, 0, s>>>(M, T, in, th, m, logl); break;
    }
    return cudaGetLastError();
}

template <int PREC>
static cudaError_t eval_d(const Model &M, const Tables &T, int warps, const double *in, int th, int m,
                          double *logl, cudaStream_t s) {
    switch (M.n_det) {
        case 1: return eval_w<PREC, 1>(M, T, warps, in, th, m, logl, s);
        case 2: return eval_w<PREC, 2>(M, T, warps, in, th, m, logl, s);
        case 3: return eval_w<PREC, 3>(M, T, warps, in, th, m, logl, s);
        default: return eval_w<PREC, 4>(M, T, warps, in, th, m, logl, s);
    }
}

cudaError_t launch_eval(const Model &M, const Tables &T, int precision, int warps, const double *in,
                        int in_is_theta, int m, double *logl, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    return precision == 1 ? eval_d<1>(M, T, warps, in, in_is_theta, m, logl, s)
                          : eval_d<0>(M, T, warps, in, in_is_theta, m, logl, s);
}

// ------------------------------------------------------------------ select
// Ascending order of n log L values, ties by index: bitonic sort of
// (order-preserving 64-bit key, index) pairs in shared memory, one CTA.
constexpr int SELECT_MAX = 4096;

__device__ __forceinline__ unsigned long long sortable_key(double x) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b & 0x8000000000000000ull) ? ~b : (b | 0x8000000000000000ull);
}

__device__ void select_body(const double *logl, int n, int *order) {
    __shared__ unsigned long long key[SELECT_MAX];
    __shared__ int idx[SELECT_MAX];
    int P = 1;
    while (P < n) P <<= 1;
    for (int i = threadIdx.x; i < P; i += blockDim.x) {
        key[i] = (i < n) ? sortable_key(logl[i]) : 0xFFFFFFFFFFFFFFFFull;
        idx[i] = (i < n) ? i : 0x7FFFFFFF;
    }
    __syncthreads();
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < P; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    const bool up = ((i & size) == 0);
                    const unsigned long long ki = key[i], kj = key[j];
                    const int ii = idx[i], ij = idx[j];
                    const bool gt = (ki > kj) || (ki == kj && ii > ij);
                    if (gt == up) { key[i] = kj; key[j] = ki; idx[i] = ij; idx[j] = ii; }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) order[i] = idx[i];
}

__global__ void __launch_bounds__(1024) k_select(const double *logl, int n, int *order) {
    select_body(logl, n, order);
}

cudaError_t launch_select(const double *logl, int n, int *order, cudaStream_t s) {
    if (n > SELECT_MAX) return cudaErrorInvalidValue;
    k_select<<<1, 1024, 0, s>>>(logl, n, order);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- evidence
// Dead points j = 1..k in ascending order: Delta_j = 1/(n-j+1),
// log w_j = log X_{j-1} + log(1 - exp(-Delta_j)), log X_j = log X_{j-1} - Delta_j,
// log Z <- logaddexp(log Z, logsumexp_j(log L_j + log w_j)). The prefix sums of
// Delta_j use a block scan; the dead records are appended at state->n_dead.
__device__ void evidence_body(const Model &M, const StepArgs &A) {
    __shared__ double scan[1024];
    __shared__ double scratch[32];
    RunState *st = A.state;
    const int n = A.n, k = A.k, d = M.dim, T = blockDim.x, t = threadIdx.x;
    const double logX0 = st->logX;
    const long long base = st->n_dead;
    double carry = 0.0;      // sum of Delta over previous chunks
    double amax = -DBL_MAX;
    // pass 1: log w_j, dead records, running max of log L_j + log w_j
    for (int c0 = 0; c0 < k; c0 += T) {
        const int j = c0 + t + 1;               // 1-based
        const double delta = (j <= k) ? 1.0 / (double)(n - j + 1) : 0.0;
        scan[t] = delta;
        __syncthreads();
        for (int o = 1; o < T; o <<= 1) {       // inclusive Hillis-Steele scan
            double v = (t >= o) ? scan[t - o] : 0.0;
            __syncthreads();
            scan[t] += v;
            __syncthreads();
        }
        const double incl = carry + scan[t];
        const double excl = incl - delta;
        if (j <= k) {
            const int src = A.order[j - 1];
            const double lw = logX0 - excl + log(-expm1(-delta));
            const double ll = A.live_logl[src];
            const long long o = base + (j - 1);
            A.dead_logl[o] = ll;
            A.dead_logw[o] = lw;
            A.dead_nlive[o] = (double)(n - j + 1);
            for (int i = 0; i < d; i++) A.dead_u[o * d + i] = A.live_u[(size_t)src * d + i];
            amax = fmax(amax, ll + lw);
        }
        const double last = scan[T - 1];
        __syncthreads();
        carry += last;
    }
    amax = block_max(amax, scratch);
    double s = 0.0;
    for (int j = t + 1; j <= k; j += T) {
        const long long o = base + (j - 1);
        s += exp(A.dead_logl[o] + A.dead_logw[o] - amax);
    }
    s = block_sum(s, scratch);
    if (t == 0) {
        const double lz_new = amax + log(s);
        const double lz = st->logZ;
        const double hi = fmax(lz, lz_new), lo = fmin(lz, lz_new);
        st->logZ = (lo == -INFINITY) ? hi : hi + log1p(exp(lo - hi));
        st->logX = logX0 - carry;
        st->lstar = A.live_logl[A.order[k - 1]];
        st->n_dead = base + k;
    }
}

__global__ void __launch_bounds__(1024) k_evidence(Model M, StepArgs A) { evidence_body(M, A); }

cudaError_t launch_evidence(const Model &M, const StepArgs &A, cudaStream_t s) {
    k_evidence<<<1, 1024, 0, s>>>(M, A);
    return cudaGetLastError();
}

// ----------------------------------------------------- covariance, Cholesky
// Unbiased covariance (1/(m-1)) of the m = n-k survivors (sorted positions
// k..n-1) in unit-cube coordinates, jittered by 1e-12 tr/d, Cholesky factor
// by warp 0 (lane i owns row i); diag(sqrt(Sigma_ii)) if it fails.
__device__ void cov_chol_body(const Model &M, const StepArgs &A) {
    __shared__ double mean[MAXD];
    __shared__ double cov[MAXD * MAXD];
    __shared__ double xs[64][MAXD + 1];     // a tile of survivors, centred
    const int d = M.dim, n = A.n, k = A.k, m = n - k;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // means: warp w sums coordinate w (and w + nw, ...) over all survivors
    for (int i = warp; i < d; i += nw) {
        double s = 0.0;
        for (int p = lane; p < m; p += 32) s += A.live_u[(size_t)A.order[k + p] * d + i];
        s = warp_sum(s);
        if (lane == 0) mean[i] = s / m;
    }
    __syncthreads();
    // covariance: thread t owns entries (i, j), j <= i, t = i (i + 1)/2 + j, and
    // accumulates them over tiles of 64 centred survivors held in shared memory
    const int npair = d * (d + 1) / 2;
    int pi = 0, pj = 0;
    if ((int)threadIdx.x < npair) {
        int t = threadIdx.x;
        while (t > pi) { t -= pi + 1; pi++; }
        pj = t;
    }
    double acc = 0.0;
    for (int p0 = 0; p0 < m; p0 += 64) {
        for (int e = threadIdx.x; e < 64 * d; e += blockDim.x) {
            const int p = e / d, i = e % d;
            xs[p][i] = (p0 + p < m) ? A.live_u[(size_t)A.order[k + p0 + p] * d + i] - mean[i] : 0.0;
        }
        __syncthreads();
        if ((int)threadIdx.x < npair) {
            const int pe = min(64, m - p0);
            for (int p = 0; p < pe; p++) acc += xs[p][pi] * xs[p][pj];
        }
        __syncthreads();
    }
    if ((int)threadIdx.x < npair) {
        cov[pi * d + pj] = acc / (m - 1);
        cov[pj * d + pi] = acc / (m - 1);
    }
    if (threadIdx.x == 0 && A.active) *A.active = A.k;     // chains of the coming slice update
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        double tr = 0.0;
        for (int i = 0; i < d; i++) tr += cov[i * d + i];
        const double jit = 1e-12 * tr / d;
        double row[MAXD];
        for (int j = 0; j < MAXD; j++) row[j] = 0.0;
        bool ok = true;
        for (int j = 0; j < d; j++) {
            // diagonal element of column j (owned by lane j), then rows i > j
            double s = (lane < d) ? cov[lane * d + j] + ((lane == j) ? jit : 0.0) : 0.0;
            for (int q = 0; q < j; q++) {
                const double ljq = __shfl_sync(0xffffffffu, row[q], j);
                s -= row[q] * ljq;
            }
            const double djj = __shfl_sync(0xffffffffu, s, j);
            if (!(djj > 0.0)) { ok = false; break; }
            const double ljj = sqrt(djj);
            if (lane == j) row[j] = ljj;
            else if (lane > j && lane < d) row[j] = s / ljj;
        }
        ok = __all_sync(0xffffffffu, ok);
        if (lane < d) {
            for (int j = 0; j < d; j++) {
                double v;
                if (ok) v = (j <= lane) ? row[j] : 0.0;
                else v = (j == lane) ? sqrt(fmax(cov[lane * d + lane] + jit, 0.0)) : 0.0;
                A.chol[lane * d + j] = v;
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_cov_chol(Model M, StepArgs A) { cov_chol_body(M, A); }

cudaError_t launch_cov_chol(const Model &M, const StepArgs &A, cudaStream_t s) {
    k_cov_chol<<<1, 256, 0, s>>>(M, A);
    return cudaGetLastError();
}

// ------------------------------------------------------------ slice update
// One CTA per chain, S warps ("slots"). Warp 0 owns the chain: the point x,
// the direction e and the bracket (lane i < d holds coordinate i). Every slice
// step draws a direction and a bracket offset, steps out to the left and to the
// right, then shrinks (Neal 2003, Sec. 4, along a hit-and-run direction).
//
// The candidates of each stage form sequences fixed by the draws alone:
// stepping out to the left visits x + (a - q) e, to the right x + (b + q) e,
// and the q-th shrink draw is determined once the earlier draws are known to be
// rejected. Each round, warp 0 plans the next S candidates of these sequences
// that lie inside the prior box and are not yet evaluated; every slot warp
// computes one candidate's coefficients and bins; warp 0 then consumes the
// results strictly in the sequential order (left stepping out, right stepping
// out, shrinkage) and keeps results it could not consume yet in a small cache.
// Evaluations the sequential order never reaches are discarded. The trajectory,
// the evaluation count and every draw are those of the sequential algorithm;
// the slots only shorten the chain's critical path.
enum { PH_NEWSTEP = 0, PH_OUT = 1, PH_SHRINK = 2, PH_DONE = 3 };
enum { KIND_L = 0, KIND_R = 1, KIND_SH = 2 };
constexpr int CACHE_MAX = 16;

struct Chain {
    double x, e, lrow[MAXD];
    double lx, a, b;
    int s, phase, nl, nr, nsh, caps, left_done, right_done;
    long long evals;
    unsigned long long bins;
    // cache of evaluated, not yet consumed candidates
    int ncache;
    int ckind[CACHE_MAX], cidx[CACHE_MAX], cbins[CACHE_MAX];
    double cval[CACHE_MAX];
};

__device__ __forceinline__ bool warp_inbox(double y, int lane, int d) {
    return __all_sync(0xffffffffu, lane >= d || (y >= 0.0 && y <= 1.0));
}

__device__ __forceinline__ int cache_find(const Chain &c, int kind, int idx) {
    for (int i = 0; i < c.ncache; i++)
        if (c.ckind[i] == kind && c.cidx[i] == idx) return i;
    return -1;
}

__device__ __forceinline__ void cache_drop(Chain &c, int i) {
    c.ncache--;
    c.ckind[i] = c.ckind[c.ncache];
    c.cidx[i] = c.cidx[c.ncache];
    c.cval[i] = c.cval[c.ncache];
    c.cbins[i] = c.cbins[c.ncache];
}

// Drop every cached result of one stepping-out side (once that side has ended,
// its later candidates are never consumed).
__device__ __forceinline__ void cache_purge(Chain &c, int kind) {
    for (int i = c.ncache - 1; i >= 0; i--)
        if (c.ckind[i] == kind) cache_drop(c, i);
}

__device__ __forceinline__ void end_side(Chain &c, bool left) {
    if (left) { c.left_done = 1; cache_purge(c, KIND_L); }
    else { c.right_done = 1; cache_purge(c, KIND_R); }
}

__device__ __forceinline__ double shrink_t(const StepArgs &A, double a, double b, int nsh, int step,
                                           int chain, uint32_t iter) {
    const uint4 w = draw(A.seed, SLOT_SHRINK0 + (uint32_t)nsh, (uint32_t)step, (uint32_t)chain, iter);
    return __dadd_rn(a, __dmul_rn(__dsub_rn(b, a), u01(w.x, w.y)));
}

// Apply every transition that needs no new evaluation: new steps (direction and
// bracket draws), cap and prior-box outcomes, and results already in the cache.
// Returns when the next transition needs an evaluation not in the cache, or the
// chain is done.
__device__ void chain_run(const Model &M, const StepArgs &A, Chain &c, int chain, uint32_t iter,
                          double lstar) {
    const int lane = threadIdx.x & 31, d = M.dim;
    for (int guard = 0; guard < (1 << 22); guard++) {
        if (c.phase == PH_DONE) return;
        if (c.phase == PH_NEWSTEP) {
            if (c.s >= A.steps) { c.phase = PH_DONE; return; }
            // direction e = L z / |z|, z ~ N(0, I) by Box-Muller, two normals per draw
            double z = 0.0;
            if (lane < d) {
                const uint4 w = draw(A.seed, (uint32_t)(lane >> 1), (uint32_t)c.s, (uint32_t)chain, iter);
                const double u1 = u01(w.x, w.y), u2 = u01(w.z, w.w);
                const double r = sqrt(-2.0 * log(u1));
                double sn, cs;
                sincos(TWO_PI_D * u2, &sn, &cs);
                z = (lane & 1) ? r * sn : r * cs;
            }
            const double nz = sqrt(warp_sum(z * z));
            double acc = 0.0;
            for (int j = 0; j < d; j++) {
                const double zj = __shfl_sync(0xffffffffu, z, j);
                if (j <= lane) acc = __dadd_rn(acc, __dmul_rn(c.lrow[j], zj));
            }
            c.e = (lane < d) ? acc / nz : 0.0;
            const uint4 w = draw(A.seed, SLOT_OFFSET, (uint32_t)c.s, (uint32_t)chain, iter);
            const double r = u01(w.x, w.y);
            c.a = -r;
            c.b = 1.0 - r;
            c.nl = c.nr = c.nsh = 0;
            c.left_done = c.right_done = 0;
            c.ncache = 0;
            c.phase = PH_OUT;
            continue;
        }
        if (c.phase == PH_OUT) {
            const bool left = !c.left_done;
            if (!left && c.right_done) { c.phase = PH_SHRINK; continue; }
            const int n = left ? c.nl : c.nr;
            if (n >= A.max_stepout) {
                end_side(c, left);
                continue;
            }
            const double t = left ? c.a : c.b;
            const double y = (lane < d) ? __dadd_rn(c.x, __dmul_rn(t, c.e)) : 0.5;
            if (!warp_inbox(y, lane, d)) {
                end_side(c, left);
                continue;
            }
            const int ci = cache_find(c, left ? KIND_L : KIND_R, n);
            if (ci < 0) return;
            const bool in = c.cval[ci] > lstar;
            c.evals++;
            c.bins += (unsigned long long)c.cbins[ci];
            cache_drop(c, ci);
            if (left) { if (in) { c.a -= 1.0; c.nl++; } else end_side(c, true); }
            else { if (in) { c.b += 1.0; c.nr++; } else end_side(c, false); }
            continue;
        }
        // PH_SHRINK
        if (c.nsh >= A.max_shrink) {
            c.caps++;
            c.s++;
            c.phase = PH_NEWSTEP;
            continue;
        }
        const double t = shrink_t(A, c.a, c.b, c.nsh, c.s, chain, iter);
        const double y = (lane < d) ? __dadd_rn(c.x, __dmul_rn(t, c.e)) : 0.5;
        if (warp_inbox(y, lane, d)) {
            const int ci = cache_find(c, KIND_SH, c.nsh);
            if (ci < 0) return;
            const double val = c.cval[ci];
            c.evals++;
            c.bins += (unsigned long long)c.cbins[ci];
            cache_drop(c, ci);
            if (val > lstar) {
                c.x = y;
                c.lx = val;
                c.s++;
                c.phase = PH_NEWSTEP;
                continue;
            }
        }
        if (t < 0.0) c.a = t; else c.b = t;
        c.nsh++;
    }
    c.phase = PH_DONE;   // unreachable with finite caps; keeps the loop bounded
}

// Plan up to S candidates to evaluate in the next round (in-box, not cached),
// continuing the current stage's sequences. Writes their coordinates to
// ysh[slot][*] and their keys to pk/pi; returns the number of slots used.
template <int S>
__device__ int chain_plan(const Model &M, const StepArgs &A, const Chain &c, int chain, uint32_t iter,
                          double (*ysh)[MAXD], int *pk, int *pidx, int depth) {
    const int lane = threadIdx.x & 31, d = M.dim;
    int ns = 0;
    const int room = CACHE_MAX - c.ncache;
    const int lim = depth < S ? depth : S;
    const int cap = lim < room ? lim : room;
    if (c.phase == PH_OUT) {
        // the side in progress first (half the slots if the other side is
        // still open), then the other side; each looks at most S candidates
        // ahead of its consumed position, so the cache holds at most 2S entries
        for (int side = 0; side < 2 && ns < cap; side++) {
            const bool left = (side == 0);
            if (left ? c.left_done : c.right_done) continue;
            const int limit = (left && !c.right_done) ? (cap + 1) / 2 : cap;
            double t = left ? c.a : c.b;
            const int n0 = left ? c.nl : c.nr;
            for (int n = n0; n < n0 + S && n < A.max_stepout && ns < limit; n++) {
                const double y = (lane < d) ? __dadd_rn(c.x, __dmul_rn(t, c.e)) : 0.5;
                if (!warp_inbox(y, lane, d)) break;
                if (cache_find(c, left ? KIND_L : KIND_R, n) < 0) {
                    if (lane < d) ysh[ns][lane] = y;
                    pk[ns] = left ? KIND_L : KIND_R;
                    pidx[ns] = n;
                    ns++;
                }
                if (left) t -= 1.0; else t += 1.0;
            }
        }
    } else if (c.phase == PH_SHRINK) {
        double a = c.a, b = c.b;
        for (int n = c.nsh; n < c.nsh + S && n < A.max_shrink && ns < cap; n++) {
            const double t = shrink_t(A, a, b, n, c.s, chain, iter);
            const double y = (lane < d) ? __dadd_rn(c.x, __dmul_rn(t, c.e)) : 0.5;
            if (warp_inbox(y, lane, d) && cache_find(c, KIND_SH, n) < 0) {
                if (lane < d) ysh[ns][lane] = y;
                pk[ns] = KIND_SH;
                pidx[ns] = n;
                ns++;
            }
            if (t < 0.0) a = t; else b = t;     // as if rejected
        }
    }
    return ns;
}

template <int PREC, int NDET, int S>
__device__ void slice_body(const Model &M, const Tables &T, const StepArgs &A, const int chain) {
    __shared__ Coef coef[S];
    __shared__ CoefMixed cm[S];
    __shared__ double ysh[S][MAXD];
    __shared__ double lval[S];
    __shared__ int nslot;
    __shared__ int jc[S];
    __shared__ double part[S][S][NDET][2];
    if (chain >= A.k) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, d = M.dim;
    const uint32_t iter = (uint32_t)A.state->iter;
    const double lstar = A.state->lstar;
    Chain c;
    int pk[S], pidx[S];
    if (warp == 0) {
        const int m = A.n - A.k;
        const uint4 w = draw(A.seed, 0u, STEP_START, (uint32_t)chain, iter);
        int idx = (int)(u01(w.x, w.y) * m);
        if (idx >= m) idx = m - 1;
        const int src = A.order[A.k + idx];
        c.x = (lane < d) ? A.live_u[(size_t)src * d + lane] : 0.0;
        c.lx = A.live_logl[src];
        for (int j = 0; j < MAXD; j++) c.lrow[j] = (lane < d && j < d) ? A.chol[lane * d + j] : 0.0;
        c.e = 0.0; c.a = 0.0; c.b = 0.0;
        c.s = 0; c.phase = PH_NEWSTEP; c.nl = c.nr = c.nsh = 0; c.caps = 0; c.evals = 0; c.bins = 0;
        c.left_done = c.right_done = 0; c.ncache = 0;
    }
    for (;;) {
        if (warp == 0) {
            chain_run(M, A, c, chain, iter, lstar);
            // plan the base depth while many chains run; the stragglers of the
            // update (fewer running chains than the tail threshold) use every warp
            int depth = S;
            if (A.active) {
                const int running = *((volatile int *)A.active);
                if (running > A.tail) depth = A.depth;
            }
            int ns = (c.phase == PH_DONE) ? 0 : chain_plan<S>(M, A, c, chain, iter, ysh, pk, pidx, depth);
            if (ns == 0 && c.phase != PH_DONE) {
                // cannot happen with the bounds above; end the chain at its
                // current (in-slice) point and flag the run state
                c.phase = PH_DONE;
                if (lane == 0) atomicOr(&A.state->status, 1);
            }
            if (lane == 0) nslot = ns;
        }
        __syncthreads();
        const int ns = nslot;
        if (ns == 0) break;
        // coefficients: warp w computes candidates 4w .. 4w+3 (8 lanes each)
        if (M.model == M_TOY) {
            if (warp < ns) point_coef_warp(M, T, ysh[warp], &coef[warp]);
        } else if (4 * warp < ns) {
            const int cnt = ns - 4 * warp < 4 ? ns - 4 * warp : 4;
            point_coef_group(M, T, ysh[4 * warp], MAXD, &coef[4 * warp], cnt, PREC == 0 ? 32 : 0);
        }
        __syncthreads();
        if (warp < ns && M.rb) {
            // relative-binning likelihood of the slot's candidate
            if (PREC == 1) {
                coef_to_mixed_warp(coef[warp], M.n_det, &cm[warp], T.rb.fid);
                __syncwarp();
            }
            const double v = rb_loglike_warp<NDET, PREC>(M, T.rb, coef[warp], cm[warp], lane);
            if (lane == 0) {
                lval[warp] = v;
                coef[warp].jcut = T.rb.nb - 1;     // bins counted for the work statistics
            }
        } else if (PREC == 1 && S > 1 && S <= 4 && M.model == M_GW && !M.rb && M.coop) {
            // mixed: all warps stride the bins for all candidates of the round
            if (warp < ns) coef_to_mixed_warp(coef[warp], M.n_det, &cm[warp]);
            if (lane == 0 && warp < ns) jc[warp] = coef[warp].jcut;
            __syncthreads();
            float zrh[S][NDET], zrl[S][NDET], zih[S][NDET], zil[S][NDET];
            bins_mixed_multi<NDET, S>(T, M.N, cm, jc, ns, threadIdx.x, S * 32, zrh, zrl, zih, zil);
#pragma unroll
            for (int sc = 0; sc < S; sc++)
#pragma unroll
                for (int dd = 0; dd < NDET; dd++) {
                    warp_sum_df(zrh[sc][dd], zrl[sc][dd]);
                    warp_sum_df(zih[sc][dd], zil[sc][dd]);
                    if (lane == 0) {
                        part[warp][sc][dd][0] = (double)zrh[sc][dd] + (double)zrl[sc][dd];
                        part[warp][sc][dd][1] = (double)zih[sc][dd] + (double)zil[sc][dd];
                    }
                }
            __syncthreads();
            if (warp == 0) {
                // lane = (candidate, detector): sum over warps, then log L per candidate
                double v = 0.0;
                const int sc = lane / NDET, dd = lane % NDET;
                if (sc < ns && lane < S * NDET) {
                    double ZR = 0.0, ZI = 0.0;
                    for (int w2 = 0; w2 < S; w2++) { ZR += part[w2][sc][dd][0]; ZI += part[w2][sc][dd][1]; }
                    v = coef[sc].gre[dd] * ZR - coef[sc].gim[dd] * ZI;
                }
                for (int sc2 = 0; sc2 < ns; sc2++) {
                    double t = (lane / NDET == sc2 && lane < S * NDET) ? v : 0.0;
                    t = warp_sum(t);
                    if (lane == 0) lval[sc2] = t - 0.5 * coef[sc2].hh;
                }
            }
        } else if (warp < ns) {
            // one candidate per slot warp: bins and warp reduction
            if (PREC == 1) {
                coef_to_mixed_warp(coef[warp], M.n_det, &cm[warp]);
                __syncwarp();
            }
            double zr[NDET], zi[NDET];
            if (PREC == 0) bins_fp64<NDET, true>(T, M.N, M.f0, M.df, coef[warp], lane, 32, zr, zi);
            else bins_mixed<NDET>(T, M.N, cm[warp], coef[warp].jcut, lane, 32, zr, zi);
            double v = 0.0;
#pragma unroll
            for (int dd = 0; dd < NDET; dd++) {
                const double ZR = warp_sum(zr[dd]), ZI = warp_sum(zi[dd]);
                v += coef[warp].gre[dd] * ZR - coef[warp].gim[dd] * ZI;
            }
            if (lane == 0) lval[warp] = (M.model == M_TOY) ? coef[warp].toy : v - 0.5 * coef[warp].hh;
        }
        __syncthreads();
        if (warp == 0) {
            for (int sl = 0; sl < ns; sl++) {
                c.ckind[c.ncache] = pk[sl];
                c.cidx[c.ncache] = pidx[sl];
                c.cval[c.ncache] = lval[sl];
                c.cbins[c.ncache] = coef[sl].jcut + 1;
                c.ncache++;
            }
        }
        // coef/lval are rewritten only after the next barrier's plan
    }
    if (warp == 0) {
        const int dst = A.order[chain];
        if (lane < d) A.live_u[(size_t)dst * d + lane] = c.x;
        if (lane == 0) {
            A.live_logl[dst] = c.lx;
            if (A.active) atomicSub(A.active, 1);
            atomicAdd(&A.state->evals, (unsigned long long)c.evals);
            atomicAdd(&A.state->caps, (unsigned long long)c.caps);
            atomicAdd(&A.state->point_bins, c.bins);
        }
    }
}

template <int PREC, int NDET, int S>
__global__ void __launch_bounds__(S * 32) k_slice(Model M, Tables T, StepArgs A) {
    slice_body<PREC, NDET, S>(M, T, A, blockIdx.x);
}

template <int PREC, int NDET>
static cudaError_t slice_w(const Model &M, const Tables &T, int slots, const StepArgs &A, cudaStream_t s) {
    switch (slots) {
        case 1: k_slice<PREC, NDET, 1><<<A.k, 32, 0, s>>>(M, T, A); break;
        case 2: k_slice<PREC, NDET, 2><<<A.k, 64, 0, s>>>(M, T, A); break;
        case 4: k_slice<PREC, NDET, 4><<<A.k, 128, 0, s>>>(M, T, A); break;
        default: k_slice<PREC, NDET, 8><<<A.k, 256, 0, s>>>(M, T, A); break;
    }
    return cudaGetLastError();
}

template <int PREC>
static cudaError_t slice_d(const Model &M, const Tables &T, int slots, const StepArgs &A, cudaStream_t s) {
    switch (M.n_det) {
        case 1: return slice_w<PREC, 1>(M, T, slots, A, s);
        case 2: return slice_w<PREC, 2>(M, T, slots, A, s);
        case 3: return slice_w<PREC, 3>(M, T, slots, A, s);
        default: return slice_w<PREC, 4>(M, T, slots, A, s);
    }
}

cudaError_t launch_slice(const Model &M, const Tables &T, int precision, int slots, const StepArgs &A,
                         cudaStream_t s) {
    return precision == 1 ? slice_d<1>(M, T, slots, A, s) : slice_d<0>(M, T, slots, A, s);
}

// ------------------------------------------------------------------ finish
__device__ void finish_body(const StepArgs &A) {
    __shared__ double scratch[32];
    double m = -DBL_MAX;
    for (int i = threadIdx.x; i < A.n; i += blockDim.x) m = fmax(m, A.live_logl[i]);
    m = block_max(m, scratch);
    if (threadIdx.x == 0) {
        RunState *st = A.state;
        const double lz = st->logZ, b = st->logX + m;
        const double hi = fmax(lz, b), lo = fmin(lz, b);
        const double tot = (lo == -INFINITY) ? hi : hi + log1p(exp(lo - hi));
        st->logl_max = m;
        st->remaining = tot - lz;
        st->done = (st->remaining < A.dlogz_stop) ? 1 : 0;
        st->iter += 1;
    }
}

__global__ void __launch_bounds__(1024) k_finish(StepArgs A) { finish_body(A); }

cudaError_t launch_finish(const StepArgs &A, cudaStream_t s) {
    k_finish<<<1, 1024, 0, s>>>(A);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ result
// Final live points (order[] ascending, computed before): Delta_j = 1/(n-j+1)
// for j = 1..n continuing from the current log X; total log Z.
__global__ void __launch_bounds__(1024) k_final_live(Model M, StepArgs A, double *fin_u, double *fin_logl,
                                                     double *fin_logw, double *fin_nlive, double *logz_total) {
    __shared__ double scan[1024];
    __shared__ double scratch[32];
    const int n = A.n, d = M.dim, T = blockDim.x, t = threadIdx.x;
    const double logX0 = A.state->logX;
    double carry = 0.0, amax = -DBL_MAX;
    for (int c0 = 0; c0 < n; c0 += T) {
        const int j = c0 + t + 1;
        const double delta = (j <= n) ? 1.0 / (double)(n - j + 1) : 0.0;
        scan[t] = delta;
        __syncthreads();
        for (int o = 1; o < T; o <<= 1) {
            double v = (t >= o) ? scan[t - o] : 0.0;
            __syncthreads();
            scan[t] += v;
            __syncthreads();
        }
        const double excl = carry + scan[t] - delta;
        if (j <= n) {
            const int src = A.order[j - 1];
            const double lw = logX0 - excl + log(-expm1(-delta));
            const double ll = A.live_logl[src];
            fin_logl[j - 1] = ll;
            fin_logw[j - 1] = lw;
            fin_nlive[j - 1] = (double)(n - j + 1);
            for (int i = 0; i < d; i++) fin_u[(size_t)(j - 1) * d + i] = A.live_u[(size_t)src * d + i];
            amax = fmax(amax, ll + lw);
        }
        const double last = scan[T - 1];
        __syncthreads();
        carry += last;
    }
    amax = block_max(amax, scratch);
    double s = 0.0;
    for (int j = t; j < n; j += T) s += exp(fin_logl[j] + fin_logw[j] - amax);
    s = block_sum(s, scratch);
    if (t == 0) {
        const double lz_new = amax + log(s), lz = A.state->logZ;
        const double hi = fmax(lz, lz_new), lo = fmin(lz, lz_new);
        *logz_total = (lo == -INFINITY) ? hi : hi + log1p(exp(lo - hi));
    }
}

cudaError_t launch_final_live(const Model &M, const StepArgs &A, double *fin_u, double *fin_logl,
                              double *fin_logw, double *fin_nlive, double *logz_total, cudaStream_t s) {
    k_final_live<<<1, 1024, 0, s>>>(M, A, fin_u, fin_logl, fin_logw, fin_nlive, logz_total);
    return cudaGetLastError();
}

// Replicate evidences for dlogZ: one block per replicate r redraws every
// shrinkage factor, log t_i = log(U_ri)/n_i, and accumulates
// log Z_r = logsumexp_i(log L_i + log X_{i-1} + log(1 - t_i)) with an online
// (max, sum) pair per thread; entries are the dead points then the final live.
__device__ __forceinline__ void lse_push(double &mx, double &sm, double a) {
    if (a > mx) { sm = sm * exp(mx - a) + 1.0; mx = a; }
    else sm += exp(a - mx);
}

__global__ void __launch_bounds__(1024) k_replicates(ResultArgs R) {
    __shared__ double scan[1024];
    __shared__ double smx[32], ssm[32];
    const int T = blockDim.x, t = threadIdx.x, r = blockIdx.x;
    const long long m = R.n_dead + R.n;
    double carry = 0.0, mx = -DBL_MAX, sm = 0.0;
    for (long long c0 = 0; c0 < m; c0 += T) {
        const long long i = c0 + t;
        double logt = 0.0, ll = 0.0;
        if (i < m) {
            const uint4 w = draw(R.seed, 0u, (uint32_t)i, (uint32_t)r, ITER_REPLICATE);
            const double nl = (i < R.n_dead) ? R.dead_nlive[i] : R.fin_nlive[i - R.n_dead];
            ll = (i < R.n_dead) ? R.dead_logl[i] : R.fin_logl[i - R.n_dead];
            logt = log(u01(w.x, w.y)) / nl;
        }
        scan[t] = logt;
        __syncthreads();
        for (int o = 1; o < T; o <<= 1) {
            double v = (t >= o) ? scan[t - o] : 0.0;
            __syncthreads();
            scan[t] += v;
            __syncthreads();
        }
        if (i < m) {
            const double logx_prev = carry + scan[t] - logt;
            lse_push(mx, sm, ll + logx_prev + log(-expm1(logt)));
        }
        const double last = scan[T - 1];
        __syncthreads();
        carry += last;
    }
    // combine (mx, sm) over the block
    const int lane = t & 31, warp = t >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        const double omx = __shfl_xor_sync(0xffffffffu, mx, o), osm = __shfl_xor_sync(0xffffffffu, sm, o);
        const double nm = fmax(mx, omx);
        sm = sm * exp(mx - nm) + osm * exp(omx - nm);
        mx = nm;
    }
    if (lane == 0) { smx[warp] = mx; ssm[warp] = sm; }
    __syncthreads();
    if (t == 0) {
        double M0 = -DBL_MAX, S0 = 0.0;
        for (int w = 0; w < (T + 31) / 32; w++) {
            const double nm = fmax(M0, smx[w]);
            S0 = S0 * exp(M0 - nm) + ssm[w] * exp(smx[w] - nm);
            M0 = nm;
        }
        R.reps[r] = M0 + log(S0);
    }
}

// dlogZ (standard deviation of the replicates), information H and Kish ESS.
__global__ void __launch_bounds__(1024) k_result_stats(ResultArgs R) {
    __shared__ double scratch[32];
    const long long m = R.n_dead + R.n;
    double s = 0.0;
    for (int r = threadIdx.x; r < R.R; r += blockDim.x) s += R.reps[r];
    const double mean = block_sum(s, scratch) / R.R;
    double v = 0.0;
    for (int r = threadIdx.x; r < R.R; r += blockDim.x) v += (R.reps[r] - mean) * (R.reps[r] - mean);
    const double var = block_sum(v, scratch) / R.R;
    double sp = 0.0, sp2 = 0.0, sh = 0.0;
    for (long long i = threadIdx.x; i < m; i += blockDim.x) {
        const double ll = (i < R.n_dead) ? R.dead_logl[i] : R.fin_logl[i - R.n_dead];
        const double lw = (i < R.n_dead) ? R.dead_logw[i] : R.fin_logw[i - R.n_dead];
        const double p = exp(lw + ll - R.logZ);
        sp += p;
        sp2 += p * p;
        sh += p * (ll - R.logZ);
    }
    sp = block_sum(sp, scratch);
    sp2 = block_sum(sp2, scratch);
    sh = block_sum(sh, scratch);
    if (threadIdx.x == 0) {
        R.out[0] = sqrt(var);
        R.out[1] = sh;
        R.out[2] = sp * sp / sp2;
        R.out[3] = mean;
    }
}

cudaError_t launch_result_stats(const ResultArgs &R, cudaStream_t s) {
    k_replicates<<<R.R, 1024, 0, s>>>(R);
    k_result_stats<<<1, 1024, 0, s>>>(R);
    return cudaGetLastError();
}

__global__ void k_theta(Model M, const double *u, long long m, double *theta) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    double th[NPARAM];
    prior_transform(M, u + i * M.dim, th);
    for (int p = 0; p < NPARAM; p++) theta[i * NPARAM + p] = th[p];
}

cudaError_t launch_theta(const Model &M, const double *u, long long m, double *theta, cudaStream_t s) {
    if (m <= 0 || M.model != M_GW) return cudaSuccess;
    k_theta<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(M, u, m, theta);
    return cudaGetLastError();
}

// Detector strain of one parameter vector: coefficients by one warp, then
// h_d(f_j) = conj(G_d) f^(-7/6) exp(-i Psi_dj) per bin in FP64 (zero above jcut).
__global__ void k_waveform_coef(Model M, Tables T, const double *theta, Coef *out) {
    __shared__ Coef c;
    Model Mt = M;
    for (int p = 0; p < NPARAM; p++) { Mt.kind[p] = K_FIXED; Mt.lo[p] = theta[p]; }
    point_coef_warp(Mt, T, theta, &c);
    __syncwarp();
    if (threadIdx.x == 0) *out = c;
}

__global__ void k_waveform_bins(Model M, Tables T, const Coef *cp, double *h_re, double *h_im) {
    const Coef &c = *cp;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M.N; j += gridDim.x * blockDim.x) {
        const double f = T.f64[j];
        double psi0 = c.c0;
        for (int m = 0; m < NB; m++) psi0 += c.a[m] * T.basis64[(size_t)m * M.N + j];
        const double amp = pow(f, -7.0 / 6.0);
        for (int d = 0; d < M.n_det; d++) {
            double re = 0.0, im = 0.0;
            if (j <= c.jcut) {
                double s, co;
                sincos(psi0 + TWO_PI_D * f * c.tau[d], &s, &co);
                re = amp * (c.gre[d] * co - c.gim[d] * s);
                im = amp * (-c.gre[d] * s - c.gim[d] * co);
            }
            h_re[(size_t)d * M.N + j] = re;
            h_im[(size_t)d * M.N + j] = im;
        }
    }
}

// ------------------------------------------------------- relative binning setup
// Coarse-bin edges: B+1 geometric frequencies f0 (f_last/f0)^(b/B), moved to the
// nearest grid index, repeated indices dropped (one thread: B is ~1e3).
__global__ void k_rb_edges(Model M, int B, int *J, int *nedge) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double flo = M.f0, fhi = __dadd_rn(M.f0, __dmul_rn((double)(M.N - 1), M.df));
    int n = 0;
    for (int b = 0; b <= B; b++) {
        const double target = flo * pow(fhi / flo, (double)b / B);
        int j = (int)floor((target - M.f0) / M.df + 0.5);
        j = j < 0 ? 0 : (j > M.N - 1 ? M.N - 1 : j);
        if (b == B) j = M.N - 1;
        if (n == 0 || j > J[n - 1]) J[n++] = j;
    }
    *nedge = n;
}

// Fiducial strain without cutoff on the fine grid: h0 = conj(G0) f^(-7/6) exp(-i Psi0).
__global__ void k_rb_h0(Model M, Tables T, const Coef *fid, double2 *h0) {
    const Coef &c = *fid;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < M.N; j += gridDim.x * blockDim.x) {
        const double f = T.f64[j];
        double psi0 = c.c0;
        for (int m = 0; m < NB; m++) psi0 += c.a[m] * T.basis64[(size_t)m * M.N + j];
        const double amp = pow(f, -7.0 / 6.0);
        for (int d = 0; d < M.n_det; d++) {
            double s, co;
            sincos(psi0 + TWO_PI_D * f * c.tau[d], &s, &co);
            h0[(size_t)d * M.N + j] = make_double2(amp * (c.gre[d] * co - c.gim[d] * s),
                                                   amp * (-c.gre[d] * s - c.gim[d] * co));
        }
    }
}

// Summary data of bin b (blockIdx.x) and detector d (blockIdx.y), plus the edge
// tables (from block (b, 0)).
__global__ void __launch_bounds__(256) k_rb_summary(Model M, const int *J, const int *nedge_p,
                                                    const double *dre, const double *dim, const double *psd,
                                                    const double2 *h0, RBTables R, double *fe, double *basis64,
                                                    float2 *basis32, float2 *fe32, double *fm, double *inv_de,
                                                    double2 *A0, double2 *A1, double *B0, double *B1, float2 *A0f,
                                                    float2 *A1f, float *B0f, float *B1f, float *inv_de_f) {
    __shared__ double scratch[32];
    const int nedge = *nedge_p, nb = nedge - 1;
    const int b = blockIdx.x, d = blockIdx.y;
    if (b >= nb) return;
    const int lo = J[b], hi = (b == nb - 1) ? J[b + 1] + 1 : J[b + 1];
    const double elo = __dadd_rn(M.f0, __dmul_rn((double)J[b], M.df));
    const double ehi = __dadd_rn(M.f0, __dmul_rn((double)J[b + 1], M.df));
    const double fmid = 0.5 * (elo + ehi);
    double a0r = 0, a0i = 0, a1r = 0, a1i = 0, b0 = 0, b1 = 0;
    for (int j = lo + threadIdx.x; j < hi; j += blockDim.x) {
        const size_t o = (size_t)d * M.N + j;
        const double f = __dadd_rn(M.f0, __dmul_rn((double)j, M.df));
        const double w = 4.0 * M.df / psd[o];
        const double2 h = h0[o];
        const double xr = dre[o] * h.x + dim[o] * h.y;      // d h0^*
        const double xi = dim[o] * h.x - dre[o] * h.y;
        const double hh = h.x * h.x + h.y * h.y;
        a0r += w * xr; a0i += w * xi;
        a1r += w * xr * (f - fmid); a1i += w * xi * (f - fmid);
        b0 += w * hh; b1 += w * hh * (f - fmid);
    }
    a0r = block_sum(a0r, scratch); a0i = block_sum(a0i, scratch);
    a1r = block_sum(a1r, scratch); a1i = block_sum(a1i, scratch);
    b0 = block_sum(b0, scratch); b1 = block_sum(b1, scratch);
    if (threadIdx.x == 0) {
        const size_t o = (size_t)d * nb + b;
        A0[o] = make_double2(a0r, a0i);
        A1[o] = make_double2(a1r, a1i);
        B0[o] = b0;
        B1[o] = b1;
        A0f[o] = make_float2((float)a0r, (float)a0i);
        A1f[o] = make_float2((float)a1r, (float)a1i);
        B0f[o] = (float)b0;
        B1f[o] = (float)b1;
        if (d == 0) {
            fm[b] = fmid;
            inv_de[b] = 1.0 / (ehi - elo);
            inv_de_f[b] = (float)(1.0 / (ehi - elo));
        }
    }
    // edge tables: edge b (and the last edge from the last bin)
    if (d == 0 && threadIdx.x < 2) {
        const int e = b + threadIdx.x;
        if (threadIdx.x == 1 && b != nb - 1) return;
        const double f = __dadd_rn(M.f0, __dmul_rn((double)J[e], M.df));
        const double lf = log(f), cb = cbrt(f), ic = 1.0 / cb;
        double Bv[NB] = {ic * ic * ic * ic * ic, 1.0 / f, ic * ic, ic, lf, cb, cb * lf, cb * cb};
        for (int m = 0; m < NB; m++) {
            basis64[(size_t)m * nedge + e] = Bv[m];
            const float h = __double2float_rn(Bv[m]);
            basis32[(size_t)m * nedge + e] = make_float2(h, __double2float_rn(Bv[m] - (double)h));
        }
        fe[e] = f;
        const float h = __double2float_rn(f);
        fe32[e] = make_float2(h, __double2float_rn(f - (double)h));
    }
}

cudaError_t launch_rb_setup(const Model &M, const Tables &T, int B, const double *theta_fid, int *J,
                            int *nedge_dev, Coef *fid, double2 *h0_tmp, const double *dre, const double *dim,
                            const double *psd, RBTables &R, double *fe, double *basis64, float2 *basis32,
                            float2 *fe32, double *fm, double *inv_de, double2 *A0, double2 *A1, double *B0,
                            double *B1, float2 *A0f, float2 *A1f, float *B0f, float *B1f, float *inv_de_f,
                            cudaStream_t s) {
    k_rb_edges<<<1, 1, 0, s>>>(M, B, J, nedge_dev);
    k_waveform_coef<<<1, 32, 0, s>>>(M, T, theta_fid, fid);
    k_rb_h0<<<min((M.N + 255) / 256, 1216), 256, 0, s>>>(M, T, fid, h0_tmp);
    dim3 grid(B, M.n_det);
    k_rb_summary<<<grid, 256, 0, s>>>(M, J, nedge_dev, dre, dim, psd, h0_tmp, R, fe, basis64, basis32, fe32,
                                      fm, inv_de, A0, A1, B0, B1, A0f, A1f, B0f, B1f, inv_de_f);
    return cudaGetLastError();
}

cudaError_t launch_point_coef(const Model &M, const Tables &T, const double *theta, Coef *out,
                              cudaStream_t s) {
    k_waveform_coef<<<1, 32, 0, s>>>(M, T, theta, out);
    return cudaGetLastError();
}

cudaError_t launch_waveform(const Model &M, const Tables &T, const double *theta, Coef *scratch,
                            double *h_re, double *h_im, cudaStream_t s) {
    k_waveform_coef<<<1, 32, 0, s>>>(M, T, theta, scratch);
    k_waveform_bins<<<min((M.N + 255) / 256, 1216), 256, 0, s>>>(M, T, scratch, h_re, h_im);
    return cudaGetLastError();
}

// ------------------------------------------------ multi-analysis iteration
// The serving loop runs one iteration of every admitted analysis with one
// launch per kernel: block a of the per-analysis kernels works on analysis a,
// and block b of the slice update on chain map[b].y of analysis map[b].x.
// Each block first copies its analysis' descriptor to shared memory.
__device__ __forceinline__ void load_desc(const Desc *g, Desc &s) {
    const int *src = (const int *)g;
    int *dst = (int *)&s;
    for (int i = threadIdx.x; i < (int)(sizeof(Desc) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    __syncthreads();
}

__global__ void __launch_bounds__(1024) k_select_multi(const Desc *D) {
    // the sort's 48 KB of shared memory leaves no room for a descriptor copy
    const StepArgs &A = D[blockIdx.x].A;
    select_body(A.live_logl, A.n, A.order);
}
__global__ void __launch_bounds__(1024) k_evidence_multi(const Desc *D) {
    __shared__ Desc d;
    load_desc(D + blockIdx.x, d);
    evidence_body(d.M, d.A);
}
__global__ void __launch_bounds__(256) k_cov_chol_multi(const Desc *D) {
    __shared__ Desc d;
    load_desc(D + blockIdx.x, d);
    cov_chol_body(d.M, d.A);
}
__global__ void __launch_bounds__(1024) k_finish_multi(const Desc *D) {
    __shared__ Desc d;
    load_desc(D + blockIdx.x, d);
    finish_body(d.A);
}
template <int PREC, int NDET, int S>
__global__ void __launch_bounds__(S * 32) k_slice_multi(const Desc *D, const int2 *map) {
    __shared__ Desc d;
    const int2 ac = map[blockIdx.x];
    load_desc(D + ac.x, d);
    slice_body<PREC, NDET, S>(d.M, d.T, d.A, ac.y);
}

template <int PREC, int NDET>
static cudaError_t slice_multi_w(const Desc *D, const int2 *map, int nblocks, int slots, cudaStream_t s) {
    switch (slots) {
        case 1: k_slice_multi<PREC, NDET, 1><<<nblocks, 32, 0, s>>>(D, map); break;
        case 2: k_slice_multi<PREC, NDET, 2><<<nblocks, 64, 0, s>>>(D, map); break;
        case 4: k_slice_multi<PREC, NDET, 4><<<nblocks, 128, 0, s>>>(D, map); break;
        default: k_slice_multi<PREC, NDET, 8><<<nblocks, 256, 0, s>>>(D, map); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_iteration_multi_head(const Desc *D, int n_an, cudaStream_t s) {
    k_select_multi<<<n_an, 1024, 0, s>>>(D);
    k_evidence_multi<<<n_an, 1024, 0, s>>>(D);
    k_cov_chol_multi<<<n_an, 256, 0, s>>>(D);
    return cudaGetLastError();
}

cudaError_t launch_slice_multi(const Desc *D, const int2 *map, int nblocks, int precision, int ndet, int slots,
                               cudaStream_t s) {
    if (nblocks <= 0) return cudaSuccess;
    if (precision == 1) {
        switch (ndet) {
            case 1: return slice_multi_w<1, 1>(D, map, nblocks, slots, s);
            case 2: return slice_multi_w<1, 2>(D, map, nblocks, slots, s);
            case 3: return slice_multi_w<1, 3>(D, map, nblocks, slots, s);
            default: return slice_multi_w<1, 4>(D, map, nblocks, slots, s);
        }
    }
    switch (ndet) {
        case 1: return slice_multi_w<0, 1>(D, map, nblocks, slots, s);
        case 2: return slice_multi_w<0, 2>(D, map, nblocks, slots, s);
        case 3: return slice_multi_w<0, 3>(D, map, nblocks, slots, s);
        default: return slice_multi_w<0, 4>(D, map, nblocks, slots, s);
    }
}

cudaError_t launch_iteration_multi_tail(const Desc *D, int n_an, cudaStream_t s) {
    k_finish_multi<<<n_an, 1024, 0, s>>>(D);
    return cudaGetLastError();
}

}  // namespace gwns
