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
// Phase basis {f^-5/3, f^-1, f^-2/3, f^-1/3, ln f, f^1/3, f^1/3 ln f, f^2/3}.
__device__ __forceinline__ void basis_at(double f, double B[NB]) {
    const double lf = log(f);
    const double c = cbrt(f);          // f^(1/3)
    const double ic = 1.0 / c;
    B[0] = ic * ic * ic * ic * ic;
    B[1] = 1.0 / f;
    B[2] = ic * ic;
    B[3] = ic;
    B[4] = lf;
    B[5] = c;
    B[6] = c * lf;
    B[7] = c * c;
}

// Taylor coefficients D[k][m] = B_m^(k)(f) df^k / k!, k = 0..TK, of the basis
// about f: binomial series for the powers, the log series for ln f, and their
// Cauchy product for f^(1/3) ln f.
__device__ __forceinline__ void basis_taylor(double f, double df, double D[TK + 1][NB]) {
    const double r = df / f;
    double B[NB];
    basis_at(f, B);
    const double pw[NB] = {-5.0 / 3.0, -1.0, -2.0 / 3.0, -1.0 / 3.0, 0.0, 1.0 / 3.0, 0.0, 2.0 / 3.0};
#pragma unroll
    for (int m = 0; m < NB; m++) {
        if (m == 4 || m == 6) continue;
        double cf = 1.0;
        D[0][m] = B[m];
        for (int k = 1; k <= TK; k++) {
            cf *= (pw[m] - (k - 1)) / k * r;
            D[k][m] = B[m] * cf;
        }
    }
    D[0][4] = B[4];
    double rk = 1.0;
    for (int k = 1; k <= TK; k++) {
        rk *= r;
        D[k][4] = ((k & 1) ? rk : -rk) / k;
    }
    for (int k = 0; k <= TK; k++) {
        double acc = 0.0;
        for (int i = 0; i <= k; i++) acc += D[i][5] * D[k - i][4];
        D[k][6] = acc;
    }
}

// Per bin: f_j, the phase basis B_m(f_j), the weighted data
// w_dj = 4 df f^(-7/6) d_dj / S_dj and the terms 4 df f^(-7/3) / S_dj of the
// <h|h> prefix sums (scanned by k_prefix_scan). Mixed form per bin: B_m(f_j),
// f_j and w_dj as floats. Tiled form: w_dj in pair-tile order over the padded
// grid (zero beyond N) and, per tile, the basis Taylor coefficients about its
// centre and the centre frequency.
__global__ void k_build_tables(Model M, const double *dre, const double *dim, const double *psd,
                               double *basis64, double *f64, double2 *w64, double *prefix, float2 *basis32,
                               float2 *f32, float2 *w32, float2 *tb0, float2 *tb1, float *tbk, float2 *fc,
                               float2 *wt) {
    const int N = M.N, lg = M.tlg;
    const int jend = lg ? M.np : N;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < jend; j += gridDim.x * blockDim.x) {
        if (lg && (j & ((1 << lg) - 1)) == 0) {
            const int t = j >> lg, nt = M.np >> lg;
            const double fcen = __dadd_rn(M.f0, __dmul_rn((double)(j + (1 << (lg - 1))), M.df));
            double D[TK + 1][NB];
            basis_taylor(fcen, M.df, D);
#pragma unroll
            for (int m = 0; m < NB; m++) {
                float h = __double2float_rn(D[0][m]);
                tb0[(size_t)m * nt + t] = make_float2(h, __double2float_rn(D[0][m] - (double)h));
                h = __double2float_rn(D[1][m]);
                tb1[(size_t)m * nt + t] = make_float2(h, __double2float_rn(D[1][m] - (double)h));
                for (int k = 2; k <= TK; k++) tbk[((size_t)(k - 2) * NB + m) * nt + t] = __double2float_rn(D[k][m]);
            }
            const float h = __double2float_rn(fcen);
            fc[t] = make_float2(h, __double2float_rn(fcen - (double)h));
        }
        if (j >= N) {
            for (int d = 0; d < M.n_det; d++) wt[(size_t)d * M.np + tile_pos2(j, lg)] = make_float2(0.f, 0.f);
            continue;
        }
        const double f = __dadd_rn(M.f0, __dmul_rn((double)j, M.df));
        double B[NB];
        basis_at(f, B);
#pragma unroll
        for (int m = 0; m < NB; m++) {
            basis64[(size_t)m * N + j] = B[m];
            if (!lg) {
                const float h = __double2float_rn(B[m]);
                basis32[(size_t)m * N + j] = make_float2(h, __double2float_rn(B[m] - (double)h));
            }
        }
        f64[j] = f;
        if (!lg) {
            const float h = __double2float_rn(f);
            f32[j] = make_float2(h, __double2float_rn(f - (double)h));
        }
        const double f76 = pow(f, -7.0 / 6.0);
        for (int d = 0; d < M.n_det; d++) {
            const size_t o = (size_t)d * N + j;
            const double sd = psd[o];
            const double wr = 4.0 * M.df * f76 * dre[o] / sd;
            const double wi = 4.0 * M.df * f76 * dim[o] / sd;
            w64[o] = make_double2(wr, wi);
            const float2 wf = make_float2(__double2float_rn(wr), __double2float_rn(wi));
            if (lg) {
                // float2 slot pos of the pair order -> float4 (Re, Re, Im, Im) of its bin pair
                const size_t pos = (size_t)d * M.np + tile_pos2(j, lg);
                float *wq = reinterpret_cast<float *>(wt) + ((pos >> 1) << 2) + (pos & 1);
                wq[0] = wf.x;
                wq[2] = wf.y;
            } else {
                w32[o] = wf;
            }
            prefix[o] = 4.0 * M.df * f76 * f76 / sd;
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
                                double *prefix, const MixedTables &X, cudaStream_t s) {
    const int n = M.tlg ? M.np : M.N;
    int blocks = min((n + 255) / 256, 152 * 8);
    k_build_tables<<<blocks, 256, 0, s>>>(M, data_re, data_im, psd, basis64, f64, w64, prefix, X.basis32,
                                          X.f32, X.w32, X.tb0, X.tb1, X.tbk, X.fc, X.wt);
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
// ------------------------------------------------------------ dispatch
// The likelihood and slice kernels are instantiated per (precision, detectors)
// in gwns_inst_p<P>_d<D>.cu.
template <int PREC>
static cudaError_t eval_d(const Model &M, const Tables &T, int warps, const double *in, int th, int m,
                          double *logl, RunState *st, cudaStream_t s) {
    switch (M.n_det) {
        case 1: return eval_launch<PREC, 1>(M, T, warps, in, th, m, logl, st, s);
        case 2: return eval_launch<PREC, 2>(M, T, warps, in, th, m, logl, st, s);
        case 3: return eval_launch<PREC, 3>(M, T, warps, in, th, m, logl, st, s);
        default: return eval_launch<PREC, 4>(M, T, warps, in, th, m, logl, st, s);
    }
}

cudaError_t launch_eval(const Model &M, const Tables &T, int precision, int warps, const double *in,
                        int in_is_theta, int m, double *logl, RunState *st, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    return precision == 1 ? eval_d<1>(M, T, warps, in, in_is_theta, m, logl, st, s)
                          : eval_d<0>(M, T, warps, in, in_is_theta, m, logl, st, s);
}

template <int PREC>
static cudaError_t slice_d(const Model &M, const Tables &T, int slots, const StepArgs &A, cudaStream_t s) {
    switch (M.n_det) {
        case 1: return slice_launch<PREC, 1>(M, T, slots, A, s);
        case 2: return slice_launch<PREC, 2>(M, T, slots, A, s);
        case 3: return slice_launch<PREC, 3>(M, T, slots, A, s);
        default: return slice_launch<PREC, 4>(M, T, slots, A, s);
    }
}

int ws_blocks_per_sm(int precision, int ndet) {
    if (precision != 1) return 0;
    switch (ndet) {
        case 1: return slice_ws_blocks_per_sm<1, 1>();
        case 2: return slice_ws_blocks_per_sm<1, 2>();
        case 3: return slice_ws_blocks_per_sm<1, 3>();
        default: return slice_ws_blocks_per_sm<1, 4>();
    }
}

cudaError_t launch_slice(const Model &M, const Tables &T, int precision, int slots, const StepArgs &A,
                         cudaStream_t s) {
    return precision == 1 ? slice_d<1>(M, T, slots, A, s) : slice_d<0>(M, T, slots, A, s);
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
        // a single survivor (k = n - 1) has no sample covariance: the unit
        // cube's prior covariance I/12 stands in
        const double v = m >= 2 ? acc / (m - 1) : (pi == pj ? 1.0 / 12.0 : 0.0);
        cov[pi * d + pj] = v;
        cov[pj * d + pi] = v;
    }
    if (threadIdx.x == 0 && A.active) *A.active = A.k;     // chains of the coming slice update
    if (threadIdx.x == 0 && A.chain_ctr) *A.chain_ctr = 0;  // next chain for the work-shared update
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
        if (A.kernel == 1) {
            // next walk length: A.steps accepted moves per walk at this
            // iteration's acceptance, within [A.steps, 64 A.steps]
            const unsigned long long acc = st->walk_acc;
            double t = 64.0 * A.steps;
            if (acc > 0) {
                t = ceil(((double)st->walk_len * (double)A.steps) * (double)A.k / (double)acc);
                t = fmin(fmax(t, (double)A.steps), 64.0 * A.steps);
            }
            st->walk_len = (int)t;
            st->walk_acc = 0;
        }
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
cudaError_t launch_iteration_multi_head(const Desc *D, int n_an, cudaStream_t s) {
    k_select_multi<<<n_an, 1024, 0, s>>>(D);
    k_evidence_multi<<<n_an, 1024, 0, s>>>(D);
    k_cov_chol_multi<<<n_an, 256, 0, s>>>(D);
    return cudaGetLastError();
}

cudaError_t launch_slice_multi(const Desc *D, const int2 *map, int nblocks, int precision, int ndet, int slots,
                               int rot, cudaStream_t s) {
    if (nblocks <= 0) return cudaSuccess;
    if (precision == 1) {
        switch (ndet) {
            case 1: return slice_multi_launch<1, 1>(D, map, nblocks, slots, rot, s);
            case 2: return slice_multi_launch<1, 2>(D, map, nblocks, slots, rot, s);
            case 3: return slice_multi_launch<1, 3>(D, map, nblocks, slots, rot, s);
            default: return slice_multi_launch<1, 4>(D, map, nblocks, slots, rot, s);
        }
    }
    switch (ndet) {
        case 1: return slice_multi_launch<0, 1>(D, map, nblocks, slots, 0, s);
        case 2: return slice_multi_launch<0, 2>(D, map, nblocks, slots, 0, s);
        case 3: return slice_multi_launch<0, 3>(D, map, nblocks, slots, 0, s);
        default: return slice_multi_launch<0, 4>(D, map, nblocks, slots, 0, s);
    }
}

cudaError_t launch_iteration_multi_tail(const Desc *D, int n_an, cudaStream_t s) {
    k_finish_multi<<<n_an, 1024, 0, s>>>(D);
    return cudaGetLastError();
}

}  // namespace gwns
