/*
 * gwns.h -- C ABI of the GB300 nested-slice-sampling library for
 * gravitational-wave parameter estimation.
 *
 * The calls follow the paper's statement of the problem (Sec. 2 and Sec. 3 of
 * "Parallel Nested Slice Sampling for Gravitational Wave Parameter
 * Estimation"): set up a likelihood from data, noise PSD and frequency grid
 * (ns_init), run nested-sampling iterations that each delete the k
 * lowest-likelihood live points and replace them with slice-sampling chains
 * (ns_step), and read back the evidence with its error and the weighted
 * posterior samples (ns_result).
 *
 * Conventions for every call:
 *   - return NS_OK (0) on success, a negative NS_ERR_* code otherwise; no C++
 *     exception crosses this boundary; ns_strerror() names each code;
 *   - "host" pointers are read (or written) before the call returns; inputs are
 *     copied, so the caller keeps ownership and may free them afterwards;
 *   - "device" pointers are CUDA global-memory pointers of the current device,
 *     accessed asynchronously on the context's stream;
 *   - all device state (tables, live set, dead list, scratch) is owned by the
 *     context and released by ns_free();
 *   - one context is not thread-safe; distinct contexts are independent.
 */
#ifndef GWNS_H
#define GWNS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- codes */
enum {
    NS_OK = 0,
    NS_ERR_INVALID_ARG = -1,   /* a null pointer, a size out of range, a bad enum */
    NS_ERR_PSD_NONPOS = -2,    /* a PSD value <= 0 or not finite */
    NS_ERR_K_RANGE = -3,       /* k outside 1 .. n_live-1 */
    NS_ERR_OOM = -4,           /* a device allocation failed */
    NS_ERR_CAPACITY = -5,      /* the caller's output buffer is too small */
    NS_ERR_TIMEOUT = -6,       /* a bounded device-side wait gave up (the work-shared slice update
                                  of mixed precision on the finest grids; ns_stats.status bit 1) */
    NS_ERR_CANCELLED = -7,     /* the request was cancelled */
    NS_ERR_CUDA = -8,          /* a CUDA runtime call failed */
    NS_ERR_STATE = -9          /* call not valid in the context's state */
};

/* --------------------------------------------------------- parameters */
/* The 11 physical parameters, in this order everywhere (theta[11]):
 * detector-frame chirp mass [Msun], mass ratio q = m2/m1 <= 1, aligned spins
 * chi1, chi2, luminosity distance [Mpc], cos(inclination), polarisation
 * angle [rad], coalescence phase [rad], geocentre coalescence time [s],
 * right ascension [rad] (Greenwich sidereal time 0), sin(declination). */
enum {
    NS_MC = 0, NS_Q, NS_CHI1, NS_CHI2, NS_DL, NS_COSI, NS_PSI, NS_PHIC, NS_TC, NS_RA,
    NS_SINDEC, NS_NPARAM
};

enum { NS_PRIOR_FIXED = 0, NS_PRIOR_UNIFORM = 1, NS_PRIOR_VOLUME = 2 };

/* Inner kernels of the update (ns_options.kernel). */
enum { NS_KERNEL_SLICE = 0, NS_KERNEL_WALK = 1 };
/* Arithmetic of the likelihood (ns_options.precision). NS_FP64: FP64 throughout.
 * NS_MIXED: per-point coefficients in double-float (pairs of floats on the FP32
 * pipe; the FP64 stage instead when the environment variable GWNS_COEF_FP64=1 is
 * set at ns_init, or for relative binning), the per-bin phase in double-float,
 * FP32 sine/cosine and products with compensated sums, the final log L in FP64
 * (paper Sec. 3's likelihood; the precision split is this library's). */
enum { NS_FP64 = 0, NS_MIXED = 1 };
enum { NS_MODEL_GW = 0, NS_MODEL_TOY = 1 };

#define NS_MAX_DET 4
#define NS_MAX_DIM 16

/* Prior over the 11 parameters. FIXED: theta = lo. UNIFORM on [lo, hi].
 * VOLUME: p(x) ~ x^2 on [lo, hi] (distance uniform in comoving volume).
 * The sampled dimension d is the number of non-FIXED entries; a unit-cube
 * point u[d] maps to the non-fixed parameters in parameter order. */
typedef struct {
    int kind[NS_NPARAM];
    double lo[NS_NPARAM];
    double hi[NS_NPARAM];
} ns_prior;

/* Strain data and detector geometry (host, copied at ns_init).
 * re/im: [n_det][N] frequency-domain data d_d(f_j); both NULL means zero data
 * (used to build injections, see ns_waveform / ns_set_data).
 * pos: [n_det][3] detector positions in metres (Earth-fixed frame);
 * xarm, yarm: [n_det][3] unit vectors of the two arms.
 * ideal = 1 replaces every detector by an idealised one with F+ = 1,
 * Fx = 0 and no time delay (pos/xarm/yarm may then be NULL). */
typedef struct {
    int n_det;
    int ideal;
    const double *re;
    const double *im;
    const double *pos;
    const double *xarm;
    const double *yarm;
} ns_data;

/* One-sided noise PSD S_d(f_j) [1/Hz], [n_det][N], host, copied, all > 0. */
typedef struct {
    const double *S;
} ns_psd;

/* Uniform frequency grid f_j = f0 + j df, j = 0 .. N-1 (both ends included).
 * coarse_bins > 0 switches the likelihood to relative binning (the paper's
 * heterodyned likelihood on a coarser frequency grid, Sec. 2-3; Zackay, Dai &
 * Venumadhav 2018) about the fiducial parameters theta_fid[11] (host, copied):
 * coarse_bins geometric bins between f0 and the last grid frequency, edges
 * moved to the nearest grid index (repeated edges dropped); per bin and
 * detector the summary data A0 = sum d h0^* w, A1 = sum d h0^* w (f - fm),
 * B0 = sum |h0|^2 w, B1 = sum |h0|^2 w (f - fm) (w = 4 df / S, h0 the fiducial
 * strain without cutoff, fm the bin centre), and for each point r = h/h0
 * interpolated linearly between the edges. Bins whose centre lies above
 * f_ISCO are dropped when the cutoff is on. */
typedef struct {
    int N;
    double f0;
    double df;
    int coarse_bins;
    const double *theta_fid;
} ns_grid;

/* Run options. Zero-initialise and set what you need; zero fields take the
 * defaults in brackets. */
typedef struct {
    int n_live;          /* live points n (required, >= 2) */
    int k;               /* points deleted per iteration [n/2] (paper Sec. 2) */
    int steps_per_dim;   /* slice steps per chain = steps_per_dim * d [5] */
    int precision;       /* NS_FP64 or NS_MIXED */
    int no_cutoff;       /* 0: waveform zero above f_ISCO; 1: no cutoff */
    int max_stepout;     /* per side [64] */
    int max_shrink;      /* shrink draws per slice step [64] */
    int model;           /* NS_MODEL_GW, or NS_MODEL_TOY (correlated Gaussian) */
    int toy_dim;         /* toy dimension d (model = NS_MODEL_TOY) */
    int warps_per_point; /* warps cooperating on one batched likelihood (1,2,4,8) [0: rule] */
    int slots;           /* candidates one chain evaluates concurrently in the slice
                            update, one warp each (1,2,4,8) [0: rule] */
    double dlogz_stop;   /* stop when log(Z + X Lmax) - log Z < this [0.1]; a negative value is
                            never met, so the run goes on to its iteration cap (ns_run's
                            max_iter, the server's max_iter) */
    uint64_t seed;       /* Philox key */
    void *stream;        /* cudaStream_t to run on [NULL: library-owned stream] */
    int kernel;          /* inner kernel of the update: NS_KERNEL_SLICE (slice sampling along
                            hit-and-run directions, paper Sec. 2) or NS_KERNEL_WALK (constrained
                            random walk of adaptive length, the acceptance-walk variant the
                            paper compares against, Sec. 3) [NS_KERNEL_SLICE] */
    double walk_scale;   /* NS_KERNEL_WALK: proposal y = x + walk_scale L z [2.38/sqrt(d)] */
    unsigned periodic;   /* bit p set (p = NS_MC..NS_SINDEC): parameter p is periodic over
                            its prior range (phi_c, psi, RA with their full-period uniform
                            priors): its unit-cube coordinate wraps mod 1 on the slice line
                            instead of leaving the prior box [0: none]. Toy model: bit i
                            is unit-cube coordinate i. The paper (Sec. 2) names better
                            handling of such parameters as future work. */
} ns_options;

typedef struct ns_ctx ns_ctx;

/* Create a context: validate, copy data and PSD to the device, build the
 * per-grid tables (basis functions of f, weighted data 4 df f^(-7/6) d / S,
 * prefix sums of 4 df f^(-7/3) / S), draw the n initial live points from the
 * prior and evaluate them. The likelihood is the Whittle log-likelihood ratio
 * against noise, log L = sum_d [<d_d|h_d> - <h_d|h_d>/2] with
 * <a|b> = 4 df Re sum_j a_j b_j^* / S_j, for a TaylorF2 signal projected on
 * each detector (paper Sec. 3 uses the same likelihood with another waveform).
 * Errors: INVALID_ARG, PSD_NONPOS, K_RANGE, OOM, CUDA. On error *out = NULL. */
int ns_init(ns_ctx **out, const ns_prior *prior, const ns_data *data, const ns_psd *psd,
            const ns_grid *grid, const ns_options *opts);

/* Replace the strain data (host [n_det][N] arrays) and re-evaluate the live
 * points. Errors: INVALID_ARG, CUDA. */
int ns_set_data(ns_ctx *ctx, const double *re, const double *im);

/* One nested-sampling iteration (paper Sec. 2): delete the k lowest live
 * points (the k-th lowest log L is the new threshold L*), update log X and
 * log Z, and replace them by k slice-sampling chains of steps_per_dim * d
 * steps each, started at uniformly chosen survivors and moving along
 * directions drawn from the survivors' covariance, with stepping out and
 * shrinkage (Neal 2003). *done (may be NULL) is set to 1 once the remaining
 * evidence fraction is below dlogz_stop. 1 <= k <= n_live - 1 (K_RANGE). */
int ns_step(ns_ctx *ctx, int k, int *done);

/* ns_step with the iteration's k dead points copied to host buffers
 * (each may be NULL): u [k][d], logl [k], logw [k] (log prior-mass weight). */
int ns_step_host(ns_ctx *ctx, int k, int *done, double *dead_u, double *dead_logl,
                 double *dead_logw);

/* Iterate ns_step(opts.k) until done or max_iter iterations. */
int ns_run(ns_ctx *ctx, int max_iter, int *iterations);

/* Weighted samples: the dead points in deletion order followed by the final
 * live points in ascending log L. All arrays host, caller-owned, cap entries.
 * theta may be NULL; u, logl, logw may be NULL. */
typedef struct {
    int cap;          /* capacity (entries) provided by the caller */
    int count;        /* entries written (or needed, on NS_ERR_CAPACITY) */
    double *theta;    /* [cap][11] physical parameters */
    double *u;        /* [cap][d] unit-cube coordinates */
    double *logl;     /* [cap] */
    double *logw;     /* [cap] log prior-mass weight; log posterior weight = logw + logl - logZ */
} ns_samples;

/* Finish the run: add the final live points to the evidence, then return
 * log Z (log Bayes factor signal vs noise), its error dlogZ (standard deviation
 * over 200 replicate shrinkage sequences t ~ Beta(n_j, 1)) and the weighted
 * samples. samples may be NULL. Does not end the run: ns_step may continue.
 * Errors: CAPACITY (samples->count = entries needed), CUDA. */
int ns_result(ns_ctx *ctx, double *logZ, double *dlogZ, ns_samples *samples);

/* Summary statistics of the last ns_result call: the information
 * H = sum_i p_i ln(L_i / Z) (p_i the posterior weights; sqrt(H / n) is the
 * classic evidence-error estimate, Skilling 2006) and the Kish effective sample
 * size (sum p_i)^2 / sum p_i^2 of the weighted samples (the ESS the paper
 * reports, Sec. 4). Host pointers, either may be NULL.
 * Errors: INVALID_ARG (no ns_result yet). */
int ns_result_info(ns_ctx *ctx, double *H, double *ess);

typedef struct {
    long long iterations;
    long long evals;        /* likelihood evaluations so far (initial draw included) */
    long long cap_hits;     /* slice steps that ended at the shrink cap */
    double logZ;            /* running log Z (dead points only) */
    double logX;            /* log prior volume enclosed by the live set */
    double lstar;           /* last threshold */
    double logl_max;        /* largest live log L */
    int done;
    int d;                  /* sampled dimension */
    int n_live;
    int n_dead;
    long long point_bins;   /* sum over slice-update evaluations of the bins each one read */
    int status;             /* 0, or bit 0: a chain ended early (internal inconsistency);
                               bit 1: a bounded wait of the work-shared slice update gave up */
    double kernel_ms[5];    /* cumulative device time of the iteration's kernels, from CUDA
                               events recorded on the context's stream inside the iteration's
                               graph: select, evidence, covariance, slice update, finish */
    int mixed_tile;         /* mixed precision: bins per lane tile of the tiled form (grids fine
                               enough for its Taylor expansion), 0 for the per-bin form */
    long long batch_evals;       /* points through the batched likelihood (ns_eval_lnl*, ns_init's
                                    initial live set) */
    long long batch_point_bins;  /* their sum of the bins each one read */
    long long scratch_bytes;     /* device bytes of the context's staging scratch, allocated by the
                                    host-buffer entry points (ns_eval_lnl_host, ns_waveform,
                                    ns_result with theta) on first use and when a call needs more */
    long long point_bins_lo;       /* of point_bins, the bins of the mixed tiled form's tile groups
                                      summed at the low Taylor degree (work-shared update) */
    long long batch_point_bins_lo; /* of batch_point_bins, the same (mixed batched likelihood on
                                      grids above 262,144 bins) */
} ns_stats;

int ns_get_stats(ns_ctx *ctx, ns_stats *st);

/* Batched likelihood of m unit-cube points, device pointers: u [m][d] in,
 * logl [m] out, on the context's stream (asynchronous). 0 <= m. */
int ns_eval_lnl(ns_ctx *ctx, const double *u, int m, double *logl);

/* Same with host pointers (copies in, evaluates, copies out, synchronises). */
int ns_eval_lnl_host(ns_ctx *ctx, const double *u, int m, double *logl);

/* Allocation-free variant of ns_eval_lnl_host, for callers that cannot call
 * cudaMalloc at this point: real-time or callback code that must not block in
 * the allocator, and hosts whose device memory is reserved by another
 * allocator (a memory pool that owns the free memory). (The paper has no
 * counterpart; this is an integration feature.) ns_eval_lnl_host stages u and
 * log L in device scratch that it allocates on first use or when m grows;
 * this entry point stages them instead in one file-scope device array of
 * NS_NOALLOC_MAX_POINTS x (NS_MAX_DIM + 1) doubles (557,056 bytes) that every
 * GPU loading the library holds until exit, and it calls no
 * cudaMalloc/cudaFree. Host pointers: u [m][d] in, logl [m] out; the values
 * are in logl when it returns, because it synchronises the context's stream.
 *   - m > NS_NOALLOC_MAX_POINTS returns NS_ERR_CAPACITY (split the batch);
 *   - the first call on a device looks up the array's device address once
 *     (cudaGetSymbolAddress) and keeps it for the process, so make that first
 *     call before any stream capture, and do not call it again on a device
 *     after cudaDeviceReset (the kept address would be stale);
 *   - all calls share the array and it keeps the last call's contents (each
 *     call overwrites the m entries it uses; nothing needs to start at zero);
 *     calls that overlap on the GPU (other threads, other contexts on other
 *     streams) race on it and must be serialised by the caller. */
#define NS_NOALLOC_MAX_POINTS 4096
int ns_eval_lnl_host_noalloc(ns_ctx *ctx, const double *u, int m, double *logl);

/* Batched likelihood of m physical parameter vectors theta [m][11] (device). */
int ns_eval_lnl_theta(ns_ctx *ctx, const double *theta, int m, double *logl);

/* Detector strain h_d(f_j) of one physical parameter vector (host theta[11]),
 * written to host h_re, h_im [n_det][N]; zero above f_ISCO unless no_cutoff. */
int ns_waveform(ns_ctx *ctx, const double *theta, double *h_re, double *h_im);

/* Prior transform of m unit-cube points (host u [m][d]) to physical
 * parameters (host theta [m][11]). */
int ns_prior_transform(ns_ctx *ctx, const double *u, int m, double *theta);

/* Network optimal SNR^2 = sum_d <h_d|h_d> of one parameter vector (host
 * theta[11]), from the closed form A^2 |Q_d|^2 P_d(jcut). */
int ns_optimal_snr2(ns_ctx *ctx, const double *theta, double *rho2);

/* Checkpoint of the run: live set, run state (log Z, log X, iteration,
 * counters) and the dead list, in a self-describing byte buffer (host,
 * caller-owned). With buf NULL, *len receives the size needed; otherwise
 * *len is the buffer's size on input and the bytes written on output
 * (CAPACITY if too small). Inputs (data, PSD, grid, options) are not stored:
 * restore into a context created with the same ones. */
int ns_checkpoint(ns_ctx *ctx, void *buf, size_t *len);

/* Resume from a checkpoint: the continuation is bit-identical to the run that
 * wrote it (same draws, same order). INVALID_ARG if the buffer does not match
 * the context's n_live and dimension. */
int ns_restore(ns_ctx *ctx, const void *buf, size_t len);

/* Live set (host, each may be NULL): u [n][d], logl [n]. */
int ns_get_live(ns_ctx *ctx, double *u, double *logl);

/* Overwrite the live set (host u [n][d], logl [n]); used to resume. */
int ns_set_live(ns_ctx *ctx, const double *u, const double *logl);

/* Autotune the slice update: time `trials` iterations (>= 1) with each slot
 * count 1, 2, 4, 8 from the same saved state (live set, run state and dead
 * list are restored afterwards, so the run continues as if untouched), keep
 * the fastest for this context, and remember it for contexts of the same grid
 * size, detector count, precision, n_live and k created later in the process
 * (used when their options leave slots at 0). The slot count never changes
 * results. *slots (may be NULL) receives the choice. */
int ns_autotune(ns_ctx *ctx, int trials, int *slots);

/* Autotune the batched likelihood (ns_eval_lnl*): time `trials` launches (>= 1)
 * on the context's live points with 1, 2, 4 and 8 warps per point, after one
 * warm-up launch each, and keep the fastest for this context (as if its
 * options had set warps_per_point). Nothing of the run changes; these launches
 * are not counted in ns_stats. *warps (may be NULL) receives the choice. */
int ns_autotune_eval(ns_ctx *ctx, int trials, int *warps);

/* Synchronise the context's stream. */
int ns_sync(ns_ctx *ctx);

void ns_free(ns_ctx *ctx);
const char *ns_strerror(int code);

/* ------------------------------------------------------------- serving */
/* A continuous-batching server of many analyses on one GPU. Requests (one
 * analysis each: prior, data, PSD, grid, options) are queued by ns_submit; each
 * ns_server_tick admits queued requests in arrival order while the number of
 * running analyses is below max_active and their estimated device footprint
 * fits the memory budget, then iterates the running analyses with one launch
 * per iteration kernel (the slice updates of all their chains interleaved in
 * the same launch), and retires the analyses that reached their stopping rule
 * (their evidence, error and samples are kept on the host; their device memory
 * is released). Analyses on grids of more than 32768 bins run ONE iteration per
 * tick on the server's stream; those on smaller grids run on a second stream of
 * the server's own (the device's highest priority), one iteration and then
 * more while the long grids' iteration is still running, so that they do not
 * wait every iteration for the slowest analysis. Every analysis keeps its own
 * live set, Philox key and iteration counter on the device, so its result does
 * not depend on which other analyses share the GPU. Not thread-safe. */
typedef struct ns_server ns_server;

typedef struct {
    int max_active;        /* analyses interleaved at once [16] */
    size_t mem_budget;     /* device bytes for running analyses [0: 80% of free memory] */
    int precision;         /* NS_FP64 or NS_MIXED for every analysis */
    int slots;             /* slice-update slots per chain for every analysis [0: 4] */
    int max_iter;          /* iteration cap per analysis [100000] */
    void *stream;          /* cudaStream_t [NULL: server-owned] */
    int max_chains;        /* admit while the running analyses' chains per iteration (their k)
                              stay within this, the first always [0: 20 per SM]: past it the
                              GPU is saturated and more analyses only lengthen each one's
                              time to result */
} ns_server_options;

typedef struct {
    ns_prior prior;
    ns_data data;
    ns_psd psd;
    ns_grid grid;
    ns_options opts;       /* precision, slots and stream are the server's */
} ns_request;

enum { NS_REQ_PENDING = 0, NS_REQ_RUNNING = 1, NS_REQ_DONE = 2, NS_REQ_CANCELLED = 3 };

typedef struct {
    int state;             /* NS_REQ_*, or a negative NS_ERR_* if its admission failed */
    double logZ, dlogZ;    /* when done */
    long long iterations, evals;
    double t_submit, t_admit, t_done;   /* seconds on the server's clock */
    size_t footprint;      /* estimated device bytes while running: at admission with a dead
                              list of 64 n entries, then grown with the dead list (which doubles
                              when a run outgrows it); memory in use is the running analyses'
                              footprints */
    int n_samples;         /* weighted samples kept (dead + final live) */
} ns_request_status;

int ns_server_create(ns_server **out, const ns_server_options *opts);
/* Copies the request's host inputs; *id identifies it. Validation errors are
 * returned here (INVALID_ARG, PSD_NONPOS, K_RANGE). */
int ns_submit(ns_server *srv, const ns_request *req, uint64_t *id);
/* Admit, iterate the running analyses (see above), retire finished ones.
 * n_running / n_pending (may be NULL) report the queue after the tick. */
int ns_server_tick(ns_server *srv, int *n_running, int *n_pending);
int ns_poll(ns_server *srv, uint64_t id, ns_request_status *st);
/* Weighted samples of a finished request (as ns_result; CAPACITY if too small). */
int ns_server_result(ns_server *srv, uint64_t id, ns_samples *samples);
/* Cancel a pending or running request (its device memory is released). */
int ns_cancel(ns_server *srv, uint64_t id);
/* Seconds on the server's clock (steady clock, zero at creation). */
double ns_server_time(ns_server *srv);
void ns_server_free(ns_server *srv);

#ifdef __cplusplus
}
#endif
#endif /* GWNS_H */
