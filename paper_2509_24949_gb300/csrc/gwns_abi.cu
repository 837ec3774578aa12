// gwns_abi.cu -- host implementation of the C ABI declared in include/gwns.h:
// context lifetime, input validation, device buffers, CUDA-graph capture of
// one nested-sampling iteration, and result assembly.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "gwns_ctx.h"

using namespace gwns;
using namespace gwns_host;


namespace gwns_host {
int cuda_fail(cudaError_t e) {
    if (e == cudaErrorMemoryAllocation) return NS_ERR_OOM;
    return NS_ERR_CUDA;
}
}  // namespace gwns_host

namespace {

constexpr int kReplicates = 200;


#define CK(call)                                   \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return cuda_fail(e_); \
    } while (0)

template <class T>
int dalloc(T **p, size_t count) {
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) { *p = nullptr; return cuda_fail(e); }
    return NS_OK;
}

void dfree(void *p) {
    if (p) cudaFree(p);
}

bool is_fin(double x) { return std::isfinite(x); }

int choose_warps(const ns_ctx *c) {
    if (c->warps > 0) return c->warps;
    if (c->M.model == M_TOY) return 1;
    // FP64: the FP64 pipe binds, so one warp per point keeps the per-point
    // overheads lowest once every SM sub-partition has a chain; mixed: more
    // warps per point hide FP32 latency. Tuned values come from the autotuner.
    const int bins = c->M.N;
    if (c->precision == NS_FP64) return bins > 32768 ? 2 : 1;
    // the rotation form (tiles of 32 bins or more) prefetches its loads and
    // needs fewer warps per point (GB300, 519,169 bins in 128-bin tiles: 8 / 4 /
    // 2 warps give 1.50 / 1.59 / 1.53 M evals/s). Up to 262,144 bins the batched
    // kernel puts 4 max(1, W/2) points in a CTA and one warp on each point's bins:
    // 64,897 bins in 32-bin tiles, 1 / 2 / 4 / 8 warps give 65.6 / 65.7 / 68.5 /
    // 60.7 M evals/s
    if (c->M.tlg >= 5) return 4;
    return bins > 16384 ? 8 : (bins > 2048 ? 4 : 2);
}

// Speculative candidate slots per chain in the slice update: several slots
// shorten a chain's critical path when the GPU is not saturated by the k
// chains' work (small grids), one slot avoids speculative work when it is.



int ensure_scratch(ns_ctx *c, size_t bytes) {
    if (bytes <= c->scratch_bytes) return NS_OK;
    CK(cudaStreamSynchronize(c->stream));
    dfree(c->scratch);
    c->scratch = nullptr;
    c->scratch_bytes = 0;
    int rc = dalloc((char **)&c->scratch, bytes);
    if (rc) return rc;
    c->scratch_bytes = bytes;
    return NS_OK;
}

// Record timing event i on the stream (as an event-record node when capturing).
int mark(ns_ctx *c, int i) {
    if (!c->timing) return NS_OK;
    CK(cudaEventRecordWithFlags(c->ev[i], c->stream, cudaEventRecordExternal));
    return NS_OK;
}

// Enqueue the five kernels of one iteration.
int enqueue_iteration(ns_ctx *c, int k) {
    StepArgs A = step_args(c, k);
    int rc;
    if ((rc = mark(c, 0))) return rc;
    CK(launch_select(c->live_logl, c->n, c->order, c->stream));
    if ((rc = mark(c, 1))) return rc;
    CK(launch_evidence(c->M, A, c->stream));
    if ((rc = mark(c, 2))) return rc;
    CK(launch_cov_chol(c->M, A, c->stream));
    if ((rc = mark(c, 3))) return rc;
    CK(launch_slice(c->M, c->T, c->precision, slots_alloc(c), A, c->stream));
    if ((rc = mark(c, 4))) return rc;
    CK(launch_finish(A, c->stream));
    if ((rc = mark(c, 5))) return rc;
    return NS_OK;
}

int capture_iteration(ns_ctx *c, int k) {
    if (c->graph && c->graph_k == k) return NS_OK;
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_iteration(c, k);
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (rc) { if (g) cudaGraphDestroy(g); return rc; }
    if (e != cudaSuccess) return cuda_fail(e);
    e = cudaGraphInstantiate(&c->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { c->graph = nullptr; return cuda_fail(e); }
    c->graph_k = k;
    return NS_OK;
}

// Relative-binning tables for the current data (edges, fiducial coefficients,
// summary data); allocates on first use.
int build_rb(ns_ctx *c) {
    const int B = c->rb_B, nd = c->M.n_det;
    const size_t ne = (size_t)B + 1, nb = B;
    int rc;
    if (!c->rb_J) {
        if ((rc = dalloc(&c->rb_J, ne)) || (rc = dalloc(&c->rb_nedge, 1)) || (rc = dalloc(&c->rb_fid, 1)) ||
            (rc = dalloc(&c->rb_fe, ne)) || (rc = dalloc(&c->rb_basis64, NB * ne)) ||
            (rc = dalloc(&c->rb_basis32, NB * ne)) || (rc = dalloc(&c->rb_fe32, ne)) ||
            (rc = dalloc(&c->rb_fm, nb)) || (rc = dalloc(&c->rb_inv_de, nb)) ||
            (rc = dalloc(&c->rb_A0, nd * nb)) || (rc = dalloc(&c->rb_A1, nd * nb)) ||
            (rc = dalloc(&c->rb_B0, nd * nb)) || (rc = dalloc(&c->rb_B1, nd * nb)) ||
            (rc = dalloc(&c->rb_A0f, nd * nb)) || (rc = dalloc(&c->rb_A1f, nd * nb)) ||
            (rc = dalloc(&c->rb_B0f, nd * nb)) || (rc = dalloc(&c->rb_B1f, nd * nb)) ||
            (rc = dalloc(&c->rb_inv_de_f, nb)))
            return rc;
    }
    double2 *h0 = nullptr;
    double *th = nullptr;
    if ((rc = dalloc(&h0, (size_t)nd * c->M.N)) || (rc = dalloc(&th, NS_NPARAM))) { dfree(h0); return rc; }
    Model M0 = c->M;
    M0.rb = 0;
    RBTables R;
    std::memset(&R, 0, sizeof(R));
    cudaError_t e = cudaMemcpyAsync(th, c->rb_theta, sizeof(double) * NS_NPARAM, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = launch_rb_setup(M0, c->T, B, th, c->rb_J, c->rb_nedge, c->rb_fid, h0, c->d_re, c->d_im, c->d_psd, R,
                            c->rb_fe, c->rb_basis64, c->rb_basis32, c->rb_fe32, c->rb_fm, c->rb_inv_de, c->rb_A0,
                            c->rb_A1, c->rb_B0, c->rb_B1, c->rb_A0f, c->rb_A1f, c->rb_B0f, c->rb_B1f,
                            c->rb_inv_de_f, c->stream);
    int nedge = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&nedge, c->rb_nedge, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dfree(h0);
    dfree(th);
    if (e != cudaSuccess) return cuda_fail(e);
    RBTables &T = c->T.rb;
    T.nedge = nedge;
    T.nb = nedge - 1;
    T.fe = c->rb_fe; T.basis64 = c->rb_basis64; T.basis32 = c->rb_basis32; T.fe32 = c->rb_fe32;
    T.fm = c->rb_fm; T.inv_de = c->rb_inv_de; T.A0 = c->rb_A0; T.A1 = c->rb_A1; T.B0 = c->rb_B0;
    T.B1 = c->rb_B1; T.A0f = c->rb_A0f; T.A1f = c->rb_A1f; T.B0f = c->rb_B0f; T.B1f = c->rb_B1f;
    T.inv_de_f = c->rb_inv_de_f; T.fid = c->rb_fid;
    c->M.rb = 1;
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; c->graph_k = -1; }
    return NS_OK;
}

int eval_points(ns_ctx *c, const double *in, int is_theta, int m, double *logl) {
    CK(launch_eval(c->M, c->T, c->precision, choose_warps(c), in, is_theta, m, logl, c->state, c->stream));
    return NS_OK;
}

}  // namespace

namespace gwns_host {
// slot counts chosen by ns_autotune, keyed by (bins, detectors, precision, n, k)
using TuneKey = std::tuple<int, int, int, int, int>;
static std::mutex g_tune_mu;
static std::map<TuneKey, int> g_tuned;

TuneKey tune_key(const ns_ctx *c) {
    return TuneKey(c->M.rb ? -c->T.rb.nb : c->M.N, c->M.n_det, c->precision, c->n, c->k_default);
}

int choose_slots(const ns_ctx *c) {
    if (c->slots > 0) return c->slots;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tuned.find(tune_key(c));
        if (it != g_tuned.end()) return it->second;
    }
    if (c->M.model == M_TOY) return 1;
    const int bins = c->M.rb ? c->T.rb.nb : c->M.N;
    // measured on GB300 (512 / 4017 / 64,897-bin workloads): FP64 binds on its
    // pipe beyond small grids (one slot plus tail speculation from 64,897 bins),
    // the mixed form on latency up to large grids
    if (c->precision == NS_FP64) return bins <= 1024 ? 4 : (bins <= 16384 ? 2 : 1);
    return bins <= 1024 ? 8 : (c->M.coop ? 2 : 4);
}

// Warps per chain CTA: twice the base depth (at most 8; 4 for the cooperative
// mixed loop), so that the last chains of an update can plan deeper.
int slots_alloc(const ns_ctx *c) {
    // tail speculation doubles the slots of a chain up to 4; wider slot
    // templates cost more registers than the deeper lookahead saves (GB300:
    // 4 -> 8 slots lost 14% FP64 and 35% mixed on the 4017-bin workload)
    const int base = choose_slots(c);
    const int s = 2 * base;
    return base >= 4 ? base : (s < 4 ? s : 4);
}

StepArgs step_args(ns_ctx *c, int k) {
    StepArgs A;
    A.live_u = c->live_u;
    A.live_logl = c->live_logl;
    A.order = c->order;
    A.chol = c->chol;
    A.dead_u = c->dead_u;
    A.dead_logl = c->dead_logl;
    A.dead_logw = c->dead_logw;
    A.dead_nlive = c->dead_nlive;
    A.state = c->state;
    A.seed = c->seed;
    A.n = c->n;
    A.k = k;
    A.steps = c->steps;
    A.max_stepout = c->max_so;
    A.max_shrink = c->max_sh;
    A.dlogz_stop = c->dlogz;
    A.active = c->active;
    A.depth = choose_slots(c);
    A.tail = c->n_sm;
    // FP64 on fine grids: every candidate's bins on two warps, strided by 64, in
    // every round. A split chosen by the number of chains still running would make
    // the reduction order, and so the last bits of log L, depend on timing. GB300,
    // 64,897 / 519,169 bins: the split is 3% / 4% faster than deeper speculation
    // in the update's tail; on 4017 bins it gains nothing and the extra per-warp
    // start phasors would cost ~10%.
    A.fp64_split = (c->precision == NS_FP64 && c->M.model == M_GW && !c->M.rb && c->M.N >= 32768 &&
                    slots_alloc(c) >= 2) ? 2 : 1;
    A.kernel = c->kernel;
    A.walk_scale = c->walk_scale;
    // the work-shared update runs where the 8-warp cooperative kernel would
    const bool ws = c->ws && c->precision == NS_MIXED && !c->M.rb && slots_alloc(c) == 4;
    A.chain_ctr = ws ? c->chain_ctr : nullptr;
    A.ws = ws ? c->ws : nullptr;
    A.ws_part = ws ? c->ws_part : nullptr;
    A.ws_nslot = ws ? c->ws_nslot : 0;
    A.ws_gchunk = c->ws_gchunk;
    A.ws_maxchunk = c->ws_maxchunk;
    // test of the timeout path: the owner waits for one chunk more than its round has,
    // the bounded wait runs out and ns_step reports NS_ERR_TIMEOUT (no GPU fault or hang)
    A.ws_test_extra = ws ? c->ws_test_extra : 0;
    // the work-shared update sums the groups from T.g_lo at the low Taylor degree
    A.lo_bin = (ws && c->M.tlg && c->T.g_lo < 0x7fffffff) ? (long long)c->T.g_lo << (c->M.tlg + 5) : (1LL << 62);
    return A;
}

int ensure_dead_capacity(ns_ctx *c, long long need) {
    if (need <= c->dead_cap) return NS_OK;
    long long cap = std::max<long long>(need, std::max<long long>(2 * c->dead_cap, 64LL * c->n));
    double *u = nullptr, *l = nullptr, *w = nullptr, *nl = nullptr;
    int rc;
    if ((rc = dalloc(&u, (size_t)cap * c->d)) || (rc = dalloc(&l, cap)) || (rc = dalloc(&w, cap)) ||
        (rc = dalloc(&nl, cap))) {
        dfree(u); dfree(l); dfree(w); dfree(nl);
        return rc;
    }
    if (c->n_dead > 0) {
        CK(cudaMemcpyAsync(u, c->dead_u, sizeof(double) * c->n_dead * c->d, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(l, c->dead_logl, sizeof(double) * c->n_dead, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(w, c->dead_logw, sizeof(double) * c->n_dead, cudaMemcpyDeviceToDevice, c->stream));
        CK(cudaMemcpyAsync(nl, c->dead_nlive, sizeof(double) * c->n_dead, cudaMemcpyDeviceToDevice, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    dfree(c->dead_u); dfree(c->dead_logl); dfree(c->dead_logw); dfree(c->dead_nlive);
    c->dead_u = u; c->dead_logl = l; c->dead_logw = w; c->dead_nlive = nl;
    c->dead_cap = cap;
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; c->graph_k = -1; }
    return NS_OK;
}
}  // namespace gwns_host

extern "C" {

const char *ns_strerror(int code) {
    switch (code) {
        case NS_OK: return "ok";
        case NS_ERR_INVALID_ARG: return "invalid argument";
        case NS_ERR_PSD_NONPOS: return "PSD value not positive and finite";
        case NS_ERR_K_RANGE: return "k outside 1 .. n_live-1";
        case NS_ERR_OOM: return "device allocation failed";
        case NS_ERR_CAPACITY: return "output buffer too small";
        case NS_ERR_TIMEOUT: return "a bounded device-side wait gave up";
        case NS_ERR_CANCELLED: return "cancelled";
        case NS_ERR_CUDA: return "CUDA runtime error";
        case NS_ERR_STATE: return "call not valid in this state";
        default: return "unknown error";
    }
}

void ns_free(ns_ctx *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->graph) cudaGraphExecDestroy(c->graph);
    for (cudaEvent_t e : c->ev)
        if (e) cudaEventDestroy(e);
    void *bufs[] = {c->d_re, c->d_im, c->d_psd, c->basis64, c->f64, c->prefix, c->w64, c->X.basis32,
                    c->X.f32, c->X.w32, c->X.tb0, c->X.tb1, c->X.tbk, c->X.fc, c->X.wt, c->live_u, c->live_logl, c->order, c->chol, c->dead_u,
                    c->dead_logl, c->dead_logw, c->dead_nlive, c->state, c->scratch, c->fin_u,
                    c->fin_logl, c->fin_logw, c->fin_nlive, c->res, c->rb_J, c->rb_nedge, c->rb_fid,
                    c->rb_fe, c->rb_basis64, c->rb_basis32, c->rb_fe32, c->rb_fm, c->rb_inv_de, c->rb_A0,
                    c->rb_A1, c->rb_B0, c->rb_B1, c->rb_A0f, c->rb_A1f, c->rb_B0f, c->rb_B1f,
                    c->rb_inv_de_f, c->active, c->chain_ctr, c->ws, c->ws_part};
    for (void *p : bufs) dfree(p);
    if (c->h_state) cudaFreeHost(c->h_state);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

static int validate(const ns_prior *prior, const ns_data *data, const ns_psd *psd, const ns_grid *grid,
                    const ns_options *o) {
    if (!o) return NS_ERR_INVALID_ARG;
    if (o->n_live < 2 || o->n_live > 4096) return NS_ERR_INVALID_ARG;
    if (o->k != 0 && (o->k < 1 || o->k > o->n_live - 1)) return NS_ERR_K_RANGE;
    if (o->precision != NS_FP64 && o->precision != NS_MIXED) return NS_ERR_INVALID_ARG;
    if (o->steps_per_dim < 0 || o->max_stepout < 0 || o->max_shrink < 0) return NS_ERR_INVALID_ARG;
    if (o->warps_per_point != 0 && o->warps_per_point != 1 && o->warps_per_point != 2 &&
        o->warps_per_point != 4 && o->warps_per_point != 8)
        return NS_ERR_INVALID_ARG;
    if (o->slots != 0 && o->slots != 1 && o->slots != 2 && o->slots != 4 && o->slots != 8)
        return NS_ERR_INVALID_ARG;
    if (o->model == NS_MODEL_TOY) {
        if (o->toy_dim < 1 || o->toy_dim > NS_MAX_DIM) return NS_ERR_INVALID_ARG;
        return NS_OK;
    }
    if (o->model != NS_MODEL_GW) return NS_ERR_INVALID_ARG;
    if (!prior || !data || !psd || !grid || !psd->S) return NS_ERR_INVALID_ARG;
    if (grid->N < 1 || !is_fin(grid->f0) || !is_fin(grid->df) || grid->df <= 0.0 || grid->f0 <= 0.0)
        return NS_ERR_INVALID_ARG;
    if (data->n_det < 1 || data->n_det > NS_MAX_DET) return NS_ERR_INVALID_ARG;
    if (grid->coarse_bins < 0 || grid->coarse_bins > 65536 || (grid->coarse_bins > 0 && !grid->theta_fid))
        return NS_ERR_INVALID_ARG;
    if (grid->coarse_bins > 0 && grid->N < 2) return NS_ERR_INVALID_ARG;
    if ((data->re == nullptr) != (data->im == nullptr)) return NS_ERR_INVALID_ARG;
    if (!data->ideal && (!data->pos || !data->xarm || !data->yarm)) return NS_ERR_INVALID_ARG;
    int dim = 0;
    for (int p = 0; p < NS_NPARAM; p++) {
        int kd = prior->kind[p];
        if (kd != NS_PRIOR_FIXED && kd != NS_PRIOR_UNIFORM && kd != NS_PRIOR_VOLUME) return NS_ERR_INVALID_ARG;
        if (!is_fin(prior->lo[p])) return NS_ERR_INVALID_ARG;
        if (kd != NS_PRIOR_FIXED) {
            if (!is_fin(prior->hi[p]) || !(prior->hi[p] > prior->lo[p])) return NS_ERR_INVALID_ARG;
            dim++;
        }
    }
    if (dim < 1 || dim > NS_MAX_DIM) return NS_ERR_INVALID_ARG;
    // physical ranges the waveform needs
    double qlo = prior->lo[NS_Q], qhi = prior->kind[NS_Q] == NS_PRIOR_FIXED ? prior->lo[NS_Q] : prior->hi[NS_Q];
    if (!(qlo > 0.0) || qhi > 1.0) return NS_ERR_INVALID_ARG;
    if (!(prior->lo[NS_MC] > 0.0) || !(prior->lo[NS_DL] > 0.0)) return NS_ERR_INVALID_ARG;
    const size_t nn = (size_t)data->n_det * grid->N;
    for (size_t i = 0; i < nn; i++)
        if (!(psd->S[i] > 0.0) || !is_fin(psd->S[i])) return NS_ERR_PSD_NONPOS;
    return NS_OK;
}

// A double as a double-float: the nearest float, then the nearest float to the rest.
static gwns::dfl host_df(double x) {
    const float h = (float)x;
    return gwns::dfl{h, (float)(x - (double)h)};
}

// The mixed form takes its per-point coefficients in double-float on the FP32
// pipe (point_coef_group_mx) unless it uses relative binning, a parameter other
// than the distance has a uniform-in-volume prior (which needs a cube root), or
// the angles psi and RA range beyond +-100 rad (the double-float sine and cosine
// reduce arguments below 2^7 pi/2). GWNS_COEF_FP64=1 keeps the FP64 stage and its
// conversion instead (the two are compared by the GPU tests).
static bool use_df_coefficients(const ns_ctx *c) {
    const Model &M = c->M;
    if (M.model != M_GW || c->precision != NS_MIXED || M.rb) return false;
    for (int p = 0; p < NS_NPARAM; p++)
        if (M.kind[p] == K_VOLUME && p != NS_DL) return false;
    for (int p : {(int)NS_PSI, (int)NS_RA})
        if (std::fabs(M.lo[p]) > 100.0 || std::fabs(M.hi[p]) > 100.0) return false;
    const char *f = std::getenv("GWNS_COEF_FP64");
    return !(f && f[0] == '1');
}

// Mixed form: the tiled form when the Taylor remainder of the basis about each
// tile's centre stays below 1e-8 rad for every point of the prior, else the
// per-bin form. The bound: the basis terms of the phase sum to at most twice
// the Newtonian phase 3/128 (pi T_sun Mc f)^(-5/3) at the lowest chirp mass and
// frequency (leading-order and 1.5PN terms dominate at f0); the degree-TK
// remainder of f^(-5/3) over half a tile h is below 4.8 (h/f0)^(TK+1) times the
// term (TK = 7); a factor 64 covers both with margin. The longest tile that
// passes, up to 128 bins, is taken: it amortises the per-tile anchor best
// (GB300, 519,169 bins: degree 6 on 64-bin tiles against degree 7 on 128-bin
// tiles, batched likelihood 1.53 -> 1.59 M evals/s, slice update 326 -> 304 ms).
static void choose_tiles(Model &M) {
    M.tlg = 0;
    M.np = M.N;
    const double mc = M.lo[P_MC] > 0.0 ? M.lo[P_MC] : 1.0;
    const double phin = 3.0 / 128.0 * std::pow(M_PI * TSUN * mc * M.f0, -5.0 / 3.0);
    for (int lg = 7; lg >= 3; lg--) {
        const double h = 0.5 * (double)(1 << lg) * M.df;
        if (64.0 * phin * std::pow(h / M.f0, TK + 1) <= 1e-8) {
            M.tlg = lg;
            const int gb = 32 << lg;
            M.np = (M.N + gb - 1) / gb * gb;
            return;
        }
    }
}

// The same bound at a tile group's lowest frequency f_g, where the phase and
// the remainder ratio h / f_g are both smaller, with the degree TK_LO (whose
// remainder constant, 3.17, is below degree 7's 4.8): the first group from which
// it passes takes TK_LO, and so do all above it. 519,169 bins at 20 Hz in
// 128-bin tiles: from 263.5 Hz, 88% of the bins.
static int low_degree_group(const Model &M) {
    if (!M.tlg) return 0x7fffffff;
    const double mc = M.lo[P_MC] > 0.0 ? M.lo[P_MC] : 1.0;
    const double h = 0.5 * (double)(1 << M.tlg) * M.df;
    const int gb = 32 << M.tlg, ng = (int)(M.np / gb);
    for (int g = 0; g < ng; g++) {
        const double f = M.f0 + (double)g * gb * M.df;
        const double phin = 3.0 / 128.0 * std::pow(M_PI * TSUN * mc * f, -5.0 / 3.0);
        if (64.0 * phin * std::pow(h / f, TK_LO + 1) <= 1e-8) return g;
    }
    return ng;
}

static int alloc_mixed(ns_ctx *c) {
    const Model &M = c->M;
    const size_t N = M.N, nd = M.n_det;
    if (M.model != M_GW) return NS_OK;
    if (!M.tlg) {
        int rc;
        if ((rc = dalloc(&c->X.basis32, NB * N)) || (rc = dalloc(&c->X.f32, N)) || (rc = dalloc(&c->X.w32, nd * N)))
            return rc;
        return NS_OK;
    }
    const size_t np = M.np, nt = np >> M.tlg;
    int rc;
    if ((rc = dalloc(&c->X.tb0, NB * nt)) || (rc = dalloc(&c->X.tb1, NB * nt)) ||
        (rc = dalloc(&c->X.tbk, (size_t)(TK - 1) * NB * nt)) || (rc = dalloc(&c->X.fc, nt)) ||
        (rc = dalloc(&c->X.wt, nd * np)))
        return rc;
    return NS_OK;
}

int ns_init(ns_ctx **out, const ns_prior *prior, const ns_data *data, const ns_psd *psd,
            const ns_grid *grid, const ns_options *o) {
    if (!out) return NS_ERR_INVALID_ARG;
    *out = nullptr;
    int rc = validate(prior, data, psd, grid, o);
    if (rc) return rc;
    ns_ctx *c = new (std::nothrow) ns_ctx();
    if (!c) return NS_ERR_OOM;
    std::memset(&c->M, 0, sizeof(Model));
    std::memset(&c->T, 0, sizeof(Tables));
    cudaGetDevice(&c->device);
    if (cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) c->n_sm = 152;
    Model &M = c->M;
    c->n = o->n_live;
    c->k_default = o->k ? o->k : o->n_live / 2;
    c->precision = o->precision;
    c->max_so = o->max_stepout ? o->max_stepout : 64;
    c->max_sh = o->max_shrink ? o->max_shrink : 64;
    c->warps = o->warps_per_point;
    c->slots = o->slots;
    // zero takes the default; a negative tolerance is never met (the run goes
    // on to its iteration cap)
    c->dlogz = o->dlogz_stop != 0.0 ? o->dlogz_stop : 0.1;
    c->seed = o->seed;
    if (o->kernel != NS_KERNEL_SLICE && o->kernel != NS_KERNEL_WALK) { delete c; return NS_ERR_INVALID_ARG; }
    c->kernel = o->kernel;
    if (o->stream) {
        c->stream = (cudaStream_t)o->stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return NS_ERR_CUDA;
        }
        c->own_stream = true;
    }
    if (o->model == NS_MODEL_TOY) {
        M.model = M_TOY;
        M.dim = o->toy_dim;
        M.periodic = o->periodic;
        M.toy_lo = -10.0;
        M.toy_hi = 10.0;
        M.toy_rho = o->toy_dim > 1 ? 0.9 : 0.0;
        // -1/2 log det(2 pi Sigma), det Sigma = (1 - rho^2)^(d-1)
        M.toy_lognorm = -0.5 * (M.dim * std::log(2.0 * M_PI) + (M.dim - 1) * std::log(1.0 - M.toy_rho * M.toy_rho));
        M.N = 1;
        M.n_det = 1;
    } else {
        M.model = M_GW;
        M.n_det = data->n_det;
        M.N = grid->N;
        M.ideal = data->ideal;
        M.cutoff = o->no_cutoff ? 0 : 1;
        M.f0 = grid->f0;
        M.df = grid->df;
        int dim = 0;
        for (int p = 0; p < NS_NPARAM; p++) {
            M.kind[p] = prior->kind[p];
            M.lo[p] = prior->lo[p];
            M.hi[p] = prior->kind[p] == NS_PRIOR_FIXED ? prior->lo[p] : prior->hi[p];
            dim += prior->kind[p] != NS_PRIOR_FIXED;
        }
        M.dim = dim;
        M.inv_df = 1.0 / M.df;
        // periodic parameters -> unit-cube coordinates
        M.periodic = 0;
        for (int p = 0, i = 0; p < NS_NPARAM; p++) {
            if (M.kind[p] == K_FIXED) continue;
            if ((o->periodic >> p) & 1u) M.periodic |= 1u << i;
            i++;
        }
        for (int p = 0; p < NS_NPARAM; p++) {
            const double lo = M.lo[p], hi = M.hi[p];
            if (M.kind[p] == K_VOLUME) {
                M.pbase[p] = lo * lo * lo;
                M.pspan[p] = hi * hi * hi - lo * lo * lo;
            } else {
                M.pbase[p] = lo;
                M.pspan[p] = hi - lo;
            }
        }
        // double-float copies for the mixed form's coefficient stage
        for (int p = 0, i = 0; p < NS_NPARAM; p++) {
            M.uidx[p] = M.kind[p] == K_FIXED ? 0 : i++;
            M.pbase_x[p] = host_df(M.pbase[p]);
            M.pspan_x[p] = M.kind[p] == K_FIXED ? gwns::dfl{0.0f, 0.0f} : host_df(M.pspan[p]);
        }
        M.df_x = host_df(M.df);
        // large grids: the mixed slice update shares each bin's table loads among
        // the round's candidates (measured faster from ~16k bins on GB300)
        M.coop = M.N >= 16384 ? 1 : 0;
        choose_tiles(M);
        if (!data->ideal)
            for (int dd = 0; dd < M.n_det; dd++)
                for (int i = 0; i < 3; i++) {
                    M.pos[dd][i] = data->pos[dd * 3 + i];
                    M.xarm[dd][i] = data->xarm[dd * 3 + i];
                    M.yarm[dd][i] = data->yarm[dd * 3 + i];
                }
    }
    c->d = M.dim;
    c->steps = (o->steps_per_dim ? o->steps_per_dim : 5) * M.dim;
    c->walk_scale = o->walk_scale > 0.0 ? o->walk_scale : 2.38 / std::sqrt((double)M.dim);
    const size_t N = M.N, nd = M.n_det, nn = nd * N;
    if ((rc = dalloc(&c->d_re, nn)) || (rc = dalloc(&c->d_im, nn)) || (rc = dalloc(&c->d_psd, nn)) ||
        (rc = dalloc(&c->basis64, NB * N)) || (rc = dalloc(&c->f64, N)) || (rc = dalloc(&c->prefix, nn)) ||
        (rc = dalloc(&c->w64, nn)) || (rc = alloc_mixed(c)) || (rc = dalloc(&c->live_u, (size_t)c->n * c->d)) ||
        (rc = dalloc(&c->live_logl, c->n)) || (rc = dalloc(&c->order, c->n)) ||
        (rc = dalloc(&c->chol, (size_t)NS_MAX_DIM * NS_MAX_DIM)) || (rc = dalloc(&c->state, 1)) ||
        (rc = dalloc(&c->fin_u, (size_t)c->n * c->d)) || (rc = dalloc(&c->fin_logl, c->n)) ||
        (rc = dalloc(&c->fin_logw, c->n)) || (rc = dalloc(&c->fin_nlive, c->n)) ||
        (rc = dalloc(&c->res, kReplicates + 8)) || (rc = dalloc(&c->active, 1))) {
        ns_free(c);
        return rc;
    }
    if (M.model == M_GW && o->precision == NS_MIXED && M.coop && M.tlg >= 5 && M.N >= 262144 &&
        !(grid && grid->coarse_bins > 0)) {
        // work-shared slice update: one slot per CTA that fits on the GPU at once;
        // chunks of 8,192 bins (2 tile groups of 128-bin tiles; GB300, 519,169 bins:
        // 257 ms per update against 263 ms with chunks of 4 groups)
        const int per_sm = gwns::ws_blocks_per_sm(NS_MIXED, M.n_det);
        if (per_sm > 0) {
            c->ws_nslot = per_sm * c->n_sm;
            c->ws_gchunk = std::max(1, 8192 >> (M.tlg + 5));
            const int ngroups = (M.np + (32 << M.tlg) - 1) >> (M.tlg + 5);
            c->ws_maxchunk = (ngroups + c->ws_gchunk - 1) / c->ws_gchunk;
            if ((rc = dalloc(&c->chain_ctr, 1)) || (rc = dalloc(&c->ws, c->ws_nslot)) ||
                (rc = dalloc(&c->ws_part, (size_t)c->ws_nslot * c->ws_maxchunk * gwns::WS_PART_PER_CHUNK))) {
                ns_free(c);
                return rc;
            }
            if (cudaMemsetAsync(c->ws, 0, sizeof(gwns::WsSlot) * c->ws_nslot, c->stream) != cudaSuccess) {
                ns_free(c);
                return NS_ERR_CUDA;
            }
            const char *stall = std::getenv("GWNS_TEST_WS_STALL");
            c->ws_test_extra = (stall && stall[0] == '1') ? 1 : 0;
        }
    }
    if (cudaMallocHost((void **)&c->h_state, sizeof(RunState)) != cudaSuccess) { ns_free(c); return NS_ERR_OOM; }
    c->timing = true;
    for (cudaEvent_t &e : c->ev)
        if (cudaEventCreate(&e) != cudaSuccess) { e = nullptr; c->timing = false; }
    if ((rc = ensure_dead_capacity(c, 64LL * c->n))) { ns_free(c); return rc; }
    cudaError_t e = cudaSuccess;
    if (M.model == M_GW) {
        e = cudaMemcpyAsync(c->d_psd, psd->S, nn * sizeof(double), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess && data->re) {
            e = cudaMemcpyAsync(c->d_re, data->re, nn * sizeof(double), cudaMemcpyHostToDevice, c->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(c->d_im, data->im, nn * sizeof(double), cudaMemcpyHostToDevice, c->stream);
        } else if (e == cudaSuccess) {
            e = cudaMemsetAsync(c->d_re, 0, nn * sizeof(double), c->stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(c->d_im, 0, nn * sizeof(double), c->stream);
        }
        if (e == cudaSuccess)
            e = launch_build_tables(M, c->d_re, c->d_im, c->d_psd, c->basis64, c->f64, c->w64, c->prefix,
                                    c->X, c->stream);
    }
    if (e != cudaSuccess) { ns_free(c); return cuda_fail(e); }
    if (M.model == M_GW && grid->coarse_bins > 0) {
        c->rb_B = grid->coarse_bins;
        for (int p = 0; p < NS_NPARAM; p++) c->rb_theta[p] = grid->theta_fid[p];
    }
    c->T.basis64 = c->basis64;
    c->T.f64 = c->f64;
    c->T.w64 = c->w64;
    c->T.prefix = c->prefix;
    c->T.basis32 = c->X.basis32;
    c->T.f32 = c->X.f32;
    c->T.w32 = c->X.w32;
    c->T.tb0 = c->X.tb0;
    c->T.tb1 = c->X.tb1;
    c->T.tbk = c->X.tbk;
    c->T.fc = c->X.fc;
    c->T.wt = c->X.wt;
    c->T.g_lo = low_degree_group(c->M);
    if (c->rb_B > 0 && (rc = build_rb(c))) { ns_free(c); return rc; }
    c->M.cdf = use_df_coefficients(c) ? 1 : 0;
    RunState s0;
    std::memset(&s0, 0, sizeof(s0));
    s0.logZ = -INFINITY;
    s0.logX = 0.0;
    s0.lstar = -INFINITY;
    s0.evals = (unsigned long long)c->n;
    s0.walk_len = 2 * c->steps;     // random walk: first length twice the target of accepted moves
    s0.walk_acc = 0;
    *c->h_state = s0;
    e = cudaMemcpyAsync(c->state, c->h_state, sizeof(RunState), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_init_live(M, c->seed, c->n, c->live_u, c->stream);
    if (e != cudaSuccess) { ns_free(c); return cuda_fail(e); }
    if ((rc = eval_points(c, c->live_u, 0, c->n, c->live_logl))) { ns_free(c); return rc; }
    if ((e = cudaStreamSynchronize(c->stream)) != cudaSuccess) { ns_free(c); return cuda_fail(e); }
    *out = c;
    return NS_OK;
}

int ns_set_data(ns_ctx *c, const double *re, const double *im) {
    if (!c || !re || !im || c->M.model != M_GW) return NS_ERR_INVALID_ARG;
    const size_t nn = (size_t)c->M.n_det * c->M.N;
    CK(cudaMemcpyAsync(c->d_re, re, nn * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_im, im, nn * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    CK(launch_build_tables(c->M, c->d_re, c->d_im, c->d_psd, c->basis64, c->f64, c->w64, c->prefix, c->X,
                           c->stream));
    int rc;
    if (c->rb_B > 0 && (rc = build_rb(c))) return rc;
    rc = eval_points(c, c->live_u, 0, c->n, c->live_logl);
    if (rc) return rc;
    CK(cudaStreamSynchronize(c->stream));
    return NS_OK;
}

static int step_impl(ns_ctx *c, int k, int *done) {
    if (!c) return NS_ERR_INVALID_ARG;
    if (k < 1 || k > c->n - 1) return NS_ERR_K_RANGE;
    int rc = ensure_dead_capacity(c, c->n_dead + k);
    if (rc) return rc;
    if ((rc = capture_iteration(c, k))) return rc;
    CK(cudaGraphLaunch(c->graph, c->stream));
    c->n_dead += k;
    CK(cudaMemcpyAsync(c->h_state, c->state, sizeof(RunState), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (c->timing) {
        for (int i = 0; i < 5; i++) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, c->ev[i], c->ev[i + 1]) == cudaSuccess) c->kernel_ms[i] += ms;
            else { cudaGetLastError(); c->timing = false; }
        }
    }
    if (done) *done = c->h_state->done;
    // status bit 1: a bounded wait of the work-shared slice update gave up
    if (c->h_state->status & 2) return NS_ERR_TIMEOUT;
    return NS_OK;
}

int ns_step(ns_ctx *c, int k, int *done) { return step_impl(c, k, done); }

int ns_step_host(ns_ctx *c, int k, int *done, double *dead_u, double *dead_logl, double *dead_logw) {
    int rc = step_impl(c, k, done);
    if (rc) return rc;
    const long long o = c->n_dead - k;
    if (dead_u) CK(cudaMemcpyAsync(dead_u, c->dead_u + o * c->d, sizeof(double) * k * c->d, cudaMemcpyDeviceToHost, c->stream));
    if (dead_logl) CK(cudaMemcpyAsync(dead_logl, c->dead_logl + o, sizeof(double) * k, cudaMemcpyDeviceToHost, c->stream));
    if (dead_logw) CK(cudaMemcpyAsync(dead_logw, c->dead_logw + o, sizeof(double) * k, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return NS_OK;
}

int ns_run(ns_ctx *c, int max_iter, int *iterations) {
    if (!c || max_iter < 0) return NS_ERR_INVALID_ARG;
    int it = 0, done = 0;
    while (it < max_iter && !done) {
        int rc = ns_step(c, c->k_default, &done);
        if (rc) return rc;
        it++;
    }
    if (iterations) *iterations = it;
    return NS_OK;
}

int ns_get_stats(ns_ctx *c, ns_stats *st) {
    if (!c || !st) return NS_ERR_INVALID_ARG;
    CK(cudaMemcpyAsync(c->h_state, c->state, sizeof(RunState), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const RunState &s = *c->h_state;
    st->iterations = s.iter;
    st->evals = (long long)s.evals;
    st->cap_hits = (long long)s.caps;
    st->logZ = s.logZ;
    st->logX = s.logX;
    st->lstar = s.lstar;
    st->logl_max = s.logl_max;
    st->done = s.done;
    st->d = c->d;
    st->n_live = c->n;
    st->n_dead = (int)c->n_dead;
    st->point_bins = (long long)s.point_bins;
    st->status = s.status;
    for (int i = 0; i < 5; i++) st->kernel_ms[i] = c->timing ? c->kernel_ms[i] : -1.0;
    st->mixed_tile = c->M.tlg ? 1 << c->M.tlg : 0;
    st->batch_evals = (long long)s.eval_points;
    st->batch_point_bins = (long long)s.eval_point_bins;
    st->point_bins_lo = (long long)s.point_bins_lo;
    st->batch_point_bins_lo = (long long)s.eval_point_bins_lo;
    st->scratch_bytes = (long long)c->scratch_bytes;
    return NS_OK;
}

int ns_result_info(ns_ctx *c, double *H, double *ess) {
    if (!c || !c->have_info) return NS_ERR_INVALID_ARG;
    if (H) *H = c->info_H;
    if (ess) *ess = c->info_ess;
    return NS_OK;
}

int ns_result(ns_ctx *c, double *logZ, double *dlogZ, ns_samples *smp) {
    if (!c) return NS_ERR_INVALID_ARG;
    const long long total = c->n_dead + c->n;
    if (smp && smp->cap < total) { smp->count = (int)total; return NS_ERR_CAPACITY; }
    StepArgs A = step_args(c, c->k_default);
    CK(launch_select(c->live_logl, c->n, c->order, c->stream));
    double *logz_total = c->res + kReplicates;
    CK(launch_final_live(c->M, A, c->fin_u, c->fin_logl, c->fin_logw, c->fin_nlive, logz_total, c->stream));
    double lz = 0.0;
    CK(cudaMemcpyAsync(&lz, logz_total, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    ResultArgs R;
    R.dead_logl = c->dead_logl; R.dead_logw = c->dead_logw; R.dead_nlive = c->dead_nlive;
    R.fin_logl = c->fin_logl; R.fin_logw = c->fin_logw; R.fin_nlive = c->fin_nlive;
    R.n_dead = c->n_dead; R.n = c->n; R.logZ = lz; R.reps = c->res; R.out = c->res + kReplicates + 1;
    R.seed = c->seed; R.R = kReplicates;
    CK(launch_result_stats(R, c->stream));
    double out4[4];
    CK(cudaMemcpyAsync(out4, R.out, sizeof(out4), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (logZ) *logZ = lz;
    if (dlogZ) *dlogZ = out4[0];
    c->info_H = out4[1];
    c->info_ess = out4[2];
    c->have_info = true;
    if (smp) {
        const long long nd = c->n_dead;
        const int d = c->d;
        if (smp->u) {
            CK(cudaMemcpyAsync(smp->u, c->dead_u, sizeof(double) * nd * d, cudaMemcpyDeviceToHost, c->stream));
            CK(cudaMemcpyAsync(smp->u + nd * d, c->fin_u, sizeof(double) * c->n * d, cudaMemcpyDeviceToHost, c->stream));
        }
        if (smp->logl) {
            CK(cudaMemcpyAsync(smp->logl, c->dead_logl, sizeof(double) * nd, cudaMemcpyDeviceToHost, c->stream));
            CK(cudaMemcpyAsync(smp->logl + nd, c->fin_logl, sizeof(double) * c->n, cudaMemcpyDeviceToHost, c->stream));
        }
        if (smp->logw) {
            CK(cudaMemcpyAsync(smp->logw, c->dead_logw, sizeof(double) * nd, cudaMemcpyDeviceToHost, c->stream));
            CK(cudaMemcpyAsync(smp->logw + nd, c->fin_logw, sizeof(double) * c->n, cudaMemcpyDeviceToHost, c->stream));
        }
        if (smp->theta && c->M.model == M_GW) {
            int rc = ensure_scratch(c, sizeof(double) * (size_t)total * (NS_NPARAM + d));
            if (rc) return rc;
            double *u_all = c->scratch, *th = c->scratch + (size_t)total * d;
            CK(cudaMemcpyAsync(u_all, c->dead_u, sizeof(double) * nd * d, cudaMemcpyDeviceToDevice, c->stream));
            CK(cudaMemcpyAsync(u_all + nd * d, c->fin_u, sizeof(double) * c->n * d, cudaMemcpyDeviceToDevice, c->stream));
            CK(launch_theta(c->M, u_all, total, th, c->stream));
            CK(cudaMemcpyAsync(smp->theta, th, sizeof(double) * total * NS_NPARAM, cudaMemcpyDeviceToHost, c->stream));
        }
        CK(cudaStreamSynchronize(c->stream));
        smp->count = (int)total;
    }
    return NS_OK;
}

int ns_eval_lnl(ns_ctx *c, const double *u, int m, double *logl) {
    if (!c || m < 0 || (m > 0 && (!u || !logl))) return NS_ERR_INVALID_ARG;
    return eval_points(c, u, 0, m, logl);
}

int ns_eval_lnl_theta(ns_ctx *c, const double *theta, int m, double *logl) {
    if (!c || m < 0 || (m > 0 && (!theta || !logl)) || c->M.model != M_GW) return NS_ERR_INVALID_ARG;
    return eval_points(c, theta, 1, m, logl);
}

int ns_eval_lnl_host(ns_ctx *c, const double *u, int m, double *logl) {
    if (!c || m < 0 || (m > 0 && (!u || !logl))) return NS_ERR_INVALID_ARG;
    if (m == 0) return NS_OK;
    int rc = ensure_scratch(c, sizeof(double) * (size_t)m * (c->d + 1));
    if (rc) return rc;
    double *du = c->scratch, *dl = c->scratch + (size_t)m * c->d;
    CK(cudaMemcpyAsync(du, u, sizeof(double) * m * c->d, cudaMemcpyHostToDevice, c->stream));
    if ((rc = eval_points(c, du, 0, m, dl))) return rc;
    CK(cudaMemcpyAsync(logl, dl, sizeof(double) * m, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return NS_OK;
}

int ns_eval_lnl_host_noalloc(ns_ctx *c, const double *u, int m, double *logl) {
    if (!c || m < 0 || (m > 0 && (!u || !logl))) return NS_ERR_INVALID_ARG;
    if (m > NS_NOALLOC_MAX_POINTS) return NS_ERR_CAPACITY;
    if (m == 0) return NS_OK;
    int prev = 0;
    CK(cudaGetDevice(&prev));
    if (prev != c->device) CK(cudaSetDevice(c->device));
    double *base = nullptr;
    cudaError_t e = noalloc_scratch_address(&base);
    int rc = NS_OK;
    if (e != cudaSuccess) {
        rc = cuda_fail(e);
    } else {
        double *du = base, *dl = base + (size_t)m * c->d;
        e = cudaMemcpyAsync(du, u, sizeof(double) * m * c->d, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) rc = eval_points(c, du, 0, m, dl);
        if (e == cudaSuccess && rc == NS_OK)
            e = cudaMemcpyAsync(logl, dl, sizeof(double) * m, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess && rc == NS_OK) e = cudaStreamSynchronize(c->stream);
        if (rc == NS_OK && e != cudaSuccess) rc = cuda_fail(e);
    }
    if (prev != c->device) cudaSetDevice(prev);
    return rc;
}

int ns_waveform(ns_ctx *c, const double *theta, double *h_re, double *h_im) {
    if (!c || !theta || !h_re || !h_im || c->M.model != M_GW) return NS_ERR_INVALID_ARG;
    const size_t nn = (size_t)c->M.n_det * c->M.N;
    const size_t need = sizeof(double) * (NS_NPARAM + 2 * nn) + sizeof(Coef) + 64;
    int rc = ensure_scratch(c, need);
    if (rc) return rc;
    double *th = c->scratch, *hr = th + NS_NPARAM, *hi = hr + nn;
    Coef *cf = (Coef *)(((uintptr_t)(hi + nn) + 15) & ~(uintptr_t)15);
    CK(cudaMemcpyAsync(th, theta, sizeof(double) * NS_NPARAM, cudaMemcpyHostToDevice, c->stream));
    CK(launch_waveform(c->M, c->T, th, cf, hr, hi, c->stream));
    CK(cudaMemcpyAsync(h_re, hr, sizeof(double) * nn, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(h_im, hi, sizeof(double) * nn, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return NS_OK;
}

int ns_prior_transform(ns_ctx *c, const double *u, int m, double *theta) {
    if (!c || m < 0 || (m > 0 && (!u || !theta)) || c->M.model != M_GW) return NS_ERR_INVALID_ARG;
    if (m == 0) return NS_OK;
    int rc = ensure_scratch(c, sizeof(double) * (size_t)m * (c->d + NS_NPARAM));
    if (rc) return rc;
    double *du = c->scratch, *dt = c->scratch + (size_t)m * c->d;
    CK(cudaMemcpyAsync(du, u, sizeof(double) * m * c->d, cudaMemcpyHostToDevice, c->stream));
    CK(launch_theta(c->M, du, m, dt, c->stream));
    CK(cudaMemcpyAsync(theta, dt, sizeof(double) * m * NS_NPARAM, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return NS_OK;
}

int ns_optimal_snr2(ns_ctx *c, const double *theta, double *rho2) {
    if (!c || !theta || !rho2 || c->M.model != M_GW) return NS_ERR_INVALID_ARG;
    int rc = ensure_scratch(c, sizeof(double) * NS_NPARAM + sizeof(Coef) + 64);
    if (rc) return rc;
    double *th = c->scratch;
    Coef *cf = (Coef *)(((uintptr_t)(th + NS_NPARAM) + 15) & ~(uintptr_t)15);
    CK(cudaMemcpyAsync(th, theta, sizeof(double) * NS_NPARAM, cudaMemcpyHostToDevice, c->stream));
    CK(launch_point_coef(c->M, c->T, th, cf, c->stream));
    CK(cudaMemcpyAsync(rho2, &cf->hh, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return NS_OK;
}

int ns_get_live(ns_ctx *c, double *u, double *logl) {
    if (!c) return NS_ERR_INVALID_ARG;
    if (u) CK(cudaMemcpyAsync(u, c->live_u, sizeof(double) * c->n * c->d, cudaMemcpyDeviceToHost, c->stream));
    if (logl) CK(cudaMemcpyAsync(logl, c->live_logl, sizeof(double) * c->n, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return NS_OK;
}

int ns_set_live(ns_ctx *c, const double *u, const double *logl) {
    if (!c || !u || !logl) return NS_ERR_INVALID_ARG;
    CK(cudaMemcpyAsync(c->live_u, u, sizeof(double) * c->n * c->d, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->live_logl, logl, sizeof(double) * c->n, cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return NS_OK;
}

int ns_autotune(ns_ctx *c, int trials, int *slots) {
    if (!c || trials < 1) return NS_ERR_INVALID_ARG;
    const int k = c->k_default;
    int rc = ensure_dead_capacity(c, c->n_dead + (long long)trials * k);
    if (rc) return rc;
    // snapshot: live set and run state (the dead list is only appended)
    const size_t nu = (size_t)c->n * c->d;
    double *su = nullptr, *sl = nullptr;
    RunState *ss = nullptr;
    if ((rc = dalloc(&su, nu)) || (rc = dalloc(&sl, c->n)) || (rc = dalloc(&ss, 1))) {
        dfree(su); dfree(sl); dfree(ss);
        return rc;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const int saved_slots = c->slots;
    const bool saved_timing = c->timing;
    const int cand[4] = {1, 2, 4, 8};
    float best_ms = 3.4e38f;
    int best = choose_slots(c);
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(su, c->live_u, sizeof(double) * nu, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sl, c->live_logl, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ss, c->state, sizeof(RunState), cudaMemcpyDeviceToDevice, c->stream);
    c->timing = false;
    for (int i = 0; i < 4 && e == cudaSuccess && rc == NS_OK; i++) {
        c->slots = cand[i];
        e = cudaEventRecord(e0, c->stream);
        for (int t = 0; t < trials && e == cudaSuccess && rc == NS_OK; t++) rc = enqueue_iteration(c, k);
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess && rc == NS_OK) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && rc == NS_OK && ms < best_ms) { best_ms = ms; best = cand[i]; }
        // restore the snapshot
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->live_u, su, sizeof(double) * nu, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->live_logl, sl, sizeof(double) * c->n, cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c->state, ss, sizeof(RunState), cudaMemcpyDeviceToDevice, c->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    c->timing = saved_timing;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dfree(su); dfree(sl); dfree(ss);
    if (rc) { c->slots = saved_slots; return rc; }
    if (e != cudaSuccess) { c->slots = saved_slots; return cuda_fail(e); }
    c->slots = best;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tuned[tune_key(c)] = best;
    }
    if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; c->graph_k = -1; }
    if (slots) *slots = best;
    return NS_OK;
}

int ns_autotune_eval(ns_ctx *c, int trials, int *warps) {
    if (!c || trials < 1) return NS_ERR_INVALID_ARG;
    const int m = c->n;
    int rc = ensure_scratch(c, sizeof(double) * (size_t)m);
    if (rc) return rc;
    double *out = c->scratch;
    const int cand[4] = {1, 2, 4, 8};
    float best_ms = 3.4e38f;
    int best = choose_warps(c);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int i = 0; i < 4 && e == cudaSuccess; i++) {
        e = launch_eval(c->M, c->T, c->precision, cand[i], c->live_u, 0, m, out, nullptr, c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
        for (int t = 0; t < trials && e == cudaSuccess; t++)
            e = launch_eval(c->M, c->T, c->precision, cand[i], c->live_u, 0, m, out, nullptr, c->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < best_ms) { best_ms = ms; best = cand[i]; }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e);
    c->warps = best;
    if (warps) *warps = best;
    return NS_OK;
}

namespace {
struct CkptHeader {
    char magic[8];          // "GWNSCKP2"
    int n, d;
    long long n_dead;
    RunState state;
};
}  // namespace

int ns_checkpoint(ns_ctx *c, void *buf, size_t *len) {
    if (!c || !len) return NS_ERR_INVALID_ARG;
    const size_t nl = (size_t)c->n, d = c->d, nd = (size_t)c->n_dead;
    const size_t need = sizeof(CkptHeader) + sizeof(double) * (nl * (d + 1) + nd * (d + 3));
    if (!buf) { *len = need; return NS_OK; }
    if (*len < need) { *len = need; return NS_ERR_CAPACITY; }
    CkptHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, "GWNSCKP2", 8);
    h.n = c->n;
    h.d = c->d;
    h.n_dead = c->n_dead;
    CK(cudaMemcpyAsync(&h.state, c->state, sizeof(RunState), cudaMemcpyDeviceToHost, c->stream));
    double *p = (double *)((char *)buf + sizeof(CkptHeader));
    CK(cudaMemcpyAsync(p, c->live_u, sizeof(double) * nl * d, cudaMemcpyDeviceToHost, c->stream));
    p += nl * d;
    CK(cudaMemcpyAsync(p, c->live_logl, sizeof(double) * nl, cudaMemcpyDeviceToHost, c->stream));
    p += nl;
    if (nd) {
        CK(cudaMemcpyAsync(p, c->dead_u, sizeof(double) * nd * d, cudaMemcpyDeviceToHost, c->stream));
        p += nd * d;
        CK(cudaMemcpyAsync(p, c->dead_logl, sizeof(double) * nd, cudaMemcpyDeviceToHost, c->stream));
        p += nd;
        CK(cudaMemcpyAsync(p, c->dead_logw, sizeof(double) * nd, cudaMemcpyDeviceToHost, c->stream));
        p += nd;
        CK(cudaMemcpyAsync(p, c->dead_nlive, sizeof(double) * nd, cudaMemcpyDeviceToHost, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    std::memcpy(buf, &h, sizeof(h));
    *len = need;
    return NS_OK;
}

int ns_restore(ns_ctx *c, const void *buf, size_t len) {
    if (!c || !buf || len < sizeof(CkptHeader)) return NS_ERR_INVALID_ARG;
    CkptHeader h;
    std::memcpy(&h, buf, sizeof(h));
    if (std::memcmp(h.magic, "GWNSCKP2", 8) != 0 || h.n != c->n || h.d != c->d || h.n_dead < 0)
        return NS_ERR_INVALID_ARG;
    const size_t nl = (size_t)c->n, d = c->d, nd = (size_t)h.n_dead;
    if (len < sizeof(CkptHeader) + sizeof(double) * (nl * (d + 1) + nd * (d + 3))) return NS_ERR_INVALID_ARG;
    int rc = ensure_dead_capacity(c, (long long)nd + c->k_default);
    if (rc) return rc;
    const double *p = (const double *)((const char *)buf + sizeof(CkptHeader));
    CK(cudaMemcpyAsync(c->live_u, p, sizeof(double) * nl * d, cudaMemcpyHostToDevice, c->stream));
    p += nl * d;
    CK(cudaMemcpyAsync(c->live_logl, p, sizeof(double) * nl, cudaMemcpyHostToDevice, c->stream));
    p += nl;
    if (nd) {
        CK(cudaMemcpyAsync(c->dead_u, p, sizeof(double) * nd * d, cudaMemcpyHostToDevice, c->stream));
        p += nd * d;
        CK(cudaMemcpyAsync(c->dead_logl, p, sizeof(double) * nd, cudaMemcpyHostToDevice, c->stream));
        p += nd;
        CK(cudaMemcpyAsync(c->dead_logw, p, sizeof(double) * nd, cudaMemcpyHostToDevice, c->stream));
        p += nd;
        CK(cudaMemcpyAsync(c->dead_nlive, p, sizeof(double) * nd, cudaMemcpyHostToDevice, c->stream));
    }
    *c->h_state = h.state;
    CK(cudaMemcpyAsync(c->state, c->h_state, sizeof(RunState), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->n_dead = h.n_dead;
    return NS_OK;
}

int ns_sync(ns_ctx *c) {
    if (!c) return NS_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(c->stream));
    return NS_OK;
}

}  // extern "C"
