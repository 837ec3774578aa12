// gwns_serve.cu -- continuous-batching server of many nested-sampling analyses
// on one GPU (ns_server_* in include/gwns.h).
//
// Each admitted analysis is an ordinary context (its own tables, live set,
// dead list and run state on the device). An iteration of a set of analyses
// takes one launch per iteration kernel: the per-analysis kernels (sort,
// evidence, covariance, stopping test) take one block per analysis, and the
// slice update takes one block per (analysis, chain) of all of them, grouped by
// detector count. Descriptors (model, tables, iteration arguments) live in a
// device array.
//
// Two lanes: analyses on grids of more than SHORT_LANE_BINS bins run on the
// server's stream, those on smaller grids on a second, higher-priority stream.
// A tick launches one iteration of the long lane and, while it runs, iterates
// the short lane again and again (each time after the previous one finished),
// so that a short analysis does not wait every iteration for the slowest long
// one. Each analysis' arithmetic is its own, so its result does not depend on
// the lanes.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <utility>
#include <new>
#include <unordered_map>
#include <vector>

#include "gwns_ctx.h"

using namespace gwns_host;

namespace {

struct Request {
    uint64_t id = 0;
    ns_prior prior;
    ns_options opts;
    int N = 0, n_det = 0, ideal = 0, coarse_bins = 0;
    double f0 = 0, df = 0;
    bool has_data = false;
    std::vector<double> re, im, pos, xarm, yarm, psd, theta_fid;
    ns_request_status st;
    ns_ctx *ctx = nullptr;
    int d = 0;
    std::vector<double> s_u, s_logl, s_logw, s_theta;
};

int sampled_dim(const Request &r) {
    int d = 0;
    for (int p = 0; p < NS_NPARAM; p++) d += r.prior.kind[p] != NS_PRIOR_FIXED;
    return d;
}

// Device bytes of an analysis apart from its dead list: FP64 basis, f,
// weighted data, prefix, data and PSD copies; the mixed form's tiled
// increments, weighted data and tile anchors (grid padded by less than 1024
// bins); live and final sets; relative-binning tables; fixed overhead.
size_t footprint_base(const Request &r) {
    const size_t N = r.N, D = r.n_det, n = r.opts.n_live, d = sampled_dim(r);
    size_t b = (72 + 48 * D) * N + (37 + 8 * D) * (N + 1024);
    b += n * (16 * d + 40);
    if (r.coarse_bins > 0) b += (size_t)(r.coarse_bins + 1) * (160 + 64 * D) + 16 * D * N;
    return b + (1u << 20);
}

// Dead-list bytes at a capacity of cap entries (u, log L, log w, n_live).
size_t dead_bytes(const Request &r, long long cap) { return (size_t)cap * (size_t)(sampled_dim(r) + 3) * 8; }

// Estimated device bytes at admission: the dead list starts at 64 n entries
// and doubles when the run outgrows it; the server then adds the growth to the
// analysis' footprint and to the memory in use (see iterate_all).
size_t footprint(const Request &r) { return footprint_base(r) + dead_bytes(r, 64LL * r.opts.n_live); }

}  // namespace

// Grids of up to this many bins run on the short lane (the 4-, 8- and 16-s
// analyses of a 20-2048 Hz stream; 32- and 64-s ones on the long lane).
constexpr int SHORT_LANE_BINS = 32768;

struct Lane {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    Desc *d_desc = nullptr;
    int desc_cap = 0;
    int2 *d_map = nullptr;
    int map_cap = 0;
};

struct ns_server {
    ns_server_options o;
    cudaStream_t stream = nullptr;   // the long lane's (lane[0].stream)
    uint64_t next_id = 1;
    size_t budget = 0, used = 0;
    long long chains = 0;          // k of the running analyses
    std::deque<uint64_t> pending;
    std::vector<uint64_t> running;
    std::unordered_map<uint64_t, Request> reqs;
    Lane lane[2];                  // 0: long grids, 1: short grids
    std::chrono::steady_clock::time_point t0;
};

namespace {

double now(const ns_server *s) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

#define SCK(call)                                      \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return cuda_fail(e_);   \
    } while (0)

void release(ns_server *s, Request &r) {
    if (r.ctx) {
        ns_free(r.ctx);
        r.ctx = nullptr;
        s->used -= r.st.footprint;
        s->chains -= r.opts.k ? r.opts.k : r.opts.n_live / 2;
    }
}

int admit(ns_server *s, Request &r) {
    ns_data data;
    data.n_det = r.n_det;
    data.ideal = r.ideal;
    data.re = r.has_data ? r.re.data() : nullptr;
    data.im = r.has_data ? r.im.data() : nullptr;
    data.pos = r.pos.empty() ? nullptr : r.pos.data();
    data.xarm = r.xarm.empty() ? nullptr : r.xarm.data();
    data.yarm = r.yarm.empty() ? nullptr : r.yarm.data();
    ns_psd psd;
    psd.S = r.psd.data();
    ns_grid grid;
    grid.N = r.N;
    grid.f0 = r.f0;
    grid.df = r.df;
    grid.coarse_bins = r.coarse_bins;
    grid.theta_fid = r.theta_fid.empty() ? nullptr : r.theta_fid.data();
    ns_options o = r.opts;
    o.precision = s->o.precision;
    o.slots = s->o.slots;
    o.stream = (void *)s->lane[r.N <= SHORT_LANE_BINS ? 1 : 0].stream;
    ns_ctx *c = nullptr;
    int rc = ns_init(&c, &r.prior, &data, &psd, &grid, &o);
    if (rc) return rc;
    r.ctx = c;
    r.d = c->d;
    s->used += r.st.footprint;
    s->chains += r.opts.k ? r.opts.k : r.opts.n_live / 2;
    // the pending copies of the inputs are no longer needed
    std::vector<double>().swap(r.re);
    std::vector<double>().swap(r.im);
    return NS_OK;
}

int retire(ns_server *s, Request &r) {
    ns_ctx *c = r.ctx;
    ns_stats st;
    int rc = ns_get_stats(c, &st);
    if (rc) return rc;
    const long long total = (long long)c->n_dead + c->n;
    r.s_u.resize((size_t)total * c->d);
    r.s_logl.resize(total);
    r.s_logw.resize(total);
    if (c->M.model == gwns::M_GW) r.s_theta.resize((size_t)total * NS_NPARAM);
    ns_samples sm;
    sm.cap = (int)total;
    sm.count = 0;
    sm.u = r.s_u.data();
    sm.logl = r.s_logl.data();
    sm.logw = r.s_logw.data();
    sm.theta = r.s_theta.empty() ? nullptr : r.s_theta.data();
    double lz = 0, dlz = 0;
    if ((rc = ns_result(c, &lz, &dlz, &sm))) return rc;
    r.st.logZ = lz;
    r.st.dlogZ = dlz;
    r.st.iterations = st.iterations;
    r.st.evals = st.evals;
    r.st.n_samples = sm.count;
    r.st.state = NS_REQ_DONE;
    r.st.t_done = now(s);
    release(s, r);
    return NS_OK;
}

// One iteration of the analyses ids, interleaved, launched on lane L's stream
// (not waited for). Their run states are copied to the host at its end.
int iterate_lane(ns_server *s, int L, const std::vector<uint64_t> &ids) {
    const int na = (int)ids.size();
    if (na == 0) return NS_OK;
    Lane &ln = s->lane[L];
    std::vector<Desc> desc(na);
    // slice-update launches grouped by (detector count, warps per chain): every
    // analysis always runs at its own width, whatever the mix. Tiled mixed grids
    // take the direct form at every tile length (GB300, the 64-analysis stream:
    // p50 / p99 4.55 / 7.7 s; with the rotation form for tiles of 32 bins or more
    // in a kernel of its own, 5.8 / 9.2 s, and 6.3 / 10.0 s on a second stream)
    std::map<std::pair<int, int>, std::vector<int2>> groups;
    for (int a = 0; a < na; a++) {
        Request &r = s->reqs[ids[a]];
        ns_ctx *c = r.ctx;
        const int k = c->k_default;
        const long long cap0 = c->dead_cap;
        int rc = ensure_dead_capacity(c, c->n_dead + k);
        if (rc) return rc;
        if (c->dead_cap != cap0) {
            // the dead list doubled: count the new size (memory in use is the
            // running analyses' actual footprints, so admission stays within
            // the budget however long the runs grow)
            const size_t fp = footprint_base(r) + dead_bytes(r, c->dead_cap);
            if (fp > r.st.footprint) {
                s->used += fp - r.st.footprint;
                r.st.footprint = fp;
            }
        }
        desc[a].M = c->M;
        desc[a].T = c->T;
        desc[a].A = step_args(c, k);
        std::vector<int2> &g = groups[std::make_pair(c->M.n_det, slots_alloc(c))];
        for (int ch = 0; ch < k; ch++) g.push_back(make_int2(a, ch));
    }
    if (na > ln.desc_cap) {
        cudaFree(ln.d_desc);
        ln.d_desc = nullptr;
        SCK(cudaMalloc((void **)&ln.d_desc, sizeof(Desc) * (size_t)na * 2));
        ln.desc_cap = na * 2;
    }
    size_t nmap = 0;
    for (auto &kv : groups) nmap += kv.second.size();
    if ((int)nmap > ln.map_cap) {
        cudaFree(ln.d_map);
        ln.d_map = nullptr;
        SCK(cudaMalloc((void **)&ln.d_map, sizeof(int2) * nmap * 2));
        ln.map_cap = (int)nmap * 2;
    }
    // pageable host sources: each copy is staged before the call returns
    SCK(cudaMemcpyAsync(ln.d_desc, desc.data(), sizeof(Desc) * na, cudaMemcpyHostToDevice, ln.stream));
    SCK(gwns::launch_iteration_multi_head(ln.d_desc, na, ln.stream));
    size_t off = 0;
    for (auto &kv : groups) {
        const std::vector<int2> &g = kv.second;
        SCK(cudaMemcpyAsync(ln.d_map + off, g.data(), sizeof(int2) * g.size(), cudaMemcpyHostToDevice, ln.stream));
        SCK(gwns::launch_slice_multi(ln.d_desc, ln.d_map + off, (int)g.size(), s->o.precision, kv.first.first,
                                     kv.first.second, 0, ln.stream));
        off += g.size();
    }
    SCK(gwns::launch_iteration_multi_tail(ln.d_desc, na, ln.stream));
    for (int a = 0; a < na; a++) {
        ns_ctx *c = s->reqs[ids[a]].ctx;
        c->n_dead += c->k_default;
        SCK(cudaMemcpyAsync(c->h_state, c->state, sizeof(RunState), cudaMemcpyDeviceToHost, ln.stream));
    }
    return NS_OK;
}

bool finished(const ns_server *s, const Request &r) {
    const RunState &st = *r.ctx->h_state;
    return st.done || st.iter >= s->o.max_iter;
}

// One tick's iterations: the long lane once; the short lane once, then again
// while the long lane's iteration is still running.
int iterate_all(ns_server *s) {
    std::vector<uint64_t> ids[2];
    for (uint64_t id : s->running) ids[s->reqs[id].N <= SHORT_LANE_BINS ? 1 : 0].push_back(id);
    int rc = iterate_lane(s, 0, ids[0]);
    if (rc) return rc;
    cudaEvent_t ev = nullptr;
    if (!ids[0].empty() && !ids[1].empty()) {
        SCK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        if (cudaEventRecord(ev, s->lane[0].stream) != cudaSuccess) {
            cudaEventDestroy(ev);
            return NS_ERR_CUDA;
        }
    }
    std::vector<uint64_t> act = ids[1];
    while (!act.empty()) {
        if ((rc = iterate_lane(s, 1, act))) break;
        if (cudaStreamSynchronize(s->lane[1].stream) != cudaSuccess) { rc = NS_ERR_CUDA; break; }
        std::vector<uint64_t> next;
        for (uint64_t id : act)
            if (!finished(s, s->reqs[id])) next.push_back(id);
        act.swap(next);
        // another round only while the long lane is still busy
        if (!ev || cudaEventQuery(ev) != cudaErrorNotReady) break;
    }
    if (ev) cudaEventDestroy(ev);
    if (rc) return rc;
    SCK(cudaStreamSynchronize(s->lane[0].stream));
    return NS_OK;
}

}  // namespace

extern "C" {

int ns_server_create(ns_server **out, const ns_server_options *o) {
    if (!out || !o) return NS_ERR_INVALID_ARG;
    *out = nullptr;
    if (o->precision != NS_FP64 && o->precision != NS_MIXED) return NS_ERR_INVALID_ARG;
    if (o->max_active < 0 || o->max_iter < 0 || o->max_chains < 0) return NS_ERR_INVALID_ARG;
    if (o->slots != 0 && o->slots != 1 && o->slots != 2 && o->slots != 4 && o->slots != 8) return NS_ERR_INVALID_ARG;
    ns_server *s = new (std::nothrow) ns_server();
    if (!s) return NS_ERR_OOM;
    s->o = *o;
    if (s->o.max_active == 0) s->o.max_active = 16;
    if (s->o.slots == 0) s->o.slots = 4;
    if (s->o.max_iter == 0) s->o.max_iter = 100000;
    if (s->o.max_chains == 0) {
        int dev = 0, nsm = 152;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) nsm = 152;
        s->o.max_chains = 20 * nsm;
    }
    if (o->stream) {
        s->lane[0].stream = (cudaStream_t)o->stream;
    } else {
        if (cudaStreamCreateWithFlags(&s->lane[0].stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete s;
            return NS_ERR_CUDA;
        }
        s->lane[0].own_stream = true;
    }
    s->stream = s->lane[0].stream;
    // the short lane's stream: the device's highest priority, so that its blocks
    // are scheduled first as the long lane's blocks retire
    int lo_pri = 0, hi_pri = 0;
    if (cudaDeviceGetStreamPriorityRange(&lo_pri, &hi_pri) != cudaSuccess) hi_pri = 0;
    if (cudaStreamCreateWithPriority(&s->lane[1].stream, cudaStreamNonBlocking, hi_pri) != cudaSuccess) {
        ns_server_free(s);
        return NS_ERR_CUDA;
    }
    s->lane[1].own_stream = true;
    if (o->mem_budget) {
        s->budget = o->mem_budget;
    } else {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { ns_server_free(s); return NS_ERR_CUDA; }
        s->budget = (size_t)(0.8 * (double)fr);
    }
    s->t0 = std::chrono::steady_clock::now();
    *out = s;
    return NS_OK;
}

double ns_server_time(ns_server *s) { return s ? now(s) : 0.0; }

int ns_submit(ns_server *s, const ns_request *q, uint64_t *id) {
    if (!s || !q || !id) return NS_ERR_INVALID_ARG;
    const ns_options &o = q->opts;
    if (o.model != NS_MODEL_GW) return NS_ERR_INVALID_ARG;
    if (o.n_live < 2 || o.n_live > 4096) return NS_ERR_INVALID_ARG;
    if (o.k != 0 && (o.k < 1 || o.k > o.n_live - 1)) return NS_ERR_K_RANGE;
    const ns_data &dt = q->data;
    const ns_grid &g = q->grid;
    if (dt.n_det < 1 || dt.n_det > NS_MAX_DET || g.N < 1 || !q->psd.S) return NS_ERR_INVALID_ARG;
    if (!dt.ideal && (!dt.pos || !dt.xarm || !dt.yarm)) return NS_ERR_INVALID_ARG;
    if ((dt.re == nullptr) != (dt.im == nullptr)) return NS_ERR_INVALID_ARG;
    if (g.coarse_bins > 0 && !g.theta_fid) return NS_ERR_INVALID_ARG;
    const size_t nn = (size_t)dt.n_det * g.N;
    for (size_t i = 0; i < nn; i++)
        if (!(q->psd.S[i] > 0.0)) return NS_ERR_PSD_NONPOS;
    Request r;
    r.id = s->next_id++;
    r.prior = q->prior;
    r.opts = o;
    r.N = g.N;
    r.f0 = g.f0;
    r.df = g.df;
    r.coarse_bins = g.coarse_bins;
    r.n_det = dt.n_det;
    r.ideal = dt.ideal;
    r.psd.assign(q->psd.S, q->psd.S + nn);
    if (dt.re) {
        r.has_data = true;
        r.re.assign(dt.re, dt.re + nn);
        r.im.assign(dt.im, dt.im + nn);
    }
    if (!dt.ideal) {
        r.pos.assign(dt.pos, dt.pos + 3 * dt.n_det);
        r.xarm.assign(dt.xarm, dt.xarm + 3 * dt.n_det);
        r.yarm.assign(dt.yarm, dt.yarm + 3 * dt.n_det);
    }
    if (g.coarse_bins > 0) r.theta_fid.assign(g.theta_fid, g.theta_fid + NS_NPARAM);
    std::memset(&r.st, 0, sizeof(r.st));
    r.st.state = NS_REQ_PENDING;
    r.st.t_submit = now(s);
    r.st.footprint = footprint(r);
    *id = r.id;
    s->reqs.emplace(r.id, std::move(r));
    s->pending.push_back(*id);
    return NS_OK;
}

int ns_server_tick(ns_server *s, int *n_running, int *n_pending) {
    if (!s) return NS_ERR_INVALID_ARG;
    // admission in arrival order, by slot count and footprint
    while (!s->pending.empty() && (int)s->running.size() < s->o.max_active) {
        Request &r = s->reqs[s->pending.front()];
        if (r.st.footprint > s->budget) {      // can never fit
            r.st.state = NS_ERR_OOM;
            s->pending.pop_front();
            continue;
        }
        if (s->used + r.st.footprint > s->budget) break;
        const int kr = r.opts.k ? r.opts.k : r.opts.n_live / 2;
        if (!s->running.empty() && s->chains + kr > s->o.max_chains) break;
        int rc = admit(s, r);
        s->pending.pop_front();
        if (rc) { r.st.state = rc; continue; }
        r.st.state = NS_REQ_RUNNING;
        r.st.t_admit = now(s);
        s->running.push_back(r.id);
    }
    int rc = iterate_all(s);
    if (rc) return rc;
    // retire analyses that reached their stopping rule or the iteration cap
    std::vector<uint64_t> keep;
    for (uint64_t id : s->running) {
        Request &r = s->reqs[id];
        if (finished(s, r)) {
            if ((rc = retire(s, r))) return rc;
        } else {
            keep.push_back(id);
        }
    }
    s->running.swap(keep);
    if (n_running) *n_running = (int)s->running.size();
    if (n_pending) *n_pending = (int)s->pending.size();
    return NS_OK;
}

int ns_poll(ns_server *s, uint64_t id, ns_request_status *st) {
    if (!s || !st) return NS_ERR_INVALID_ARG;
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return NS_ERR_INVALID_ARG;
    *st = it->second.st;
    if (it->second.ctx) {
        const RunState &rs = *it->second.ctx->h_state;
        st->iterations = rs.iter;
        st->evals = (long long)rs.evals;
    }
    return NS_OK;
}

int ns_server_result(ns_server *s, uint64_t id, ns_samples *sm) {
    if (!s || !sm) return NS_ERR_INVALID_ARG;
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return NS_ERR_INVALID_ARG;
    Request &r = it->second;
    if (r.st.state != NS_REQ_DONE) return NS_ERR_STATE;
    const int n = r.st.n_samples;
    if (sm->cap < n) { sm->count = n; return NS_ERR_CAPACITY; }
    if (sm->u) std::memcpy(sm->u, r.s_u.data(), sizeof(double) * (size_t)n * r.d);
    if (sm->logl) std::memcpy(sm->logl, r.s_logl.data(), sizeof(double) * n);
    if (sm->logw) std::memcpy(sm->logw, r.s_logw.data(), sizeof(double) * n);
    if (sm->theta && !r.s_theta.empty()) std::memcpy(sm->theta, r.s_theta.data(), sizeof(double) * (size_t)n * NS_NPARAM);
    sm->count = n;
    return NS_OK;
}

int ns_cancel(ns_server *s, uint64_t id) {
    if (!s) return NS_ERR_INVALID_ARG;
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return NS_ERR_INVALID_ARG;
    Request &r = it->second;
    if (r.st.state == NS_REQ_PENDING) {
        s->pending.erase(std::remove(s->pending.begin(), s->pending.end(), id), s->pending.end());
    } else if (r.st.state == NS_REQ_RUNNING) {
        for (Lane &ln : s->lane)
            if (ln.stream) cudaStreamSynchronize(ln.stream);
        release(s, r);
        s->running.erase(std::remove(s->running.begin(), s->running.end(), id), s->running.end());
    } else {
        return NS_ERR_STATE;
    }
    r.st.state = NS_REQ_CANCELLED;
    r.st.t_done = now(s);
    return NS_OK;
}

void ns_server_free(ns_server *s) {
    if (!s) return;
    for (Lane &ln : s->lane)
        if (ln.stream) cudaStreamSynchronize(ln.stream);
    for (auto &kv : s->reqs) release(s, kv.second);
    for (Lane &ln : s->lane) {
        if (ln.d_desc) cudaFree(ln.d_desc);
        if (ln.d_map) cudaFree(ln.d_map);
        if (ln.own_stream && ln.stream) cudaStreamDestroy(ln.stream);
    }
    delete s;
}

}  // extern "C"
