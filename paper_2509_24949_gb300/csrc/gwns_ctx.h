// gwns_ctx.h -- the context of one analysis (device buffers, options, the
// iteration graph) and the host helpers shared by the C ABI (gwns_abi.cu) and
// the serving loop (gwns_serve.cu).
#pragma once
#include <cuda_runtime.h>

#include "../../include/gwns.h"
#include "gwns_kernels.cuh"

using gwns::Coef;
using gwns::Desc;
using gwns::MixedTables;
using gwns::Model;
using gwns::RBTables;
using gwns::RunState;
using gwns::StepArgs;
using gwns::Tables;

struct ns_ctx {
    Model M;
    Tables T;
    int n = 0, d = 0, k_default = 0, steps = 0, precision = 0, max_so = 64, max_sh = 64, warps = 0;
    int slots = 0;
    double dlogz = 0.1;
    uint64_t seed = 0;
    double info_H = 0.0, info_ess = 0.0;   // of the last ns_result
    bool have_info = false;
    int kernel = 0;            // NS_KERNEL_SLICE or NS_KERNEL_WALK
    double walk_scale = 0.0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int device = 0;
    // device buffers
    double *d_re = nullptr, *d_im = nullptr, *d_psd = nullptr;
    double *basis64 = nullptr, *f64 = nullptr, *prefix = nullptr;
    double2 *w64 = nullptr;
    MixedTables X = {};   // mixed-form tables (per-bin or tiled)
    double *live_u = nullptr, *live_logl = nullptr;
    int *order = nullptr;
    int *active = nullptr;           // running-chain counter of the slice update
    // work-shared slice update (mixed precision, grids of 262,144 bins or more)
    int *chain_ctr = nullptr;
    gwns::WsSlot *ws = nullptr;
    double *ws_part = nullptr;
    int ws_nslot = 0, ws_gchunk = 0, ws_maxchunk = 0;
    int ws_test_extra = 0;           // GWNS_TEST_WS_STALL set at ns_init: see step_args
    int n_sm = 152;
    double *chol = nullptr;
    double *dead_u = nullptr, *dead_logl = nullptr, *dead_logw = nullptr, *dead_nlive = nullptr;
    long long dead_cap = 0;
    RunState *state = nullptr;
    RunState *h_state = nullptr;     // pinned
    double *scratch = nullptr;       // eval / waveform scratch
    size_t scratch_bytes = 0;
    // relative-binning tables
    int rb_B = 0;
    double rb_theta[NS_NPARAM];
    int *rb_J = nullptr, *rb_nedge = nullptr;
    Coef *rb_fid = nullptr;
    double *rb_fe = nullptr, *rb_basis64 = nullptr, *rb_fm = nullptr, *rb_inv_de = nullptr;
    double *rb_B0 = nullptr, *rb_B1 = nullptr;
    double2 *rb_A0 = nullptr, *rb_A1 = nullptr;
    float2 *rb_basis32 = nullptr, *rb_fe32 = nullptr, *rb_A0f = nullptr, *rb_A1f = nullptr;
    float *rb_B0f = nullptr, *rb_B1f = nullptr, *rb_inv_de_f = nullptr;
    // result buffers
    double *fin_u = nullptr, *fin_logl = nullptr, *fin_logw = nullptr, *fin_nlive = nullptr;
    double *res = nullptr;           // [R + 8]
    // graph of one iteration, with timing events between its kernels
    cudaGraphExec_t graph = nullptr;
    int graph_k = -1;
    cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    bool timing = false;
    double kernel_ms[5] = {0, 0, 0, 0, 0};
    long long n_dead = 0;
};

namespace gwns_host {
int cuda_fail(cudaError_t e);
int choose_slots(const ns_ctx *c);
int slots_alloc(const ns_ctx *c);
StepArgs step_args(ns_ctx *c, int k);
int ensure_dead_capacity(ns_ctx *c, long long need);
}  // namespace gwns_host
