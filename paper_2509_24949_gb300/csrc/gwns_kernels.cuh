// gwns_kernels.cuh -- kernel launch interface between the C ABI (gwns_abi.cu)
// and the kernels (gwns_kernels.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "gwns_device.cuh"

namespace gwns {

// Run state kept on the device (read by the kernels of one iteration, so that
// an iteration can be replayed from a CUDA graph without host arguments).
struct RunState {
    double logZ;        // running log evidence of the dead points
    double logX;        // log prior volume inside the live set
    double lstar;       // current threshold
    double logl_max;    // largest live log L (after the last iteration)
    double remaining;   // log(Z + X Lmax) - log Z
    unsigned long long evals;
    unsigned long long caps;
    unsigned long long point_bins;   // sum over evaluations in k_slice of (jcut + 1)
    long long n_dead;
    long long iter;
    int done;
    int status;
    int walk_len;                    // random-walk kernel: proposals per walk this iteration
    int pad_;
    unsigned long long walk_acc;     // random-walk kernel: accepted moves of this iteration's walks
    unsigned long long eval_points;      // points through the batched likelihood (k_eval)
    unsigned long long eval_point_bins;  // their sum of (jcut + 1)
    unsigned long long point_bins_lo;       // of point_bins, those in tile groups at the Taylor degree TK_LO
    unsigned long long eval_point_bins_lo;  // of eval_point_bins, the same
};

// Work-shared slice update (mixed precision, fine tiled grids): one slot per
// persistent CTA. A round's tile groups are cut into fixed chunks of
// ws_gchunk groups; the owner publishes the round's candidates in its slot and
// any warp of the launch (its own, or of CTAs with no chain left) claims chunks
// through the claim word and adds its partial sums to the slot's partials.
struct WsSlot {
    unsigned long long word;   // seq (bits 40..63) | chunks of the round (20..39) | next chunk (0..19)
    int done;                  // chunks of the round whose partials are written
    int ns;                    // candidates of the round
    int jc[4];                 // their last bins
    int pad[2];
    CoefMixed cm[4];           // their mixed-precision coefficients
};

constexpr int WS_PART_PER_CHUNK = 4 * MAXDET * 2;   // doubles: [candidate][detector][re, im]

struct StepArgs {
    double *live_u;       // [n][d]
    double *live_logl;    // [n]
    int *order;           // [n] ascending by (log L, index)
    double *chol;         // [d][d] lower-triangular factor of the survivors' covariance
    double *dead_u;       // [cap][d]
    double *dead_logl;    // [cap]
    double *dead_logw;    // [cap]
    double *dead_nlive;   // [cap] live count at removal (n - j + 1)
    RunState *state;
    uint64_t seed;
    int n, k, steps, max_stepout, max_shrink;
    double dlogz_stop;
    int *active;          // chains of the current slice update still running
    int depth;            // candidates planned per round while many chains run
    int tail;             // below this many running chains, plan as many as there are warps
    int fp64_split;       // FP64: warps per candidate's bins in every round (1, or 2 on fine grids:
                          // always the same split, so results do not depend on timing)
    int kernel;           // 0 slice sampling, 1 random walk
    double walk_scale;    // random walk: y = x + walk_scale L z
    // work-shared slice update (ws != nullptr): persistent CTAs take chains from
    // chain_ctr; ws_nslot slots, partials [ws_nslot][ws_maxchunk][WS_PART_PER_CHUNK]
    int *chain_ctr;
    WsSlot *ws;
    double *ws_part;
    int ws_nslot, ws_gchunk, ws_maxchunk;
    int ws_test_extra;    // test hook: chunks the owner waits for beyond its round's (0 in use)
    long long lo_bin;     // first bin of the tile groups this launch sums at the Taylor degree TK_LO
                          // (bin accounting only; past every grid when none)
};

// One analysis' iteration arguments, for the multi-analysis launches.
struct Desc {
    Model M;
    Tables T;
    StepArgs A;
};

// Copy of an analysis' descriptor into shared memory by the whole block
// (multi-analysis launches); ends with a barrier.
__device__ __forceinline__ void load_desc(const Desc *g, Desc &s) {
    const int *src = (const int *)g;
    int *dst = (int *)&s;
    for (int i = threadIdx.x; i < (int)(sizeof(Desc) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    __syncthreads();
}

// Writable mixed-form tables (per-bin or tiled set, by Model::tlg).
struct MixedTables {
    float2 *basis32, *f32, *w32;
    float2 *tb0, *tb1;
    float *tbk;
    float2 *fc, *wt;
};

struct ResultArgs {
    const double *dead_logl, *dead_logw, *dead_nlive;
    const double *fin_logl, *fin_logw, *fin_nlive;   // [n] final live points, ascending
    long long n_dead;
    int n;
    double logZ;          // total log Z
    double *reps;         // [R]
    double *out;          // [4]: dlogZ, H, ESS, mean of replicates
    uint64_t seed;
    int R;
};

// Staging for the allocation-free host-buffer likelihood entry: up to
// NOALLOC_MAX_POINTS points of up to MAXD coordinates plus their log L.
constexpr int NOALLOC_MAX_POINTS = 4096;
constexpr size_t NOALLOC_DOUBLES = (size_t)NOALLOC_MAX_POINTS * (MAXD + 1);
// Device address of that staging array on the current device (looked up once
// per device and cached; never allocates).
cudaError_t noalloc_scratch_address(double **ptr);

// Likelihood and slice-update launchers per (precision, detectors), defined in
// gwns_slice.cuh and instantiated in gwns_inst_p<P>_d<D>.cu.
template <int PREC, int NDET>
cudaError_t eval_launch(const Model &M, const Tables &T, int warps, const double *in, int th, int m,
                        double *logl, RunState *st, cudaStream_t s);
template <int PREC, int NDET>
cudaError_t slice_launch(const Model &M, const Tables &T, int slots, const StepArgs &A, cudaStream_t s);
template <int PREC, int NDET>
cudaError_t slice_multi_launch(const Desc *D, const int2 *map, int nblocks, int slots, int rot, cudaStream_t s);
template <int PREC, int NDET>
int slice_ws_blocks_per_sm();
// CTAs of the work-shared slice update per SM for this precision and detector count.
int ws_blocks_per_sm(int precision, int ndet);

// Launchers (return cudaGetLastError()).
cudaError_t launch_build_tables(const Model &M, const double *data_re, const double *data_im,
                                const double *psd, double *basis64, double *f64, double2 *w64,
                                double *prefix, const MixedTables &X, cudaStream_t s);
cudaError_t launch_init_live(const Model &M, uint64_t seed, int n, double *live_u, cudaStream_t s);
cudaError_t launch_eval(const Model &M, const Tables &T, int precision, int warps, const double *in,
                        int in_is_theta, int m, double *logl, RunState *st, cudaStream_t s);
cudaError_t launch_select(const double *logl, int n, int *order, cudaStream_t s);
cudaError_t launch_evidence(const Model &M, const StepArgs &A, cudaStream_t s);
cudaError_t launch_cov_chol(const Model &M, const StepArgs &A, cudaStream_t s);
cudaError_t launch_slice(const Model &M, const Tables &T, int precision, int warps, const StepArgs &A,
                         cudaStream_t s);
cudaError_t launch_finish(const StepArgs &A, cudaStream_t s);
cudaError_t launch_final_live(const Model &M, const StepArgs &A, double *fin_u, double *fin_logl,
                              double *fin_logw, double *fin_nlive, double *logz_total, cudaStream_t s);
cudaError_t launch_result_stats(const ResultArgs &R, cudaStream_t s);
cudaError_t launch_iteration_multi_head(const Desc *D, int n_an, cudaStream_t s);
// rot = 1: the analyses of the launch are mixed, with tiles of 32 bins or more
// (rotation-form kernel); 0: direct-form kernel.
cudaError_t launch_slice_multi(const Desc *D, const int2 *map, int nblocks, int precision, int ndet, int slots,
                               int rot, cudaStream_t s);
cudaError_t launch_iteration_multi_tail(const Desc *D, int n_an, cudaStream_t s);
cudaError_t launch_theta(const Model &M, const double *u, long long m, double *theta, cudaStream_t s);
cudaError_t launch_rb_setup(const Model &M, const Tables &T, int B, const double *theta_fid, int *J,
                            int *nedge_dev, Coef *fid, double2 *h0_tmp, const double *dre, const double *dim,
                            const double *psd, RBTables &R, double *fe, double *basis64, float2 *basis32,
                            float2 *fe32, double *fm, double *inv_de, double2 *A0, double2 *A1, double *B0,
                            double *B1, float2 *A0f, float2 *A1f, float *B0f, float *B1f, float *inv_de_f,
                            cudaStream_t s);
cudaError_t launch_point_coef(const Model &M, const Tables &T, const double *theta, Coef *out,
                              cudaStream_t s);
cudaError_t launch_waveform(const Model &M, const Tables &T, const double *theta, Coef *scratch,
                            double *h_re, double *h_im, cudaStream_t s);

}  // namespace gwns
