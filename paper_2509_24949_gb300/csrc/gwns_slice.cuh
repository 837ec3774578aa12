// gwns_slice.cuh -- the per-candidate likelihood and the slice-sampling
// update (paper Sec. 2) as templates over precision and detector count. Each
// gwns_inst_p<P>_d<D>.cu translation unit instantiates one (precision,
// detectors) pair, so the kernels compile in parallel.
#pragma once
#include "gwns_kernels.cuh"

namespace gwns {

// The warp sums of one candidate's double-float sums zh/zl[d][re, im] by the
// transposing butterfly (warp_sum_df_many; lanes 2v hold value v = 2 d + re/im),
// written as doubles to out[v] (2 NDET entries).
template <int NDET>
__device__ __forceinline__ void warp_sums_df_to(const float (&zh)[NDET][2], const float (&zl)[NDET][2],
                                                double *out) {
    const int lane = threadIdx.x & 31;
    float vh[16], vl[16];
#pragma unroll
    for (int d = 0; d < NDET; d++)
#pragma unroll
        for (int ri = 0; ri < 2; ri++) { vh[2 * d + ri] = zh[d][ri]; vl[2 * d + ri] = zl[d][ri]; }
    float rh, rl;
    warp_sum_df_many<2 * NDET>(vh, vl, rh, rl);
    const int v = lane >> 1;
    if ((lane & 1) == 0 && v < 2 * NDET) out[v] = (double)rh + (double)rl;
}

// The same sums combined with G_d: returns sum_d (Re G_d Re Z_d - gim_d Im Z_d)
// on lane 0 (the detector terms of log L), from the transposed warp sums: the
// lane holding value v multiplies it by its factor, then lanes 0, 2, .., 14 add.
template <int NDET>
__device__ __forceinline__ double warp_detector_terms_df(const float (&zh)[NDET][2], const float (&zl)[NDET][2],
                                                         const Coef &c) {
    const int lane = threadIdx.x & 31;
    float vh[16], vl[16];
#pragma unroll
    for (int d = 0; d < NDET; d++)
#pragma unroll
        for (int ri = 0; ri < 2; ri++) { vh[2 * d + ri] = zh[d][ri]; vl[2 * d + ri] = zl[d][ri]; }
    float rh, rl;
    warp_sum_df_many<2 * NDET>(vh, vl, rh, rl);
    const int v = lane >> 1, dd = v >> 1;
    double t = 0.0;
    if ((lane & 1) == 0 && v < 2 * NDET) {
        const double z = (double)rh + (double)rl;
        t = (v & 1) ? -c.gim[dd] * z : c.gre[dd] * z;
    }
#pragma unroll
    for (int o = 2; o < 16; o <<= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    return t;
}

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
#pragma unroll
        for (int d = 0; d < NDET; d++) {
            zr[d] = warp_sum(zr[d]);
            zi[d] = warp_sum(zi[d]);
        }
    } else if (M.tlg) {
        // tiled form: warp w takes tile groups w, w + W, ...
        float zh[1][NDET][2], zl[1][NDET][2];
        if (M.tlg >= 5)
            tile_bins<NDET, 1, true, true, true>(T, M.tlg, M.np, &cm, &coef.jcut, 1, warp, W, zh, zl);
        else
            tile_bins<NDET, 1, false>(T, M.tlg, M.np, &cm, &coef.jcut, 1, warp, W, zh, zl);
        warp_sums_df_to<NDET>(zh[0], zl[0], red[warp]);
    } else {
        float zh[NDET][2], zl[NDET][2];
        bins_mixed<NDET>(T, M.N, cm, coef.jcut, threadIdx.x, W * 32, zh, zl);
        warp_sums_df_to<NDET>(zh, zl, red[warp]);
    }
    if (PREC == 0 && lane == 0) {
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
    if (precision == 1 && M.cdf && !in_is_theta) {
        point_coef_group_mx(M, T, in, 0, coef, cm, 1, M.tlg >= 5);
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
    if (precision == 1) coef_to_mixed_warp(*coef, M.n_det, M.df, cm, M.rb ? T.rb.fid : nullptr, M.tlg >= 5);
    (void)lane;
}

// Points per CTA of the batched likelihood: the coefficient stage packs up to
// four points into one warp pass (8 lanes each), so the per-point FP64 work that
// binds the mixed form on grids of a few thousand bins is shared. GB300, 8192
// prior draws of the 64,897-bin workload: 4.0e7 -> 5.9e7 evals/s. Where the
// bins bind (the FP64 form; 519,169 bins) the coarser grid of CTAs cost 4-9%,
// and there, as for physical-parameter and toy inputs, a CTA takes one point.
constexpr int EVAL_PPC = 4;

template <int PREC, int NDET, int W>
__global__ void __launch_bounds__(W * 32) k_eval(Model M, Tables T, const double *in, int in_is_theta,
                                                 int m, int ppc, double *logl, RunState *st) {
    __shared__ Coef coef[EVAL_PPC];
    __shared__ CoefMixed cm[EVAL_PPC];
    __shared__ double red[W][2 * MAXDET];
    __shared__ double lval;
    __shared__ double pt[EVAL_PPC][NPARAM + MAXD];
    const int i0 = blockIdx.x * ppc;
    if (i0 >= m) return;
    const int np = m - i0 < ppc ? m - i0 : ppc;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int stride_in = in_is_theta ? NPARAM : M.dim;
    for (int t = threadIdx.x; t < np * stride_in; t += W * 32)
        pt[t / stride_in][t % stride_in] = in[(size_t)i0 * stride_in + t];
    __syncthreads();
    if (warp == 0) {
        if (ppc == 1) {
            warp_point_coef(M, T, pt[0], in_is_theta, PREC, &coef[0], &cm[0]);
        } else {
            point_coef_group(M, T, pt[0], NPARAM + MAXD, coef, np, 0);
            __syncwarp();
            if (PREC == 1)
                for (int p = 0; p < np; p++)
                    coef_to_mixed_warp(coef[p], M.n_det, M.df, &cm[p], M.rb ? T.rb.fid : nullptr, M.tlg >= 5);
        }
    }
    __syncthreads();
    for (int p = 0; p < np; p++) {
        if (M.rb) {
            // relative-binning sums: one warp
            if (warp == 0) {
                const double v = rb_loglike_warp<NDET, PREC>(M, T.rb, coef[p], cm[p], lane);
                if (lane == 0) {
                    logl[i0 + p] = v;
                    if (st) atomicAdd(&st->eval_points, 1ull);
                }
            }
            continue;
        }
        cta_loglike_bins<PREC, NDET, W>(M, T, coef[p], cm[p], red, &lval);
        if (threadIdx.x == 0) {
            logl[i0 + p] = lval;
            if (st) {
                atomicAdd(&st->eval_points, 1ull);
                if (M.model != M_TOY) {
                    atomicAdd(&st->eval_point_bins, (unsigned long long)(coef[p].jcut + 1));
                    // the rotation form here sums the groups from T.g_lo at the low Taylor degree
                    if (PREC == 1 && M.tlg >= 5) {
                        const long long lo = (long long)coef[p].jcut + 1 - ((long long)T.g_lo << (M.tlg + 5));
                        if (lo > 0) atomicAdd(&st->eval_point_bins_lo, (unsigned long long)lo);
                    }
                }
            }
        }
        __syncthreads();    // red and lval serve the next point
    }
}

// Batched likelihood, mixed precision, unit-cube points on grids of up to
// 262,144 bins (where the per-point FP64 work weighs most): 4 max(1, W/2)
// points per CTA. The coefficient stage runs as its two halves on two warps per
// group of four points (mass and phase on one, sky and detectors on the other,
// independent FP64 chains on two SM sub-partitions), joined by the first; then
// each point's bins are summed by one warp (points dealt to the warps in turn),
// reduced in double-float, and only the final log L is formed in FP64. GB300,
// 8192 prior draws of the 64,897-bin workload: the previous kernel (coefficients
// of four points on one warp, the other warp waiting, every point's tile groups
// shared by both warps and reduced in FP64) reached 5.75e7 evals/s.
template <int NDET, int W>
__global__ void __launch_bounds__(W * 32) k_eval_batch(Model M, Tables T, const double *in, int m, double *logl,
                                                       RunState *st) {
    constexpr int NG = W >= 2 ? W / 2 : 1;
    constexpr int PPC = 4 * NG;
    __shared__ Coef coef[PPC];
    __shared__ CoefMixed cm[PPC];
    __shared__ double pt[PPC][MAXD];
    const int i0 = blockIdx.x * PPC;
    if (i0 >= m) return;
    const int np = m - i0 < PPC ? m - i0 : PPC;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int d = M.dim;
    for (int t = threadIdx.x; t < np * d; t += W * 32) pt[t / d][t % d] = in[(size_t)i0 * d + t];
    __syncthreads();
    const int grp = W >= 2 ? warp >> 1 : warp;
    const bool lead = W >= 2 ? (warp & 1) == 0 : true;
    const int cnt = (grp < NG && 4 * grp < np) ? min(4, np - 4 * grp) : 0;
    if (cnt > 0) {
        if (M.cdf)
            point_coef_group_mx(M, T, pt[4 * grp], MAXD, &coef[4 * grp], &cm[4 * grp], cnt, M.tlg >= 5,
                                W >= 2 ? 1 + (warp & 1) : 0);
        else
            point_coef_group(M, T, pt[4 * grp], MAXD, &coef[4 * grp], cnt, 0, W >= 2 ? 1 + (warp & 1) : 0);
    }
    __syncthreads();
    if (cnt > 0 && lead) {
        if (W >= 2) point_coef_join(M, T, &coef[4 * grp], cnt);
        __syncwarp();
        if (!M.cdf)
            for (int p = 4 * grp; p < 4 * grp + cnt; p++)
                coef_to_mixed_warp(coef[p], M.n_det, M.df, &cm[p], nullptr, M.tlg >= 5);
    }
    __syncthreads();
    unsigned long long n_pts = 0, n_pb = 0;     // this warp's counts, added once at the end
    for (int p = warp; p < np; p += W) {
        double t;       // on lane 0: sum over detectors of Re(G_d Z_d)
        if (M.tlg) {
            float zh[1][NDET][2], zl[1][NDET][2];
            if (M.tlg >= 5)
                tile_bins<NDET, 1, true, true>(T, M.tlg, M.np, &cm[p], &coef[p].jcut, 1, 0, 1, zh, zl);
            else
                tile_bins<NDET, 1, false>(T, M.tlg, M.np, &cm[p], &coef[p].jcut, 1, 0, 1, zh, zl);
            t = warp_detector_terms_df<NDET>(zh[0], zl[0], coef[p]);
        } else {
            float zh[NDET][2], zl[NDET][2];
            bins_mixed<NDET>(T, M.N, cm[p], coef[p].jcut, lane, 32, zh, zl);
            t = warp_detector_terms_df<NDET>(zh, zl, coef[p]);
        }
        if (lane == 0) {
            const double v = t - 0.5 * coef[p].hh;
            logl[i0 + p] = v;
            n_pts++;
            n_pb += (unsigned long long)(coef[p].jcut + 1);
        }
    }
    if (st && lane == 0 && n_pts) {
        atomicAdd(&st->eval_points, n_pts);
        atomicAdd(&st->eval_point_bins, n_pb);
    }
}

template <int PREC, int NDET>
cudaError_t eval_launch(const Model &M, const Tables &T, int warps, const double *in, int th, int m,
                        double *logl, RunState *st, cudaStream_t s) {
    const int nbins = M.rb ? T.rb.nb : M.N;
    if constexpr (PREC == 1) {
        if (M.model == M_GW && !th && !M.rb && nbins <= 262144) {
            const int ppc = 4 * (warps >= 2 ? warps / 2 : 1);
            const int gb = (m + ppc - 1) / ppc;
            switch (warps) {
                case 1: k_eval_batch<NDET, 1><<<gb, 32, 0, s>>>(M, T, in, m, logl, st); break;
                case 2: k_eval_batch<NDET, 2><<<gb, 64, 0, s>>>(M, T, in, m, logl, st); break;
                case 4: k_eval_batch<NDET, 4><<<gb, 128, 0, s>>>(M, T, in, m, logl, st); break;
                default: k_eval_batch<NDET, 8><<<gb, 256, 0, s>>>(M, T, in, m, logl, st); break;
            }
            return cudaGetLastError();
        }
    }
    const int ppc = (PREC == 1 && M.model == M_GW && !th && nbins <= 262144) ? EVAL_PPC : 1;
    const int g = (m + ppc - 1) / ppc;
    switch (warps) {
        case 1: k_eval<PREC, NDET, 1><<<g, 32, 0, s>>>(M, T, in, th, m, ppc, logl, st); break;
        case 2: k_eval<PREC, NDET, 2><<<g, 64, 0, s>>>(M, T, in, th, m, ppc, logl, st); break;
        case 4: k_eval<PREC, NDET, 4><<<g, 128, 0, s>>>(M, T, in, th, m, ppc, logl, st); break;
        default: k_eval<PREC, NDET, 8><<<g, 256, 0, s>>>(M, T, in, th, m, ppc, logl, st); break;
    }
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
enum { PH_NEWSTEP = 0, PH_OUT = 1, PH_SHRINK = 2, PH_DONE = 3, PH_WALK = 4 };
enum { KIND_L = 0, KIND_R = 1, KIND_SH = 2, KIND_W = 3 };
constexpr int CACHE_MAX = 16;

struct Chain {
    double x, e, lrow[MAXD];
    double lx, a, b;
    int s, phase, nl, nr, nsh, caps, left_done, right_done;
    long long evals;
    unsigned long long bins, bins_lo;   // bins read by the consumed evaluations; of those, in low-degree groups
    // cache of evaluated, not yet consumed candidates
    int ncache;
    int ckind[CACHE_MAX], cidx[CACHE_MAX], cbins[CACHE_MAX];
    double cval[CACHE_MAX];
    double cy[CACHE_MAX];      // random walk: the evaluated proposal (lane's coordinate)
};

// A consumed evaluation's bins (jcut + 1 of them): all, and those at or past lo_bin.
__device__ __forceinline__ void count_bins(Chain &c, int bins, long long lo_bin) {
    c.bins += (unsigned long long)bins;
    if ((long long)bins > lo_bin) c.bins_lo += (unsigned long long)((long long)bins - lo_bin);
}

// Lane i's coordinate of the candidate x + t e (lanes >= d: 0.5, inside the
// box); periodic coordinates wrap into [0, 1).
__device__ __forceinline__ double line_y(const Model &M, const Chain &c, double t, int lane, int d) {
    if (lane >= d) return 0.5;
    double y = __dadd_rn(c.x, __dmul_rn(t, c.e));
    if ((M.periodic >> lane) & 1u) y = __dsub_rn(y, floor(y));
    return y;
}

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
    c.cy[i] = c.cy[c.ncache];
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

// Hit-and-run direction of slice step s: lane i < d gets coordinate i of
// L z / |z|, z ~ N(0, I) by Box-Muller (two normals per draw); lrow is the
// lane's row of the Cholesky factor L.
__device__ __forceinline__ double slice_direction(const StepArgs &A, const double *lrow, int chain, uint32_t iter,
                                                  int s, int lane, int d) {
    double z = 0.0;
    if (lane < d) {
        const uint4 w = draw(A.seed, (uint32_t)(lane >> 1), (uint32_t)s, (uint32_t)chain, iter);
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
        if (j <= lane) acc = __dadd_rn(acc, __dmul_rn(lrow[j], zj));
    }
    return (lane < d) ? acc / nz : 0.0;
}

// Apply every transition that needs no new evaluation: new steps (direction and
// bracket draws), cap and prior-box outcomes, and results already in the cache.
// Returns when the next transition needs an evaluation not in the cache, or the
// chain is done.
static __device__ void chain_run(const Model &M, const StepArgs &A, Chain &c, int chain, uint32_t iter,
                                 double lstar, const double *e_pre, int e_pre_step) {
    const int lane = threadIdx.x & 31, d = M.dim;
    for (int guard = 0; guard < (1 << 22); guard++) {
        if (c.phase == PH_DONE) return;
        if (c.phase == PH_NEWSTEP) {
            if (c.s >= A.steps) { c.phase = PH_DONE; return; }
            // direction (computed ahead by a spare warp when it could be)
            if (e_pre_step == c.s) c.e = (lane < d) ? e_pre[lane] : 0.0;
            else c.e = slice_direction(A, c.lrow, chain, iter, c.s, lane, d);
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
            const double y = line_y(M, c, t, lane, d);
            if (!warp_inbox(y, lane, d)) {
                end_side(c, left);
                continue;
            }
            const int ci = cache_find(c, left ? KIND_L : KIND_R, n);
            if (ci < 0) return;
            const bool in = c.cval[ci] > lstar;
            c.evals++;
            count_bins(c, c.cbins[ci], A.lo_bin);
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
        const double y = line_y(M, c, t, lane, d);
        if (warp_inbox(y, lane, d)) {
            const int ci = cache_find(c, KIND_SH, c.nsh);
            if (ci < 0) return;
            const double val = c.cval[ci];
            c.evals++;
            count_bins(c, c.cbins[ci], A.lo_bin);
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
                const double y = line_y(M, c, t, lane, d);
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
            const double y = line_y(M, c, t, lane, d);
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

// ------------------------------------------------------------ random walk
// The random-walk inner kernel (acceptance walk): from the chain's start point,
// walk_len proposals y = x + scale L z_p, z_p ~ N(0, I) from the draws of
// proposal p (the slice directions' slots with p in place of the step); a
// proposal inside the prior box (periodic coordinates wrapped) and above L*
// is accepted. The walk length is fixed within an iteration and rescaled
// between iterations (k_finish). Speculation: the proposals after the current
// one are evaluated from the current point, as if it were rejected; an
// acceptance discards them. c.s counts accepted moves, c.nsh the proposal.
__device__ __forceinline__ double walk_disp(const StepArgs &A, const Chain &c, int chain, uint32_t iter, int p,
                                            int lane, int d) {
    double z = 0.0;
    if (lane < d) {
        const uint4 w = draw(A.seed, (uint32_t)(lane >> 1), (uint32_t)p, (uint32_t)chain, iter);
        const double u1 = u01(w.x, w.y), u2 = u01(w.z, w.w);
        const double r = sqrt(-2.0 * log(u1));
        double sn, cs;
        sincos(TWO_PI_D * u2, &sn, &cs);
        z = (lane & 1) ? r * sn : r * cs;
    }
    double acc = 0.0;
    for (int j = 0; j < d; j++) {
        const double zj = __shfl_sync(0xffffffffu, z, j);
        if (j <= lane) acc = __dadd_rn(acc, __dmul_rn(c.lrow[j], zj));
    }
    return __dmul_rn(acc, A.walk_scale);
}

__device__ __forceinline__ double walk_y(const Model &M, const Chain &c, double disp, int lane, int d) {
    if (lane >= d) return 0.5;
    double y = __dadd_rn(c.x, disp);
    if ((M.periodic >> lane) & 1u) y = __dsub_rn(y, floor(y));
    return y;
}

static __device__ void walk_run(const Model &M, const StepArgs &A, Chain &c, int chain, uint32_t iter,
                                double lstar, int walk_len) {
    const int lane = threadIdx.x & 31, d = M.dim;
    for (int guard = 0; guard < (1 << 22); guard++) {
        if (c.phase == PH_DONE) return;
        if (c.nsh >= walk_len) { c.phase = PH_DONE; return; }
        // an evaluated proposal comes with its point (planned from the current
        // point: the cache is emptied at every acceptance); otherwise compute
        // it, skip it outside the box, or wait for its evaluation
        const int ci = cache_find(c, KIND_W, c.nsh);
        double y;
        if (ci >= 0) {
            y = (lane < d) ? c.cy[ci] : 0.5;
        } else {
            y = walk_y(M, c, walk_disp(A, c, chain, iter, c.nsh, lane, d), lane, d);
            if (!warp_inbox(y, lane, d)) { c.nsh++; continue; }
            return;
        }
        const double val = c.cval[ci];
        c.evals++;
        count_bins(c, c.cbins[ci], A.lo_bin);
        cache_drop(c, ci);
        if (val > lstar) {
            c.x = y;
            c.lx = val;
            c.s++;
            cache_purge(c, KIND_W);
        }
        c.nsh++;
    }
    c.phase = PH_DONE;
}

template <int S>
__device__ int walk_plan(const Model &M, const StepArgs &A, const Chain &c, int chain, uint32_t iter,
                         double (*ysh)[MAXD], int *pk, int *pidx, int depth, int walk_len) {
    const int lane = threadIdx.x & 31, d = M.dim;
    const int room = CACHE_MAX - c.ncache;
    const int lim = depth < S ? depth : S;
    const int cap = lim < room ? lim : room;
    int ns = 0;
    for (int p = c.nsh; p < c.nsh + S && p < walk_len && ns < cap; p++) {
        if (cache_find(c, KIND_W, p) >= 0) continue;
        const double y = walk_y(M, c, walk_disp(A, c, chain, iter, p, lane, d), lane, d);
        if (warp_inbox(y, lane, d)) {
            if (lane < d) ysh[ns][lane] = y;
            pk[ns] = KIND_W;
            pidx[ns] = p;
            ns++;
        }
    }
    return ns;
}

// ------------------------------------------------- work-shared slice update
// Mixed precision on fine tiled grids (the 519,169-bin workload): when fewer
// chains remain than CTA slots, the update's last chains would run alone on
// otherwise idle SMs. Instead, persistent CTAs take chains from a counter, and
// each round's candidates are evaluated in fixed chunks of ws_gchunk tile
// groups. The owner publishes the round in its slot (coefficients, then the
// claim word); its own warps and the warps of CTAs without a chain claim
// chunks through the word, each chunk's sums are computed by one warp and
// written to the slot's partials, and the owner adds them in chunk order. The
// decomposition does not depend on who computes a chunk, so results do not
// depend on timing. No warp waits on a CTA that has not claimed work: the
// owner waits only for chunks already claimed (their warps are running), and
// helpers stop once no chain is running. Both waits are bounded; on a timeout
// the run state's status gets bit 1 and the host reports NS_ERR_TIMEOUT.
constexpr long long WS_WAIT_LIMIT = 1ll << 24;   // owner polls of the done count (~100 ns apart)
constexpr long long WS_IDLE_LIMIT = 1ll << 22;   // consecutive helper polls without work (~1 us each)

__device__ __forceinline__ unsigned long long ws_word(unsigned long long seq, int n, int next) {
    return (seq << 40) | ((unsigned long long)n << 20) | (unsigned long long)next;
}

// Lane 0: claim the next chunk of a slot's round; -1 if none is left. A stale
// view of the word is harmless: the atomic's return value names the round and
// chunk actually claimed, and a round's data stay in place until all its
// claimed chunks are done.
__device__ __forceinline__ int ws_claim(WsSlot *s) {
    const unsigned long long w = *((volatile unsigned long long *)&s->word);
    if ((w & 0xFFFFFull) >= ((w >> 20) & 0xFFFFFull)) return -1;
    const unsigned long long old = atomicAdd(&s->word, 1ull);
    const int n = (int)((old >> 20) & 0xFFFFFull), nx = (int)(old & 0xFFFFFull);
    return nx < n ? nx : -1;
}

// One warp: the sums of chunk c (tile groups c G .. c G + G - 1) for the ns
// candidates, reduced over the warp; lane 0 writes out[candidate][detector][re, im].
template <int NDET>
__device__ __forceinline__ void ws_chunk(const Model &M, const Tables &T, const CoefMixed *cm, const int *jc,
                                         int ns, int c, int G, double *out) {
    const int lane = threadIdx.x & 31;
    const int g0 = c * G, g1 = g0 + G;
    for (int c0 = 0; c0 < ns; c0++) {
        float zh[1][NDET][2], zl[1][NDET][2];
        tile_bins<NDET, 1, true, true, true>(T, M.tlg, M.np, cm + c0, jc + c0, 1, g0, 1, zh, zl, g1);
        // value v = (detector, re/im), summed over the warp at once
        float vh[16], vl[16];
#pragma unroll
        for (int dd = 0; dd < NDET; dd++)
#pragma unroll
            for (int ri = 0; ri < 2; ri++) {
                vh[dd * 2 + ri] = zh[0][dd][ri];
                vl[dd * 2 + ri] = zl[0][dd][ri];
            }
        float rh, rl;
        warp_sum_df_many<2 * NDET>(vh, vl, rh, rl);
        const int v = lane >> 1, dd = v >> 1, ri = v & 1;
        if ((lane & 1) == 0 && v < 2 * NDET)
            out[(c0 * MAXDET + dd) * 2 + ri] = (double)rh + (double)rl;
    }
}

// One warp: find a slot (other than skip) with an unclaimed chunk, claim it
// and compute it into that slot's partials. Returns 1 if it did a chunk. The
// round's coefficients are staged in this warp's shared buffer.
template <int NDET, int W>
__device__ int ws_take_any(const Model &M, const Tables &T, const StepArgs &A, int skip) {
    __shared__ CoefMixed hcm[W][4];
    __shared__ int hjc[W][4];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nslot = A.ws_nslot;
    const int start = (int)(((unsigned)blockIdx.x * 37u + (unsigned)warp * 11u) % (unsigned)nslot);
    int found = -1;
    for (int base = 0; base < nslot && found < 0; base += 32) {
        const int j = base + lane;
        int s = start + j;
        if (s >= nslot) s -= nslot;
        bool open = false;
        if (j < nslot && s != skip) {
            const unsigned long long w = *((volatile unsigned long long *)&A.ws[s].word);
            open = (w & 0xFFFFFull) < ((w >> 20) & 0xFFFFFull);
        }
        const unsigned b = __ballot_sync(0xffffffffu, open);
        if (b) found = __shfl_sync(0xffffffffu, s, __ffs(b) - 1);
    }
    int c = -1;
    if (found >= 0 && lane == 0) c = ws_claim(A.ws + found);
    c = __shfl_sync(0xffffffffu, c, 0);
    if (c < 0) return 0;
    __threadfence();
    WsSlot *sl = A.ws + found;
    const int ns = __ldcg(&sl->ns);
    const int nwords = ns * (int)(sizeof(CoefMixed) / sizeof(int));
    for (int i = lane; i < nwords; i += 32) ((int *)hcm[warp])[i] = __ldcg(((const int *)sl->cm) + i);
    if (lane < ns) hjc[warp][lane] = __ldcg(&sl->jc[lane]);
    __syncwarp();
    ws_chunk<NDET>(M, T, hcm[warp], hjc[warp], ns, c, A.ws_gchunk,
                   A.ws_part + ((size_t)found * A.ws_maxchunk + c) * WS_PART_PER_CHUNK);
    __threadfence();
    if (lane == 0) atomicAdd(&sl->done, 1);
    __syncwarp();
    return 1;
}

// Owner CTA (all threads): publish the round's ns candidates (coefficients cm,
// last bins jc, in shared memory), take part in its chunks, then warp 0 waits
// for the chunks helpers took and writes the sums over chunks, in chunk order,
// to zs[candidate][detector][re, im] (shared).
template <int NDET, int W>
__device__ void ws_owner_round(const Model &M, const Tables &T, const StepArgs &A, const CoefMixed *cm,
                               const int *jc, int ns, double (*zs)[NDET][2]) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WsSlot *slot = A.ws + blockIdx.x;
    double *part = A.ws_part + (size_t)blockIdx.x * A.ws_maxchunk * WS_PART_PER_CHUNK;
    int jmax = -1;
    for (int c = 0; c < ns; c++) jmax = max(jmax, jc[c]);
    const int G = A.ws_gchunk;
    const int ng = jmax < 0 ? 0 : (jmax >> (M.tlg + 5)) + 1;
    const int nch = min((ng + G - 1) / G, A.ws_maxchunk);
    const int nwords = ns * (int)(sizeof(CoefMixed) / sizeof(int));
    for (int i = threadIdx.x; i < nwords; i += W * 32) ((int *)slot->cm)[i] = ((const int *)cm)[i];
    if (threadIdx.x < ns) slot->jc[threadIdx.x] = jc[threadIdx.x];
    if (threadIdx.x == 0) {
        slot->ns = ns;
        slot->done = 0;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned long long w = *((volatile unsigned long long *)&slot->word);
        atomicExch(&slot->word, ws_word((w >> 40) + 1, nch, 0));
    }
    __syncthreads();
    // every warp claims the round's chunks; warp 0 then waits for the chunks
    // other CTAs took (GB300, 519,169 bins: letting the other warps take other
    // rounds' chunks meanwhile was slower, 264 -> 297 ms per update, as a
    // chain's next round then waits for its warps to come back)
    for (int guard = 0; guard < (1 << 20); guard++) {
        int c = -1;
        if (lane == 0) c = ws_claim(slot);
        c = __shfl_sync(0xffffffffu, c, 0);
        if (c < 0) break;
        ws_chunk<NDET>(M, T, cm, jc, ns, c, G, part + (size_t)c * WS_PART_PER_CHUNK);
        __threadfence();
        if (lane == 0) atomicAdd(&slot->done, 1);
    }
    if (warp == 0 && lane == 0) {
        // ws_test_extra (a test hook, 0 in use) makes the owner wait for chunks
        // nobody computes, so that the bounded wait runs out
        for (long long it = 0; *((volatile int *)&slot->done) < nch + A.ws_test_extra; it++) {
            if (it > WS_WAIT_LIMIT) {
                atomicOr(&A.state->status, 2);
                break;
            }
            __nanosleep(100);
        }
    }
    __syncthreads();
    if (warp == 0) {
        __threadfence();
        const int sc = lane / NDET, dd = lane - sc * NDET;
        if (lane < ns * NDET) {
            double zr = 0.0, zi = 0.0;
            for (int c = 0; c < nch; c++) {
                const double *p = part + (size_t)c * WS_PART_PER_CHUNK + (sc * MAXDET + dd) * 2;
                zr += __ldcg(p);
                zi += __ldcg(p + 1);
            }
            zs[sc][dd][0] = zr;
            zs[sc][dd][1] = zi;
        }
    }
}

// A CTA without a chain left: each warp takes chunks of any running chain's
// round until no chain is running.
template <int NDET, int W>
__device__ void ws_help(const Model &M, const Tables &T, const StepArgs &A) {
    const int lane = threadIdx.x & 31;
    long long idle = 0;
    for (;;) {
        if (*((volatile int *)A.active) <= 0) break;
        if (ws_take_any<NDET, W>(M, T, A, -1)) {
            idle = 0;
            continue;
        }
        if (++idle > WS_IDLE_LIMIT) {
            if (lane == 0) atomicOr(&A.state->status, 2);
            break;
        }
        __nanosleep(200);
    }
}

// Forms of the tiled mixed sums a kernel compiles. FORM_BOTH chooses at run
// time: rotation (tile_bins_rot) on tiles of 32 bins or more, direct on
// shorter ones. FORM_DIRECT and FORM_ROT compile one form only (the serving
// kernel, which runs many analyses per launch, spilled registers with both);
// FORM_ROT kernels run only grids with tiles of 32 bins or more.
enum { FORM_DIRECT = 0, FORM_BOTH = 1, FORM_ROT = 2 };

template <int FORM>
__device__ __forceinline__ bool form_rot(const Model &M) {
    if constexpr (FORM == FORM_ROT) return true;
    else if constexpr (FORM == FORM_DIRECT) return false;
    else return M.tlg >= 5;
}

template <int NDET, int NC, int FORM>
__device__ __forceinline__ void tile_bins_form(const Model &M, const Tables &T, const CoefMixed *cm,
                                               const int *jc, int nc, int g0, int gstride,
                                               float zh[NC][NDET][2], float zl[NC][NDET][2]) {
    if constexpr (FORM == FORM_ROT) {
        tile_bins<NDET, NC, true>(T, M.tlg, M.np, cm, jc, nc, g0, gstride, zh, zl);
    } else if constexpr (FORM == FORM_DIRECT) {
        tile_bins<NDET, NC, false>(T, M.tlg, M.np, cm, jc, nc, g0, gstride, zh, zl);
    } else {
        if (M.tlg >= 5) tile_bins<NDET, NC, true>(T, M.tlg, M.np, cm, jc, nc, g0, gstride, zh, zl);
        else tile_bins<NDET, NC, false>(T, M.tlg, M.np, cm, jc, nc, g0, gstride, zh, zl);
    }
}

template <int PREC, int NDET, int S, int W = S, int FORM = FORM_BOTH, bool WS = false>
__device__ void slice_body(const Model &M, const Tables &T, const StepArgs &A, const int chain) {
    __shared__ Coef coef[S];
    __shared__ CoefMixed cm[S];
    __shared__ double ysh[S][MAXD];
    __shared__ double lval[S];
    __shared__ int nslot, tailmode;
    __shared__ double e_next[MAXD];         // direction of slice step e_next_step, computed ahead
    __shared__ int e_next_step, cur_step;
    __shared__ int jc[S];
    __shared__ double part[W][S][NDET][2];
    if (chain >= A.k) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, d = M.dim;
    const uint32_t iter = (uint32_t)A.state->iter;
    const double lstar = A.state->lstar;
    const int walk_len = A.state->walk_len;
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
        c.s = 0; c.phase = A.kernel == 1 ? PH_WALK : PH_NEWSTEP; c.nl = c.nr = c.nsh = 0; c.caps = 0;
        c.evals = 0; c.bins = 0; c.bins_lo = 0;
        c.left_done = c.right_done = 0; c.ncache = 0;
        if (lane == 0) e_next_step = -1;
    }
    for (;;) {
        if (warp == 0) {
            // a bounded wait of the work-shared update gave up (status bit 1):
            // every chain ends at its current point, so that the launch ends
            if (WS && (*((volatile int *)&A.state->status) & 2)) c.phase = PH_DONE;
            if (A.kernel == 1) walk_run(M, A, c, chain, iter, lstar, walk_len);
            else chain_run(M, A, c, chain, iter, lstar, e_next, e_next_step);
            // plan the base depth while many chains run; the stragglers of the
            // update (fewer running chains than the tail threshold) use every warp.
            // FP64 on fine grids splits every candidate's bins over two warps in
            // every round instead (FP64 branch below), with at most W/2 candidates.
            int depth = S, tail = 1;
            if (A.active) {
                const int running = *((volatile int *)A.active);
                if (running > A.tail) { depth = A.depth; tail = 0; }
            }
            if (PREC == 0 && A.fp64_split == 2 && W >= 2) {
                depth = A.depth < W / 2 ? A.depth : W / 2;
                tail = 2;
            }
            int ns = (c.phase == PH_DONE) ? 0
                   : A.kernel == 1 ? walk_plan<S>(M, A, c, chain, iter, ysh, pk, pidx, depth, walk_len)
                                   : chain_plan<S>(M, A, c, chain, iter, ysh, pk, pidx, depth);
            if (ns == 0 && c.phase != PH_DONE) {
                // cannot happen with the bounds above; end the chain at its
                // current (in-slice) point and flag the run state
                c.phase = PH_DONE;
                if (lane == 0) atomicOr(&A.state->status, 1);
            }
            if (lane == 0) { nslot = ns; tailmode = tail; cur_step = c.s; }
        }
        __syncthreads();
        const int ns = nslot;
        if (ns == 0) break;
        // coefficients: candidates 4j .. 4j+3 (8 lanes each) by one warp, or,
        // with two warps per group of four, the mass/phase half on warp 2j and
        // the sky/detector half on warp 2j + 1 (independent FP64 chains on two
        // sub-partitions), joined after the barrier
        if (M.model == M_TOY) {
            if (warp < ns) point_coef_warp(M, T, ysh[warp], &coef[warp]);
            __syncthreads();
        } else if (S >= 2) {
            const int grp = warp >> 1;
            if (4 * grp < ns && 2 * grp + 1 < W) {
                const int cnt = ns - 4 * grp < 4 ? ns - 4 * grp : 4;
                if (PREC == 1 && M.cdf)
                    point_coef_group_mx(M, T, ysh[4 * grp], MAXD, &coef[4 * grp], &cm[4 * grp], cnt,
                                        form_rot<FORM>(M), 1 + (warp & 1));
                else
                    point_coef_group(M, T, ysh[4 * grp], MAXD, &coef[4 * grp], cnt, PREC == 0 ? 32 : 0,
                                     1 + (warp & 1));
            } else if (warp == W - 1 && A.kernel == 0) {
                // a warp without coefficients computes the next slice step's direction
                const int s1 = cur_step + 1;
                if (s1 < A.steps && e_next_step != s1) {
                    double lrow[MAXD];
                    for (int j = 0; j < MAXD; j++) lrow[j] = (lane < d && j < d) ? A.chol[lane * d + j] : 0.0;
                    const double e1 = slice_direction(A, lrow, chain, iter, s1, lane, d);
                    if (lane < d) e_next[lane] = e1;
                    __syncwarp();
                    if (lane == 0) e_next_step = s1;
                }
            }
            __syncthreads();
            if (warp == 0) point_coef_join(M, T, coef, ns);
            __syncthreads();
        } else {
            if (4 * warp < ns) {
                const int cnt = ns - 4 * warp < 4 ? ns - 4 * warp : 4;
                if (PREC == 1 && M.cdf)
                    point_coef_group_mx(M, T, ysh[4 * warp], MAXD, &coef[4 * warp], &cm[4 * warp], cnt,
                                        form_rot<FORM>(M));
                else
                    point_coef_group(M, T, ysh[4 * warp], MAXD, &coef[4 * warp], cnt, PREC == 0 ? 32 : 0);
            }
            __syncthreads();
        }
        if (warp < ns && M.rb) {
            // relative-binning likelihood of the slot's candidate
            if (PREC == 1) {
                coef_to_mixed_warp(coef[warp], M.n_det, M.df, &cm[warp], T.rb.fid);
                __syncwarp();
            }
            const double v = rb_loglike_warp<NDET, PREC>(M, T.rb, coef[warp], cm[warp], lane);
            if (lane == 0) {
                lval[warp] = v;
                coef[warp].jcut = T.rb.nb - 1;     // bins counted for the work statistics
            }
        } else if (PREC == 1 && S > 1 && S <= 4 && M.model == M_GW && !M.rb && M.coop) {
            // mixed, every warp on every candidate of the round: the tiled form
            // shares out the tile groups (two candidates per pass on one table
            // load), the per-bin form strides the bins
            if (warp < ns && !M.cdf) coef_to_mixed_warp(coef[warp], M.n_det, M.df, &cm[warp], nullptr, form_rot<FORM>(M));
            if (lane == 0 && warp < ns) jc[warp] = coef[warp].jcut;
            __syncthreads();
            if (WS) {
                // work-shared: fixed chunks of tile groups, computed by this CTA's
                // warps and by helper CTAs, summed in chunk order into part[0]
                ws_owner_round<NDET, W>(M, T, A, cm, jc, ns, part[0]);
            } else if (M.tlg) {
                // the (candidate pair, tile group) items of the round are dealt out
                // to the warps in turn, pair after pair, so that every warp has
                // work when a candidate spans fewer groups than there are warps
                int off = 0;
                for (int c0 = 0; c0 < ns; c0 += 2) {
                    float zh[2][NDET][2], zl[2][NDET][2];
                    const int nc = ns - c0 < 2 ? ns - c0 : 2;
                    const int jm = nc == 2 ? max(jc[c0], jc[c0 + 1]) : jc[c0];
                    const int ng = jm < 0 ? 0 : (jm >> (M.tlg + 5)) + 1;
                    const int g0 = ((warp - off) % W + W) % W;
                    off += ng;
                    tile_bins_form<NDET, 2, FORM>(M, T, cm + c0, jc + c0, nc, g0, W, zh, zl);
                    // the pair's 4 NDET sums at once (transposing butterfly): lane 2v
                    // holds value v = (2 (candidate NDET + detector) + re/im)
                    float vh[16], vl[16];
#pragma unroll
                    for (int sc = 0; sc < 2; sc++)
#pragma unroll
                        for (int dd = 0; dd < NDET; dd++)
#pragma unroll
                            for (int ri = 0; ri < 2; ri++) {
                                vh[(sc * NDET + dd) * 2 + ri] = zh[sc][dd][ri];
                                vl[(sc * NDET + dd) * 2 + ri] = zl[sc][dd][ri];
                            }
                    float rh, rl;
                    warp_sum_df_many<4 * NDET>(vh, vl, rh, rl);
                    const int v = lane >> 1, q = v >> 1, sc = q / NDET, dd = q - sc * NDET;
                    if ((lane & 1) == 0 && v < 4 * NDET && c0 + sc < S)
                        part[warp][c0 + sc][dd][v & 1] = (double)rh + (double)rl;
                }
            } else {
                float zrh[S][NDET], zrl[S][NDET], zih[S][NDET], zil[S][NDET];
                bins_mixed_multi<NDET, S>(T, M.N, cm, jc, ns, threadIdx.x, W * 32, zrh, zrl, zih, zil);
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
            }
            __syncthreads();
            if (warp == 0) {
                // lane = (candidate, detector): sum over warps, then log L per candidate
                double v = 0.0;
                const int sc = lane / NDET, dd = lane % NDET;
                if (sc < ns && lane < S * NDET) {
                    double ZR = 0.0, ZI = 0.0;
                    for (int w2 = 0; w2 < (WS ? 1 : W); w2++) { ZR += part[w2][sc][dd][0]; ZI += part[w2][sc][dd][1]; }
                    v = coef[sc].gre[dd] * ZR - coef[sc].gim[dd] * ZI;
                }
                const double t = group_sum_down<NDET>(v);
                if (dd == 0 && sc < ns && lane < S * NDET) lval[sc] = t - 0.5 * coef[sc].hh;
            }
        } else if (PREC == 0 && W > 1 && M.model == M_GW && !M.rb && tailmode == 2) {
            // FP64 on fine grids: each candidate's bins on two warps (warps on
            // different SM sub-partitions issue FP64 independently), bin j on
            // lane j mod 32 of warp (j / 32) mod 2; the two warp sums meet in
            // shared memory in a fixed order, whatever the round.
            const int lg = 1;
            const int wpc = 1 << lg, cand = warp >> lg, sub = warp & (wpc - 1);
            if (cand < ns) {
                double zr[NDET], zi[NDET];
                bins_fp64<NDET, true>(T, M.N, M.f0, M.df, coef[cand], sub * 32 + lane, wpc * 32, zr, zi, lg);
#pragma unroll
                for (int dd = 0; dd < NDET; dd++) {
                    const double ZR = warp_sum(zr[dd]), ZI = warp_sum(zi[dd]);
                    if (lane == 0) { part[warp][0][dd][0] = ZR; part[warp][0][dd][1] = ZI; }
                }
            }
            __syncthreads();
            if (warp == 0) {
                // lane = (candidate, detector): sum over the candidate's warps
                double v = 0.0;
                const int sc = lane / NDET, dd = lane % NDET;
                if (sc < ns && lane < S * NDET) {
                    double ZR = 0.0, ZI = 0.0;
                    for (int w2 = 0; w2 < wpc; w2++) {
                        ZR += part[sc * wpc + w2][0][dd][0];
                        ZI += part[sc * wpc + w2][0][dd][1];
                    }
                    v = coef[sc].gre[dd] * ZR - coef[sc].gim[dd] * ZI;
                }
                const double t = group_sum_down<NDET>(v);
                if (dd == 0 && sc < ns && lane < S * NDET) lval[sc] = t - 0.5 * coef[sc].hh;
            }
        } else if (warp < ns) {
            // one candidate per slot warp: bins and warp reduction
            double v = 0.0;
            if (PREC == 0) {
                double zr[NDET], zi[NDET];
                bins_fp64<NDET, true>(T, M.N, M.f0, M.df, coef[warp], lane, 32, zr, zi);
#pragma unroll
                for (int dd = 0; dd < NDET; dd++) {
                    const double ZR = warp_sum(zr[dd]), ZI = warp_sum(zi[dd]);
                    v += coef[warp].gre[dd] * ZR - coef[warp].gim[dd] * ZI;
                }
            } else if (M.tlg) {
                if (!M.cdf) coef_to_mixed_warp(coef[warp], M.n_det, M.df, &cm[warp], nullptr, form_rot<FORM>(M));
                if (lane == 0) jc[warp] = coef[warp].jcut;
                __syncwarp();
                float zh[1][NDET][2], zl[1][NDET][2];
                tile_bins_form<NDET, 1, FORM>(M, T, &cm[warp], &jc[warp], 1, 0, 1, zh, zl);
                v = warp_detector_terms_df<NDET>(zh[0], zl[0], coef[warp]);
            } else {
                if (!M.cdf) coef_to_mixed_warp(coef[warp], M.n_det, M.df, &cm[warp], nullptr, form_rot<FORM>(M));
                __syncwarp();
                float zh[NDET][2], zl[NDET][2];
                bins_mixed<NDET>(T, M.N, cm[warp], coef[warp].jcut, lane, 32, zh, zl);
                v = warp_detector_terms_df<NDET>(zh, zl, coef[warp]);
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
                c.cy[c.ncache] = (lane < d) ? ysh[sl][lane] : 0.5;
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
            atomicAdd(&A.state->point_bins_lo, c.bins_lo);
            if (A.kernel == 1) atomicAdd(&A.state->walk_acc, (unsigned long long)c.s);
        }
    }
}

// At most 128 registers, so that 512 threads of chains fit on an SM: measured
// on GB300 against the uncapped 168 (3 CTAs of 4 warps per SM), c1 FP64 10.9 ->
// 9.8 ms, c1 mixed 4.7 -> 3.4 ms, c4 mixed 631 -> 550 ms per slice update, in
// spite of ~100 bytes of spills in the mixed tile loop.
#define SLICE_MIN_BLOCKS(PREC, S) (16 / (S))

template <int PREC, int NDET, int S, int W = S>
__global__ void __launch_bounds__(W * 32, SLICE_MIN_BLOCKS(PREC, W)) k_slice(Model M, Tables T, StepArgs A) {
    slice_body<PREC, NDET, S, W>(M, T, A, blockIdx.x);
}

// The work-shared slice update: persistent CTAs (as many as fit on the GPU at
// once) take chains until none is left, then help the running ones.
template <int NDET>
__global__ void __launch_bounds__(256, SLICE_MIN_BLOCKS(1, 8)) k_slice_ws(Model M, Tables T, StepArgs A) {
    __shared__ int s_chain;
    for (int guard = 0; guard < (1 << 20); guard++) {
        if (threadIdx.x == 0) s_chain = atomicAdd(A.chain_ctr, 1);
        __syncthreads();
        const int chain = s_chain;
        __syncthreads();
        if (chain >= A.k) break;
        slice_body<1, NDET, 4, 8, FORM_ROT, true>(M, T, A, chain);
        __syncthreads();
    }
    ws_help<NDET, 8>(M, T, A);
}

// CTAs of the work-shared slice update that fit on one SM (0: not used for
// this precision).
template <int PREC, int NDET>
int slice_ws_blocks_per_sm() {
    if constexpr (PREC == 1) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_slice_ws<NDET>, 256, 0) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return nb;
    } else {
        return 0;
    }
}

template <int PREC, int NDET>
cudaError_t slice_launch(const Model &M, const Tables &T, int slots, const StepArgs &A, cudaStream_t s) {
    // on grids of 262,144 bins or more in tiles of 32 bins or more the tiled
    // mixed form with cooperative bins takes 8 warps for 4 slots: as many warps
    // per SM as 4-warp CTAs, twice as many per chain, so the update's last chains
    // finish sooner (GB300, 519,169 bins: 536 -> 467 ms per slice update; on
    // 64,897 bins, where an evaluation has a few tile groups, 15.2 -> 17.5 ms,
    // hence the threshold)
    if (PREC == 1 && slots == 4 && M.model == M_GW && M.coop && M.tlg >= 5 && !M.rb &&
        M.N >= 262144) {
        if constexpr (PREC == 1) {
            if (A.ws) {
                k_slice_ws<NDET><<<A.ws_nslot, 256, 0, s>>>(M, T, A);
                return cudaGetLastError();
            }
        }
        k_slice<PREC, NDET, 4, 8><<<A.k, 256, 0, s>>>(M, T, A);
        return cudaGetLastError();
    }
    switch (slots) {
        case 1: k_slice<PREC, NDET, 1><<<A.k, 32, 0, s>>>(M, T, A); break;
        case 2: k_slice<PREC, NDET, 2><<<A.k, 64, 0, s>>>(M, T, A); break;
        case 4: k_slice<PREC, NDET, 4><<<A.k, 128, 0, s>>>(M, T, A); break;
        default: k_slice<PREC, NDET, 8><<<A.k, 256, 0, s>>>(M, T, A); break;
    }
    return cudaGetLastError();
}

// Many analyses in one launch (serving), one form of the tiled mixed sums per
// kernel: the direct form for every analysis (FP64, per-bin and short-tile
// grids) or the rotation form for mixed grids with tiles of 32 bins or more.
// A kernel with both forms spilled registers (serving stream p50 4.0 -> 5.8 s).
template <int PREC, int NDET, int S, int FORM>
__global__ void __launch_bounds__(S * 32, SLICE_MIN_BLOCKS(PREC, S)) k_slice_multi(const Desc *D, const int2 *map) {
    __shared__ Desc d;
    const int2 ac = map[blockIdx.x];
    load_desc(D + ac.x, d);
    slice_body<PREC, NDET, S, S, FORM>(d.M, d.T, d.A, ac.y);
}

template <int PREC, int NDET, int FORM>
cudaError_t slice_multi_launch_form(const Desc *D, const int2 *map, int nblocks, int slots, cudaStream_t s) {
    switch (slots) {
        case 1: k_slice_multi<PREC, NDET, 1, FORM><<<nblocks, 32, 0, s>>>(D, map); break;
        case 2: k_slice_multi<PREC, NDET, 2, FORM><<<nblocks, 64, 0, s>>>(D, map); break;
        case 4: k_slice_multi<PREC, NDET, 4, FORM><<<nblocks, 128, 0, s>>>(D, map); break;
        default: k_slice_multi<PREC, NDET, 8, FORM><<<nblocks, 256, 0, s>>>(D, map); break;
    }
    return cudaGetLastError();
}

template <int PREC, int NDET>
cudaError_t slice_multi_launch(const Desc *D, const int2 *map, int nblocks, int slots, int rot, cudaStream_t s) {
    if constexpr (PREC == 1) {
        if (rot) return slice_multi_launch_form<PREC, NDET, FORM_ROT>(D, map, nblocks, slots, s);
    }
    return slice_multi_launch_form<PREC, NDET, FORM_DIRECT>(D, map, nblocks, slots, s);
}

// Explicit instantiation of the launchers of one (precision, detectors) pair.
#define GWNS_INSTANTIATE(P, D)                                                                       \
    template int slice_ws_blocks_per_sm<P, D>();                                                     \
    template cudaError_t eval_launch<P, D>(const Model &, const Tables &, int, const double *, int, int, \
                                           double *, RunState *, cudaStream_t);                     \
    template cudaError_t slice_launch<P, D>(const Model &, const Tables &, int, const StepArgs &,     \
                                            cudaStream_t);                                          \
    template cudaError_t slice_multi_launch<P, D>(const Desc *, const int2 *, int, int, int, cudaStream_t);

}  // namespace gwns
