"""Nested-sampling outer loop of the oracle (TEST INFRASTRUCTURE ONLY).

One iteration (paper Sec. 2: classic nested sampling with a vectorised slice
sampling update, deleting k of the n live points per iteration), written in
the order the method takes its steps:

1. sort the live log-likelihoods ascending (ties by index); the k lowest die,
   and the threshold L* is the k-th lowest value;
2. evidence bookkeeping for the dead points in ascending order: with
   Delta_j = 1/(n-j+1), log w_j = log X + log(1 - exp(-Delta_j)),
   log X -= Delta_j, log Z = logaddexp(log Z, log L_j + log w_j)
   (the expected log-shrinkage of removing the j-th point of n-j+1);
3. mean and covariance of the n-k survivors in unit-cube coordinates, with a
   jittered Cholesky factor (paper Sec. 2: the particle covariance tunes the
   direction proposals);
4. k independent slice-sampling chains (C code), each started at a uniformly
   chosen survivor, replace the dead points in place (static memory);
5. stop once log(Z + X max L_live) - log Z < dlogz.

The final live points are then added in ascending order with the same
Delta_j = 1/(n-j+1) rule. dlogZ is the standard deviation of log Z over
replicate runs whose shrinkage factors are redrawn, t ~ Beta(n_j, 1); the
information H gives the secondary estimate sqrt(H/n). ESS is Kish's
(sum w)^2 / sum w^2.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

from . import initial_points, lib, replicate_uniforms, _ptr, _f64


@dataclasses.dataclass
class NSState:
    live_u: np.ndarray      # [n, d]
    live_logl: np.ndarray   # [n]
    logX: float = 0.0
    logZ: float = -math.inf
    it: int = 0
    evals: int = 0
    caps: int = 0
    walk_len: int = 0       # random-walk kernel: proposals per walk this iteration (0: not set yet)
    dead_u: List[np.ndarray] = dataclasses.field(default_factory=list)
    dead_logl: List[np.ndarray] = dataclasses.field(default_factory=list)
    dead_logw: List[np.ndarray] = dataclasses.field(default_factory=list)
    dead_nlive: List[np.ndarray] = dataclasses.field(default_factory=list)


def initial_state(problem, n_live: int, seed: int, nthreads: Optional[int] = None) -> NSState:
    u = initial_points(seed, n_live, problem.dim)
    return NSState(live_u=u, live_logl=problem.loglike(u, nthreads), evals=n_live)


def survivor_cholesky(surv_u: np.ndarray) -> np.ndarray:
    """Cholesky factor of the survivors' covariance (unbiased, 1/(m-1)),
    jittered by 1e-12 tr(Sigma)/d on the diagonal; diag(sqrt(Sigma_ii)) if the
    factorisation fails. A single survivor (k = n - 1) has no sample
    covariance: the unit cube's prior covariance I/12 stands in (reading; the
    paper deletes half the population)."""
    m, d = surv_u.shape
    if m < 2:
        sigma = np.eye(d) / 12.0
        sigma = sigma + 1e-12 * np.trace(sigma) / d * np.eye(d)
        return np.linalg.cholesky(sigma)
    mu = surv_u.mean(axis=0)
    xc = surv_u - mu
    sigma = xc.T @ xc / (m - 1)
    sigma = sigma + 1e-12 * np.trace(sigma) / d * np.eye(d)
    try:
        return np.linalg.cholesky(sigma)
    except np.linalg.LinAlgError:
        return np.diag(np.sqrt(np.maximum(np.diag(sigma), 0.0)))


def walk_scale_default(d: int) -> float:
    """Random-walk proposal scale on top of the survivors' Cholesky factor:
    2.38 / sqrt(d) (Roberts, Gelman and Gilks 1997)."""
    return 2.38 / math.sqrt(d)


def iterate(problem, st: NSState, k: int, steps: int, seed: int, *, max_stepout: int = 64,
            max_shrink: int = 64, nthreads: Optional[int] = None, kernel: str = "slice",
            walk_scale: Optional[float] = None) -> dict:
    """One nested-sampling iteration in place on st. Returns its details."""
    n, d = st.live_u.shape
    order = np.argsort(st.live_logl, kind="stable")       # ascending, ties by index
    dead = order[:k]
    surv = order[k:]
    lstar = float(st.live_logl[order[k - 1]])
    logw = np.zeros(k)
    for j in range(1, k + 1):
        delta = 1.0 / (n - j + 1)
        logw[j - 1] = st.logX + math.log(-math.expm1(-delta))
        st.logX -= delta
        st.logZ = float(np.logaddexp(st.logZ, st.live_logl[dead[j - 1]] + logw[j - 1]))
    st.dead_u.append(st.live_u[dead].copy())
    st.dead_logl.append(st.live_logl[dead].copy())
    st.dead_logw.append(logw)
    st.dead_nlive.append(n - np.arange(k, dtype=np.float64))

    surv_u = _f64(st.live_u[surv])
    surv_logl = _f64(st.live_logl[surv])
    chol = _f64(survivor_cholesky(surv_u))
    new_u = np.zeros((k, d))
    new_logl = np.zeros(k)
    caps = np.zeros(1, dtype=np.int32)
    nt = nthreads if nthreads else lib().or_max_threads()
    if kernel == "walk":
        # walks of fixed length within the iteration (first: 2 x the target of
        # `steps` accepted moves), rescaled between iterations
        scale = walk_scale if walk_scale else walk_scale_default(d)
        if st.walk_len == 0:
            st.walk_len = 2 * steps
        acc = np.zeros(1, dtype=np.int64)
        ev = lib().or_evolve_walk(problem.c, nt, seed, st.it, k, _ptr(surv_u), _ptr(surv_logl),
                                  n - k, _ptr(chol), lstar, st.walk_len, scale,
                                  _ptr(new_u), _ptr(new_logl), _ptr(acc))
        st.walk_len = int(lib().or_walk_next(st.walk_len, steps, k, int(acc[0])))
    else:
        ev = lib().or_evolve(problem.c, nt, seed, st.it, k, _ptr(surv_u), _ptr(surv_logl),
                             n - k, _ptr(chol), lstar, steps, max_stepout, max_shrink,
                             _ptr(new_u), _ptr(new_logl), _ptr(caps))
    st.live_u[dead] = new_u
    st.live_logl[dead] = new_logl
    st.evals += int(ev)
    st.caps += int(caps[0])
    st.it += 1
    return dict(lstar=lstar, dead=dead, chol=chol, new_u=new_u, new_logl=new_logl, evals=int(ev))


def remaining_fraction(st: NSState) -> float:
    """log(Z + X max L_live) - log Z."""
    lmax = float(np.max(st.live_logl))
    return float(np.logaddexp(st.logZ, st.logX + lmax) - st.logZ)


def finalize(st: NSState, seed: int, replicates: int = 200) -> dict:
    n, d = st.live_u.shape
    order = np.argsort(st.live_logl, kind="stable")
    logX = st.logX
    logZ = st.logZ
    logw = np.zeros(n)
    for j in range(1, n + 1):
        delta = 1.0 / (n - j + 1)
        logw[j - 1] = logX + math.log(-math.expm1(-delta))
        logX -= delta
        logZ = float(np.logaddexp(logZ, st.live_logl[order[j - 1]] + logw[j - 1]))
    all_u = np.concatenate(st.dead_u + [st.live_u[order]]) if st.dead_u else st.live_u[order]
    all_logl = np.concatenate(st.dead_logl + [st.live_logl[order]])
    all_logw = np.concatenate(st.dead_logw + [logw])
    all_nlive = np.concatenate(st.dead_nlive + [n - np.arange(n, dtype=np.float64)])
    # information and Kish ESS
    logp = all_logw + all_logl - logZ
    p = np.exp(logp)
    H = float(np.sum(p * (all_logl - logZ)))
    ess = float(np.sum(p) ** 2 / np.sum(p ** 2))
    # replicate shrinkage draws: log t_i = log(U)/n_i
    m = all_logl.shape[0]
    reps = np.zeros(replicates)
    for r in range(replicates):
        U = replicate_uniforms(seed, r, m)
        logt = np.log(U) / all_nlive
        logx = np.cumsum(logt)
        logx_prev = np.concatenate([[0.0], logx[:-1]])
        lw = logx_prev + np.log(-np.expm1(logt))
        a = lw + all_logl
        amax = np.max(a)
        reps[r] = amax + math.log(np.sum(np.exp(a - amax)))
    return dict(logZ=logZ, dlogZ=float(np.std(reps)), dlogZ_info=math.sqrt(max(H, 0.0) / n),
                H=H, ess=ess, samples_u=all_u, logl=all_logl, logw=all_logw, nlive=all_nlive,
                replicates=reps)


def run(problem, *, n_live: int, k: int, steps: int, seed: int, dlogz: float = 0.1,
        max_iter: int = 100000, max_stepout: int = 64, max_shrink: int = 64,
        nthreads: Optional[int] = None, replicates: int = 200, kernel: str = "slice",
        walk_scale: Optional[float] = None) -> dict:
    """Full nested-sampling run; returns the finalize() dict plus counters."""
    st = initial_state(problem, n_live, seed, nthreads)
    while st.it < max_iter:
        iterate(problem, st, k, steps, seed, max_stepout=max_stepout, max_shrink=max_shrink,
                nthreads=nthreads, kernel=kernel, walk_scale=walk_scale)
        if remaining_fraction(st) < dlogz:
            break
    res = finalize(st, seed, replicates)
    res.update(iterations=st.it, evals=st.evals, caps=st.caps)
    return res


def equal_weight_resample(samples: np.ndarray, logw_post: np.ndarray, seed: int) -> np.ndarray:
    """Systematic resampling to equal-weight samples (post-processing)."""
    p = np.exp(logw_post - np.max(logw_post))
    p /= p.sum()
    n = int(round(1.0 / np.sum(p ** 2)))
    rng = np.random.default_rng(seed)
    pos = (rng.random() + np.arange(n)) / n
    idx = np.searchsorted(np.cumsum(p), pos)
    idx = np.minimum(idx, len(p) - 1)
    return samples[idx]
