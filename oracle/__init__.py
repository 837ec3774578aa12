"""Plain FP64 CPU oracle for the nested-slice-sampling hot path.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers. The library never imports
this package, and this package never imports the library: the only shared
module is ``gwinputs`` (seeded raw inputs, no method arithmetic).

The likelihood, waveform, antenna patterns, Philox generator and slice-sampling
chains live in ``gwns_oracle.c`` (plain C, compiled with ``-ffp-contract=off``);
the nested-sampling outer loop (deletion of the k lowest points, evidence
bookkeeping, covariance and Cholesky factor) is in ``oracle/ns.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Optional

import numpy as np

import gwinputs as gi

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gwns_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libgwns_oracle.so")
_lock = threading.Lock()
_lib = None

MODEL_GW, MODEL_TOY = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle's C code (plain gcc, OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(ctypes.Structure):
    _fields_ = [
        ("model", ctypes.c_int),
        ("n_det", ctypes.c_int), ("N", ctypes.c_int),
        ("f0", ctypes.c_double), ("df", ctypes.c_double),
        ("psd", ctypes.c_void_p), ("d_re", ctypes.c_void_p), ("d_im", ctypes.c_void_p),
        ("pos", ctypes.c_void_p), ("xarm", ctypes.c_void_p), ("yarm", ctypes.c_void_p),
        ("ideal", ctypes.c_int), ("cutoff", ctypes.c_int),
        ("kind", ctypes.c_void_p), ("lo", ctypes.c_void_p), ("hi", ctypes.c_void_p),
        ("toy_d", ctypes.c_int), ("toy_prec", ctypes.c_void_p),
        ("toy_lognorm", ctypes.c_double), ("toy_lo", ctypes.c_double), ("toy_hi", ctypes.c_double),
        ("rb_nedge", ctypes.c_int), ("rb_J", ctypes.c_void_p), ("rb_sum", ctypes.c_void_p * 6),
        ("rb_theta_fid", ctypes.c_void_p),
        ("periodic", ctypes.c_uint),
    ]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.POINTER(_Problem)
            dp = ctypes.c_void_p
            L.or_dim.argtypes = [P]; L.or_dim.restype = ctypes.c_int
            L.or_theta_from_u.argtypes = [P, dp, dp]; L.or_theta_from_u.restype = None
            L.or_pn_phi.argtypes = [ctypes.c_double] * 5 + [dp]; L.or_pn_phi.restype = None
            L.or_fisco.argtypes = [dp]; L.or_fisco.restype = ctypes.c_double
            L.or_phase.argtypes = [dp, ctypes.c_double]; L.or_phase.restype = ctypes.c_double
            L.or_amplitude.argtypes = [dp, ctypes.c_double]; L.or_amplitude.restype = ctypes.c_double
            L.or_polarizations.argtypes = [dp, ctypes.c_double, dp, dp]; L.or_polarizations.restype = None
            L.or_antenna.argtypes = [dp, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double, dp, dp]
            L.or_antenna.restype = None
            L.or_delay.argtypes = [dp, ctypes.c_double, ctypes.c_double]; L.or_delay.restype = ctypes.c_double
            L.or_strain.argtypes = [P, dp, ctypes.c_int, dp, dp]; L.or_strain.restype = None
            L.or_inner.argtypes = [P, ctypes.c_int, dp, dp, dp, dp]; L.or_inner.restype = ctypes.c_double
            L.or_loglike_theta.argtypes = [P, dp]; L.or_loglike_theta.restype = ctypes.c_double
            L.or_loglike_u.argtypes = [P, dp]; L.or_loglike_u.restype = ctypes.c_double
            L.or_loglike_batch.argtypes = [P, dp, ctypes.c_int, dp, ctypes.c_int]
            L.or_loglike_batch.restype = None
            L.or_loglike_theta_batch.argtypes = [P, dp, ctypes.c_int, dp, ctypes.c_int]
            L.or_loglike_theta_batch.restype = None
            L.or_philox4x32_10.argtypes = [dp, dp, dp]; L.or_philox4x32_10.restype = None
            L.or_u01.argtypes = [ctypes.c_uint32, ctypes.c_uint32]; L.or_u01.restype = ctypes.c_double
            L.or_initial_points.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_int, dp]
            L.or_initial_points.restype = None
            L.or_replicate_uniform.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_longlong]
            L.or_replicate_uniform.restype = ctypes.c_double
            L.or_replicate_uniforms.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_longlong, dp]
            L.or_replicate_uniforms.restype = None
            L.or_evolve.argtypes = [P, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                    dp, dp, ctypes.c_int, dp, ctypes.c_double, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_int, dp, dp, dp]
            L.or_evolve.restype = ctypes.c_longlong
            L.or_evolve_chains.argtypes = [P, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                           ctypes.c_int, dp, dp, ctypes.c_int, dp, ctypes.c_double,
                                           ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp]
            L.or_evolve_chains.restype = ctypes.c_longlong
            L.or_evolve_walk.argtypes = [P, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                         dp, dp, ctypes.c_int, dp, ctypes.c_double, ctypes.c_int,
                                         ctypes.c_double, dp, dp, dp]
            L.or_evolve_walk.restype = ctypes.c_longlong
            L.or_walk_next.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_longlong]
            L.or_walk_next.restype = ctypes.c_int
            L.or_max_threads.argtypes = []; L.or_max_threads.restype = ctypes.c_int
            L.or_rb_edges.argtypes = [P, ctypes.c_int, dp]; L.or_rb_edges.restype = ctypes.c_int
            L.or_rb_summary.argtypes = [P, dp, dp, ctypes.c_int] + [dp] * 6
            L.or_rb_summary.restype = None
            L.or_loglike_rb.argtypes = [P, dp, dp, ctypes.c_int] + [dp] * 6 + [dp]
            L.or_loglike_rb.restype = ctypes.c_double
            _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


class Problem:
    """A GW (or toy) likelihood problem as the oracle sees it.

    Arrays are held here so that the C structure's pointers stay valid."""

    def __init__(self, *, model=MODEL_GW, f0=0.0, df=1.0, psd=None, data=None, pos=None,
                 xarm=None, yarm=None, ideal=False, cutoff=True, kind=None, lo=None, hi=None,
                 toy_d=0, toy_rho=gi.TOY_RHO):
        self.model = model
        self.cutoff = bool(cutoff)
        self.ideal = bool(ideal)
        if model == MODEL_GW:
            self.psd = _f64(psd)
            self.n_det, self.N = self.psd.shape
            data = np.asarray(data, dtype=np.complex128).reshape(self.n_det, self.N)
            self.d_re = _f64(data.real)
            self.d_im = _f64(data.imag)
            self.pos = _f64(pos if pos is not None else np.zeros((self.n_det, 3)))
            self.xarm = _f64(xarm if xarm is not None else np.zeros((self.n_det, 3)))
            self.yarm = _f64(yarm if yarm is not None else np.zeros((self.n_det, 3)))
            self.kind = np.ascontiguousarray(np.asarray(kind, dtype=np.int32))
            self.lo = _f64(lo)
            self.hi = _f64(hi)
            self.f0, self.df = float(f0), float(df)
            self.toy_prec = _f64(np.zeros(1))
            self.toy_d = 0
            self.toy_lognorm = 0.0
        else:
            self.n_det, self.N, self.f0, self.df = 0, 0, 0.0, 1.0
            self.psd = self.d_re = self.d_im = self.pos = self.xarm = self.yarm = _f64(np.zeros(1))
            self.kind = np.zeros(gi.NPARAM, dtype=np.int32)
            self.lo = self.hi = _f64(np.zeros(gi.NPARAM))
            sigma = gi.toy_covariance(toy_d, toy_rho)
            self.toy_d = int(toy_d)
            self.toy_prec = _f64(np.linalg.inv(sigma))
            sign, logdet = np.linalg.slogdet(2.0 * np.pi * sigma)
            self.toy_lognorm = -0.5 * logdet
        self._c = _Problem(
            model, self.n_det, self.N, self.f0, self.df, _ptr(self.psd), _ptr(self.d_re),
            _ptr(self.d_im), _ptr(self.pos), _ptr(self.xarm), _ptr(self.yarm), int(self.ideal),
            int(self.cutoff), _ptr(self.kind), _ptr(self.lo), _ptr(self.hi), self.toy_d,
            _ptr(self.toy_prec), self.toy_lognorm, gi.TOY_BOX[0], gi.TOY_BOX[1])

    @property
    def c(self):
        return ctypes.byref(self._c)

    def set_periodic(self, params) -> int:
        """Mark parameters as periodic (indices in gwinputs' parameter order; for
        the toy model, unit-cube coordinates): their unit-cube coordinates wrap
        mod 1 on the slice line instead of leaving the prior box. Returns the
        mask over unit-cube coordinates."""
        params = set(int(p) for p in params)
        mask = 0
        if self.model == MODEL_TOY:
            for i in params:
                mask |= 1 << i
        else:
            i = 0
            for p in range(gi.NPARAM):
                if int(self.kind[p]) == gi.PRIOR_FIXED:
                    continue
                if p in params:
                    mask |= 1 << i
                i += 1
        self._c.periodic = mask
        return mask

    @property
    def dim(self) -> int:
        return int(lib().or_dim(self.c))

    def data(self) -> np.ndarray:
        return self.d_re + 1j * self.d_im

    # -- likelihood --------------------------------------------------------
    def theta(self, u) -> np.ndarray:
        u = _f64(np.atleast_2d(u))
        out = np.zeros((u.shape[0], gi.NPARAM))
        for i in range(u.shape[0]):
            lib().or_theta_from_u(self.c, _ptr(u[i]), _ptr(out[i]))
        return out

    def loglike(self, u, nthreads: Optional[int] = None) -> np.ndarray:
        u = _f64(np.atleast_2d(u))
        out = np.zeros(u.shape[0])
        nt = nthreads if nthreads else lib().or_max_threads()
        lib().or_loglike_batch(self.c, _ptr(u), u.shape[0], _ptr(out), nt)
        return out

    def loglike_theta(self, theta, nthreads: Optional[int] = None) -> np.ndarray:
        th = _f64(np.atleast_2d(theta))
        out = np.zeros(th.shape[0])
        nt = nthreads if nthreads else lib().or_max_threads()
        lib().or_loglike_theta_batch(self.c, _ptr(th), th.shape[0], _ptr(out), nt)
        return out

    def strain(self, theta, det: int) -> np.ndarray:
        th = _f64(theta)
        re = np.zeros(self.N)
        im = np.zeros(self.N)
        lib().or_strain(self.c, _ptr(th), det, _ptr(re), _ptr(im))
        return re + 1j * im

    def inner(self, det: int, a, b) -> float:
        a = np.asarray(a, dtype=np.complex128)
        b = np.asarray(b, dtype=np.complex128)
        ar, ai, br, bi = _f64(a.real), _f64(a.imag), _f64(b.real), _f64(b.imag)
        return float(lib().or_inner(self.c, det, _ptr(ar), _ptr(ai), _ptr(br), _ptr(bi)))

    def snr2(self, theta) -> float:
        """Network optimal SNR^2 = sum_d <h_d|h_d>."""
        return sum(self.inner(d, self.strain(theta, d), self.strain(theta, d)) for d in range(self.n_det))


# -- single-quantity helpers (used by the pins) ------------------------------
def pn_phi(eta, delta, chi1, chi2, v) -> np.ndarray:
    out = np.zeros(8)
    lib().or_pn_phi(float(eta), float(delta), float(chi1), float(chi2), float(v), _ptr(out))
    return out


def phase(theta, f) -> float:
    return float(lib().or_phase(_ptr(_f64(theta)), float(f)))


def amplitude(theta, f) -> float:
    return float(lib().or_amplitude(_ptr(_f64(theta)), float(f)))


def fisco(theta) -> float:
    return float(lib().or_fisco(_ptr(_f64(theta))))


def polarizations(theta, f):
    hp = np.zeros(2)
    hc = np.zeros(2)
    lib().or_polarizations(_ptr(_f64(theta)), float(f), _ptr(hp), _ptr(hc))
    return complex(hp[0], hp[1]), complex(hc[0], hc[1])


def antenna(xarm, yarm, ra, sindec, psi):
    fp = np.zeros(1)
    fc = np.zeros(1)
    lib().or_antenna(_ptr(_f64(xarm)), _ptr(_f64(yarm)), float(ra), float(sindec), float(psi),
                     _ptr(fp), _ptr(fc))
    return float(fp[0]), float(fc[0])


def delay(pos, ra, sindec) -> float:
    return float(lib().or_delay(_ptr(_f64(pos)), float(ra), float(sindec)))


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def u01(a: int, b: int) -> float:
    return float(lib().or_u01(a, b))


def initial_points(seed: int, n: int, d: int) -> np.ndarray:
    out = np.zeros((n, d))
    lib().or_initial_points(seed, n, d, _ptr(out))
    return out


def replicate_uniform(seed: int, replicate: int, dead_index: int) -> float:
    return float(lib().or_replicate_uniform(seed, replicate, dead_index))


def replicate_uniforms(seed: int, replicate: int, m: int) -> np.ndarray:
    out = np.zeros(m)
    lib().or_replicate_uniforms(seed, replicate, m, _ptr(out))
    return out


def max_threads() -> int:
    return int(lib().or_max_threads())


# -- building an analysis from a workload -------------------------------------
def make_problem(w: gi.Workload, *, cutoff: bool = True, max_draws: int = 1000):
    """Build the synthetic analysis of a workload with the oracle's waveform.

    Returns (problem, theta_inj). The data are noise (if the workload has
    noise) plus the injected signal; the injection's distance is rescaled so
    that the network optimal SNR equals w.snr (c0: the fixed distance itself is
    set that way)."""
    f = w.freqs()
    psd = np.tile(gi.psd_analytic(f), (w.n_det, 1))
    if w.ideal:
        pos = xarm = yarm = np.zeros((w.n_det, 3))
    else:
        pos, xarm, yarm = gi.detectors(w.seed_geometry, w.n_det)
    kind, lo, hi = w.kind.copy(), w.lo.copy(), w.hi.copy()
    zero = np.zeros((w.n_det, w.N), dtype=np.complex128)
    tmp = Problem(f0=w.f0, df=w.df, psd=psd, data=zero, pos=pos, xarm=xarm, yarm=yarm,
                  ideal=w.ideal, cutoff=cutoff, kind=kind, lo=lo, hi=hi)
    if w.fixed_injection is not None:
        th = w.fixed_injection.copy()
        rho = np.sqrt(tmp.snr2(th))
        th[gi.P_DL] *= rho / w.snr
        if w.dl_from_snr:
            lo[gi.P_DL] = hi[gi.P_DL] = th[gi.P_DL]
    else:
        cands = gi.unit_cube(w.seed_injection, max_draws, tmp.dim)
        th = None
        for u in cands:
            t = tmp.theta(u)[0]
            rho = np.sqrt(tmp.snr2(t))
            dl = t[gi.P_DL] * rho / w.snr
            if lo[gi.P_DL] <= dl <= hi[gi.P_DL]:
                t[gi.P_DL] = dl
                th = t
                break
        if th is None:
            raise RuntimeError("no injection candidate reaches the target SNR inside the prior")
    signal = np.stack([tmp.strain(th, d) for d in range(w.n_det)])
    data = signal.copy()
    if w.noise:
        data = data + gi.noise(w.seed_noise, psd, w.df)
    pb = Problem(f0=w.f0, df=w.df, psd=psd, data=data, pos=pos, xarm=xarm, yarm=yarm,
                 ideal=w.ideal, cutoff=cutoff, kind=kind, lo=lo, hi=hi)
    return pb, th


class RelativeBinning:
    """Relative-binning (heterodyned) likelihood of a problem about a fiducial
    parameter vector, on B geometric coarse bins."""

    def __init__(self, problem: Problem, theta_fid, B: int = 1024):
        self.pb = problem
        self.theta_fid = _f64(theta_fid)
        J = np.zeros(B + 1, dtype=np.int32)
        ne = lib().or_rb_edges(problem.c, B, _ptr(J))
        self.J = np.ascontiguousarray(J[:ne])
        nb = ne - 1
        nd = problem.n_det
        self.sums = [np.zeros(nd * nb) for _ in range(6)]
        lib().or_rb_summary(problem.c, _ptr(self.theta_fid), _ptr(self.J), ne,
                            *[_ptr(a) for a in self.sums])

    @property
    def n_bins(self) -> int:
        return len(self.J) - 1

    def loglike_theta(self, theta) -> np.ndarray:
        th = _f64(np.atleast_2d(theta))
        return np.array([lib().or_loglike_rb(self.pb.c, _ptr(self.theta_fid), _ptr(self.J), len(self.J),
                                             *[_ptr(a) for a in self.sums], _ptr(_f64(t))) for t in th])

    def loglike(self, u) -> np.ndarray:
        return self.loglike_theta(self.pb.theta(u))

    def problem(self) -> "Problem":
        """A copy of the problem whose likelihood (batched, and inside the
        sampler's chains) is this relative-binning one."""
        pb = self.pb
        q = Problem(f0=pb.f0, df=pb.df, psd=pb.psd, data=pb.data(), pos=pb.pos, xarm=pb.xarm,
                    yarm=pb.yarm, ideal=pb.ideal, cutoff=pb.cutoff, kind=pb.kind, lo=pb.lo, hi=pb.hi)
        q._rb = self
        q._c.rb_nedge = len(self.J)
        q._c.rb_J = _ptr(self.J)
        for i in range(6):
            q._c.rb_sum[i] = _ptr(self.sums[i])
        q._c.rb_theta_fid = _ptr(self.theta_fid)
        return q


def toy_problem(d: int) -> Problem:
    return Problem(model=MODEL_TOY, toy_d=d)
