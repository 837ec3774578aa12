"""Python binding of libgwns.so (the C ABI in include/gwns.h).

Argument marshalling only: every step of the likelihood and of the nested
sampling iteration runs in the library's CUDA kernels. Importing this package
loads the in-tree shared library and raises if it has not been built
(``python -c "import __graft_entry__ as g; g.build()"``); there is no CPU path.
PyTorch is used only for device buffers (tensor ``data_ptr()``) and streams.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import _build

_LIB = None

NS_OK = 0
NS_FP64, NS_MIXED = 0, 1
NS_MODEL_GW, NS_MODEL_TOY = 0, 1
NS_KERNEL_SLICE, NS_KERNEL_WALK = 0, 1
NPARAM = 11
NS_MAX_DET = 4
NOALLOC_MAX_POINTS = 4096


class GWNSError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {lib().ns_strerror(code).decode()} ({code})")


class _Prior(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int * NPARAM), ("lo", ctypes.c_double * NPARAM),
                ("hi", ctypes.c_double * NPARAM)]


class _Data(ctypes.Structure):
    _fields_ = [("n_det", ctypes.c_int), ("ideal", ctypes.c_int), ("re", ctypes.c_void_p),
                ("im", ctypes.c_void_p), ("pos", ctypes.c_void_p), ("xarm", ctypes.c_void_p),
                ("yarm", ctypes.c_void_p)]


class _Psd(ctypes.Structure):
    _fields_ = [("S", ctypes.c_void_p)]


class _Grid(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("f0", ctypes.c_double), ("df", ctypes.c_double),
                ("coarse_bins", ctypes.c_int), ("theta_fid", ctypes.c_void_p)]


class _Options(ctypes.Structure):
    _fields_ = [("n_live", ctypes.c_int), ("k", ctypes.c_int), ("steps_per_dim", ctypes.c_int),
                ("precision", ctypes.c_int), ("no_cutoff", ctypes.c_int),
                ("max_stepout", ctypes.c_int), ("max_shrink", ctypes.c_int),
                ("model", ctypes.c_int), ("toy_dim", ctypes.c_int),
                ("warps_per_point", ctypes.c_int), ("slots", ctypes.c_int),
                ("dlogz_stop", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("stream", ctypes.c_void_p), ("kernel", ctypes.c_int),
                ("walk_scale", ctypes.c_double), ("periodic", ctypes.c_uint)]


class _Samples(ctypes.Structure):
    _fields_ = [("cap", ctypes.c_int), ("count", ctypes.c_int), ("theta", ctypes.c_void_p),
                ("u", ctypes.c_void_p), ("logl", ctypes.c_void_p), ("logw", ctypes.c_void_p)]


class _Stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_longlong), ("evals", ctypes.c_longlong),
                ("cap_hits", ctypes.c_longlong), ("logZ", ctypes.c_double),
                ("logX", ctypes.c_double), ("lstar", ctypes.c_double),
                ("logl_max", ctypes.c_double), ("done", ctypes.c_int), ("d", ctypes.c_int),
                ("n_live", ctypes.c_int), ("n_dead", ctypes.c_int), ("point_bins", ctypes.c_longlong),
                ("status", ctypes.c_int), ("kernel_ms", ctypes.c_double * 5), ("mixed_tile", ctypes.c_int),
                ("batch_evals", ctypes.c_longlong), ("batch_point_bins", ctypes.c_longlong),
                ("scratch_bytes", ctypes.c_longlong),
                ("point_bins_lo", ctypes.c_longlong), ("batch_point_bins_lo", ctypes.c_longlong)]


class _ServerOptions(ctypes.Structure):
    _fields_ = [("max_active", ctypes.c_int), ("mem_budget", ctypes.c_size_t), ("precision", ctypes.c_int),
                ("slots", ctypes.c_int), ("max_iter", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("max_chains", ctypes.c_int)]


class _Request(ctypes.Structure):
    _fields_ = [("prior", _Prior), ("data", _Data), ("psd", _Psd), ("grid", _Grid), ("opts", _Options)]


class _ReqStatus(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int), ("logZ", ctypes.c_double), ("dlogZ", ctypes.c_double),
                ("iterations", ctypes.c_longlong), ("evals", ctypes.c_longlong),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
                ("footprint", ctypes.c_size_t), ("n_samples", ctypes.c_int)]


NS_REQ_PENDING, NS_REQ_RUNNING, NS_REQ_DONE, NS_REQ_CANCELLED = 0, 1, 2, 3


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libgwns.so (raises if it was not built)."""
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise ImportError(f"libgwns.so is not built ({path}); run __graft_entry__.build()")
        L = ctypes.CDLL(path)
        vp, ip, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        P = ctypes.POINTER
        L.ns_strerror.argtypes = [ip]; L.ns_strerror.restype = ctypes.c_char_p
        L.ns_init.argtypes = [P(vp), P(_Prior), P(_Data), P(_Psd), P(_Grid), P(_Options)]
        L.ns_set_data.argtypes = [vp, vp, vp]
        L.ns_step.argtypes = [vp, ip, P(ip)]
        L.ns_step_host.argtypes = [vp, ip, P(ip), vp, vp, vp]
        L.ns_run.argtypes = [vp, ip, P(ip)]
        L.ns_result.argtypes = [vp, P(dp), P(dp), P(_Samples)]
        L.ns_get_stats.argtypes = [vp, P(_Stats)]
        L.ns_result_info.argtypes = [vp, P(dp), P(dp)]
        L.ns_eval_lnl.argtypes = [vp, vp, ip, vp]
        L.ns_eval_lnl_host.argtypes = [vp, vp, ip, vp]
        L.ns_eval_lnl_theta.argtypes = [vp, vp, ip, vp]
        L.ns_eval_lnl_host_noalloc.argtypes = [vp, vp, ip, vp]
        L.ns_waveform.argtypes = [vp, vp, vp, vp]
        L.ns_prior_transform.argtypes = [vp, vp, ip, vp]
        L.ns_optimal_snr2.argtypes = [vp, vp, P(dp)]
        L.ns_get_live.argtypes = [vp, vp, vp]
        L.ns_set_live.argtypes = [vp, vp, vp]
        L.ns_sync.argtypes = [vp]
        L.ns_autotune.argtypes = [vp, ip, P(ip)]
        L.ns_autotune_eval.argtypes = [vp, ip, P(ip)]
        L.ns_checkpoint.argtypes = [vp, vp, P(ctypes.c_size_t)]
        L.ns_restore.argtypes = [vp, vp, ctypes.c_size_t]
        L.ns_free.argtypes = [vp]; L.ns_free.restype = None
        L.ns_server_create.argtypes = [P(vp), P(_ServerOptions)]
        L.ns_submit.argtypes = [vp, P(_Request), P(ctypes.c_uint64)]
        L.ns_server_tick.argtypes = [vp, P(ip), P(ip)]
        L.ns_poll.argtypes = [vp, ctypes.c_uint64, P(_ReqStatus)]
        L.ns_server_result.argtypes = [vp, ctypes.c_uint64, P(_Samples)]
        L.ns_cancel.argtypes = [vp, ctypes.c_uint64]
        L.ns_server_time.argtypes = [vp]; L.ns_server_time.restype = ctypes.c_double
        L.ns_server_free.argtypes = [vp]; L.ns_server_free.restype = None
        for name in ("ns_server_create", "ns_submit", "ns_server_tick", "ns_poll", "ns_server_result",
                     "ns_cancel"):
            getattr(L, name).restype = ctypes.c_int
        for name in ("ns_init", "ns_set_data", "ns_step", "ns_step_host", "ns_run", "ns_result",
                     "ns_get_stats", "ns_eval_lnl", "ns_eval_lnl_host", "ns_eval_lnl_theta",
                     "ns_eval_lnl_host_noalloc",
                     "ns_waveform", "ns_prior_transform", "ns_optimal_snr2", "ns_get_live", "ns_set_live", "ns_sync",
                     "ns_autotune", "ns_autotune_eval", "ns_checkpoint", "ns_restore"):
            getattr(L, name).restype = ctypes.c_int
        _LIB = L
    return _LIB


def _check(rc: int, what: str):
    if rc != NS_OK:
        raise GWNSError(rc, what)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


class Sampler:
    """One nested-sampling context (ns_init .. ns_free)."""

    def __init__(self, *, kind=None, lo=None, hi=None, data=None, psd=None, f0=20.0, df=1.0,
                 pos=None, xarm=None, yarm=None, ideal=False, n_live=100, k=0, steps_per_dim=5,
                 precision=NS_FP64, no_cutoff=False, max_stepout=0, max_shrink=0,
                 model=NS_MODEL_GW, toy_dim=0, warps_per_point=0, slots=0, dlogz_stop=0.1, seed=0,
                 stream=None, coarse_bins=0, theta_fid=None, periodic=(), kernel=0, walk_scale=0.0):
        """periodic: parameter indices (NS_* order; toy model: unit-cube
        coordinates) whose coordinates wrap mod 1 on the slice line."""
        L = lib()
        self._keep = []
        pr = _Prior()
        dt = _Data()
        ps = _Psd()
        gr = _Grid()
        if model == NS_MODEL_GW:
            kind = np.asarray(kind, dtype=np.int32)
            for p in range(NPARAM):
                pr.kind[p] = int(kind[p])
                pr.lo[p] = float(lo[p])
                pr.hi[p] = float(hi[p])
            psd = _f64(psd)
            n_det, N = psd.shape
            self._keep.append(psd)
            ps.S = _ptr(psd)
            dt.n_det = n_det
            dt.ideal = int(bool(ideal))
            if data is not None:
                data = np.asarray(data, dtype=np.complex128).reshape(n_det, N)
                re, im = _f64(data.real), _f64(data.imag)
                self._keep += [re, im]
                dt.re, dt.im = _ptr(re), _ptr(im)
            if not ideal:
                arrs = [_f64(pos).reshape(n_det, 3), _f64(xarm).reshape(n_det, 3), _f64(yarm).reshape(n_det, 3)]
                self._keep += arrs
                dt.pos, dt.xarm, dt.yarm = (_ptr(a) for a in arrs)
            gr.N, gr.f0, gr.df = N, float(f0), float(df)
            if coarse_bins:
                tf = _f64(theta_fid)
                self._keep.append(tf)
                gr.coarse_bins, gr.theta_fid = int(coarse_bins), _ptr(tf)
            self.n_det, self.N = n_det, N
        else:
            self.n_det, self.N = 0, 0
        opt = _Options(n_live, k, steps_per_dim, precision, int(bool(no_cutoff)), max_stepout,
                       max_shrink, model, toy_dim, warps_per_point, slots, dlogz_stop, seed,
                       None if stream is None else int(stream), int(kernel), float(walk_scale),
                       sum(1 << int(p) for p in set(periodic)))
        ctx = ctypes.c_void_p()
        _check(L.ns_init(ctypes.byref(ctx), ctypes.byref(pr), ctypes.byref(dt), ctypes.byref(ps),
                         ctypes.byref(gr), ctypes.byref(opt)), "ns_init")
        self._ctx = ctx
        self._keep = []
        self.n_live = n_live
        self.k = k if k else n_live // 2
        self.precision = precision
        self.model = model
        st = self.stats()
        self.dim = st["d"]

    # ------------------------------------------------------------ lifetime
    def close(self):
        if getattr(self, "_ctx", None):
            lib().ns_free(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------ sampling
    def set_data(self, data):
        data = np.asarray(data, dtype=np.complex128).reshape(self.n_det, self.N)
        re, im = _f64(data.real), _f64(data.imag)
        _check(lib().ns_set_data(self._ctx, _ptr(re), _ptr(im)), "ns_set_data")

    def step(self, k: Optional[int] = None) -> bool:
        done = ctypes.c_int(0)
        _check(lib().ns_step(self._ctx, int(k if k else self.k), ctypes.byref(done)), "ns_step")
        return bool(done.value)

    def step_host(self, k: Optional[int] = None, out_u=None, out_logl=None, out_logw=None) -> bool:
        done = ctypes.c_int(0)
        _check(lib().ns_step_host(self._ctx, int(k if k else self.k), ctypes.byref(done), _ptr(out_u),
                                  _ptr(out_logl), _ptr(out_logw)), "ns_step_host")
        return bool(done.value)

    def run(self, max_iter: int = 100000) -> int:
        it = ctypes.c_int(0)
        _check(lib().ns_run(self._ctx, max_iter, ctypes.byref(it)), "ns_run")
        return it.value

    def stats(self) -> dict:
        s = _Stats()
        _check(lib().ns_get_stats(self._ctx, ctypes.byref(s)), "ns_get_stats")
        out = {name: getattr(s, name) for name, _ in _Stats._fields_}
        out["kernel_ms"] = list(s.kernel_ms)
        return out

    def result(self, samples: bool = True) -> dict:
        lz, dlz = ctypes.c_double(), ctypes.c_double()
        if not samples:
            _check(lib().ns_result(self._ctx, ctypes.byref(lz), ctypes.byref(dlz), None), "ns_result")
            return dict(logZ=lz.value, dlogZ=dlz.value, **self._info())
        st = self.stats()
        cap = st["n_dead"] + self.n_live
        u = np.zeros((cap, self.dim))
        logl = np.zeros(cap)
        logw = np.zeros(cap)
        theta = np.zeros((cap, NPARAM)) if self.model == NS_MODEL_GW else None
        sm = _Samples(cap, 0, _ptr(theta), _ptr(u), _ptr(logl), _ptr(logw))
        _check(lib().ns_result(self._ctx, ctypes.byref(lz), ctypes.byref(dlz), ctypes.byref(sm)), "ns_result")
        out = dict(logZ=lz.value, dlogZ=dlz.value, u=u, logl=logl, logw=logw, count=sm.count, **self._info())
        if theta is not None:
            out["theta"] = theta
        return out

    def _info(self) -> dict:
        h, e = ctypes.c_double(), ctypes.c_double()
        _check(lib().ns_result_info(self._ctx, ctypes.byref(h), ctypes.byref(e)), "ns_result_info")
        return dict(H=h.value, ess=e.value)

    # ---------------------------------------------------------- likelihood
    def eval_lnl(self, u, out=None):
        """Device batched log L: u is a CUDA float64 tensor [m, d] (or a host array)."""
        if isinstance(u, np.ndarray):
            u = _f64(u).reshape(-1, self.dim)
            res = np.zeros(u.shape[0])
            _check(lib().ns_eval_lnl_host(self._ctx, _ptr(u), u.shape[0], _ptr(res)), "ns_eval_lnl_host")
            return res
        import torch
        assert u.is_cuda and u.dtype == torch.float64 and u.is_contiguous()
        m = u.shape[0]
        if out is None:
            out = torch.empty(m, dtype=torch.float64, device=u.device)
        # order torch's producers before the library's stream, and the
        # library's writes before torch's consumers
        torch.cuda.current_stream(u.device).synchronize()
        _check(lib().ns_eval_lnl(self._ctx, u.data_ptr(), m, out.data_ptr()), "ns_eval_lnl")
        self.sync()
        return out

    def eval_lnl_host_noalloc(self, u) -> np.ndarray:
        """Host-buffer batched log L that allocates no device memory (at most
        NOALLOC_MAX_POINTS points per call; see include/gwns.h)."""
        u = _f64(u).reshape(-1, self.dim)
        res = np.zeros(u.shape[0])
        _check(lib().ns_eval_lnl_host_noalloc(self._ctx, _ptr(u), u.shape[0], _ptr(res)),
               "ns_eval_lnl_host_noalloc")
        return res

    def eval_lnl_theta(self, theta, out=None):
        import torch
        assert theta.is_cuda and theta.dtype == torch.float64 and theta.is_contiguous()
        m = theta.shape[0]
        if out is None:
            out = torch.empty(m, dtype=torch.float64, device=theta.device)
        torch.cuda.current_stream(theta.device).synchronize()
        _check(lib().ns_eval_lnl_theta(self._ctx, theta.data_ptr(), m, out.data_ptr()), "ns_eval_lnl_theta")
        self.sync()
        return out

    def waveform(self, theta) -> np.ndarray:
        th = _f64(theta)
        re = np.zeros((self.n_det, self.N))
        im = np.zeros((self.n_det, self.N))
        _check(lib().ns_waveform(self._ctx, _ptr(th), _ptr(re), _ptr(im)), "ns_waveform")
        return re + 1j * im

    def theta(self, u) -> np.ndarray:
        u = _f64(u).reshape(-1, self.dim)
        th = np.zeros((u.shape[0], NPARAM))
        _check(lib().ns_prior_transform(self._ctx, _ptr(u), u.shape[0], _ptr(th)), "ns_prior_transform")
        return th

    def snr2(self, theta) -> float:
        r = ctypes.c_double()
        _check(lib().ns_optimal_snr2(self._ctx, _ptr(_f64(theta)), ctypes.byref(r)), "ns_optimal_snr2")
        return r.value

    def live(self):
        u = np.zeros((self.n_live, self.dim))
        l = np.zeros(self.n_live)
        _check(lib().ns_get_live(self._ctx, _ptr(u), _ptr(l)), "ns_get_live")
        return u, l

    def set_live(self, u, logl):
        u, l = _f64(u), _f64(logl)
        _check(lib().ns_set_live(self._ctx, _ptr(u), _ptr(l)), "ns_set_live")

    def sync(self):
        _check(lib().ns_sync(self._ctx), "ns_sync")

    def checkpoint(self) -> bytes:
        n = ctypes.c_size_t(0)
        _check(lib().ns_checkpoint(self._ctx, None, ctypes.byref(n)), "ns_checkpoint")
        buf = ctypes.create_string_buffer(n.value)
        _check(lib().ns_checkpoint(self._ctx, buf, ctypes.byref(n)), "ns_checkpoint")
        return buf.raw[: n.value]

    def restore(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(lib().ns_restore(self._ctx, buf, len(blob)), "ns_restore")

    def autotune(self, trials: int = 2) -> int:
        """Pick the fastest slice-update slot count on this workload (results unchanged)."""
        s = ctypes.c_int()
        _check(lib().ns_autotune(self._ctx, trials, ctypes.byref(s)), "ns_autotune")
        return s.value

    def autotune_eval(self, trials: int = 3) -> int:
        """Pick the fastest warps per point for the batched likelihood."""
        w = ctypes.c_int()
        _check(lib().ns_autotune_eval(self._ctx, trials, ctypes.byref(w)), "ns_autotune_eval")
        return w.value


def _fill_inputs(kind, lo, hi, data, psd, f0, df, pos, xarm, yarm, ideal, coarse_bins, theta_fid, keep):
    pr, dt, ps, gr = _Prior(), _Data(), _Psd(), _Grid()
    kind = np.asarray(kind, dtype=np.int32)
    for p in range(NPARAM):
        pr.kind[p], pr.lo[p], pr.hi[p] = int(kind[p]), float(lo[p]), float(hi[p])
    psd = _f64(psd)
    n_det, N = psd.shape
    keep.append(psd)
    ps.S = _ptr(psd)
    dt.n_det, dt.ideal = n_det, int(bool(ideal))
    if data is not None:
        data = np.asarray(data, dtype=np.complex128).reshape(n_det, N)
        re, im = _f64(data.real), _f64(data.imag)
        keep += [re, im]
        dt.re, dt.im = _ptr(re), _ptr(im)
    if not ideal:
        arrs = [_f64(pos).reshape(n_det, 3), _f64(xarm).reshape(n_det, 3), _f64(yarm).reshape(n_det, 3)]
        keep += arrs
        dt.pos, dt.xarm, dt.yarm = (_ptr(a) for a in arrs)
    gr.N, gr.f0, gr.df = N, float(f0), float(df)
    if coarse_bins:
        tf = _f64(theta_fid)
        keep.append(tf)
        gr.coarse_bins, gr.theta_fid = int(coarse_bins), _ptr(tf)
    return pr, dt, ps, gr


class Server:
    """Continuous-batching server of many analyses (ns_server_* in gwns.h)."""

    def __init__(self, *, max_active=16, mem_budget=0, precision=NS_MIXED, slots=0, max_iter=0, stream=None,
                 max_chains=0):
        o = _ServerOptions(max_active, mem_budget, precision, slots, max_iter,
                           None if stream is None else int(stream), max_chains)
        h = ctypes.c_void_p()
        _check(lib().ns_server_create(ctypes.byref(h), ctypes.byref(o)), "ns_server_create")
        self._h = h

    def submit(self, *, kind, lo, hi, data, psd, f0, df, pos=None, xarm=None, yarm=None, ideal=False,
               n_live=100, k=0, steps_per_dim=5, no_cutoff=False, dlogz_stop=0.1, seed=0,
               coarse_bins=0, theta_fid=None) -> int:
        keep = []
        pr, dt, ps, gr = _fill_inputs(kind, lo, hi, data, psd, f0, df, pos, xarm, yarm, ideal,
                                      coarse_bins, theta_fid, keep)
        opt = _Options(n_live, k, steps_per_dim, 0, int(bool(no_cutoff)), 0, 0, NS_MODEL_GW, 0, 0, 0,
                       dlogz_stop, seed, None)
        req = _Request(pr, dt, ps, gr, opt)
        rid = ctypes.c_uint64()
        _check(lib().ns_submit(self._h, ctypes.byref(req), ctypes.byref(rid)), "ns_submit")
        return rid.value

    def tick(self):
        r, p = ctypes.c_int(), ctypes.c_int()
        _check(lib().ns_server_tick(self._h, ctypes.byref(r), ctypes.byref(p)), "ns_server_tick")
        return r.value, p.value

    def poll(self, rid: int) -> dict:
        st = _ReqStatus()
        _check(lib().ns_poll(self._h, rid, ctypes.byref(st)), "ns_poll")
        return {name: getattr(st, name) for name, _ in _ReqStatus._fields_}

    def result(self, rid: int, dim: int) -> dict:
        st = self.poll(rid)
        n = st["n_samples"]
        u, logl, logw, theta = np.zeros((n, dim)), np.zeros(n), np.zeros(n), np.zeros((n, NPARAM))
        sm = _Samples(n, 0, _ptr(theta), _ptr(u), _ptr(logl), _ptr(logw))
        _check(lib().ns_server_result(self._h, rid, ctypes.byref(sm)), "ns_server_result")
        return dict(u=u, logl=logl, logw=logw, theta=theta, logZ=st["logZ"], dlogZ=st["dlogZ"])

    def cancel(self, rid: int):
        _check(lib().ns_cancel(self._h, rid), "ns_cancel")

    def time(self) -> float:
        return lib().ns_server_time(self._h)

    def run_until_idle(self, max_ticks: int = 1000000):
        for _ in range(max_ticks):
            r, p = self.tick()
            if r == 0 and p == 0:
                return
        raise RuntimeError("server did not drain")

    def close(self):
        if getattr(self, "_h", None):
            lib().ns_server_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def sampler_for_workload(w, data=None, precision=NS_FP64, **kw) -> Sampler:
    """A Sampler for a gwinputs.Workload (seeded detectors and analytic PSD)."""
    import gwinputs as gi
    f = w.freqs()
    psd = np.tile(gi.psd_analytic(f), (w.n_det, 1))
    if w.ideal:
        pos = xarm = yarm = None
    else:
        pos, xarm, yarm = gi.detectors(w.seed_geometry, w.n_det)
    args = dict(kind=w.kind, lo=w.lo, hi=w.hi, data=data, psd=psd, f0=w.f0, df=w.df, pos=pos,
                xarm=xarm, yarm=yarm, ideal=w.ideal, n_live=w.n_live, k=w.k,
                steps_per_dim=w.steps_per_dim, precision=precision, dlogz_stop=w.dlogz_stop,
                seed=w.seed_sampler)
    args.update(kw)
    return Sampler(**args)


def make_analysis(w, precision=NS_FP64, max_draws: int = 1000, **kw):
    """Build a workload's synthetic data with the library's own waveform
    (injection drawn from the prior, distance scaled to the target SNR) and
    return (sampler, theta_inj)."""
    import gwinputs as gi
    probe = sampler_for_workload(w, data=None, precision=NS_FP64, n_live=2, k=1, **{
        k_: v for k_, v in kw.items() if k_ not in ("n_live", "k")})
    kind, lo, hi = w.kind.copy(), w.lo.copy(), w.hi.copy()

    def snr(th):
        return float(np.sqrt(probe.snr2(th)))

    if w.fixed_injection is not None:
        th = w.fixed_injection.copy()
        th[gi.P_DL] *= snr(th) / w.snr
        if w.dl_from_snr:
            lo[gi.P_DL] = hi[gi.P_DL] = th[gi.P_DL]
    else:
        th = None
        cands = probe.theta(gi.unit_cube(w.seed_injection, max_draws, w.dim))
        for t in cands:
            t = t.copy()
            dl = t[gi.P_DL] * snr(t) / w.snr
            if lo[gi.P_DL] <= dl <= hi[gi.P_DL]:
                t[gi.P_DL] = dl
                th = t
                break
        if th is None:
            raise RuntimeError("no injection candidate reaches the target SNR inside the prior")
    data = probe.waveform(th)
    probe.close()
    if w.noise:
        f = w.freqs()
        data = data + gi.noise(w.seed_noise, np.tile(gi.psd_analytic(f), (w.n_det, 1)), w.df)
    import copy
    w2 = copy.copy(w)
    w2.kind, w2.lo, w2.hi = kind, lo, hi
    return sampler_for_workload(w2, data=data, precision=precision, **kw), th
