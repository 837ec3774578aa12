"""The allocation-free host-buffer likelihood entry point.

Some callers cannot call cudaMalloc when they evaluate the likelihood:
real-time or callback code that must not block in the allocator, or hosts
whose device memory belongs to another allocator. ns_eval_lnl_host_noalloc
serves them from a fixed device array instead of allocated scratch. This file
is collected last so that a run stopping at the first failure has already run
every other test."""
import ctypes

import numpy as np
import pytest

import gwinputs as gi
import oracle

pytestmark = pytest.mark.gpu


def _sampler(gw):
    w = gi.workload("c1")
    w.N = 1500
    pb, th = oracle.make_problem(w)
    sp = gw.Sampler(kind=pb.kind, lo=pb.lo, hi=pb.hi, data=pb.data(), psd=pb.psd, f0=pb.f0, df=pb.df,
                    pos=pb.pos, xarm=pb.xarm, yarm=pb.yarm, n_live=16, precision=gw.NS_FP64)
    return sp, pb


def _noalloc(gw, sp, u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    out = np.zeros(u.shape[0])
    rc = gw.lib().ns_eval_lnl_host_noalloc(sp._ctx, u.ctypes.data, u.shape[0], out.ctypes.data)
    return rc, out


def test_noalloc_allocates_no_scratch(gw):
    """On a fresh context the entry point leaves the context's staging scratch
    unallocated, over two calls; the allocating host entry point then does
    allocate it."""
    sp, pb = _sampler(gw)
    assert sp.stats()["scratch_bytes"] == 0
    for seed, m in [(11, 900), (12, 4096)]:
        rc, got = _noalloc(gw, sp, gi.unit_cube(seed, m, pb.dim))
        assert rc == 0 and np.all(np.isfinite(got))
        assert sp.stats()["scratch_bytes"] == 0
    sp.eval_lnl(gi.unit_cube(13, 50, pb.dim))
    assert sp.stats()["scratch_bytes"] > 0
    sp.close()


def test_noalloc_matches_host_entry_on_consecutive_calls(gw):
    sp, pb = _sampler(gw)
    for call, (seed, m) in enumerate([(101, 700), (202, 333)]):
        u = gi.unit_cube(seed, m, pb.dim)
        rc, got = _noalloc(gw, sp, u)
        assert rc == 0, gw.lib().ns_strerror(rc)
        want = sp.eval_lnl(u)              # the existing host-buffer entry point
        err = np.abs(got - want) / np.maximum(1.0, np.abs(want))
        assert np.max(err) < 1e-9, (call, np.max(err))
    sp.close()


def test_noalloc_limits(gw):
    sp, pb = _sampler(gw)
    rc, _ = _noalloc(gw, sp, np.zeros((0, pb.dim)))
    assert rc == 0
    too_many = gw.NOALLOC_MAX_POINTS + 1
    rc, _ = _noalloc(gw, sp, np.full((too_many, pb.dim), 0.5))
    assert rc == -5          # NS_ERR_CAPACITY
    rc, got = _noalloc(gw, sp, np.full((gw.NOALLOC_MAX_POINTS, pb.dim), 0.5))
    assert rc == 0 and np.all(got == got[0])
    sp.close()
