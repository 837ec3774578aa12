"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.

Tolerances: FP64 log L within 1e-9 relative (of max(|log L|, 1)); mixed
precision within 1e-3 absolute; waveforms within 1e-10 of the peak strain.
"""
import math

import numpy as np
import pytest
from scipy import stats

import gwinputs as gi
import oracle
from oracle import ns as ons

pytestmark = pytest.mark.gpu

FP64_RTOL = 1e-9
MIXED_ATOL = 1e-3


def sampler_from(g, pb, precision=0, **kw):
    args = dict(kind=pb.kind, lo=pb.lo, hi=pb.hi, data=pb.data(), psd=pb.psd, f0=pb.f0, df=pb.df,
                pos=pb.pos, xarm=pb.xarm, yarm=pb.yarm, ideal=pb.ideal, no_cutoff=not pb.cutoff,
                precision=precision)
    args.update(kw)
    return g.Sampler(**args)


_PROBLEMS = {}


def problem(name, **over):
    key = (name, tuple(sorted(over.items())))
    if key not in _PROBLEMS:
        w = gi.workload(name, **over)
        _PROBLEMS[key] = (w,) + oracle.make_problem(w)
    return _PROBLEMS[key]


def pts_for(pb, th_inj, count=160, seed=17):
    u = gi.unit_cube(seed, count, pb.dim)
    # prior corners and faces
    u[0] = 1e-12
    u[1] = 1.0 - 1e-12
    u[2, ::2] = 1e-12
    u[3, 1::2] = 1.0 - 1e-12
    return u


@pytest.mark.parametrize("name,over", [
    ("c0", {}),
    ("c1", {}),
    ("c1", {"N": 1013}),            # ragged tail
    ("c1", {"N": 33, "df": 4.0}),    # tiny grid
    ("c1", {"n_det": 1}),
    ("c1", {"n_det": 2}),
])
@pytest.mark.parametrize("warps", [1, 4])
def test_lnl_fp64_parity(gw, name, over, warps):
    w, pb, th = problem(name, **over)
    u = pts_for(pb, th)
    want = pb.loglike(u)
    with sampler_from(gw, pb, 0, n_live=8, warps_per_point=warps) as sp:
        got = sp.eval_lnl(u)
    err = np.abs(got - want) / np.maximum(1.0, np.abs(want))
    assert np.max(err) < FP64_RTOL, (np.max(err), np.argmax(err))


@pytest.mark.parametrize("name,over", [("c0", {}), ("c1", {}), ("c1", {"N": 1013}),
                                       ("c1", {"N": 33, "df": 4.0}), ("c1", {"N": 8000, "df": 0.03125}),
                                       ("c1", {"N": 3001, "df": 0.03125}), ("c1", {"N": 3001, "df": 0.0625}),
                                       ("c1", {"N": 1500, "df": 0.125})])
@pytest.mark.parametrize("warps", [1, 2, 8])
def test_lnl_mixed_parity(gw, name, over, warps):
    """Coarse grids take the per-bin mixed form, fine ones the tiled form:
    df = 1/32 Hz 32-bin tiles (rotation), 1/16 Hz 16-bin and 1/8 Hz 8-bin
    tiles (direct), some with a ragged last group."""
    w, pb, th = problem(name, **over)
    u = pts_for(pb, th)
    want = pb.loglike(u)
    with sampler_from(gw, pb, 1, n_live=8, warps_per_point=warps) as sp:
        got = sp.eval_lnl(u)
    assert np.max(np.abs(got - want)) < MIXED_ATOL, np.max(np.abs(got - want))


@pytest.mark.parametrize("name,over,tile", [("c0", {"N": 12000, "df": 1 / 128}, 128),
                                            ("c1", {"N": 12000, "df": 1 / 128, "n_det": 2}, 128),
                                            ("c1", {"N": 12000, "df": 1 / 128}, 128),
                                            ("c1", {"N": 12000, "df": 1 / 128, "n_det": 4}, 128),
                                            ("c1", {"N": 6000, "df": 1 / 64}, 64)])
@pytest.mark.parametrize("warps", [1, 4])
def test_lnl_mixed_rotation_parity(gw, name, over, tile, warps):
    """128- and 64-bin tiles (df = 1/128, 1/64 Hz): detector 0 by its own sine
    and cosine per bin, detectors 1..3 by their rotation against it; cutoffs
    inside the grid for the heavier draws and a ragged last tile group."""
    w, pb, th = problem(name, **over)
    u = pts_for(pb, th)
    want = pb.loglike(u)
    with sampler_from(gw, pb, 1, n_live=8, warps_per_point=warps) as sp:
        assert sp.stats()["mixed_tile"] == tile
        got = sp.eval_lnl(u)
        import torch
        g_inj = sp.eval_lnl_theta(torch.tensor(th[None], dtype=torch.float64, device="cuda")).item()
    assert np.max(np.abs(got - want)) < MIXED_ATOL, np.max(np.abs(got - want))
    # the injection, where <d|h> is largest
    assert abs(g_inj - pb.loglike_theta(th)[0]) < MIXED_ATOL


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", ["c2", "c4"])
def test_lnl_full_size_sampled(gw, name, precision):
    """Full-size grids (64,897 and 519,169 bins): sampled points, including the
    injection, against the oracle evaluated one by one."""
    w, pb, th = problem(name)
    u = gi.unit_cube(23, 6, pb.dim)
    want = pb.loglike(u)
    with sampler_from(gw, pb, precision, n_live=8) as sp:
        got = sp.eval_lnl(u)
        import torch
        tt = torch.tensor(th[None, :], dtype=torch.float64, device="cuda")
        got_inj = sp.eval_lnl_theta(tt).cpu().numpy()[0]
    want_inj = pb.loglike_theta(th)[0]
    if precision == 0:
        assert np.max(np.abs(got - want) / np.maximum(1, np.abs(want))) < FP64_RTOL
        assert abs(got_inj - want_inj) / max(1, abs(want_inj)) < FP64_RTOL
    else:
        assert np.max(np.abs(got - want)) < MIXED_ATOL
        assert abs(got_inj - want_inj) < MIXED_ATOL


@pytest.mark.parametrize("name,over", [("c0", {}), ("c1", {}), ("c1", {"N": 8000, "df": 0.03125}),
                                       ("c1", {"N": 3001, "df": 0.0625}),
                                       ("c1", {"N": 12000, "df": 1 / 128, "n_det": 4}), ("c2", {})])
def test_mixed_coefficients_double_float_against_fp64_stage(gw, name, over, monkeypatch):
    """The mixed form's per-point coefficients in double-float on the FP32 pipe
    (the default) against the FP64 stage and its conversion to (hi, lo) floats
    (GWNS_COEF_FP64=1), on the per-bin form, the direct and the rotation tiled
    forms: the same log L to within 1e-4, both within 1e-3 of the oracle, and
    the same bins read (cutoff indices) point for point. The injection too."""
    import torch
    w, pb, th = problem(name, **over)
    u = pts_for(pb, th, count=512)
    want = pb.loglike(u)
    got = {}
    for mode in ("df", "fp64"):
        if mode == "fp64":
            monkeypatch.setenv("GWNS_COEF_FP64", "1")
        else:
            monkeypatch.delenv("GWNS_COEF_FP64", raising=False)
        with sampler_from(gw, pb, 1, n_live=8) as sp:
            st0 = sp.stats()
            v = sp.eval_lnl(u)
            st1 = sp.stats()
            g_inj = sp.eval_lnl_theta(torch.tensor(th[None], dtype=torch.float64, device="cuda")).item()
        got[mode] = (v, st1["batch_point_bins"] - st0["batch_point_bins"], g_inj)
    (a, pa, ia), (b, pbn, ib) = got["df"], got["fp64"]
    assert pa == pbn
    assert np.max(np.abs(a - b)) < 1e-4, np.max(np.abs(a - b))
    assert np.max(np.abs(a - want)) < MIXED_ATOL, np.max(np.abs(a - want))
    assert abs(ia - ib) < MIXED_ATOL


def test_lnl_device_pointer_path(gw):
    import torch
    w, pb, th = problem("c1")
    u = gi.unit_cube(3, 64, pb.dim)
    with sampler_from(gw, pb, 0, n_live=8) as sp:
        dev = torch.tensor(u, dtype=torch.float64, device="cuda")
        got = sp.eval_lnl(dev).cpu().numpy()
        empty = sp.eval_lnl(torch.zeros((0, pb.dim), dtype=torch.float64, device="cuda"))
    assert empty.numel() == 0
    want = pb.loglike(u)
    assert np.max(np.abs(got - want) / np.maximum(1, np.abs(want))) < FP64_RTOL


def test_waveform_and_snr_parity(gw):
    w, pb, th = problem("c1")
    with sampler_from(gw, pb, 0, n_live=8) as sp:
        h = sp.waveform(th)
        rho2 = sp.snr2(th)
        theta = sp.theta(gi.unit_cube(4, 50, pb.dim))
    for d in range(pb.n_det):
        ho = pb.strain(th, d)
        assert np.max(np.abs(h[d] - ho)) < 1e-10 * np.max(np.abs(ho))
    assert rho2 == pytest.approx(pb.snr2(th), rel=1e-10, abs=0)
    assert np.max(np.abs(theta - pb.theta(gi.unit_cube(4, 50, pb.dim)))) < 1e-10


def test_injection_identity_gpu(gw):
    """Noise-free data: log L(theta_inj) = rho^2/2 on the GPU too."""
    import torch
    w, pb, th = problem("c1", noise=False)
    for prec, tol in ((0, 1e-9 * 200), (1, MIXED_ATOL)):
        with sampler_from(gw, pb, prec, n_live=8) as sp:
            v = sp.eval_lnl_theta(torch.tensor(th[None], dtype=torch.float64, device="cuda")).item()
        assert abs(v - w.snr ** 2 / 2) < tol


def test_no_cutoff_and_empty_band(gw):
    """The no-cutoff option, and points whose f_ISCO lies below the first bin
    (jcut = -1, log L = 0)."""
    w, pb, th = problem("c1", N=500)
    pb2 = oracle.Problem(f0=pb.f0, df=pb.df, psd=pb.psd, data=pb.data(), pos=pb.pos, xarm=pb.xarm,
                         yarm=pb.yarm, cutoff=False, kind=pb.kind, lo=pb.lo, hi=pb.hi)
    u = gi.unit_cube(8, 40, pb.dim)
    with sampler_from(gw, pb2, 0, n_live=8) as sp:
        got = sp.eval_lnl(u)
    want = pb2.loglike(u)
    assert np.max(np.abs(got - want) / np.maximum(1, np.abs(want))) < FP64_RTOL
    # grid starting at 400 Hz: heavy systems have f_ISCO < 400 Hz
    pb3 = oracle.Problem(f0=400.0, df=pb.df, psd=pb.psd, data=pb.data(), pos=pb.pos, xarm=pb.xarm,
                         yarm=pb.yarm, cutoff=True, kind=pb.kind, lo=pb.lo, hi=pb.hi)
    with sampler_from(gw, pb3, 0, n_live=8) as sp:
        got = sp.eval_lnl(u)
    want = pb3.loglike(u)
    assert np.sum(want == 0.0) > 5
    assert np.max(np.abs(got - want) / np.maximum(1, np.abs(want))) < FP64_RTOL


# ------------------------------------------------------------ sampler parity
def _ns_pair(gw, name, n_live, k, precision=0, slots=0, **over):
    w, pb, th = problem(name, **over)
    sp = sampler_from(gw, pb, precision, n_live=n_live, k=k, steps_per_dim=w.steps_per_dim,
                      seed=w.seed_sampler, slots=slots)
    st = ons.initial_state(pb, n_live, w.seed_sampler)
    return w, pb, sp, st


@pytest.mark.parametrize("slots", [1, 2, 4, 8])
@pytest.mark.parametrize("name,n_live,k,iters", [("c0", 200, 100, 4), ("c1", 120, 60, 2)])
def test_ns_iterations_match_oracle(gw, name, n_live, k, iters, slots):
    """Same Philox draws on both sides: the live set after each iteration and
    the evidence bookkeeping match the oracle's, whatever the number of
    speculative candidate slots per chain."""
    w, pb, sp, st = _ns_pair(gw, name, n_live, k, slots=slots)
    u0, l0 = sp.live()
    assert np.max(np.abs(u0 - st.live_u)) == 0.0
    assert np.max(np.abs(l0 - st.live_logl) / np.maximum(1, np.abs(st.live_logl))) < FP64_RTOL
    for it in range(iters):
        info = ons.iterate(pb, st, k, w.steps_per_dim * pb.dim, w.seed_sampler)
        sp.step(k)
        gu, gl = sp.live()
        s = sp.stats()
        assert s["lstar"] == pytest.approx(info["lstar"], rel=1e-9, abs=1e-9)
        assert np.max(np.abs(gu - st.live_u)) < 1e-9, (it, np.max(np.abs(gu - st.live_u)))
        assert np.max(np.abs(gl - st.live_logl) / np.maximum(1, np.abs(st.live_logl))) < 1e-8
        assert s["logX"] == pytest.approx(st.logX, rel=1e-12)
        assert s["logZ"] == pytest.approx(st.logZ, rel=1e-9, abs=1e-9)
        assert s["evals"] == st.evals
        assert s["status"] == 0
    sp.close()


@pytest.mark.parametrize("slots", [1, 2])
def test_periodic_iterations_match_oracle(gw, slots):
    """phi_c, psi and RA wrapping on the slice line: GPU and oracle follow the
    same trajectories (a fresh problem, so no other test sees the mask)."""
    w = gi.workload("c1")
    pb, th = oracle.make_problem(w)
    pb.set_periodic((gi.P_PHIC, gi.P_PSI, gi.P_RA))
    n_live, k = 120, 60
    st = ons.initial_state(pb, n_live, w.seed_sampler)
    with sampler_from(gw, pb, 0, n_live=n_live, k=k, steps_per_dim=w.steps_per_dim, seed=w.seed_sampler,
                      slots=slots, periodic=(gi.P_PHIC, gi.P_PSI, gi.P_RA)) as sp:
        for it in range(2):
            ons.iterate(pb, st, k, w.steps_per_dim * pb.dim, w.seed_sampler)
            sp.step(k)
            gu, gl = sp.live()
            assert np.max(np.abs(gu - st.live_u)) < 1e-9, it
            assert np.max(np.abs(gl - st.live_logl) / np.maximum(1, np.abs(st.live_logl))) < 1e-8
            assert sp.stats()["evals"] == st.evals


def test_bench_configuration_iteration_matches_oracle(gw):
    """The benchmarked configuration itself (3 detectors, 4017 bins, 1000 live
    points, 500 chains of 55 steps, FP64, the default slot rule and launch):
    the live set after one iteration matches the oracle's."""
    w, pb, th = problem("c1")
    st = ons.initial_state(pb, w.n_live, w.seed_sampler)
    with sampler_from(gw, pb, 0, n_live=w.n_live, k=w.k, steps_per_dim=w.steps_per_dim,
                      seed=w.seed_sampler) as sp:
        ons.iterate(pb, st, w.k, w.steps_per_dim * pb.dim, w.seed_sampler)
        sp.step()
        gu, gl = sp.live()
        s = sp.stats()
    assert np.max(np.abs(gu - st.live_u)) < 1e-9
    assert np.max(np.abs(gl - st.live_logl) / np.maximum(1, np.abs(st.live_logl))) < 1e-8
    assert s["evals"] == st.evals and s["status"] == 0


@pytest.mark.parametrize("slots", [0, 2])
@pytest.mark.parametrize("name,n_live,k,spd", [("c2", 400, 200, 2), ("c4", 20, 10, 1)])
def test_fp64_iteration_on_the_large_grids_matches_oracle(gw, name, n_live, k, spd, slots):
    """FP64 slice update on the 64,897- and 519,169-bin grids (3 detectors,
    11 parameters) with the default slot rule (one slot there) and with two:
    after one iteration the live set, threshold, evidence and evaluation count
    equal the oracle's. On the 64,897-bin grid 200 chains run, more than there
    are SMs, so chains run both while the GPU is full and in the update's tail."""
    w, pb, th = problem(name)
    st = ons.initial_state(pb, n_live, w.seed_sampler)
    with sampler_from(gw, pb, 0, n_live=n_live, k=k, steps_per_dim=spd, seed=w.seed_sampler,
                      slots=slots) as sp:
        u0, l0 = sp.live()
        assert np.max(np.abs(u0 - st.live_u)) == 0.0
        assert np.max(np.abs(l0 - st.live_logl) / np.maximum(1, np.abs(st.live_logl))) < FP64_RTOL
        info = ons.iterate(pb, st, k, spd * pb.dim, w.seed_sampler)
        sp.step(k)
        gu, gl = sp.live()
        s = sp.stats()
    assert s["lstar"] == pytest.approx(info["lstar"], rel=1e-9, abs=1e-9)
    assert np.max(np.abs(gu - st.live_u)) < 1e-9
    assert np.max(np.abs(gl - st.live_logl) / np.maximum(1, np.abs(st.live_logl))) < 1e-8
    assert s["logZ"] == pytest.approx(st.logZ, rel=1e-9, abs=1e-9)
    assert s["evals"] == st.evals and s["status"] == 0


@pytest.mark.parametrize("name,precision,half", [("c1", 0, 3), ("c1", 1, 3), ("c4", 1, 1)])
def test_runs_at_the_benchmark_population_are_bit_identical(gw, name, precision, half):
    """Two fresh runs at the workload's own population (1000 live points and
    500 chains on 4017 bins; 2000 and 1000 on 519,169 bins, where the mixed
    update is work-shared: chains finish in a timing-dependent order and the
    CTAs left without a chain help the running ones with chunks of their tile
    groups) give bit-identical live sets and log Z, and so does a run resumed
    from a checkpoint taken halfway."""
    w, pb, th = problem(name)
    args = dict(n_live=w.n_live, k=w.k, steps_per_dim=w.steps_per_dim, seed=w.seed_sampler)
    runs = []
    for r in range(2):
        with sampler_from(gw, pb, precision, **args) as sp:
            for _ in range(half):
                sp.step()
            blob = sp.checkpoint() if r == 0 else None
            for _ in range(half):
                sp.step()
            runs.append((sp.live(), sp.stats(), blob))
            assert runs[-1][1]["status"] == 0
    (ua, la), sa, blob = runs[0]
    (ub, lb), sb, _ = runs[1]
    assert np.array_equal(ua, ub) and np.array_equal(la, lb)
    assert sa["logZ"] == sb["logZ"] and sa["evals"] == sb["evals"]
    with sampler_from(gw, pb, precision, **args) as sp:
        sp.restore(blob)
        for _ in range(half):
            sp.step()
        uc, lc = sp.live()
        sc = sp.stats()
    assert np.array_equal(ua, uc) and np.array_equal(la, lc)
    assert sa["logZ"] == sc["logZ"] and sa["evals"] == sc["evals"]


def test_ns_step_host_dead_points(gw):
    w, pb, sp, st = _ns_pair(gw, "c0", 100, 50)
    k, d = 50, pb.dim
    du, dl, dw = np.zeros((k, d)), np.zeros(k), np.zeros(k)
    order = np.argsort(st.live_logl, kind="stable")
    sp.step_host(k, du, dl, dw)
    ons.iterate(pb, st, k, w.steps_per_dim * d, w.seed_sampler)
    assert np.max(np.abs(du - st.dead_u[0])) == 0.0
    assert np.max(np.abs(dw - st.dead_logw[0])) < 1e-12
    sp.close()


def test_toy_evidence_gpu(gw):
    """Correlated-Gaussian toy, analytic log Z = -d ln 20."""
    d = 4
    truth = -d * math.log(20.0)
    hits = 0
    for s in range(6):
        with gw.Sampler(model=gw.NS_MODEL_TOY, toy_dim=d, n_live=200, k=100, steps_per_dim=5,
                        seed=300 + s) as sp:
            sp.run()
            r = sp.result(samples=False)
        hits += abs(r["logZ"] - truth) < 3 * r["dlogZ"]
    assert hits >= 5


@pytest.mark.parametrize("slots", [1, 2, 4])
@pytest.mark.parametrize("name,n_live,k,iters", [("c0", 200, 100, 3), ("c1", 120, 60, 2)])
def test_walk_iterations_match_oracle(gw, name, n_live, k, iters, slots):
    """The random-walk inner kernel: same proposals, same accepted moves, same
    walk-length adaptation on both sides."""
    w, pb, th = problem(name)
    st = ons.initial_state(pb, n_live, w.seed_sampler)
    with sampler_from(gw, pb, 0, n_live=n_live, k=k, steps_per_dim=w.steps_per_dim, seed=w.seed_sampler,
                      slots=slots, kernel=gw.NS_KERNEL_WALK) as sp:
        for it in range(iters):
            ons.iterate(pb, st, k, w.steps_per_dim * pb.dim, w.seed_sampler, kernel="walk")
            sp.step(k)
            gu, gl = sp.live()
            s = sp.stats()
            assert np.max(np.abs(gu - st.live_u)) < 1e-9, it
            assert np.max(np.abs(gl - st.live_logl) / np.maximum(1, np.abs(st.live_logl))) < 1e-8
            assert s["evals"] == st.evals and s["status"] == 0
            assert s["logZ"] == pytest.approx(st.logZ, rel=1e-9, abs=1e-9)


def test_walk_toy_run_matches_oracle_run(gw):
    """Whole toy run with the random walk: same iterations and evidence as the
    oracle's, and log Z within 3 dlogZ of the analytic -d ln 20."""
    d = 4
    pb = oracle.toy_problem(d)
    ref = ons.run(pb, n_live=100, k=50, steps=5 * d, seed=43, kernel="walk")
    with gw.Sampler(model=gw.NS_MODEL_TOY, toy_dim=d, n_live=100, k=50, steps_per_dim=5, seed=43,
                    kernel=gw.NS_KERNEL_WALK) as sp:
        it = sp.run()
        r = sp.result()
    assert it == ref["iterations"]
    assert r["logZ"] == pytest.approx(ref["logZ"], rel=1e-10, abs=1e-10)
    assert abs(r["logZ"] + d * math.log(20.0)) < 3 * r["dlogZ"] + 0.05


def test_toy_run_matches_oracle_run(gw):
    """Whole toy run: same seed, same draws, same evidence and replicates."""
    d = 4
    pb = oracle.toy_problem(d)
    ref = ons.run(pb, n_live=100, k=50, steps=5 * d, seed=42, replicates=200)
    with gw.Sampler(model=gw.NS_MODEL_TOY, toy_dim=d, n_live=100, k=50, steps_per_dim=5, seed=42) as sp:
        it = sp.run()
        r = sp.result()
    assert it == ref["iterations"]
    assert r["logZ"] == pytest.approx(ref["logZ"], rel=1e-10, abs=1e-10)
    assert r["dlogZ"] == pytest.approx(ref["dlogZ"], rel=1e-8)
    assert r["H"] == pytest.approx(ref["H"], rel=1e-9)
    assert r["ess"] == pytest.approx(ref["ess"], rel=1e-9)
    assert np.max(np.abs(r["logl"] - ref["logl"])) < 1e-9
    assert np.max(np.abs(r["logw"] - ref["logw"])) < 1e-9


def _mixed_log_z_pairs(gw, pb, n_live, k, steps_per_dim, seed0, pairs=8):
    """Mixed minus FP64 log Z over seed pairs on the same data (pair i: both
    forms with sampler seed seed0 + 1000 (i + 1)). The two forms follow the same
    trajectory only until an accept/reject decision that a ~1e-5 log L
    difference flips; after it they scatter like independent runs, by several
    times dlogZ. Returns the differences."""
    d = []
    for i in range(pairs):
        z = []
        for prec in (0, 1):
            with sampler_from(gw, pb, prec, n_live=n_live, k=k, steps_per_dim=steps_per_dim,
                              seed=seed0 + 1000 * (i + 1)) as sp:
                sp.run()
                z.append(sp.result(samples=False)["logZ"])
        d.append(z[1] - z[0])
    return np.array(d)


def _assert_mixed_log_z_agrees(d):
    """The mean mixed - FP64 difference is consistent with zero: within four
    standard errors of the pairs' own scatter (plus 0.02 for pairs that never
    diverged)."""
    se = d.std(ddof=1) / math.sqrt(len(d))
    assert abs(d.mean()) < 4 * se + 0.02, (d.mean(), se, d)


@pytest.mark.parametrize("precision", [0, 1])
def test_c0_run_against_oracle(gw, precision):
    """Single-detector workload end to end and per-parameter posterior KS
    p > 0.01 against the oracle's run. FP64: the oracle's run itself (same
    draws). Mixed: log Z agrees with the FP64 form's over 8 seed pairs."""
    w, pb, th = problem("c0")
    ref = ons.run(pb, n_live=w.n_live, k=w.k, steps=w.steps_per_dim * pb.dim, seed=w.seed_sampler)
    with sampler_from(gw, pb, precision, n_live=w.n_live, k=w.k, steps_per_dim=w.steps_per_dim,
                      seed=w.seed_sampler) as sp:
        sp.run()
        r = sp.result()
    if precision == 0:
        assert r["logZ"] == pytest.approx(ref["logZ"], abs=1e-6)
    else:
        _assert_mixed_log_z_agrees(_mixed_log_z_pairs(gw, pb, w.n_live, w.k, w.steps_per_dim, w.seed_sampler))
    lw_g = r["logw"] + r["logl"] - r["logZ"]
    lw_o = ref["logw"] + ref["logl"] - ref["logZ"]
    sg = ons.equal_weight_resample(r["u"], lw_g, 1)
    so = ons.equal_weight_resample(ref["samples_u"], lw_o, 2)
    for i in range(pb.dim):
        assert stats.ks_2samp(sg[:, i], so[:, i]).pvalue > 0.01


def test_errors(gw):
    w, pb, th = problem("c0")
    with pytest.raises(gw.GWNSError) as e:
        sampler_from(gw, pb, 0, n_live=1)
    assert e.value.code == -1
    bad = pb.psd.copy()
    bad[0, 7] = 0.0
    with pytest.raises(gw.GWNSError) as e:
        gw.Sampler(kind=pb.kind, lo=pb.lo, hi=pb.hi, data=pb.data(), psd=bad, f0=pb.f0, df=pb.df,
                   ideal=True, n_live=10)
    assert e.value.code == -2
    with sampler_from(gw, pb, 0, n_live=10) as sp:
        with pytest.raises(gw.GWNSError) as e:
            sp.step(10)
        assert e.value.code == -3
        with pytest.raises(gw.GWNSError) as e:
            sp.step(-1)
        assert e.value.code == -3


@pytest.mark.parametrize("n_live,k", [(2, 1), (40, 39), (4096, 2048)])
def test_population_extremes_match_oracle(gw, n_live, k):
    """The smallest population (2 live points, 1 deleted), one survivor per
    iteration (k = n - 1) and the largest population the one-CTA sort takes
    (4096): iterations match the oracle's."""
    w, pb, sp, st = _ns_pair(gw, "c0", n_live, k)
    with sp:
        for it in range(2):
            ons.iterate(pb, st, k, w.steps_per_dim * pb.dim, w.seed_sampler)
            sp.step(k)
            gu, gl = sp.live()
            assert np.max(np.abs(gu - st.live_u)) < 1e-9, it
            assert np.max(np.abs(gl - st.live_logl) / np.maximum(1, np.abs(st.live_logl))) < 1e-8
            s = sp.stats()
            assert s["logZ"] == pytest.approx(st.logZ, rel=1e-9, abs=1e-9)
            assert s["evals"] == st.evals and s["status"] == 0


def test_population_above_the_limit_is_refused(gw):
    w, pb, th = problem("c0")
    with pytest.raises(gw.GWNSError) as e:
        sampler_from(gw, pb, 0, n_live=4097)
    assert e.value.code == -1


# ---------------------------------------------------------- relative binning
@pytest.mark.parametrize("precision", [0, 1])
def test_relative_binning_parity(gw, precision):
    w, pb, th = problem("c1")
    rb = oracle.RelativeBinning(pb, th, B=256)
    u = pts_for(pb, th, count=80)
    want = rb.loglike(u)
    with sampler_from(gw, pb, precision, n_live=8, coarse_bins=256, theta_fid=th) as sp:
        got = sp.eval_lnl(u)
    if precision == 0:
        assert np.max(np.abs(got - want) / np.maximum(1, np.abs(want))) < FP64_RTOL
    else:
        assert np.max(np.abs(got - want)) < MIXED_ATOL


@pytest.mark.parametrize("precision", [0, 1])
def test_relative_binning_full_size(gw, precision):
    """519,169-bin grid on 1024 geometric coarse bins about the injection:
    sampled points and the injection itself against the oracle, and the
    coarse result at the fiducial point against the full-grid one."""
    import torch
    w, pb, th = problem("c4")
    rb = oracle.RelativeBinning(pb, th, B=1024)
    u = gi.unit_cube(29, 6, pb.dim)
    want = rb.loglike(u)
    with sampler_from(gw, pb, precision, n_live=8, coarse_bins=1024, theta_fid=th) as sp:
        got = sp.eval_lnl(u)
        g_inj = sp.eval_lnl_theta(torch.tensor(th[None], dtype=torch.float64, device="cuda")).item()
    w_inj = rb.loglike_theta(th)[0]
    full_inj = pb.loglike_theta(th)[0]
    if precision == 0:
        assert np.max(np.abs(got - want) / np.maximum(1, np.abs(want))) < FP64_RTOL
        assert abs(g_inj - w_inj) / abs(w_inj) < FP64_RTOL
    else:
        assert np.max(np.abs(got - want)) < MIXED_ATOL
        assert abs(g_inj - w_inj) < MIXED_ATOL
    # bin-granular cutoff: a fraction of a coarse bin of signal at most
    assert abs(w_inj - full_inj) < 0.02 * abs(full_inj)


def test_relative_binning_iterations_match_oracle(gw):
    w, pb, th = problem("c1")
    rb = oracle.RelativeBinning(pb, th, B=256)
    pbr = rb.problem()
    n_live, k = 120, 60
    st = ons.initial_state(pbr, n_live, w.seed_sampler)
    with sampler_from(gw, pb, 0, n_live=n_live, k=k, steps_per_dim=w.steps_per_dim, seed=w.seed_sampler,
                      coarse_bins=256, theta_fid=th) as sp:
        for it in range(2):
            ons.iterate(pbr, st, k, w.steps_per_dim * pb.dim, w.seed_sampler)
            sp.step(k)
            gu, gl = sp.live()
            assert np.max(np.abs(gu - st.live_u)) < 1e-9
            assert np.max(np.abs(gl - st.live_logl) / np.maximum(1, np.abs(st.live_logl))) < 1e-8


def test_autotune_keeps_the_trajectory(gw):
    """Autotuning times each slot count from a saved state and restores it:
    the run continues exactly as the oracle's."""
    w, pb, sp, st = _ns_pair(gw, "c1", 120, 60)
    chosen = sp.autotune(trials=1)
    assert chosen in (1, 2, 4, 8)
    for it in range(2):
        ons.iterate(pb, st, 60, w.steps_per_dim * pb.dim, w.seed_sampler)
        sp.step(60)
    gu, gl = sp.live()
    assert np.max(np.abs(gu - st.live_u)) < 1e-9
    s = sp.stats()
    assert s["iterations"] == 2 and s["evals"] == st.evals
    sp.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_autotune_eval_keeps_parity(gw, precision):
    """The batched likelihood's warps-per-point autotuner picks one of 1, 2, 4,
    8; its launches are not counted, and the likelihood then still matches the
    oracle (8000 bins at 1/32 Hz: 32-bin tiles in the mixed form)."""
    w, pb, th = problem("c1", N=8000, df=0.03125)
    u = pts_for(pb, th)
    want = pb.loglike(u)
    with sampler_from(gw, pb, precision, n_live=64) as sp:
        before = sp.stats()["batch_evals"]
        chosen = sp.autotune_eval(trials=2)
        assert chosen in (1, 2, 4, 8)
        assert sp.stats()["batch_evals"] == before
        got = sp.eval_lnl(u)
    if precision == 0:
        assert np.max(np.abs(got - want) / np.maximum(1.0, np.abs(want))) < FP64_RTOL
    else:
        assert np.max(np.abs(got - want)) < MIXED_ATOL


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("kernel", [0, 1])
def test_checkpoint_resume_is_bit_identical(gw, precision, kernel):
    """A run resumed from a checkpoint continues bit-identically (for the
    random walk this includes the adapted walk length)."""
    w, pb, th = problem("c0")
    args = dict(n_live=100, k=50, steps_per_dim=w.steps_per_dim, seed=w.seed_sampler, kernel=kernel)
    with sampler_from(gw, pb, precision, **args) as a:
        for _ in range(3):
            a.step()
        blob = a.checkpoint()
        for _ in range(4):
            a.step()
        ua, la = a.live()
        ra = a.result()
    with sampler_from(gw, pb, precision, **args) as b:
        b.restore(blob)
        for _ in range(4):
            b.step()
        ub, lb = b.live()
        rb = b.result()
    assert np.array_equal(ua, ub) and np.array_equal(la, lb)
    assert ra["logZ"] == rb["logZ"] and np.array_equal(ra["logw"], rb["logw"])


def test_shrink_cap_keeps_the_chain_in_the_slice(gw):
    """A stuck chain (no shrink draw allowed) keeps its current point, counts a
    cap hit per step and the run goes on."""
    w, pb, th = problem("c0")
    with sampler_from(gw, pb, 0, n_live=60, k=30, steps_per_dim=2, seed=3, max_shrink=1) as sp:
        lstar_prev = -np.inf
        for _ in range(3):
            sp.step()
            s = sp.stats()
            _, l = sp.live()
            assert np.all(l > s["lstar"]) and s["lstar"] >= lstar_prev
            lstar_prev = s["lstar"]
        assert s["cap_hits"] > 0 and s["status"] == 0


@pytest.mark.parametrize("slots", [2, 4])
def test_mixed_large_grid_cooperative_bins(gw, slots):
    """Grids of 16k bins or more use the cooperative mixed bin loop (all warps,
    all candidates of a round): same per-point tolerance against the oracle,
    through the sampler (live points after one iteration are re-evaluated by
    the oracle)."""
    w, pb, th = problem("c2")
    with sampler_from(gw, pb, 1, n_live=60, k=30, steps_per_dim=2, seed=5, slots=slots) as sp:
        sp.step()
        u, l = sp.live()
    want = pb.loglike(u)
    assert np.max(np.abs(l - want)) < MIXED_ATOL


@pytest.mark.parametrize("name,over,tile", [("c1", {}, 0), ("c1", {"N": 8000, "df": 0.03125}, 32),
                                            ("c1", {"N": 3001, "df": 0.0625}, 16),
                                            ("c2", {}, 32), ("c4", {}, 128), ("c1", {"N": 33, "df": 4.0}, 0)])
def test_mixed_form_choice(gw, name, over, tile):
    """The tiled form is taken where the Taylor remainder bound allows (the
    longest such tile), the per-bin form elsewhere."""
    w, pb, th = problem(name, **over)
    with sampler_from(gw, pb, 1, n_live=8) as sp:
        assert sp.stats()["mixed_tile"] == tile


def test_mixed_wide_ctas_on_the_largest_grid(gw):
    """The 519,169-bin grid runs the work-shared mixed slice update (8-warp
    persistent CTAs; 128-bin tiles by rotation, in chunks of two tile groups
    computed by the chain's own CTA and by the CTAs left without a chain, here
    almost all of them; the groups above 276 Hz at Taylor degree 3): live points
    after one iteration agree with the oracle per point, no bounded wait gave
    up, and the update counted bins at the low degree."""
    w, pb, th = problem("c4")
    with sampler_from(gw, pb, 1, n_live=24, k=12, steps_per_dim=1, seed=11) as sp:
        assert sp.stats()["mixed_tile"] == 128
        s0 = sp.stats()
        sp.step()
        u, l = sp.live()
        s1 = sp.stats()
        assert s1["status"] == 0
    pbins, lo = s1["point_bins"] - s0["point_bins"], s1["point_bins_lo"] - s0["point_bins_lo"]
    assert 0 < lo < pbins
    want = pb.loglike(u)
    assert np.max(np.abs(l - want)) < MIXED_ATOL


def _low_degree_first_bin(w, tile):
    """First bin of the first 32-tile group whose degree-3 Taylor remainder
    passes the tiled form's bound at the group's lowest frequency f_g:
    64 (3/128) (pi T_sun Mc_lo f_g)^(-5/3) (h / f_g)^4 <= 1e-8, h half a tile."""
    tsun = 4.925490947641267e-6
    gb, h = 32 * tile, 0.5 * tile * w.df
    ng = -(-w.N // gb)
    for g in range(ng):
        f = w.f0 + g * gb * w.df
        phin = 3.0 / 128.0 * (np.pi * tsun * w.lo[0] * f) ** (-5.0 / 3.0)
        if 64.0 * phin * (h / f) ** 4 <= 1e-8:
            return g * gb
    return ng * gb


def test_every_group_at_the_low_degree(gw):
    """A 519,169-bin grid from 300 Hz (injection at SNR 6): the degree-3 bound
    already passes at f0, so every tile group of the batched likelihood and of
    the work-shared update takes degree 3. Per-point log L against the oracle,
    for prior draws and for the live set after one iteration; every counted bin
    is a low-degree bin."""
    w, pb, th = problem("c4", f0=300.0, snr=6.0)
    assert _low_degree_first_bin(w, 128) == 0
    u = gi.unit_cube(31, 16, pb.dim)
    with sampler_from(gw, pb, 1, n_live=24, k=12, steps_per_dim=1, seed=5) as sp:
        assert sp.stats()["mixed_tile"] == 128
        s0 = sp.stats()
        got = sp.eval_lnl(u)
        s1 = sp.stats()
        assert s1["batch_point_bins_lo"] - s0["batch_point_bins_lo"] == \
            s1["batch_point_bins"] - s0["batch_point_bins"] > 0
        sp.step()
        s2 = sp.stats()
        assert s2["status"] == 0
        assert s2["point_bins_lo"] - s1["point_bins_lo"] == s2["point_bins"] - s1["point_bins"] > 0
        uu, l = sp.live()
    assert np.max(np.abs(got - pb.loglike(u))) < MIXED_ATOL
    assert np.max(np.abs(l - pb.loglike(uu))) < MIXED_ATOL


def test_low_degree_bins_are_counted(gw):
    """The mixed batched likelihood on the 519,169-bin grid sums the tile groups
    from 276 Hz up at Taylor degree 3 and counts their bins: per point, the bins
    from that group's first bin up to its f_ISCO cutoff (from the oracle), and
    in all the bins up to the cutoff."""
    w, pb, th = problem("c4")
    u = gi.unit_cube(29, 64, pb.dim)
    theta = pb.theta(u)
    f = w.f0 + np.arange(w.N) * w.df
    jcut = np.array([np.searchsorted(f, oracle.fisco(t), side="right") - 1 for t in theta])
    lo_bin = _low_degree_first_bin(w, 128)
    assert abs(w.f0 + lo_bin * w.df - 276.0) < 1e-9
    with sampler_from(gw, pb, 1, n_live=8) as sp:
        assert sp.stats()["mixed_tile"] == 128
        s0 = sp.stats()
        got = sp.eval_lnl(u)
        s1 = sp.stats()
    assert s1["batch_point_bins"] - s0["batch_point_bins"] == int(np.sum(jcut + 1))
    want_lo = int(np.sum(np.maximum(jcut + 1 - lo_bin, 0)))
    assert 0 < want_lo < int(np.sum(jcut + 1))
    assert s1["batch_point_bins_lo"] - s0["batch_point_bins_lo"] == want_lo
    assert np.max(np.abs(got - pb.loglike(u))) < MIXED_ATOL


def test_work_shared_wait_timeout_is_reported(gw, monkeypatch):
    """The work-shared update's waits are bounded. With the test hook
    GWNS_TEST_WS_STALL=1 (read at ns_init) each chain's owner waits for one
    chunk more than its round has; the wait runs out after some seconds, the
    chains end at their current points, and ns_step returns NS_ERR_TIMEOUT with
    status bit 1 set. Nothing faults: a context created without the hook then
    runs normally."""
    import time
    w, pb, th = problem("c4")
    monkeypatch.setenv("GWNS_TEST_WS_STALL", "1")
    sp = sampler_from(gw, pb, 1, n_live=8, k=2, steps_per_dim=1, seed=3)
    monkeypatch.delenv("GWNS_TEST_WS_STALL")
    t0 = time.time()
    with pytest.raises(gw.GWNSError) as err:
        sp.step()
    assert err.value.code == -6          # NS_ERR_TIMEOUT
    assert sp.stats()["status"] & 2
    sp.close()
    assert time.time() - t0 < 120
    with sampler_from(gw, pb, 1, n_live=8, k=2, steps_per_dim=1, seed=3) as sp2:
        sp2.step()
        assert sp2.stats()["status"] == 0


@pytest.mark.parametrize("slots", [1, 2, 4])
def test_mixed_tiled_form_in_slice_update(gw, slots):
    """A fine grid below the cooperative size (8000 bins at 1/32 Hz, 32-bin
    tiles): each slot warp runs the direct tiled form on its own candidate;
    live points after one iteration agree with the oracle per point."""
    w, pb, th = problem("c1", N=8000, df=0.03125)
    with sampler_from(gw, pb, 1, n_live=60, k=30, steps_per_dim=2, seed=7, slots=slots) as sp:
        sp.step()
        u, l = sp.live()
    want = pb.loglike(u)
    assert np.max(np.abs(l - want)) < MIXED_ATOL


def test_mixed_rotation_in_slice_update(gw):
    """Eight one-warp slots on 128-bin tiles: each slot warp sums its
    candidate's tiles by rotation; live points after one iteration agree with
    the oracle per point."""
    w, pb, th = problem("c1", N=12000, df=1 / 128)
    with sampler_from(gw, pb, 1, n_live=60, k=30, steps_per_dim=2, seed=7, slots=8) as sp:
        assert sp.stats()["mixed_tile"] == 128
        sp.step()
        u, l = sp.live()
        assert sp.stats()["status"] == 0
    want = pb.loglike(u)
    assert np.max(np.abs(l - want)) < MIXED_ATOL


@pytest.mark.parametrize("precision", [0, 1])
def test_c1_model_run_against_oracle(gw, precision):
    """The 3-detector, 11-parameter, 4017-bin model (300 live points, 150
    deleted per iteration): a per-parameter two-sample KS test of the
    posteriors against the oracle's run at p > 0.01. FP64: the oracle's run
    itself (same draws). Mixed: log Z agrees with the FP64 form's over 8 seed
    pairs (a single run against the oracle's would pass or fail with the seed:
    the run-to-run scatter is several times dlogZ)."""
    w, pb, th = problem("c1")
    n_live, k = 300, 150
    ref = ons.run(pb, n_live=n_live, k=k, steps=w.steps_per_dim * pb.dim, seed=w.seed_sampler)
    with sampler_from(gw, pb, precision, n_live=n_live, k=k, steps_per_dim=w.steps_per_dim,
                      seed=w.seed_sampler) as sp:
        sp.run()
        r = sp.result()
    if precision == 1:
        _assert_mixed_log_z_agrees(_mixed_log_z_pairs(gw, pb, n_live, k, w.steps_per_dim, w.seed_sampler))
    lw_g = r["logw"] + r["logl"] - r["logZ"]
    lw_o = ref["logw"] + ref["logl"] - ref["logZ"]
    sg = ons.equal_weight_resample(r["u"], lw_g, 1)
    so = ons.equal_weight_resample(ref["samples_u"], lw_o, 2)
    for i in range(pb.dim):
        assert stats.ks_2samp(sg[:, i], so[:, i]).pvalue > 0.01, i
    if precision == 0:
        # same draws, FP64 on both sides: the same run
        assert r["logZ"] == pytest.approx(ref["logZ"], abs=1e-6)
