"""Pins of the CPU oracle to things other than itself: published known-answer
vectors, closed forms, textbook special cases, mathematical identities and
distributional facts. None of these tests needs a GPU."""
import math
import os

import numpy as np
import pytest
from scipy import stats

import gwinputs as gi
import oracle
from oracle import ns as ons

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TSUN = 4.925490947641267e-6
C_SI = 299792458.0
MPC = 3.085677581491367e22


# ----------------------------------------------------------------- Philox
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        ctr = [int(x, 16) for x in r[0:4]]
        key = [int(x, 16) for x in r[4:6]]
        want = [int(x, 16) for x in r[6:10]]
        assert list(oracle.philox(ctr, key)) == want


def test_u01_open_interval_and_resolution():
    assert oracle.u01(0, 0) == 0.5 * 2.0 ** -52
    assert oracle.u01(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 0.5 * 2.0 ** -52
    assert 0.0 < oracle.u01(0, 0) < oracle.u01(0xFFFFFFFF, 0xFFFFFFFF) < 1.0


def test_initial_points_uniform():
    u = oracle.initial_points(123, 4000, 5)
    assert u.shape == (4000, 5)
    for i in range(5):
        assert stats.kstest(u[:, i], "uniform").pvalue > 1e-3


# ------------------------------------------------------- TaylorF2 phasing
def _energy_flux_coeffs(eta):
    ns = {"pi": math.pi, "gammaE": 0.5772156649015329, "ln2": math.log(2.0), "eta": eta}
    out = {}
    for line in open(os.path.join(GOLDEN, "pn_energy_flux.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        name, expr = line.split(None, 1)
        out[name] = float(eval(expr.replace("^", "**"), {"__builtins__": {}}, ns))
    return out


def _phase_from_energy_balance(eta, v):
    """TaylorF2 phase (up to a constant and a term linear in f) derived from the
    energy-balance equations dt/dv = -E'(v)/F(v), dphi/dv = v^3 dt/dv and the
    stationary-phase relation Psi = 2 pi f t - 2 phi (M = 1 units), by series
    re-expansion of 1/F and term-by-term integration."""
    c = _energy_flux_coeffs(eta)
    b = {0: 1.0, 1: 0.0, 2: c["f2"], 3: c["f3"], 4: c["f4"], 5: c["f5"], 6: c["f6"], 7: c["f7"]}
    b6l = c["f6l"]
    inv = {0: 1.0}
    inv_l = {0: 0.0}      # coefficient of ln v
    for k in range(1, 8):
        inv[k] = -sum(b[i] * inv[k - i] for i in range(1, k + 1))
        inv_l[k] = -sum(b[i] * inv_l[k - i] for i in range(1, k + 1)) - (b6l * inv[k - 6] if k >= 6 else 0.0)
    num = {0: 1.0, 1: 0.0, 2: 2 * c["e2"], 3: 0.0, 4: 3 * c["e4"], 5: 0.0, 6: 4 * c["e6"], 7: 0.0}
    a = {k: sum(num[i] * inv[k - i] for i in range(k + 1)) for k in range(8)}
    al = {k: sum(num[i] * inv_l[k - i] for i in range(k + 1)) for k in range(8)}
    assert all(abs(al[k]) < 1e-14 for k in range(8) if k != 6)
    pref = 5.0 / (32.0 * eta)
    lv = np.log(v)
    # t(v) and phi(v) by term-by-term integration of pref * sum_k a_k v^(k-9)
    t = np.zeros_like(v)
    phi = np.zeros_like(v)
    for k in range(8):
        t += pref * a[k] * v ** (k - 8) / (k - 8)
        if k == 5:
            phi += pref * a[k] * lv
        else:
            phi += pref * a[k] * v ** (k - 5) / (k - 5)
    t += pref * al[6] * (-lv / (2 * v ** 2) - 1.0 / (4 * v ** 2))
    phi += pref * al[6] * (v * lv - v)
    return 2.0 * v ** 3 * t - 2.0 * phi


@pytest.mark.parametrize("mc,q", [(25.0, 0.8), (10.0, 0.25), (1.2, 1.0)])
def test_phasing_matches_energy_balance(mc, q):
    th = np.zeros(gi.NPARAM)
    th[gi.P_MC], th[gi.P_Q], th[gi.P_DL], th[gi.P_COSI] = mc, q, 100.0, 1.0
    eta = q / (1 + q) ** 2
    M = mc * eta ** -0.6 * TSUN
    fisco = 1.0 / (6 ** 1.5 * math.pi * M)
    f = np.linspace(20.0, min(fisco, 1000.0), 400)
    v = np.cbrt(math.pi * M * f)
    psi_o = np.array([oracle.phase(th, x) for x in f])
    psi_d = _phase_from_energy_balance(eta, v) - math.pi / 4
    r = psi_o - psi_d
    A = np.stack([np.ones_like(f), f], axis=1)
    coef, *_ = np.linalg.lstsq(A, r, rcond=None)
    resid = r - A @ coef
    assert np.max(np.abs(resid)) < 1e-6 * max(1.0, np.max(np.abs(psi_o)) * 1e-6), np.max(np.abs(resid))


def test_newtonian_phase_spa_time():
    """d Psi_N/df = 2 pi t(f) with t(f) = t_c - (5/256) T_Mc (pi T_Mc f)^(-8/3)."""
    eta = 0.2
    f = np.linspace(30.0, 300.0, 50)
    mc = 20.0
    tmc = mc * TSUN
    M = tmc * eta ** -0.6
    h = 1e-3
    def psi_n(ff):
        v = np.cbrt(math.pi * M * ff)
        return 3.0 / (128 * eta * v ** 5) * oracle.pn_phi(eta, math.sqrt(1 - 4 * eta), 0, 0, v)[0]
    dpsi = np.array([(psi_n(x + h) - psi_n(x - h)) / (2 * h) for x in f])
    t = -(5.0 / 256.0) * tmc * (math.pi * tmc * f) ** (-8.0 / 3.0)
    np.testing.assert_allclose(dpsi, 2 * math.pi * t, rtol=1e-6)


def test_spin_terms_mass_weighted_form():
    """beta = (1/12) sum_i [113 (m_i/M)^2 + 75 eta] chi_i and
    sigma = (eta/48)(721 - 247) chi1 chi2 for aligned spins (Cutler & Flanagan 1994 form)."""
    for q, c1, c2 in [(0.8, 0.3, -0.2), (0.3, -0.45, 0.4), (1.0, 0.1, 0.1)]:
        eta = q / (1 + q) ** 2
        m1, m2 = 1.0 / (1 + q), q / (1 + q)
        beta = (113 * m1 ** 2 + 75 * eta) * c1 / 12 + (113 * m2 ** 2 + 75 * eta) * c2 / 12
        sigma = eta / 48 * (721 - 247) * c1 * c2
        v = 0.2
        delta = (1 - q) / (1 + q)
        p = oracle.pn_phi(eta, delta, c1, c2, v)
        p0 = oracle.pn_phi(eta, delta, 0.0, 0.0, v)
        assert p[3] - p0[3] == pytest.approx(4 * beta, rel=1e-13, abs=1e-13)
        assert p[4] - p0[4] == pytest.approx(-10 * sigma, rel=1e-13, abs=1e-13)


def _spin_orbit_terms(eta, m1, m2, chi1, chi2):
    ns = {"eta": eta, "S": m1 * m1 * chi1 + m2 * m2 * chi2, "Sig": m2 * chi2 - m1 * chi1, "d": m1 - m2}
    out = {}
    for line in open(os.path.join(GOLDEN, "pn_spin_orbit.txt")):
        if not line.strip() or line.startswith("#"):
            continue
        name, expr = line.split(None, 1)
        out[name] = float(eval(expr, {"__builtins__": {}}, ns))
    return out


def _energy_balance_series(eta, so):
    """Coefficients a_k (k <= 5) of -E'(v)/F(v) / (v^-9 (5/32)/eta), the
    integrand of the energy balance, with the spin-orbit terms `so` added."""
    c = _energy_flux_coeffs(eta)
    b = {0: 1.0, 1: 0.0, 2: c["f2"], 3: c["f3"] + so.get("f3s", 0.0), 4: c["f4"], 5: c["f5"] + so.get("f5s", 0.0)}
    inv = {0: 1.0}
    for k in range(1, 6):
        inv[k] = -sum(b[i] * inv[k - i] for i in range(1, k + 1))
    num = {0: 1.0, 1: 0.0, 2: 2 * c["e2"], 3: 2.5 * so.get("e3s", 0.0), 4: 3 * c["e4"],
           5: 3.5 * so.get("e5s", 0.0)}
    return {k: sum(num[i] * inv[k - i] for i in range(k + 1)) for k in range(6)}


@pytest.mark.parametrize("q,chi1,chi2", [(0.8, 0.3, 0.0), (0.3, 0.0, 0.4), (0.5, -0.45, 0.2), (1.0, 0.2, -0.1)])
def test_spin_orbit_phasing_matches_energy_balance(q, chi1, chi2):
    """The 1.5PN and 2.5PN spin-orbit phase terms (4 beta and -gamma) from the
    spin-orbit parts of the energy and flux: term-by-term integration of the
    energy balance gives psi_3 = 4 a_3 and, from the ln v term of the 2.5PN
    order, psi_5 = -(40/9) a_5 (the same steps as the non-spinning pin)."""
    eta = q / (1 + q) ** 2
    m1, m2 = 1.0 / (1 + q), q / (1 + q)
    a = _energy_balance_series(eta, _spin_orbit_terms(eta, m1, m2, chi1, chi2))
    a0 = _energy_balance_series(eta, {})
    v = 0.21
    delta = (1 - q) / (1 + q)
    p = oracle.pn_phi(eta, delta, chi1, chi2, v)
    p0 = oracle.pn_phi(eta, delta, 0.0, 0.0, v)
    log_factor = 1.0 + 3.0 * math.log(v * math.sqrt(6.0))
    assert p[3] - p0[3] == pytest.approx(4 * (a[3] - a0[3]), rel=1e-12, abs=1e-12)
    assert (p[5] - p0[5]) / log_factor == pytest.approx(-40.0 / 9.0 * (a[5] - a0[5]), rel=1e-12, abs=1e-12)


# ----------------------------------------------------------------- amplitude
def test_amplitude_matches_time_domain_chirp():
    """Face-on |h_+(f)| = h0(f) / (2 sqrt(fdot)) with the quadrupole chirp
    h0 = 4 c T_Mc^(5/3) (pi f)^(2/3) / D and fdot = (96/5) pi^(8/3) T_Mc^(5/3) f^(11/3)."""
    th = np.zeros(gi.NPARAM)
    th[gi.P_MC], th[gi.P_Q], th[gi.P_DL], th[gi.P_COSI] = 18.0, 0.7, 410.0, 1.0
    tmc = th[gi.P_MC] * TSUN
    D = th[gi.P_DL] * MPC
    for f in [20.0, 55.5, 131.0]:
        hp, hc = oracle.polarizations(th, f)
        h0 = 4 * C_SI * tmc ** (5 / 3) * (math.pi * f) ** (2 / 3) / D
        fdot = 96 / 5 * math.pi ** (8 / 3) * tmc ** (5 / 3) * f ** (11 / 3)
        assert abs(hp) == pytest.approx(h0 / (2 * math.sqrt(fdot)), rel=1e-12, abs=0)
        # circular polarisation face-on: h_x = -i h_+
        assert hc == pytest.approx(-1j * hp, rel=1e-12, abs=0)


def test_polarizations_edge_on():
    """Edge-on (cos i = 0): the cross polarisation vanishes and |h_+| is half
    the face-on amplitude of the quadrupole chirp, h0 / (4 sqrt(fdot))."""
    th = np.zeros(gi.NPARAM)
    th[gi.P_MC], th[gi.P_Q], th[gi.P_DL], th[gi.P_COSI], th[gi.P_PHIC] = 18.0, 0.7, 410.0, 0.0, 0.4
    tmc = th[gi.P_MC] * TSUN
    D = th[gi.P_DL] * MPC
    for f in [20.0, 55.5, 131.0]:
        hp, hc = oracle.polarizations(th, f)
        h0 = 4 * C_SI * tmc ** (5 / 3) * (math.pi * f) ** (2 / 3) / D
        fdot = 96 / 5 * math.pi ** (8 / 3) * tmc ** (5 / 3) * f ** (11 / 3)
        assert hc == 0
        assert abs(hp) == pytest.approx(h0 / (4 * math.sqrt(fdot)), rel=1e-12, abs=0)


def test_polarizations_orientation_average_is_four_fifths():
    """Averaged over an isotropic orientation (cos i uniform on [-1, 1]), the
    polarisation power (|h_+|^2 + |h_x|^2) / |h_+(face-on)|^2 is 4/5 (the
    quadrupole radiation pattern (1 + cos^2 i)^2/4 + cos^2 i). Gauss-Legendre
    quadrature over the oracle's own polarisations; a wrong power of cos i in
    either polarisation changes the average."""
    th = np.zeros(gi.NPARAM)
    th[gi.P_MC], th[gi.P_Q], th[gi.P_DL], th[gi.P_PHIC] = 27.0, 0.55, 800.0, 2.1
    x, w = np.polynomial.legendre.leggauss(8)
    for f in [25.0, 90.0]:
        th[gi.P_COSI] = 1.0
        ref = abs(oracle.polarizations(th, f)[0]) ** 2
        avg = 0.0
        for ci, wi in zip(x, w):
            th[gi.P_COSI] = ci
            hp, hc = oracle.polarizations(th, f)
            avg += 0.5 * wi * (abs(hp) ** 2 + abs(hc) ** 2) / ref
        assert avg == pytest.approx(0.8, rel=1e-13)
        # and the two polarisations separately: <(1 + c^2)^2/4> = 7/15, <c^2> = 1/3
        ap = sum(0.5 * wi * abs(oracle.polarizations(np.where(np.arange(gi.NPARAM) == gi.P_COSI, ci, th), f)[0]) ** 2
                 for ci, wi in zip(x, w)) / ref
        ac = sum(0.5 * wi * abs(oracle.polarizations(np.where(np.arange(gi.NPARAM) == gi.P_COSI, ci, th), f)[1]) ** 2
                 for ci, wi in zip(x, w)) / ref
        assert ap == pytest.approx(7 / 15, rel=1e-13)
        assert ac == pytest.approx(1 / 3, rel=1e-13)


def test_equal_mass_limit_is_finite():
    """q -> 1: (m1 - m2)/M -> 0 and the likelihood stays finite."""
    w = gi.workload("c1")
    w.N = 200
    pb, th = oracle.make_problem(w)
    u = np.full((1, pb.dim), 1.0 - 1e-12)
    assert np.isfinite(pb.loglike(u)[0])
    th2 = th.copy()
    th2[gi.P_Q] = 1.0
    assert np.isfinite(pb.loglike_theta(th2)[0])


def test_isco_frequency():
    th = np.zeros(gi.NPARAM)
    th[gi.P_MC], th[gi.P_Q] = 10.0, 1.0
    M = 10.0 * 0.25 ** -0.6  # solar masses
    # f_ISCO = c^3 / (6^(3/2) pi G M) ~ 4397 Hz / (M / Msun)
    assert oracle.fisco(th) == pytest.approx(1.0 / (6 ** 1.5 * math.pi * M * TSUN), rel=1e-14)
    assert oracle.fisco(th) * M == pytest.approx(4397.0, rel=1e-3)


# --------------------------------------------------------- antenna, delays
def _rand_unit(rng):
    x = rng.standard_normal(3)
    return x / np.linalg.norm(x)


def test_antenna_psi_invariance_and_bounds():
    pos, xa, ya = gi.detectors(7, 3)
    rng = np.random.default_rng(3)
    for _ in range(20):
        ra, sd = rng.uniform(0, 2 * math.pi), rng.uniform(-1, 1)
        vals = []
        for psi in np.linspace(0, math.pi, 7):
            fp, fc = oracle.antenna(xa[0], ya[0], ra, sd, psi)
            vals.append(fp * fp + fc * fc)
        assert np.ptp(vals) < 1e-13
        assert vals[0] <= 1.0 + 1e-14


def _textbook_pattern(cos_th, phi, psi):
    """F+ and Fx of an L-shaped detector with arms along x and y, for a source
    at polar angle th and azimuth phi in the detector frame and polarisation
    angle psi: the standard interferometer response of the gravitational-wave
    literature (e.g. Sathyaprakash and Schutz, Living Rev. Rel. 12 (2009) 2,
    eq. 34), written here from that statement."""
    a = 0.5 * (1.0 + cos_th * cos_th) * math.cos(2 * phi)
    b = cos_th * math.sin(2 * phi)
    return a * math.cos(2 * psi) - b * math.sin(2 * psi), a * math.sin(2 * psi) + b * math.cos(2 * psi)


def test_antenna_textbook_pole_detector():
    """Arms along x and y at the north pole: F+ and Fx each equal the textbook
    pattern with th = pi/2 - dec, phi = RA and the textbook polarisation angle
    pi/2 - psi (the wave frame of Anderson et al. 2001 measures psi from the
    other axis and in the opposite sense). Swapping F+ and Fx or flipping the
    sign of either fails this."""
    x, y = np.array([1.0, 0, 0]), np.array([0, 1.0, 0])
    rng = np.random.default_rng(5)
    for _ in range(40):
        ra, sd, psi = rng.uniform(0, 2 * math.pi), rng.uniform(-1, 1), rng.uniform(0, math.pi)
        fp, fc = oracle.antenna(x, y, ra, sd, psi)
        want_p, want_c = _textbook_pattern(sd, ra, 0.5 * math.pi - psi)
        assert fp == pytest.approx(want_p, abs=1e-13)
        assert fc == pytest.approx(want_c, abs=1e-13)
    # special directions, with the textbook angle psi' = pi/2 - psi: overhead
    # (th = 0) F+ = cos 2psi' = -cos 2psi and Fx = sin 2psi' = sin 2psi
    for psi in (0.0, 0.3, 1.1):
        fp, fc = oracle.antenna(x, y, 0.0, 1.0, psi)
        assert fp == pytest.approx(-math.cos(2 * psi), abs=1e-14)
        assert fc == pytest.approx(math.sin(2 * psi), abs=1e-14)
    # in the arms' plane along the x arm (th = pi/2, phi = 0) only the y arm
    # responds: half the overhead response
    for psi in (0.2, 0.9):
        fp, fc = oracle.antenna(x, y, 0.0, 0.0, psi)
        assert fp == pytest.approx(-0.5 * math.cos(2 * psi), abs=1e-14)
        assert fc == pytest.approx(0.5 * math.sin(2 * psi), abs=1e-14)
    # along the diagonal between the arms in their plane (phi = pi/4): no response
    for psi in (0.2, 0.9):
        fp, fc = oracle.antenna(x, y, 0.25 * math.pi, 0.0, psi)
        assert fp == pytest.approx(0.0, abs=1e-14)
        assert fc == pytest.approx(0.0, abs=1e-14)


def test_antenna_rotated_arms_shift_the_azimuth():
    """Arms rotated by alpha about the local vertical (pole detector): the
    pattern is the textbook one at azimuth phi - alpha."""
    rng = np.random.default_rng(8)
    for alpha in (0.4, 1.3, -2.0):
        x = np.array([math.cos(alpha), math.sin(alpha), 0.0])
        y = np.array([-math.sin(alpha), math.cos(alpha), 0.0])
        for _ in range(10):
            ra, sd, psi = rng.uniform(0, 2 * math.pi), rng.uniform(-1, 1), rng.uniform(0, math.pi)
            fp, fc = oracle.antenna(x, y, ra, sd, psi)
            want_p, want_c = _textbook_pattern(sd, ra - alpha, 0.5 * math.pi - psi)
            assert fp == pytest.approx(want_p, abs=1e-13)
            assert fc == pytest.approx(want_c, abs=1e-13)


def test_antenna_sky_average_is_one_fifth():
    """Averaged over an isotropic sky and polarisation angle, <F+^2> = <Fx^2> =
    1/5 and <F+ Fx> = 0 for any orthogonal-arm detector (quadrature: Gauss-
    Legendre in sin dec, trapezoid in RA and psi, exact for these trigonometric
    polynomials)."""
    pos, xa, ya = gi.detectors(13, 2)
    xg, wg = np.polynomial.legendre.leggauss(12)
    ras = np.linspace(0, 2 * math.pi, 16, endpoint=False)
    psis = np.linspace(0, math.pi, 8, endpoint=False)
    for i in range(2):
        spp = scc = spc = 0.0
        for sd, wsd in zip(xg, wg):
            for ra in ras:
                for psi in psis:
                    fp, fc = oracle.antenna(xa[i], ya[i], ra, sd, psi)
                    wt = 0.5 * wsd / (len(ras) * len(psis))
                    spp += wt * fp * fp
                    scc += wt * fc * fc
                    spc += wt * fp * fc
        assert spp == pytest.approx(0.2, abs=1e-12)
        assert scc == pytest.approx(0.2, abs=1e-12)
        assert spc == pytest.approx(0.0, abs=1e-12)


def test_antenna_zenith_and_delay():
    pos, xa, ya = gi.detectors(11, 3)
    for i in range(3):
        u = pos[i] / np.linalg.norm(pos[i])
        ra = math.atan2(u[1], u[0])
        sd = u[2]
        fp, fc = oracle.antenna(xa[i], ya[i], ra, sd, 0.3)
        assert fp * fp + fc * fc == pytest.approx(1.0, rel=1e-12)
        assert oracle.delay(pos[i], ra, sd) == pytest.approx(-gi.EARTH_RADIUS_M / C_SI, rel=1e-12)
        # antipodal source arrives later by the same amount
        assert oracle.delay(pos[i], ra + math.pi, -sd) == pytest.approx(gi.EARTH_RADIUS_M / C_SI, rel=1e-12)
    rng = np.random.default_rng(2)
    for _ in range(50):
        ra, sd = rng.uniform(0, 2 * math.pi), rng.uniform(-1, 1)
        dts = [oracle.delay(pos[i], ra, sd) for i in range(3)]
        for i in range(3):
            for j in range(3):
                assert abs(dts[i] - dts[j]) <= np.linalg.norm(pos[i] - pos[j]) / C_SI + 1e-15


# --------------------------------------------------------- inner products
def _c1_small(N=None, noise=True, seed_noise=2001):
    w = gi.workload("c1")
    if N is not None:
        w.N = N
    w.noise = noise
    w.seed_noise = seed_noise
    return oracle.make_problem(w)


def test_noise_normalisation_and_inner_product_variance():
    """E<n|n> = 2N (chi^2 with 2 dof per bin) and Var<n|h> = <h|h>."""
    pb, th = _c1_small(N=1200, noise=False)
    h = pb.strain(th, 0)
    hh = pb.inner(0, h, h)
    nn, nh = [], []
    for s in range(300):
        n = gi.noise(9000 + s, pb.psd[:1], pb.df)[0]
        nn.append(pb.inner(0, n, n))
        nh.append(pb.inner(0, n, h))
    assert np.mean(nn) == pytest.approx(2 * pb.N, rel=0.01)
    assert np.var(nh) == pytest.approx(hh, rel=0.2)
    assert abs(np.mean(nh)) < 4 * math.sqrt(hh / 300)


def test_injection_identity_noise_free():
    """Noise-free data d = h(theta_inj): log L(theta_inj) = rho^2 / 2."""
    for name in ["c0", "c1"]:
        w = gi.workload(name)
        w.noise = False
        pb, th = oracle.make_problem(w)
        ll = pb.loglike_theta(th)[0]
        rho2 = pb.snr2(th)
        assert rho2 == pytest.approx(w.snr ** 2, rel=1e-12)
        assert ll == pytest.approx(rho2 / 2, rel=1e-12)


def test_loglike_equals_residual_form():
    """log L = -<d-h|d-h>/2 + <d|d>/2 summed over detectors."""
    pb, th0 = _c1_small()
    u = gi.unit_cube(77, 5, pb.dim)
    for ui in u:
        th = pb.theta(ui)[0]
        total = 0.0
        for d in range(pb.n_det):
            h = pb.strain(th, d)
            dd = pb.data()[d]
            total += -0.5 * pb.inner(d, dd - h, dd - h) + 0.5 * pb.inner(d, dd, dd)
        assert pb.loglike_theta(th)[0] == pytest.approx(total, rel=1e-9, abs=1e-9)


def test_hh_closed_form_tiny_grid():
    """<h|h> = A^2 |Q|^2 4 df sum_{f_j <= f_ISCO} f_j^(-7/3) / S_j on an N = 33 grid."""
    w = gi.workload("c1")
    w.N, w.df, w.noise = 33, 4.0, False
    pb, th = oracle.make_problem(w)
    f = w.freqs()
    for d in range(3):
        fp, fc = oracle.antenna(pb.xarm[d], pb.yarm[d], th[gi.P_RA], th[gi.P_SINDEC], th[gi.P_PSI])
        ci = th[gi.P_COSI]
        q2 = (fp * (1 + ci * ci) / 2) ** 2 + (fc * ci) ** 2
        A = oracle.amplitude(th, 1.0)
        mask = f <= oracle.fisco(th)
        want = A * A * q2 * 4 * w.df * np.sum(f[mask] ** (-7 / 3) / pb.psd[d][mask])
        h = pb.strain(th, d)
        assert pb.inner(d, h, h) == pytest.approx(want, rel=1e-12, abs=0)


# ---------------------------------------------------------------- prior
def test_prior_transform_distributions():
    pb, _ = _c1_small(N=64)
    u = gi.unit_cube(5, 3000, pb.dim)
    th = pb.theta(u)
    lo, hi = pb.lo[gi.P_DL], pb.hi[gi.P_DL]
    cdf = lambda x: (np.clip(x, lo, hi) ** 3 - lo ** 3) / (hi ** 3 - lo ** 3)
    assert stats.kstest(th[:, gi.P_DL], cdf).pvalue > 1e-3
    mc = th[:, gi.P_MC]
    assert stats.kstest((mc - 10) / 30, "uniform").pvalue > 1e-3


# --------------------------------------------------------- slice sampling
def test_chains_without_constraint_are_uniform():
    """With L* = -inf every point of the cube is in the slice, so the chains
    sample the uniform distribution."""
    pb = oracle.toy_problem(3)
    k, d = 2000, 3
    surv = oracle.initial_points(1, 500, d)
    surv_l = pb.loglike(surv)
    chol = np.linalg.cholesky(np.cov(surv.T))
    new_u = np.zeros((k, d))
    new_l = np.zeros(k)
    caps = np.zeros(1, dtype=np.int32)
    oracle.lib().or_evolve(pb.c, 4, 99, 0, k, oracle._ptr(surv), oracle._ptr(surv_l), 500,
                           oracle._ptr(np.ascontiguousarray(chol)), -np.inf, 6, 64, 64,
                           oracle._ptr(new_u), oracle._ptr(new_l), oracle._ptr(caps))
    for i in range(d):
        assert stats.kstest(new_u[:, i], "uniform").pvalue > 1e-3
    assert caps[0] == 0


def test_periodic_coordinates_wrap_on_the_slice_line():
    """All coordinates periodic and L* = -inf: no candidate ever leaves the
    (wrapped) box, so stepping out runs to its cap on both sides and every
    slice step costs exactly 2 * max_stepout + 1 evaluations; the chains
    still sample the uniform distribution on the torus."""
    d, k, steps, cap = 3, 1500, 4, 8
    pb = oracle.toy_problem(d)
    assert pb.set_periodic(range(d)) == 0b111
    surv = oracle.initial_points(1, 500, d)
    surv_l = pb.loglike(surv)
    chol = np.ascontiguousarray(np.linalg.cholesky(np.cov(surv.T)))
    new_u, new_l = np.zeros((k, d)), np.zeros(k)
    caps = np.zeros(1, dtype=np.int32)
    ev = oracle.lib().or_evolve(pb.c, 4, 7, 0, k, oracle._ptr(surv), oracle._ptr(surv_l), 500,
                                oracle._ptr(chol), -np.inf, steps, cap, 64,
                                oracle._ptr(new_u), oracle._ptr(new_l), oracle._ptr(caps))
    assert ev == k * steps * (2 * cap + 1)
    assert np.all((new_u >= 0.0) & (new_u <= 1.0))
    for i in range(d):
        assert stats.kstest(new_u[:, i], "uniform").pvalue > 1e-3
    # without wrapping the box stops stepping out early
    pb.set_periodic(())
    ev2 = oracle.lib().or_evolve(pb.c, 4, 7, 0, k, oracle._ptr(surv), oracle._ptr(surv_l), 500,
                                 oracle._ptr(chol), -np.inf, steps, cap, 64,
                                 oracle._ptr(new_u), oracle._ptr(new_l), oracle._ptr(caps))
    assert ev2 < ev


def test_gw_likelihood_is_periodic_in_the_wrapped_parameters():
    """phi_c (period 2 pi), psi (period pi: F+ and Fx are unchanged under
    psi -> psi + pi) and RA (period 2 pi) with their full-period uniform
    priors: log L takes the same value on opposite faces of the unit cube, which
    is what makes wrapping these coordinates exact."""
    w = gi.workload("c1", N=513)
    pb, th = oracle.make_problem(w)
    order = [p for p in range(gi.NPARAM) if pb.kind[p] != gi.PRIOR_FIXED]
    u = gi.unit_cube(31, 12, pb.dim)
    for p in (gi.P_PHIC, gi.P_PSI, gi.P_RA):
        i = order.index(p)
        a, b = u.copy(), u.copy()
        a[:, i], b[:, i] = 0.0, 1.0
        la, lb = pb.loglike(a), pb.loglike(b)
        assert np.max(np.abs(la - lb) / np.maximum(1.0, np.abs(la))) < 1e-9, p
    # and not in a non-periodic one (the chirp mass)
    i = order.index(gi.P_MC)
    a, b = u.copy(), u.copy()
    a[:, i], b[:, i] = 0.0, 1.0
    assert np.max(np.abs(pb.loglike(a) - pb.loglike(b))) > 1.0


def _walk(pb, surv, lstar, k, walk, seed=3, scale=None):
    d = pb.dim
    surv_l = pb.loglike(surv)
    chol = np.ascontiguousarray(np.linalg.cholesky(np.cov(surv.T)))
    new_u, new_l = np.zeros((k, d)), np.zeros(k)
    acc = np.zeros(1, dtype=np.int64)
    ev = oracle.lib().or_evolve_walk(pb.c, 4, seed, 0, k, oracle._ptr(surv), oracle._ptr(surv_l), len(surv),
                                     oracle._ptr(chol), lstar, walk, scale or ons.walk_scale_default(d),
                                     oracle._ptr(new_u), oracle._ptr(new_l), oracle._ptr(acc))
    return new_u, new_l, ev, int(acc[0])


def test_random_walk_without_constraint_is_uniform():
    """L* = -inf: the walk is a Metropolis chain for the uniform prior (symmetric
    proposals, rejection outside the box), so it stays uniform; every in-box
    proposal is evaluated and accepted, so evaluations = accepted moves."""
    d, k, walk = 3, 2000, 6
    pb = oracle.toy_problem(d)
    surv = oracle.initial_points(1, 500, d)
    u, l, ev, acc = _walk(pb, surv, -np.inf, k, walk)
    for i in range(d):
        assert stats.kstest(u[:, i], "uniform").pvalue > 1e-3
    assert ev == acc and 0 < acc < k * walk


def test_walk_length_rule():
    """Between iterations the walk length is rescaled towards the target of
    accepted moves per walk: walk * target * k / accepted, rounded up and kept
    within [target, 64 target]."""
    L = oracle.lib()
    assert L.or_walk_next(110, 55, 500, 500 * 55) == 110          # on target
    assert L.or_walk_next(110, 55, 500, 500 * 55 // 2) == 220     # half the moves: twice the length
    assert L.or_walk_next(110, 55, 500, 10 ** 9) == 55            # floor
    assert L.or_walk_next(110, 55, 500, 1) == 64 * 55             # ceiling
    assert L.or_walk_next(110, 55, 500, 0) == 64 * 55
    assert L.or_walk_next(100, 55, 3, 7) == math.ceil(100 * 55 * 3 / 7)


def test_random_walk_samples_the_constrained_prior():
    """Toy Gaussian with L > L*: the walk leaves the uniform law on the
    ellipsoid x^T P x < r*^2 invariant, so (x^T P x / r*^2)^(d/2) ~ U(0, 1)."""
    d = 4
    pb = oracle.toy_problem(d)
    prec = np.linalg.inv(gi.toy_covariance(d, gi.TOY_RHO))
    r2 = 9.0
    lstar = -0.5 * r2 + pb.toy_lognorm
    # survivors: uniform in the ellipsoid (rejection from the prior box)
    u = oracle.initial_points(2, 200000, d)
    x = gi.TOY_BOX[0] + (gi.TOY_BOX[1] - gi.TOY_BOX[0]) * u
    q = np.einsum("ni,ij,nj->n", x, prec, x)
    surv = np.ascontiguousarray(u[q < r2][:400])
    new_u, new_l, ev, acc = _walk(pb, surv, lstar, 3000, 6 * d)
    x = gi.TOY_BOX[0] + (gi.TOY_BOX[1] - gi.TOY_BOX[0]) * new_u
    q = np.einsum("ni,ij,nj->n", x, prec, x)
    assert np.all(q < r2) and np.all(new_l > lstar)
    assert stats.kstest((q / r2) ** (d / 2), "uniform").pvalue > 1e-3


def test_survivor_covariance():
    """L L^T is numpy's unbiased sample covariance (up to the 1e-12 tr/d
    jitter); a single survivor falls back to the unit cube's covariance I/12."""
    rng = np.random.default_rng(5)
    surv = rng.uniform(size=(37, 5))
    L = ons.survivor_cholesky(surv)
    want = np.cov(surv.T)
    assert np.allclose(L @ L.T, want + 1e-12 * np.trace(want) / 5 * np.eye(5), rtol=1e-12, atol=1e-15)
    assert np.allclose(np.tril(L), L)
    L1 = ons.survivor_cholesky(surv[:1])
    assert np.allclose(L1 @ L1.T, np.eye(5) / 12.0, rtol=1e-10)


def test_chains_sample_the_constrained_prior():
    """Toy Gaussian with L > L*: the constrained prior is uniform in the
    ellipsoid x^T P x < r*^2, so (x^T P x / r*^2)^(d/2) ~ U(0, 1)."""
    d = 4
    pb = oracle.toy_problem(d)
    st = ons.initial_state(pb, 400, 11)
    for _ in range(6):  # move inside the box, far from its edges
        ons.iterate(pb, st, 200, 5 * d, 11)
    order = np.argsort(st.live_logl, kind="stable")
    k = 200
    lstar = st.live_logl[order[k - 1]]
    surv = np.ascontiguousarray(st.live_u[order[k:]])
    surv_l = np.ascontiguousarray(st.live_logl[order[k:]])
    chol = np.ascontiguousarray(ons.survivor_cholesky(surv))
    kk = 3000
    new_u = np.zeros((kk, d))
    new_l = np.zeros(kk)
    caps = np.zeros(1, dtype=np.int32)
    oracle.lib().or_evolve(pb.c, 4, 5, 1000, kk, oracle._ptr(surv), oracle._ptr(surv_l), 400 - k,
                           oracle._ptr(chol), lstar, 5 * d, 64, 64, oracle._ptr(new_u),
                           oracle._ptr(new_l), oracle._ptr(caps))
    x = -10 + 20 * new_u
    qf = np.einsum("ni,ij,nj->n", x, pb.toy_prec, x)
    r2star = 2 * (pb.toy_lognorm - lstar)
    assert np.all(new_l > lstar)
    assert np.all(qf < r2star * (1 + 1e-12))
    assert stats.kstest((qf / r2star) ** (d / 2), "uniform").pvalue > 1e-3


# --------------------------------------------------------- evidence
@pytest.mark.parametrize("d", [4])
def test_toy_evidence_analytic(d):
    """Analytic log Z = -d ln 20 for a normalised Gaussian well inside [-10,10]^d."""
    pb = oracle.toy_problem(d)
    truth = -d * math.log(20.0)
    # information of the posterior N(0, Sigma) against the uniform prior on the
    # box: H = d ln 20 - ln det(2 pi e Sigma)/2
    h_true = d * math.log(20.0) - 0.5 * np.linalg.slogdet(2 * math.pi * math.e * gi.toy_covariance(d))[1]
    hits = 0
    seeds = range(6)
    hs = []
    for s in seeds:
        r = ons.run(pb, n_live=200, k=100, steps=5 * d, seed=100 + s, replicates=50)
        sig = max(r["dlogZ"], 1e-3)
        hits += abs(r["logZ"] - truth) < 3 * sig
        assert 0.5 * r["dlogZ_info"] < r["dlogZ"] < 2.5 * r["dlogZ_info"]
        hs.append(r["H"])
    assert hits >= 5
    # per run the estimate scatters by ~0.13 at n = 200 (measured over seeds)
    assert np.all(np.abs(np.array(hs) - h_true) < 0.6)
    assert abs(np.mean(hs) - h_true) < 0.2


def _closed_form_state(n, k, iters, dead_level, live_level, d=2):
    """A run state built without the sampler: `iters` iterations of k deletions
    from n live points, every dead point at log L = dead_level, the final live
    points at live_level; the enclosed prior mass after the j-th deletion of an
    iteration is X_j = X_{j-1} exp(-1/(n - j + 1)), so the weight of that point
    is X_{j-1} - X_j. Returns the state and the closed-form X sequence."""
    logx = [0.0]
    st = ons.NSState(live_u=np.full((n, d), 0.5), live_logl=np.full(n, float(live_level)))
    for _ in range(iters):
        lw = []
        for j in range(1, k + 1):
            x0 = logx[-1]
            x1 = x0 - 1.0 / (n - j + 1)
            lw.append(math.log(math.exp(x0) - math.exp(x1)))
            logx.append(x1)
        st.dead_u.append(np.full((k, d), 0.5))
        st.dead_logl.append(np.full(k, float(dead_level)))
        st.dead_logw.append(np.array(lw))
        st.dead_nlive.append(n - np.arange(k, dtype=np.float64))
    st.logX = logx[-1]
    st.logZ = float(np.logaddexp.reduce(np.concatenate(st.dead_logw) + dead_level))
    return st, logx


@pytest.mark.parametrize("dead_level,live_level", [(0.0, 0.0), (0.0, 6.0), (-3.0, 2.5)])
def test_finalize_closed_forms(dead_level, live_level):
    """finalize() against closed forms on two-level likelihoods: the final live
    points add the mass X_k - X_end, X_end = X_k exp(-sum_{j=1..n} 1/j); with
    mass M_dead = 1 - X_k at L_dead and M_live = X_k - X_end at L_live,
    Z = M_dead L_dead + M_live L_live, H = sum_g (M_g L_g / Z) ln(L_g / Z), and
    the Kish ESS is (sum w L)^2 / sum (w L)^2 over the individual weights."""
    n, k, iters = 40, 20, 5
    st, logx = _closed_form_state(n, k, iters, dead_level, live_level)
    r = ons.finalize(st, seed=1, replicates=8)
    x_k = math.exp(logx[-1])
    x_end = x_k * math.exp(-sum(1.0 / j for j in range(1, n + 1)))
    m_dead, m_live = 1.0 - x_k, x_k - x_end
    Z = m_dead * math.exp(dead_level) + m_live * math.exp(live_level)
    assert r["logZ"] == pytest.approx(math.log(Z), abs=1e-12)
    H = (m_dead * math.exp(dead_level) / Z * (dead_level - math.log(Z))
         + m_live * math.exp(live_level) / Z * (live_level - math.log(Z)))
    assert r["H"] == pytest.approx(H, abs=1e-12)
    # individual weights: the dead ones from the closed-form X sequence, the
    # live ones continuing it with Delta_j = 1/(n - j + 1)
    xs = list(np.exp(logx))
    for j in range(1, n + 1):
        xs.append(xs[-1] * math.exp(-1.0 / (n - j + 1)))
    w = -np.diff(np.array(xs))
    lv = np.concatenate([np.full(k * iters, dead_level), np.full(n, live_level)])
    wl = w * np.exp(lv)
    assert r["ess"] == pytest.approx(wl.sum() ** 2 / np.sum(wl ** 2), rel=1e-12)
    assert len(r["logw"]) == k * iters + n
    assert np.allclose(np.exp(r["logw"]), w, rtol=1e-12, atol=0)


def test_log_x_shrinkage_statistics():
    """Estimated ln X against the true prior volume X(L*) of the toy: the
    residual has mean ~0 and variance ~ sum_j 1/(n-j+1)^2."""
    d = 4
    pb = oracle.toy_problem(d)
    sigma = gi.toy_covariance(d)
    logdet = np.linalg.slogdet(2 * math.pi * sigma)[1]
    vd = math.pi ** (d / 2) / math.gamma(d / 2 + 1)
    resid, var = [], []
    n, k = 200, 100
    for s in range(8):
        st = ons.initial_state(pb, n, 500 + s)
        for it in range(12):
            info = ons.iterate(pb, st, k, 5 * d, 500 + s)
            r2 = -2 * info["lstar"] - logdet
            logx_true = math.log(vd) + d / 2 * math.log(r2) + 0.5 * np.linalg.slogdet(sigma)[1] - d * math.log(20)
            if it == 11:
                resid.append(logx_true - st.logX)
                var.append(sum(1.0 / (n - j + 1) ** 2 for j in range(1, k + 1)) * (it + 1))
    resid = np.array(resid)
    sd = math.sqrt(np.mean(var))
    assert abs(np.mean(resid)) < 3 * sd / math.sqrt(len(resid)) + 0.05
    assert 0.3 * sd < np.std(resid) < 2.5 * sd


def test_detector_strain_is_delayed_geocentre_waveform():
    """A detector sees the geocentre signal delayed by its dt: its strain equals
    F+ h_+ + Fx h_x evaluated with t_c -> t_c + dt (same Fourier convention as
    the coalescence time inside the phase)."""
    w = gi.workload("c1")
    w.N, w.noise = 300, False
    pb, th = oracle.make_problem(w)
    f = w.freqs()
    for d in range(3):
        fp, fc = oracle.antenna(pb.xarm[d], pb.yarm[d], th[gi.P_RA], th[gi.P_SINDEC], th[gi.P_PSI])
        dt = oracle.delay(pb.pos[d], th[gi.P_RA], th[gi.P_SINDEC])
        assert abs(dt) > 1e-3
        th2 = th.copy()
        th2[gi.P_TC] += dt
        h = pb.strain(th, d)
        for j in range(0, 300, 37):
            if f[j] > oracle.fisco(th):
                continue
            hp, hc = oracle.polarizations(th2, f[j])
            assert h[j] == pytest.approx(fp * hp + fc * hc, rel=1e-9, abs=0)


# --------------------------------------------------------- relative binning
def _rb_problem():
    w = gi.workload("c1")
    w.N = 4017
    pb, th = oracle.make_problem(w)
    nocut = oracle.Problem(f0=pb.f0, df=pb.df, psd=pb.psd, data=pb.data(), pos=pb.pos, xarm=pb.xarm,
                           yarm=pb.yarm, cutoff=False, kind=pb.kind, lo=pb.lo, hi=pb.hi)
    return pb, nocut, th


def test_relative_binning_exact_at_fiducial():
    """At theta = theta_fid, r = 1 and the coarse sums reproduce the full-grid
    inner products exactly (no cutoff: every fine bin is in some coarse bin)."""
    pb, nocut, th = _rb_problem()
    rb = oracle.RelativeBinning(nocut, th, B=256)
    assert rb.J[0] == 0 and rb.J[-1] == pb.N - 1 and np.all(np.diff(rb.J) > 0)
    assert rb.loglike_theta(th)[0] == pytest.approx(nocut.loglike_theta(th)[0], rel=1e-11)


def test_relative_binning_close_near_fiducial():
    """Near the fiducial point the linear interpolation of h/h0 inside each
    coarse bin is accurate; the error grows away from it."""
    pb, nocut, th = _rb_problem()
    rb = oracle.RelativeBinning(nocut, th, B=256)
    near, far = [], []
    rng = np.random.default_rng(4)
    for _ in range(8):
        t = th.copy()
        t[gi.P_MC] *= 1 + 1e-4 * rng.standard_normal()
        t[gi.P_TC] += 1e-4 * rng.standard_normal()
        t[gi.P_PHIC] += 0.1 * rng.standard_normal()
        near.append(abs(rb.loglike_theta(t)[0] - nocut.loglike_theta(t)[0]))
        t2 = th.copy()
        t2[gi.P_MC] *= 1 + 3e-2
        far.append(abs(rb.loglike_theta(t2)[0] - nocut.loglike_theta(t2)[0]))
    assert max(near) < 1e-3
    assert max(far) > 10 * max(near)
