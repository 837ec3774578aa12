"""Seeded synthetic inputs shared by the CPU oracle, the tests and the benchmark.

This module holds no arithmetic of the method itself (no waveform, no antenna
pattern, no likelihood, no sampler step). It only produces the raw ingredients
of a synthetic analysis:

* the frequency grid (f0, df, N) with f_j = f0 + j*df, both endpoints included;
* the analytic noise PSD S(f) = 1e-46 [(f/30)^-4 + 2 + 2 (f/200)^2], used for
  every detector (the workload recipe of the five benchmark configurations);
* synthetic detector geometry: positions on a 6371 km sphere and orthogonal,
  seeded unit-vector arms in the local tangent plane;
* stationary Gaussian noise with Re and Im i.i.d. N(0, S/(4 df)) (one-sided PSD
  convention, so that E<n|n> = 2N);
* prior boxes over the 11 physical parameters, and unit-cube injection
  candidates (each side maps them through its own prior transform and scales
  the distance to the target network SNR with its own waveform).

The paper (Sec. 3) analyses GW150914 with two real detectors and an
IMRPhenomD waveform; none of that data is available, so these seeded inputs
stand in for it with the shapes of the five workload configurations below.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np

# Physical parameter order used by every layer (oracle, library, tests).
PARAM_NAMES = ("mc", "q", "chi1", "chi2", "dl", "cosi", "psi", "phic", "tc", "ra", "sindec")
NPARAM = len(PARAM_NAMES)
P_MC, P_Q, P_CHI1, P_CHI2, P_DL, P_COSI, P_PSI, P_PHIC, P_TC, P_RA, P_SINDEC = range(NPARAM)

# Prior kinds: FIXED (value = lo), UNIFORM on [lo, hi], VOLUME (p(x) ~ x^2 on [lo, hi]).
PRIOR_FIXED, PRIOR_UNIFORM, PRIOR_VOLUME = 0, 1, 2

EARTH_RADIUS_M = 6.371e6

TWO_PI = 2.0 * math.pi


@dataclasses.dataclass
class Workload:
    """Everything needed to build one synthetic analysis, except the signal."""

    name: str
    n_det: int
    ideal: bool              # True: one idealised detector with F+=1, Fx=0, no delay
    f0: float
    df: float
    N: int
    kind: np.ndarray         # int32[11]
    lo: np.ndarray           # float64[11]
    hi: np.ndarray           # float64[11]
    n_live: int
    k: int
    steps_per_dim: int
    snr: float
    noise: bool
    seed_geometry: int
    seed_noise: int
    seed_injection: int
    seed_sampler: int
    fixed_injection: Optional[np.ndarray] = None   # physical 11-vector (C0 only)
    dl_from_snr: bool = False                      # C0: distance fixed so that SNR(theta_inj) = snr
    dlogz_stop: float = 0.1

    @property
    def dim(self) -> int:
        return int(np.sum(self.kind != PRIOR_FIXED))

    def freqs(self) -> np.ndarray:
        j = np.arange(self.N, dtype=np.float64)
        return self.f0 + j * self.df


def psd_analytic(f: np.ndarray) -> np.ndarray:
    """S(f) = 1e-46 [(f/30)^-4 + 2 + 2 (f/200)^2] (one-sided, 1/Hz)."""
    f = np.asarray(f, dtype=np.float64)
    return 1e-46 * ((f / 30.0) ** -4 + 2.0 + 2.0 * (f / 200.0) ** 2)


def detectors(seed: int, n_det: int):
    """Seeded synthetic detectors: positions on the Earth sphere, orthogonal arms.

    For detector i: u_i is a normalised Gaussian 3-vector, r_i = R_E u_i; X_i is
    the normalised projection of a Gaussian vector onto the plane orthogonal to
    u_i; Y_i = u_i x X_i.
    Returns (pos[n_det,3] metres, xarm[n_det,3], yarm[n_det,3]).
    """
    rng = np.random.default_rng(seed)
    pos = np.zeros((n_det, 3))
    xarm = np.zeros((n_det, 3))
    yarm = np.zeros((n_det, 3))
    for i in range(n_det):
        u = rng.standard_normal(3)
        u /= np.linalg.norm(u)
        g = rng.standard_normal(3)
        x = g - np.dot(g, u) * u
        x /= np.linalg.norm(x)
        y = np.cross(u, x)
        pos[i] = EARTH_RADIUS_M * u
        xarm[i] = x
        yarm[i] = y
    return pos, xarm, yarm


def noise(seed: int, psd: np.ndarray, df: float) -> np.ndarray:
    """Complex Gaussian noise, Re and Im i.i.d. N(0, S/(4 df)); shape of psd."""
    rng = np.random.default_rng(seed)
    sigma = np.sqrt(psd / (4.0 * df))
    re = rng.standard_normal(psd.shape) * sigma
    im = rng.standard_normal(psd.shape) * sigma
    return re + 1j * im


def unit_cube(seed: int, count: int, dim: int) -> np.ndarray:
    """Seeded uniform draws in [0,1)^dim (injection candidates, test points)."""
    rng = np.random.default_rng(seed)
    return rng.random((count, dim))


def _prior_11(mc=(10.0, 40.0), dl=(100.0, 2000.0)):
    kind = np.full(NPARAM, PRIOR_UNIFORM, dtype=np.int32)
    lo = np.zeros(NPARAM)
    hi = np.zeros(NPARAM)
    box = {
        P_MC: mc, P_Q: (0.25, 1.0), P_CHI1: (-0.5, 0.5), P_CHI2: (-0.5, 0.5),
        P_DL: dl, P_COSI: (-1.0, 1.0), P_PSI: (0.0, math.pi), P_PHIC: (0.0, TWO_PI),
        P_TC: (-0.1, 0.1), P_RA: (0.0, TWO_PI), P_SINDEC: (-1.0, 1.0),
    }
    for p, (a, b) in box.items():
        lo[p], hi[p] = a, b
    kind[P_DL] = PRIOR_VOLUME
    return kind, lo, hi


def _prior_c0():
    kind = np.full(NPARAM, PRIOR_FIXED, dtype=np.int32)
    lo = np.zeros(NPARAM)
    hi = np.zeros(NPARAM)
    for p, (a, b) in {P_MC: (10.0, 40.0), P_Q: (0.25, 1.0), P_TC: (-0.1, 0.1),
                      P_PHIC: (0.0, TWO_PI)}.items():
        kind[p] = PRIOR_UNIFORM
        lo[p], hi[p] = a, b
    # fixed values: no spin, face-on (cos i = 1), psi = 0, ra = 0, sin dec = 0;
    # the distance is set by the data builder so that SNR(theta_inj) = 20.
    lo[P_COSI] = hi[P_COSI] = 1.0
    lo[P_DL] = hi[P_DL] = 100.0
    return kind, lo, hi


def _uniform_grid(f_lo: float, f_hi: float, duration: float):
    df = 1.0 / duration
    N = int(round((f_hi - f_lo) * duration)) + 1
    return f_lo, df, N


def workload(name: str, **over) -> Workload:
    """The five benchmark workloads (c0..c4) and small variants for tests.

    c0: one idealised detector, 4 params, 20-512 Hz on 512 uniform bins,
        noise-free injection at SNR 20, n=200, k=100, 5*d steps.
    c1: 3 detectors, 11 params, 4 s at 20-1024 Hz (4017 bins), noise, SNR 20,
        n=1000, k=500.
    c2: as c1 with 32 s at 20-2048 Hz (64,897 bins), n=2000, k=1000.
    c3: one serving request template (durations 4..64 s at 20-2048 Hz).
    c4: 256 s at 20-2048 Hz (519,169 bins), chirp mass U[1.1,1.5], SNR 30,
        n=2000, k=1000, distance floor lowered to 10 Mpc so that SNR 30 is
        reachable inside the prior.
    """
    c = int(name[1]) if name[0] == "c" and name[1:].isdigit() else None
    if name == "c0":
        kind, lo, hi = _prior_c0()
        w = Workload(name="c0", n_det=1, ideal=True, f0=20.0, df=492.0 / 511.0, N=512,
                     kind=kind, lo=lo, hi=hi, n_live=200, k=100, steps_per_dim=5,
                     snr=20.0, noise=False, seed_geometry=1000, seed_noise=2000,
                     seed_injection=3000, seed_sampler=4000,
                     fixed_injection=_c0_injection(), dl_from_snr=True)
    elif name in ("c1", "c2", "c4") or name.startswith("c3"):
        if name == "c1":
            f0, df, N = _uniform_grid(20.0, 1024.0, 4.0)
            n_live, snr = 1000, 20.0
            kind, lo, hi = _prior_11()
        elif name == "c2":
            f0, df, N = _uniform_grid(20.0, 2048.0, 32.0)
            n_live, snr = 2000, 20.0
            kind, lo, hi = _prior_11()
        elif name == "c4":
            f0, df, N = _uniform_grid(20.0, 2048.0, 256.0)
            n_live, snr = 2000, 30.0
            kind, lo, hi = _prior_11(mc=(1.1, 1.5), dl=(10.0, 2000.0))
        else:
            duration = float(over.pop("duration", 4.0))
            f0, df, N = _uniform_grid(20.0, 2048.0, duration)
            n_live, snr = int(over.pop("n_live_c3", 1000)), float(over.pop("snr_c3", 20.0))
            kind, lo, hi = _prior_11()
            c = 3
        w = Workload(name=name, n_det=3, ideal=False, f0=f0, df=df, N=N, kind=kind,
                     lo=lo, hi=hi, n_live=n_live, k=n_live // 2, steps_per_dim=5,
                     snr=snr, noise=True, seed_geometry=1000 + c, seed_noise=2000 + c,
                     seed_injection=3000 + c, seed_sampler=4000 + c)
    else:
        raise ValueError(f"unknown workload {name!r}")
    for key, val in over.items():
        if not hasattr(w, key):
            raise ValueError(f"unknown workload field {key!r}")
        setattr(w, key, val)
    return w


def _c0_injection() -> np.ndarray:
    th = np.zeros(NPARAM)
    th[P_MC], th[P_Q], th[P_TC], th[P_PHIC] = 25.0, 0.8, 0.0, 1.0
    th[P_COSI] = 1.0
    th[P_DL] = 100.0
    return th


def serving_stream(seed: int = 4003, count: int = 64, rate_hz: float = 2.0) -> List[Dict]:
    """Request mix of the serving workload: Poisson arrivals at rate_hz,
    durations from {4,8,16,32,64} s, n_live ~ U{500..2000}, SNR ~ U[10,40]."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=count))
    durations = rng.choice([4.0, 8.0, 16.0, 32.0, 64.0], size=count)
    n_live = rng.integers(500, 2001, size=count)
    snr = rng.uniform(10.0, 40.0, size=count)
    return [dict(arrival_s=float(t[i]), duration=float(durations[i]), n_live=int(n_live[i]),
                 snr=float(snr[i]), seed_offset=i) for i in range(count)]


# Toy likelihood: correlated Gaussian N(x; 0, Sigma), Sigma_ij = rho^|i-j|,
# on the prior box [-10, 10]^d. Analytic log Z = -d ln 20 (truncation < 1e-15).
TOY_RHO = 0.9
TOY_BOX = (-10.0, 10.0)


def toy_covariance(d: int, rho: float = TOY_RHO) -> np.ndarray:
    i = np.arange(d)
    return rho ** np.abs(i[:, None] - i[None, :])
