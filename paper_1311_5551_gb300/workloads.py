"""Seeded synthetic inputs for the QED Monte-Carlo step.

This module holds only initial conditions and unit conversions: no step of the method's
arithmetic lives here.  It serves both the CUDA path (through ``bench.py`` and the tests)
and the FP64 oracle (through the tests), so that both consume identical inputs.

Units: momenta in m_e c, fields in the Schwinger field E_s, time in hbar/(m_e c^2),
length in hbar/(m_e c) (reduced Compton wavelength).  The workloads follow the paper's
test problems (Table "test_info", Sec. 4) and the head-on, rotating-field and batched set-ups
built on them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# CODATA 2018
HBAR = 1.054571817e-34
M_E = 9.1093837015e-31
C_LIGHT = 299792458.0
Q_E = 1.602176634e-19
TIME_UNIT_S = HBAR / (M_E * C_LIGHT**2)          # 1.28809e-21 s
LENGTH_UNIT_M = HBAR / (M_E * C_LIGHT)           # 3.86159e-13 m
E_SCHWINGER = M_E**2 * C_LIGHT**3 / (Q_E * HBAR)  # 1.32329e18 V/m

FIELD_UNIFORM, FIELD_ROTATING_E, FIELD_PLANE_LP, FIELD_PLANE_CP = 0, 1, 2, 3


def omega_of_wavelength(lam_m: float) -> float:
    """Angular frequency (and wavenumber, c = 1) of light of wavelength lam_m, in code units."""
    return 2.0 * math.pi * LENGTH_UNIT_M / lam_m


def sin2_length_from_fwhm(fwhm_s: float) -> float:
    """Full duration of a sin^2 field envelope whose intensity (sin^4) has the given FWHM."""
    s1 = math.asin(2.0 ** -0.25) / math.pi
    return fwhm_s / (1.0 - 2.0 * s1)


@dataclass
class FieldSpec:
    kind: int = FIELD_UNIFORM
    E: tuple = (0.0, 0.0, 0.0)
    B: tuple = (0.0, 0.0, 0.0)   # c*B
    E0: float = 0.0
    omega: float = 0.0
    phase0: float = 0.0
    phi_start: float = 0.0
    phi_len: float = 0.0

    def as_dict(self):
        return dict(kind=self.kind, E=tuple(self.E), B=tuple(self.B), E0=self.E0, omega=self.omega,
                    phase0=self.phase0, phi_start=self.phi_start, phi_len=self.phi_len)


@dataclass
class Workload:
    name: str
    x: np.ndarray                # (n, 3) float64 initial positions of the electrons
    u: np.ndarray                # (n, 3) float64 initial momenta u^{-1/2}
    field: FieldSpec
    dt: float
    n_steps: int
    seed: int
    emit_photons: bool = True
    make_pairs: bool = True
    drain_photons: bool = False
    window_x0: float = 0.0       # moving-window origin at t = 0 (x only)
    window_v: float = 0.0        # moving-window velocity along x (units of c)
    extra: dict = field(default_factory=dict)

    @property
    def n(self):
        return len(self.x)


def uniform_b(n: int = 10_000, gamma0: float = 1000.0, cB: float | None = None, n_steps: int = 2000,
              seed: int = 1, steps_per_gyro: float = 1000.0, make_pairs: bool = False,
              drain_photons: bool = True) -> Workload:
    """Test problem 1 (Table "test_info"): electrons with gamma0 moving perpendicular to a
    uniform magnetic field with c|B|/E_s = 1/gamma0 (eta0 = 1), dt = 1e-3 gyro-period,
    photons deleted right after emission (Sec. 3.1)."""
    if cB is None:
        cB = 1.0 / gamma0
    p0 = math.sqrt(gamma0 * gamma0 - 1.0)
    x = np.zeros((n, 3))
    u = np.zeros((n, 3))
    u[:, 0] = p0
    gyro = 2.0 * math.pi * gamma0 / cB
    return Workload("uniform_B", x, u, FieldSpec(FIELD_UNIFORM, B=(0.0, 0.0, cB)), gyro / steps_per_gyro,
                    n_steps, seed, True, make_pairs, drain_photons)


def dt_qed(field_max: float) -> float:
    """Delta t_QED = 1 / Max(lambda_gamma) of Sec. 3.1 (time units hbar/(m c^2)): the largest photon
    emission rate, (sqrt3 alpha/pi) Max(E, cB) h0 with h0 = 5 pi/3, for fields in units of E_s."""
    alpha = 7.2973525693e-3
    return 1.0 / ((math.sqrt(3.0) * alpha / math.pi) * field_max * (5.0 * math.pi / 3.0))


def cp_head_on(n: int = 10_000, gamma0: float = 4120.0, E0: float = 1.22e-4, lam_m: float = 1e-6,
               dt_over_dtqed: float = 0.3, t_end_s: float = 3e-15, seed: int = 6,
               make_pairs: bool = True, drain_photons: bool = False) -> Workload:
    """Test problem 2 (Table "test_info"): electrons with gamma0 = 4120 moving along -x into a
    circularly polarised plane wave of constant amplitude E = cB = 1.22e-4 E_s travelling along +x
    (a = 50 at lambda = 1 um; eta0 = gamma0 (1 + beta0) E0 = 1.0); the figures of the test are
    taken at t0 = 3 fs."""
    omega = omega_of_wavelength(lam_m)
    dt = dt_over_dtqed * dt_qed(E0)
    x = np.zeros((n, 3))
    u = np.zeros((n, 3))
    u[:, 0] = -math.sqrt(gamma0 * gamma0 - 1.0)
    n_steps = int(math.ceil(t_end_s / TIME_UNIT_S / dt))
    return Workload("cp_head_on", x, u, FieldSpec(FIELD_PLANE_CP, E0=E0, omega=omega), dt, n_steps, seed, True,
                    make_pairs, drain_photons, extra=dict(a0=E0 / omega, gamma_mean=gamma0, lam_m=lam_m))


def head_on(n: int = 1_000_000, gamma_mean: float = 2000.0, gamma_rms_frac: float = 0.05,
            divergence: float = 1e-3, a0: float = 100.0, lam_m: float = 1e-6, fwhm_s: float = 30e-15,
            steps_per_lambda: float = 100.0, n_steps: int = 4000, meet_step: int | None = None,
            bunch_rms_m: float = 1e-6, seed: int = 2, polarization: int = FIELD_PLANE_LP,
            rng: np.random.Generator | None = None) -> Workload:
    """Electron beam (moving along -x) colliding head-on with a plane-wave pulse moving along
    +x: sin^2 field envelope with the given intensity FWHM, dt = lambda/(steps_per_lambda c).
    The bunch centre meets the pulse centre at step ``meet_step`` (default: mid-run)."""
    rng = rng if rng is not None else np.random.default_rng(seed)
    omega = omega_of_wavelength(lam_m)
    dt = 2.0 * math.pi / omega / steps_per_lambda
    E0 = a0 * omega
    L = sin2_length_from_fwhm(fwhm_s) / TIME_UNIT_S
    phi_len = omega * L
    meet = n_steps // 2 if meet_step is None else meet_step
    t_meet = meet * dt
    phi_start = omega * t_meet - 0.5 * phi_len           # pulse centre at x = 0 at t_meet
    gam = gamma_mean * (1.0 + gamma_rms_frac * rng.standard_normal(n))
    gam = np.maximum(gam, 1.5)
    pmag = np.sqrt(gam * gam - 1.0)
    thy = divergence * rng.standard_normal(n)
    thz = divergence * rng.standard_normal(n)
    u = np.empty((n, 3))
    u[:, 0] = -pmag * np.cos(thy) * np.cos(thz)
    u[:, 1] = pmag * np.sin(thy) * np.cos(thz)
    u[:, 2] = pmag * np.sin(thz)
    sig = bunch_rms_m / LENGTH_UNIT_M
    beta0 = math.sqrt(1.0 - 1.0 / gamma_mean**2)
    x0c = beta0 * t_meet                                  # bunch centre reaches x = 0 at t_meet
    x = sig * rng.standard_normal((n, 3))
    x[:, 0] += x0c
    fld = FieldSpec(polarization, E0=E0, omega=omega, phi_start=phi_start, phi_len=phi_len)
    return Workload("head_on", x, u, fld, dt, n_steps, seed, True, True, False,
                    window_x0=x0c, window_v=-1.0,
                    extra=dict(a0=a0, gamma_mean=gamma_mean, lam_m=lam_m, fwhm_s=fwhm_s))


def rotating_e(n: int = 10_000, E0: float = 1e-3, lam_m: float = 0.8e-6, steps_per_lambda: float = 200.0,
               n_steps: int = 4000, cube_m: float = 1e-6, seed: int = 3) -> Workload:
    """Electrons at rest, uniformly placed, in a rotating electric field of magnitude E0
    (the field at the node of a circularly polarised standing wave), B = 0."""
    rng = np.random.default_rng(seed)
    omega = omega_of_wavelength(lam_m)
    dt = 2.0 * math.pi / omega / steps_per_lambda
    x = (rng.random((n, 3)) - 0.5) * (cube_m / LENGTH_UNIT_M)
    u = np.zeros((n, 3))
    return Workload("rotating_E", x, u, FieldSpec(FIELD_ROTATING_E, E0=E0, omega=omega), dt, n_steps, seed,
                    True, True, False)


def scan(n_scenarios: int = 256, n_min: float = 1e3, n_max: float = 1e6, a0_range=(10.0, 500.0),
         gamma_range=(200.0, 4000.0), fwhm_range_s=(15e-15, 60e-15), n_steps: int = 4000, seed: int = 4,
         scale: float = 1.0, only=None) -> list[Workload]:
    """Batched parameter scan of head-on collisions: particle counts log-uniform in
    [n_min, n_max] (times ``scale``), a0, gamma0 and pulse FWHM uniform in their ranges.  With
    ``only`` (scenario indices) just those scenarios are built, in that order; their draws are
    the same as in the whole scan."""
    rng = np.random.default_rng(seed)
    params = []
    for s in range(n_scenarios):
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max))) * scale))
        n = max(n, 1)
        a0 = rng.uniform(*a0_range)
        g0 = rng.uniform(*gamma_range)
        fw = rng.uniform(*fwhm_range_s)
        params.append((n, a0, g0, fw))
    out = []
    for s in (range(n_scenarios) if only is None else only):
        n, a0, g0, fw = params[s]
        w = head_on(n=n, gamma_mean=g0, a0=a0, fwhm_s=fw, n_steps=n_steps, seed=seed,
                    rng=np.random.default_rng([seed, s]))
        w.name = f"scan[{s}]"
        w.extra["scenario"] = s
        out.append(w)
    return out


@dataclass
class RequestSpec:
    """One head-on collision request, drawn but not yet built: ``workload()`` makes its particle
    arrays (a request stream at full size would not fit in host memory all at once)."""
    k: int
    n: int
    a0: float
    gamma0: float
    n_steps: int
    seed: int

    def workload(self) -> Workload:
        w = head_on(n=self.n, gamma_mean=self.gamma0, a0=self.a0, n_steps=self.n_steps, seed=self.seed,
                    rng=np.random.default_rng([self.seed, self.k]))
        w.name = f"request[{self.k}]"
        w.extra["scenario"] = self.k
        return w


def request_specs(rate_hz: float = 200.0, duration_s: float = 60.0, n_min: float = 1e3, n_max: float = 2e6,
                  steps_range=(2000, 8000), seed: int = 5, scale: float = 1.0):
    """Poisson arrivals of head-on collision requests: (arrival time in s, RequestSpec), particle
    counts log-uniform in [n_min, n_max] (times ``scale``), a0 uniform in [10, 500], gamma0
    uniform in [200, 4000], steps uniform in steps_range."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t > duration_s:
            break
        k = len(out)
        n = max(1, int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max))) * scale)))
        a0 = rng.uniform(10.0, 500.0)
        g0 = rng.uniform(200.0, 4000.0)
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        out.append((t, RequestSpec(k, n, a0, g0, steps, seed)))
    return out


def requests(rate_hz: float = 200.0, duration_s: float = 60.0, n_min: float = 1e3, n_max: float = 2e6,
             steps_range=(2000, 8000), seed: int = 5, scale: float = 1.0):
    """Poisson arrivals of head-on collision requests (arrival time in s, Workload), built."""
    return [(t, r.workload()) for t, r in request_specs(rate_hz, duration_s, n_min, n_max, steps_range, seed, scale)]
