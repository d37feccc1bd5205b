"""Plain FP64 CPU oracle of the QED Monte-Carlo particle step (arXiv:1311.5551).

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` import this package.  The product (the CUDA library and its binding) never
imports, links or calls it, and it never imports the product.

The arithmetic lives in ``qed_oracle.c`` (plain C, IEEE double, compiled without
multiply-add contraction); this module compiles it with gcc and wraps it with ctypes.
``rr.py`` holds the deterministic and classical radiation-reaction solutions of Sec. 2.4.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import dataclasses
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qed_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")

ALPHA = 7.2973525693e-3
ELECTRON, POSITRON, PHOTON = 0, 1, 2
FIELD_UNIFORM, FIELD_ROTATING_E, FIELD_PLANE_LP, FIELD_PLANE_CP, FIELD_GRID = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP only parallelises the table rows)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None
_dp = C.POINTER(C.c_double)
_u32p = C.POINTER(C.c_uint32)


class _Tables(C.Structure):
    _fields_ = [("n_eta", C.c_int), ("n_xi", C.c_int), ("n_chi", C.c_int), ("n_f", C.c_int),
                ("ln_eta_min", C.c_double), ("ln_eta_max", C.c_double),
                ("ln_chi_min", C.c_double), ("ln_chi_max", C.c_double), ("energy_cut", C.c_double),
                ("ln_h", _dp), ("g", _dp), ("zeta_lo", _dp), ("zeta_hi", _dp), ("P", _dp), ("Q", _dp),
                ("ln_T", _dp), ("Pf", _dp)]


class _Field(C.Structure):
    _fields_ = [("kind", C.c_int), ("E", C.c_double * 3), ("B", C.c_double * 3), ("E0", C.c_double),
                ("omega", C.c_double), ("phase0", C.c_double), ("phi_start", C.c_double),
                ("phi_len", C.c_double), ("grid", _dp), ("n", C.c_int * 3), ("shape", C.c_int),
                ("origin", C.c_double * 3), ("spacing", C.c_double * 3)]


class _StepParams(C.Structure):
    _fields_ = [("dt", C.c_double), ("t0", C.c_double), ("step", C.c_uint64), ("seed", C.c_uint64),
                ("scenario", C.c_uint64), ("emit_photons", C.c_int), ("make_pairs", C.c_int),
                ("drain_photons", C.c_int), ("recoil_energy", C.c_int), ("field", _Field)]


class _Species(C.Structure):
    _fields_ = [("x", _dp), ("y", _dp), ("z", _dp), ("ux", _dp), ("uy", _dp), ("uz", _dp), ("tau", _dp),
                ("id", _u32p), ("n", C.c_int64), ("cap", C.c_int64), ("next_id", C.c_uint32), ("w", _dp)]


class _MergeParams(C.Structure):
    _fields_ = [("origin", C.c_double * 3), ("cell", C.c_double * 3), ("n_cells", C.c_int * 3), ("n_face", C.c_int),
                ("n_sub", C.c_int), ("min_group", C.c_int)]


class _Ledger(C.Structure):
    _fields_ = [("n", C.c_double * 3), ("energy", C.c_double * 3), ("emitted_n", C.c_double),
                ("emitted_energy", C.c_double), ("dropped_n", C.c_double), ("emit_defect", C.c_double),
                ("pairs_n", C.c_double), ("pair_energy", C.c_double), ("pair_defect", C.c_double),
                ("drained_n", C.c_double), ("drained_energy", C.c_double), ("oor_eta", C.c_double),
                ("oor_chi", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        d, i, u64 = C.c_double, C.c_int, C.c_uint64
        for name, res, args in [
            ("orc_besselk", d, [d, d]), ("orc_besselk_int", d, [d, d]), ("orc_F", d, [d, d]),
            ("orc_F_classical", d, [d, d]), ("orc_h", d, [d]), ("orc_g", d, [d]), ("orc_g_fit", d, [d]),
            ("orc_T", d, [d]), ("orc_pf_unnorm", d, [d, d]), ("orc_k", d, [d]),
            ("orc_tables_build", i, [C.POINTER(_Tables)]),
            ("orc_lookup_h", d, [C.POINTER(_Tables), d, C.POINTER(i)]),
            ("orc_lookup_T", d, [C.POINTER(_Tables), d, C.POINTER(i)]),
            ("orc_sample_xi", i, [C.POINTER(_Tables), d, d, _dp]),
            ("orc_sample_f", d, [C.POINTER(_Tables), d, d]),
            ("orc_philox4x64", None, [C.POINTER(u64), C.POINTER(u64), C.POINTER(u64)]),
            ("orc_u01", d, [u64]),
            ("orc_field_eval", None, [C.POINTER(_Field), d, _dp, _dp, _dp]),
            ("orc_boris", None, [d, d, _dp, _dp, _dp]),
            ("orc_eta", d, [_dp, d, _dp, _dp]), ("orc_chi", d, [_dp, d, _dp, _dp]),
            ("orc_rate_photon", d, [C.POINTER(_Tables), d, d, C.POINTER(i)]),
            ("orc_rate_pair", d, [C.POINTER(_Tables), d, d, C.POINTER(i)]),
            ("orc_step", i, [C.POINTER(_Tables), C.POINTER(_StepParams), C.POINTER(C.POINTER(_Species)),
                             C.POINTER(_Species), C.POINTER(_Ledger)]),
            ("orc_init_tau", None, [C.POINTER(_Species), i, u64, u64]),
            ("orc_merge_photons", C.c_int64, [C.POINTER(_Species), C.POINTER(_MergeParams)]),
            ("orc_merge", C.c_int64, [C.POINTER(_Species), C.POINTER(_MergeParams), i]),
            ("orc_species_totals", None, [C.POINTER(_Species), i, C.POINTER(C.c_double)]),
        ]:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


# ----------------------------------------------------------------- scalar special functions
def besselk(nu, x):
    return lib().orc_besselk(float(nu), float(x))


def besselk_int(nu, y):
    return lib().orc_besselk_int(float(nu), float(y))


def F(eta, chi):
    return lib().orc_F(float(eta), float(chi))


def F_classical(eta, chi):
    return lib().orc_F_classical(float(eta), float(chi))


def h(eta):
    return lib().orc_h(float(eta))


def g(eta):
    return lib().orc_g(float(eta))


def g_fit(eta):
    return lib().orc_g_fit(float(eta))


def T(chi):
    return lib().orc_T(float(chi))


def pf_unnorm(f, chi):
    return lib().orc_pf_unnorm(float(f), float(chi))


def k_norm(chi):
    return lib().orc_k(float(chi))


def philox4x64(ctr, key):
    c = (C.c_uint64 * 4)(*[int(v) & (2**64 - 1) for v in ctr])
    k = (C.c_uint64 * 2)(*[int(v) & (2**64 - 1) for v in key])
    o = (C.c_uint64 * 4)()
    lib().orc_philox4x64(c, k, o)
    return [int(v) for v in o]


def u01(word):
    return lib().orc_u01(int(word))


# ----------------------------------------------------------------------------- tables
@dataclass
class TableParams:
    """256 log-spaced eta in [1e-4, 1e2] and 256 chi points (the paper's test set-up);
    the T and P_f tables span chi in [1e-2, 1e2]; 128 f points on [0, 1/2]."""
    n_eta: int = 256
    eta_min: float = 1e-4
    eta_max: float = 1e2
    n_xi: int = 256
    n_chi: int = 256
    chi_min: float = 1e-2
    chi_max: float = 1e2
    n_f: int = 128
    energy_cut: float = 1e-9


TABLE_KEYS = ("ln_h", "g", "zeta_lo", "zeta_hi", "P", "Q", "ln_T", "Pf")


class Tables:
    """Oracle look-up tables, built by direct Bessel-function quadrature."""

    def __init__(self, params: TableParams | None = None, arrays: dict | None = None):
        self.params = p = params or TableParams()
        if arrays is None:
            arrays = {"ln_h": np.zeros(p.n_eta), "g": np.zeros(p.n_eta), "zeta_lo": np.zeros(p.n_eta),
                      "zeta_hi": np.zeros(p.n_eta),
                      "P": np.zeros((p.n_eta, p.n_xi)), "Q": np.zeros((p.n_eta, p.n_xi)),
                      "ln_T": np.zeros(p.n_chi), "Pf": np.zeros((p.n_chi, p.n_f))}
            build_now = True
        else:
            arrays = {k: np.ascontiguousarray(v, dtype=np.float64) for k, v in arrays.items()}
            build_now = False
        self.a = arrays
        self._s = _Tables(p.n_eta, p.n_xi, p.n_chi, p.n_f, np.log(p.eta_min), np.log(p.eta_max),
                          np.log(p.chi_min), np.log(p.chi_max), p.energy_cut,
                          *[arrays[k].ctypes.data_as(_dp) for k in TABLE_KEYS])
        if build_now:
            rc = lib().orc_tables_build(C.byref(self._s))
            if rc != 0:
                raise RuntimeError("orc_tables_build failed")

    def save(self, path):
        np.savez(path, **self.a, params=np.array([self.params.n_eta, self.params.eta_min, self.params.eta_max,
                                                  self.params.n_xi, self.params.n_chi, self.params.chi_min,
                                                  self.params.chi_max, self.params.n_f, self.params.energy_cut]))

    @classmethod
    def load(cls, path):
        z = np.load(path)
        v = z["params"]
        p = TableParams(int(v[0]), v[1], v[2], int(v[3]), int(v[4]), v[5], v[6], int(v[7]), v[8])
        return cls(p, {k: z[k] for k in TABLE_KEYS})

    # look-ups -------------------------------------------------------------------------
    def h(self, eta):
        o = C.c_int()
        return lib().orc_lookup_h(C.byref(self._s), float(eta), C.byref(o))

    def T(self, chi):
        o = C.c_int()
        return lib().orc_lookup_T(C.byref(self._s), float(chi), C.byref(o))

    def sample_xi(self, eta, U):
        """xi = 2chi/eta of the emitted photon, or None below the cut-off."""
        x = C.c_double()
        ok = lib().orc_sample_xi(C.byref(self._s), float(eta), float(U), C.byref(x))
        return x.value if ok else None

    def sample_f(self, chi, U):
        return lib().orc_sample_f(C.byref(self._s), float(chi), float(U))

    def rate_photon(self, eta, gamma):
        o = C.c_int()
        return lib().orc_rate_photon(C.byref(self._s), float(eta), float(gamma), C.byref(o))

    def rate_pair(self, chi, eps):
        o = C.c_int()
        return lib().orc_rate_pair(C.byref(self._s), float(chi), float(eps), C.byref(o))


# ----------------------------------------------------------------------------- fields
@dataclass
class Field:
    kind: int = FIELD_UNIFORM
    E: tuple = (0.0, 0.0, 0.0)
    B: tuple = (0.0, 0.0, 0.0)
    E0: float = 0.0
    omega: float = 0.0
    phase0: float = 0.0
    phi_start: float = 0.0
    phi_len: float = 0.0
    # FIELD_GRID: float64 array of shape (6, nz, ny, nx) (Ex, Ey, Ez, cBx, cBy, cBz), Yee-staggered
    grid: object = None
    shape: int = 1
    origin: tuple = (0.0, 0.0, 0.0)
    spacing: tuple = (1.0, 1.0, 1.0)

    def c(self):
        g, n = None, (0, 0, 0)
        if self.grid is not None:
            self._grid = np.ascontiguousarray(self.grid, dtype=np.float64)  # kept alive with the Field
            g = self._grid.ctypes.data_as(_dp)
            n = (self._grid.shape[3], self._grid.shape[2], self._grid.shape[1])
        return _Field(self.kind, (C.c_double * 3)(*self.E), (C.c_double * 3)(*self.B), self.E0, self.omega,
                      self.phase0, self.phi_start, self.phi_len, g, (C.c_int * 3)(*n), int(self.shape),
                      (C.c_double * 3)(*self.origin), (C.c_double * 3)(*self.spacing))


def field_eval(fd: Field, t, x):
    xa = (C.c_double * 3)(*x)
    E = (C.c_double * 3)()
    B = (C.c_double * 3)()
    f = fd.c()
    lib().orc_field_eval(C.byref(f), float(t), xa, E, B)
    return np.array(E[:]), np.array(B[:])


def boris(q, dt, E, B, u):
    ua = (C.c_double * 3)(*u)
    lib().orc_boris(float(q), float(dt), (C.c_double * 3)(*E), (C.c_double * 3)(*B), ua)
    return np.array(ua[:])


def eta_of(u, gamma, E, B):
    return lib().orc_eta((C.c_double * 3)(*u), float(gamma), (C.c_double * 3)(*E), (C.c_double * 3)(*B))


def chi_of(k, eps, E, B):
    return lib().orc_chi((C.c_double * 3)(*k), float(eps), (C.c_double * 3)(*E), (C.c_double * 3)(*B))


# ----------------------------------------------------------------------------- particles
class Species:
    """SoA particle store in FP64 (positions, momenta, optical depth, id)."""

    def __init__(self, cap: int):
        self.cap = int(cap)
        self.arr = {k: np.zeros(self.cap) for k in ("x", "y", "z", "ux", "uy", "uz", "tau")}
        self.arr["id"] = np.zeros(self.cap, dtype=np.uint32)
        self.arr["w"] = np.ones(self.cap)
        self._s = _Species(*[self.arr[k].ctypes.data_as(_dp) for k in ("x", "y", "z", "ux", "uy", "uz", "tau")],
                           self.arr["id"].ctypes.data_as(_u32p), 0, self.cap, 0, self.arr["w"].ctypes.data_as(_dp))

    @property
    def n(self):
        return int(self._s.n)

    @property
    def next_id(self):
        return int(self._s.next_id)

    def set(self, x, u, tau=None, ids=None, w=None):
        x = np.asarray(x, dtype=np.float64)
        u = np.asarray(u, dtype=np.float64)
        n = len(x)
        if n > self.cap:
            raise ValueError("capacity")
        for c, k in enumerate(("x", "y", "z")):
            self.arr[k][:n] = x[:, c]
        for c, k in enumerate(("ux", "uy", "uz")):
            self.arr[k][:n] = u[:, c]
        self.arr["tau"][:n] = 0.0 if tau is None else tau
        self.arr["id"][:n] = np.arange(n, dtype=np.uint32) if ids is None else ids
        self.arr["w"][:n] = 1.0 if w is None else w
        self._s.n = n
        self._s.next_id = n if ids is None else int(np.max(ids)) + 1 if n else 0

    def init_tau(self, kind, seed, scenario=0):
        lib().orc_init_tau(C.byref(self._s), int(kind), int(seed), int(scenario))

    def get(self, key):
        return self.arr[key][: self.n].copy()

    def x(self):
        return np.stack([self.get("x"), self.get("y"), self.get("z")], axis=1)

    def u(self):
        return np.stack([self.get("ux"), self.get("uy"), self.get("uz")], axis=1)

    def totals(self, photon=False):
        """(sum w, sum w energy, sum w momentum[3]) of the held particles."""
        out = (C.c_double * 5)()
        lib().orc_species_totals(C.byref(self._s), int(photon), out)
        return out[0], out[1], np.array(out[2:5])

    def merge(self, origin, cell, n_cells, n_face=8, n_sub=4, min_group=4, photon=True):
        """Merge this species' particles (see orc_merge); returns the groups merged."""
        mp = _MergeParams((C.c_double * 3)(*origin), (C.c_double * 3)(*cell), (C.c_int * 3)(*n_cells), int(n_face),
                          int(n_sub), int(min_group))
        return int(lib().orc_merge(C.byref(self._s), C.byref(mp), int(bool(photon))))

    def energy(self, photon=False):
        u = self.u()
        u2 = np.sum(u * u, axis=1)
        return np.sqrt(u2) if photon else np.sqrt(1.0 + u2)


@dataclass
class StepParams:
    dt: float
    t0: float = 0.0
    seed: int = 1
    scenario: int = 0
    emit_photons: bool = True
    make_pairs: bool = True
    drain_photons: bool = False
    recoil_energy: bool = False
    field: Field = dataclasses.field(default_factory=Field)


LEDGER_KEYS = [k for k, _ in _Ledger._fields_]


def step(tables: Tables, params: StepParams, step_index: int, electrons: Species, positrons: Species,
         photons: Species, drained: Species | None = None) -> dict:
    """One Monte-Carlo step of all three species (Sec. 3); returns the step ledger."""
    sp = _StepParams(params.dt, params.t0, int(step_index), int(params.seed), int(params.scenario),
                     int(params.emit_photons), int(params.make_pairs), int(params.drain_photons),
                     int(params.recoil_energy), params.field.c())
    arr = (C.POINTER(_Species) * 3)(C.pointer(electrons._s), C.pointer(positrons._s), C.pointer(photons._s))
    led = _Ledger()
    rc = lib().orc_step(C.byref(tables._s), C.byref(sp), arr, C.pointer(drained._s) if drained else None,
                        C.byref(led))
    if rc != 0:
        raise RuntimeError("oracle step: capacity exceeded")
    out = {}
    for k, _ in _Ledger._fields_:
        v = getattr(led, k)
        out[k] = list(v) if not isinstance(v, float) else v
    return out
