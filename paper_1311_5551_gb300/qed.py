"""Thin Python binding of the C ABI in ``include/qed.h`` (ctypes; argument marshalling only).

Every step of the QED Monte-Carlo path runs in the CUDA library; PyTorch supplies device memory
(through the caching allocator, passed to the library as a ``qed_allocator``) and streams.
Loading fails loudly when the compiled library is missing: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

ELECTRON, POSITRON, PHOTON = 0, 1, 2
FP64, MIXED = 0, 1
FIELD_UNIFORM, FIELD_ROTATING_E, FIELD_PLANE_LP, FIELD_PLANE_CP, FIELD_GRID = 0, 1, 2, 3, 4
STATUS = {0: "QED_OK", 1: "QED_ERR_INVALID_ARG", 2: "QED_ERR_OOM", 3: "QED_ERR_CAPACITY", 4: "QED_ERR_TIMEOUT",
          5: "QED_ERR_CUDA", 6: "QED_ERR_NUMERIC"}
(QED_OK, QED_ERR_INVALID_ARG, QED_ERR_OOM, QED_ERR_CAPACITY, QED_ERR_TIMEOUT, QED_ERR_CUDA,
 QED_ERR_NUMERIC) = range(7)


class QedError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


# ------------------------------------------------------------------------------ C structs
class TableParams(C.Structure):
    _fields_ = [("n_eta", C.c_int), ("eta_min", C.c_double), ("eta_max", C.c_double), ("n_xi", C.c_int),
                ("n_chi", C.c_int), ("chi_min", C.c_double), ("chi_max", C.c_double), ("n_f", C.c_int),
                ("energy_cut", C.c_double)]


_dp = C.POINTER(C.c_double)


class TableArrays(C.Structure):
    _fields_ = [(k, _dp) for k in ("ln_h", "g", "zeta_lo", "zeta_hi", "P", "Q", "ln_T", "Pf")]


class Allocator(C.Structure):
    _fields_ = [("alloc", C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)),
                ("free", C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)),
                ("user", C.c_void_p)]


class MergeParams(C.Structure):
    _fields_ = [("origin", C.c_double * 3), ("cell", C.c_double * 3), ("n_cells", C.c_int32 * 3),
                ("n_face", C.c_int32), ("n_sub", C.c_int32), ("min_group", C.c_int32)]


class Soa(C.Structure):
    _fields_ = [("x", C.c_void_p), ("y", C.c_void_p), ("z", C.c_void_p), ("ux", C.c_void_p), ("uy", C.c_void_p),
                ("uz", C.c_void_p), ("tau", C.c_void_p), ("id", C.c_void_p)]


class SpeciesView(C.Structure):
    _fields_ = [("arrays", Soa), ("capacity", C.c_size_t), ("kind", C.c_int), ("precision", C.c_int)]


class FieldDesc(C.Structure):
    _fields_ = [("kind", C.c_int), ("E", C.c_double * 3), ("B", C.c_double * 3), ("E0", C.c_double),
                ("omega", C.c_double), ("phase0", C.c_double), ("phi_start", C.c_double), ("phi_len", C.c_double),
                ("grid", C.c_void_p), ("n", C.c_int32 * 3), ("shape", C.c_int32), ("origin", C.c_double * 3),
                ("spacing", C.c_double * 3)]


class StepParamsC(C.Structure):
    _fields_ = [("dt", C.c_double), ("t0", C.c_double), ("step", C.c_uint64), ("seed", C.c_uint64),
                ("scenario", C.c_uint64), ("field", FieldDesc), ("emit_photons", C.c_int), ("make_pairs", C.c_int),
                ("drain_photons", C.c_int), ("recoil_energy", C.c_int), ("window_x0", C.c_double),
                ("window_v", C.c_double)]


class Ledger(C.Structure):
    _fields_ = [("n", C.c_double * 3), ("energy", C.c_double * 3), ("emitted_n", C.c_double),
                ("emitted_energy", C.c_double), ("dropped_n", C.c_double), ("emit_defect", C.c_double),
                ("pairs_n", C.c_double), ("pair_energy", C.c_double), ("pair_defect", C.c_double),
                ("drained_n", C.c_double), ("drained_energy", C.c_double), ("oor_eta", C.c_double),
                ("oor_chi", C.c_double)]

    def as_dict(self):
        out = {}
        for k, _ in self._fields_:
            v = getattr(self, k)
            out[k] = list(v) if not isinstance(v, float) else v
        return out


EXPORTS = ["qed_tables_build", "qed_tables_from_arrays", "qed_tables_export", "qed_tables_free",
           "qed_species_alloc", "qed_species_free", "qed_species_upload", "qed_species_download",
           "qed_species_count", "qed_species_view_get", "qed_species_save", "qed_species_restore",
           "qed_species_init_tau", "qed_species_compact", "qed_species_set_weights", "qed_species_get_weights",
           "qed_species_totals", "qed_species_merge",
           "qed_step", "qed_run", "qed_run_multistep", "qed_read_ledger", "qed_drain_new_particles", "qed_check",
           "qed_step_emit_noalloc",
           "qed_batch_create", "qed_batch_attach", "qed_batch_detach", "qed_batch_run", "qed_batch_remaining",
           "qed_batch_config", "qed_batch_multistep", "qed_batch_tune", "qed_batch_free",
           "qed_eval_particles", "qed_sample", "qed_philox", "qed_work_read", "qed_work_read_split", "qed_timing_enable", "qed_timing_read_multistep", "qed_timing_read",
           "qed_selftest_wait", "qed_launch_count", "qed_version", "qed_last_error"]

_lib = None


def lib_path():
    return _build.lib_path()


def load_library(path: str | None = None):
    """Load the compiled library; raises if it has not been built (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"QED CUDA library not found at {path}: run paper_1311_5551_gb300.build.build() "
                           "(or __graft_entry__.build()) first")
    L = C.CDLL(path)
    vp, sz, st, u64 = C.c_void_p, C.c_size_t, C.c_int, C.c_uint64
    sig = {
        "qed_tables_build": (st, [C.POINTER(TableParams), C.POINTER(Allocator), vp, C.POINTER(vp)]),
        "qed_tables_from_arrays": (st, [C.POINTER(TableParams), C.POINTER(TableArrays), C.POINTER(Allocator), vp,
                                        C.POINTER(vp)]),
        "qed_tables_export": (st, [vp, C.POINTER(TableArrays)]),
        "qed_tables_free": (None, [vp]),
        "qed_species_alloc": (st, [C.c_int, C.c_int, sz, sz, C.POINTER(Allocator), vp, C.POINTER(vp)]),
        "qed_species_free": (None, [vp]),
        "qed_species_upload": (st, [vp, C.POINTER(Soa), sz, C.c_uint32, vp]),
        "qed_species_download": (st, [vp, C.POINTER(Soa), sz, C.POINTER(sz), vp]),
        "qed_species_count": (st, [vp, C.POINTER(sz), vp]),
        "qed_species_view_get": (st, [vp, C.POINTER(SpeciesView)]),
        "qed_species_save": (st, [vp, vp, sz, C.POINTER(sz), vp]),
        "qed_species_restore": (st, [vp, vp, sz, vp]),
        "qed_species_init_tau": (st, [vp, u64, u64, vp]),
        "qed_species_compact": (st, [vp, vp]),
        "qed_species_set_weights": (st, [vp, vp, sz, vp]),
        "qed_species_get_weights": (st, [vp, vp, sz, C.POINTER(sz), vp]),
        "qed_species_totals": (st, [vp, C.POINTER(C.c_double), vp]),
        "qed_species_merge": (st, [vp, C.POINTER(MergeParams), C.POINTER(C.c_uint64), vp]),
        "qed_step": (st, [vp, C.POINTER(vp), C.POINTER(StepParamsC), vp]),
        "qed_run": (st, [vp, C.POINTER(vp), C.POINTER(StepParamsC), u64, vp]),
        "qed_read_ledger": (st, [C.POINTER(vp), C.POINTER(Ledger), vp]),
        "qed_drain_new_particles": (st, [vp, C.POINTER(Soa), sz, C.POINTER(sz), vp]),
        "qed_check": (st, [C.POINTER(vp), C.c_int, vp]),
        "qed_batch_create": (st, [vp, C.c_int, C.c_int, C.POINTER(Allocator), vp, C.POINTER(vp)]),
        "qed_batch_attach": (st, [vp, C.c_int, C.POINTER(vp), C.POINTER(StepParamsC), u64, vp]),
        "qed_batch_detach": (st, [vp, C.c_int, vp]),
        "qed_batch_run": (st, [vp, u64, vp]),
        "qed_batch_remaining": (st, [vp, C.POINTER(C.c_uint32), vp]),
        "qed_batch_config": (st, [vp, C.c_int, C.c_int]),
        "qed_batch_tune": (st, [vp, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), vp]),
        "qed_batch_multistep": (st, [vp, C.c_int]),
        "qed_batch_free": (None, [vp]),
        "qed_step_emit_noalloc": (st, [vp, C.c_int, C.POINTER(Soa), sz, C.POINTER(Soa), sz, vp,
                                       C.POINTER(StepParamsC), vp]),
        "qed_eval_particles": (st, [vp, C.c_int, C.c_int, C.POINTER(FieldDesc), C.c_double, C.c_double, C.c_double,
                                    sz] + [vp] * 11 + [vp]),
        "qed_sample": (st, [vp, C.c_int, C.c_int, sz, vp, vp, vp, vp, vp]),
        "qed_philox": (st, [sz, vp, C.POINTER(C.c_uint64), vp, vp]),
        "qed_work_read": (st, [vp, C.POINTER(C.c_uint64), C.c_int, vp]),
        "qed_work_read_split": (st, [vp, C.POINTER(C.c_uint64), C.c_int, vp]),
        "qed_run_multistep": (st, [vp, C.POINTER(vp), C.POINTER(StepParamsC), u64, C.c_int, vp]),
        "qed_timing_enable": (st, [C.c_int]),
        "qed_timing_read": (st, [C.POINTER(C.c_double), C.POINTER(C.c_uint64), C.c_int]),
        "qed_timing_read_multistep": (st, [C.POINTER(C.c_double), C.POINTER(C.c_uint64), C.c_int]),
        "qed_selftest_wait": (st, [C.c_uint32, C.POINTER(C.c_uint32), vp]),
        "qed_launch_count": (u64, []),
        "qed_version": (C.c_char_p, []),
        "qed_last_error": (C.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def lib():
    return load_library()


def _check(code):
    if code != 0:
        raise QedError(code, lib().qed_last_error().decode())


def selftest_wait(polls: int = 1000, stream=None) -> int:
    """Bits of the bounded-wait self-test (3: a completed wait succeeded, a never-completed one gave up)."""
    out = C.c_uint32()
    _check(lib().qed_selftest_wait(int(polls), C.byref(out), _stream_ptr(stream)))
    return int(out.value)


def launch_count() -> int:
    return int(lib().qed_launch_count())


def work_read(electrons, reset=False, stream=None):
    """(e+- pushes, photon pushes, particles created) since the last reset, steps with these electrons."""
    out = (C.c_uint64 * 3)()
    _check(lib().qed_work_read(electrons._h, out, int(reset), _stream_ptr(stream)))
    return int(out[0]), int(out[1]), int(out[2])


def work_read_split(electrons, reset=False, stream=None):
    """work_read() plus the e+- and photon pushes made by multi-step passes (part of the first two)
    and the per-step kernel's photon pushes that changed (and stored) the optical depth."""
    out = (C.c_uint64 * 6)()
    _check(lib().qed_work_read_split(electrons._h, out, int(reset), _stream_ptr(stream)))
    return tuple(int(v) for v in out)


def timing_enable(on: bool):
    _check(lib().qed_timing_enable(int(on)))


def timing_read(reset=True):
    ms, n = C.c_double(), C.c_uint64()
    _check(lib().qed_timing_read(C.byref(ms), C.byref(n), int(reset)))
    return float(ms.value), int(n.value)


def timing_read_multistep(reset=True):
    """(ms, passes) of the multi-step probe and commit launches timed since the last reset."""
    ms, n = C.c_double(), C.c_uint64()
    _check(lib().qed_timing_read_multistep(C.byref(ms), C.byref(n), int(reset)))
    return float(ms.value), int(n.value)


# ------------------------------------------------------------------------------ torch plumbing
def _torch():
    import torch

    return torch


def _stream_ptr(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


_ALLOC_KEEP = []


def torch_allocator(on_alloc=None, on_free=None):
    """A qed_allocator backed by PyTorch's caching allocator; on_alloc(ptr, nbytes) and
    on_free(ptr, nbytes), if given, see every allocation and release (accounting)."""
    torch = _torch()

    @C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
    def _alloc(nbytes, stream, user):
        try:
            ptr = int(torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0)))
        except Exception:  # reported to the library as NULL (QED_ERR_OOM)
            return None
        if on_alloc is not None:
            on_alloc(ptr, int(nbytes))
        return ptr

    @C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
    def _free(ptr, nbytes, stream, user):
        if on_free is not None:
            on_free(int(ptr), int(nbytes))
        torch.cuda.caching_allocator_delete(int(ptr))

    a = Allocator(_alloc, _free, None)
    _ALLOC_KEEP.append((a, _alloc, _free))
    return a


_DEFAULT_ALLOC = None


def default_allocator():
    global _DEFAULT_ALLOC
    if _DEFAULT_ALLOC is None:
        _DEFAULT_ALLOC = torch_allocator()
    return _DEFAULT_ALLOC


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


# ------------------------------------------------------------------------------ tables
@dataclass
class TableSpec:
    n_eta: int = 256
    eta_min: float = 1e-4
    eta_max: float = 1e2
    n_xi: int = 256
    n_chi: int = 256
    chi_min: float = 1e-2
    chi_max: float = 1e2
    n_f: int = 128
    energy_cut: float = 1e-9

    def c(self):
        return TableParams(self.n_eta, self.eta_min, self.eta_max, self.n_xi, self.n_chi, self.chi_min, self.chi_max,
                           self.n_f, self.energy_cut)


TABLE_KEYS = ("ln_h", "g", "zeta_lo", "zeta_hi", "P", "Q", "ln_T", "Pf")


class Tables:
    """Device look-up tables (Sec. 3); built by the library's own quadrature or loaded from arrays."""

    def __init__(self, spec: TableSpec | None = None, arrays: dict | None = None, stream=None):
        self.spec = spec or TableSpec()
        self._h = C.c_void_p()
        p = self.spec.c()
        if arrays is None:
            _check(lib().qed_tables_build(C.byref(p), C.byref(default_allocator()), _stream_ptr(stream),
                                          C.byref(self._h)))
        else:
            keep = {k: np.ascontiguousarray(arrays[k], dtype=np.float64) for k in TABLE_KEYS if k in arrays}
            ta = TableArrays(*[keep[k].ctypes.data_as(_dp) if k in keep else None for k in TABLE_KEYS])
            _check(lib().qed_tables_from_arrays(C.byref(p), C.byref(ta), C.byref(default_allocator()),
                                                _stream_ptr(stream), C.byref(self._h)))

    def export(self) -> dict:
        s = self.spec
        out = {"ln_h": np.zeros(s.n_eta), "g": np.zeros(s.n_eta), "zeta_lo": np.zeros(s.n_eta),
               "zeta_hi": np.zeros(s.n_eta), "P": np.zeros((s.n_eta, s.n_xi)), "Q": np.zeros((s.n_eta, s.n_xi)),
               "ln_T": np.zeros(s.n_chi), "Pf": np.zeros((s.n_chi, s.n_f))}
        ta = TableArrays(*[out[k].ctypes.data_as(_dp) for k in TABLE_KEYS])
        _check(lib().qed_tables_export(self._h, C.byref(ta)))
        return out

    def close(self):
        if self._h:
            lib().qed_tables_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------------------ species
class Species:
    """SoA particles of one kind in device memory owned by the library (PyTorch-allocated)."""

    def __init__(self, kind: int, precision: int, capacity: int, append_capacity: int | None = None, stream=None,
                 allocator: Allocator | None = None):
        """``allocator``: a qed_allocator (see torch_allocator) that every device allocation of this
        species goes through, including later ones (weights, compaction, merging scratch);
        PyTorch's caching allocator by default."""
        self.kind, self.precision, self.capacity = kind, precision, int(capacity)
        self.append_capacity = int(append_capacity if append_capacity is not None else max(1024, capacity // 4))
        self._alloc = allocator if allocator is not None else default_allocator()
        self._h = C.c_void_p()
        _check(lib().qed_species_alloc(kind, precision, self.capacity, self.append_capacity,
                                       C.byref(self._alloc), _stream_ptr(stream), C.byref(self._h)))

    @property
    def real_dtype(self):
        return np.float32 if self.precision == MIXED else np.float64

    def upload(self, x, u, tau=None, ids=None, next_id=None, stream=None):
        """Copy particles in (numpy arrays or torch tensors, host or device, shape (n,3))."""
        torch = _torch()
        td = torch.float32 if self.precision == MIXED else torch.float64
        x = torch.as_tensor(x).to(td)
        u = torch.as_tensor(u).to(td)
        n = x.shape[0]
        cols = [x[:, c].contiguous() for c in range(3)] + [u[:, c].contiguous() for c in range(3)]
        t = torch.as_tensor(tau).to(torch.float64).contiguous() if tau is not None else None
        i = torch.as_tensor(ids).to(torch.int32).contiguous() if ids is not None else None
        s = Soa(*[_ptr(c) for c in cols], _ptr(t), _ptr(i))
        nid = int(next_id) if next_id is not None else (int(torch.as_tensor(ids).max()) + 1 if ids is not None and n
                                                         else n)
        _check(lib().qed_species_upload(self._h, C.byref(s), n, nid, _stream_ptr(stream)))
        # keep the sources alive until the copies have run
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()

    def upload_soa(self, soa: Soa, n: int, next_id: int, stream=None):
        _check(lib().qed_species_upload(self._h, C.byref(soa), n, next_id, _stream_ptr(stream)))

    def init_tau(self, seed: int, scenario: int = 0, stream=None):
        _check(lib().qed_species_init_tau(self._h, seed, scenario, _stream_ptr(stream)))

    def save(self, stream=None) -> np.ndarray:
        """Bit-exact checkpoint of the held particles (stored form) as a host byte array."""
        need = C.c_size_t()
        _check(lib().qed_species_save(self._h, None, 0, C.byref(need), _stream_ptr(stream)))
        buf = np.empty(need.value, dtype=np.uint8)
        _check(lib().qed_species_save(self._h, buf.ctypes.data_as(C.c_void_p), buf.nbytes, C.byref(need),
                                      _stream_ptr(stream)))
        return buf

    def restore(self, buf: np.ndarray, stream=None):
        _check(lib().qed_species_restore(self._h, buf.ctypes.data_as(C.c_void_p), buf.nbytes, _stream_ptr(stream)))
        _torch().cuda.synchronize()

    def set_weights(self, w, stream=None):
        """Macroparticle weights of the held particles (host array, species precision)."""
        w = np.ascontiguousarray(w, dtype=self.real_dtype)
        _check(lib().qed_species_set_weights(self._h, w.ctypes.data_as(C.c_void_p), len(w), _stream_ptr(stream)))
        _torch().cuda.synchronize()

    def weights(self, stream=None) -> np.ndarray:
        n = self.count(stream)
        w = np.empty(n, dtype=self.real_dtype)
        got = C.c_size_t()
        _check(lib().qed_species_get_weights(self._h, w.ctypes.data_as(C.c_void_p), n, C.byref(got),
                                             _stream_ptr(stream)))
        return w[: got.value]

    def totals(self, stream=None):
        """(sum w, sum w energy, sum w momentum[3]) in FP64."""
        out = (C.c_double * 5)()
        _check(lib().qed_species_totals(self._h, out, _stream_ptr(stream)))
        return out[0], out[1], np.array(out[2:5])

    def merge(self, origin, cell, n_cells, n_face=8, n_sub=4, min_group=4, stream=None) -> int:
        """Macroparticle merging of this species (qed_species_merge); returns the groups merged."""
        mp = MergeParams((C.c_double * 3)(*origin), (C.c_double * 3)(*cell), (C.c_int32 * 3)(*n_cells), int(n_face),
                         int(n_sub), int(min_group))
        g = C.c_uint64()
        _check(lib().qed_species_merge(self._h, C.byref(mp), C.byref(g), _stream_ptr(stream)))
        return int(g.value)

    def compact(self, stream=None):
        """Remove converted photons, keeping the order of the survivors."""
        _check(lib().qed_species_compact(self._h, _stream_ptr(stream)))

    def count(self, stream=None) -> int:
        n = C.c_size_t()
        _check(lib().qed_species_count(self._h, C.byref(n), _stream_ptr(stream)))
        return int(n.value)

    def view(self):
        v = SpeciesView()
        _check(lib().qed_species_view_get(self._h, C.byref(v)))
        return v

    def download(self, stream=None) -> dict:
        """Host copy of the held particles: x, u (n,3) in the species precision, tau, id."""
        n = self.count(stream)
        dt = self.real_dtype
        cols = [np.empty(n, dtype=dt) for _ in range(6)]
        tau = np.empty(n, dtype=np.float64)
        ids = np.empty(n, dtype=np.uint32)
        s = Soa(*[c.ctypes.data_as(C.c_void_p) for c in cols], tau.ctypes.data_as(C.c_void_p),
                ids.ctypes.data_as(C.c_void_p))
        got = C.c_size_t()
        _check(lib().qed_species_download(self._h, C.byref(s), n, C.byref(got), _stream_ptr(stream)))
        return {"x": np.stack(cols[:3], axis=1), "u": np.stack(cols[3:], axis=1), "tau": tau, "id": ids}

    def close(self):
        if self._h:
            lib().qed_species_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------------------ stepping
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
    # FIELD_GRID: contiguous device tensor of shape (6, nz, ny, nx) (Ex, Ey, Ez, cBx, cBy, cBz), in
    # the species precision, Yee-staggered; it must stay alive while steps that use it run
    grid: object = None
    shape: int = 1
    origin: tuple = (0.0, 0.0, 0.0)
    spacing: tuple = (1.0, 1.0, 1.0)

    def c(self):
        ptr, n = None, (0, 0, 0)
        if self.grid is not None:
            if not self.grid.is_cuda or not self.grid.is_contiguous() or self.grid.dim() != 4 or self.grid.shape[0] != 6:
                raise ValueError("grid must be a contiguous CUDA tensor of shape (6, nz, ny, nx)")
            ptr = self.grid.data_ptr()
            n = (self.grid.shape[3], self.grid.shape[2], self.grid.shape[1])
        return FieldDesc(self.kind, (C.c_double * 3)(*self.E), (C.c_double * 3)(*self.B), self.E0, self.omega,
                         self.phase0, self.phi_start, self.phi_len, ptr, (C.c_int32 * 3)(*n), int(self.shape),
                         (C.c_double * 3)(*self.origin), (C.c_double * 3)(*self.spacing))


@dataclass
class StepParams:
    dt: float
    t0: float = 0.0
    seed: int = 1
    scenario: int = 0
    field: Field = field(default_factory=Field)
    emit_photons: bool = True
    make_pairs: bool = True
    drain_photons: bool = False
    recoil_energy: bool = False
    window_x0: float = 0.0
    window_v: float = 0.0

    def c(self, step):
        return StepParamsC(self.dt, self.t0, int(step), int(self.seed), int(self.scenario), self.field.c(),
                           int(self.emit_photons), int(self.make_pairs), int(self.drain_photons),
                           int(self.recoil_energy), self.window_x0, self.window_v)


def _check_grid(fld, precision):
    """A grid field's tensor must be in the species precision (the library reads it as such)."""
    if fld is None or fld.grid is None:
        return
    want = _torch().float32 if precision == MIXED else _torch().float64
    if fld.grid.dtype != want:
        raise ValueError(f"grid field tensor must be {want} for this precision, got {fld.grid.dtype}")


def _sp_array(species):
    return (C.c_void_p * 4)(*[s._h if s is not None else None for s in species])


def run(tables: Tables, species, params: StepParams, step: int, n_steps: int = 1, stream=None):
    """n_steps Monte-Carlo steps of (electrons, positrons, photons[, drain]) from step index ``step``."""
    sp = list(species) + [None] * (4 - len(species))
    _check_grid(params.field, sp[0].precision)
    p = params.c(step)
    _check(lib().qed_run(tables._h, _sp_array(sp), C.byref(p), int(n_steps), _stream_ptr(stream)))


def run_multistep(tables: Tables, species, params: StepParams, step: int, n_steps: int, chunk: int = 16,
                  stream=None):
    """As run(), taking event-free stretches of up to ``chunk`` steps in one pass (same particles)."""
    sp = list(species) + [None] * (4 - len(species))
    _check_grid(params.field, sp[0].precision)
    p = params.c(step)
    _check(lib().qed_run_multistep(tables._h, _sp_array(sp), C.byref(p), int(n_steps), int(chunk),
                                   _stream_ptr(stream)))


def read_ledger(species, stream=None) -> dict:
    led = Ledger()
    sp = list(species) + [None] * (4 - len(species))
    _check(lib().qed_read_ledger(_sp_array(sp), C.byref(led), _stream_ptr(stream)))
    return led.as_dict()


_SOA_KEYS = ("x", "y", "z", "ux", "uy", "uz", "tau", "id")


def noalloc_arg_errors(precision: int, electrons: dict, n: int, photons: dict, photon_counter,
                       require_cuda: bool = True) -> list[str]:
    """Why the arguments of step_emit_noalloc would let the kernels read or write outside the
    caller's tensors (empty when they are fine).  The C entry point sees only raw pointers, the
    electron count and the photon capacity (photons["x"].numel()), so every array is checked here:
    on the current CUDA device (require_cuda), contiguous, long enough, and of the element type
    the precision implies (float32 or float64 coordinates, 8-byte tau, 4-byte ids); the counter
    holds at least 3 four-byte words."""
    errs = []
    rbytes = 4 if precision == MIXED else 8
    if precision not in (FP64, MIXED):
        return [f"unknown precision {precision}"]
    if n < 0:
        errs.append("n must be >= 0")
    cur = None
    if require_cuda:
        torch = _torch()
        cur = torch.cuda.current_device() if torch.cuda.is_available() else None

    def check(name, t, min_len, nbytes, floating):
        if t is None:
            errs.append(f"{name} is missing")
            return
        if require_cuda and (not t.is_cuda or t.device.index != cur):
            errs.append(f"{name} must be a tensor on the current CUDA device")
        if not t.is_contiguous():
            errs.append(f"{name} must be contiguous")
        if t.element_size() != nbytes or (floating is not None and t.dtype.is_floating_point != floating):
            errs.append(f"{name} has dtype {t.dtype}, needs {nbytes}-byte "
                        f"{'float' if floating else 'integer' if floating is False else 'words'}")
        if t.numel() < min_len:
            errs.append(f"{name} holds {t.numel()} elements, needs {min_len}")

    for side, arrays, length in (("electrons", electrons, n), ("photons", photons, None)):
        if length is None:
            x = arrays.get("x")
            length = x.numel() if x is not None else 0
        for k in _SOA_KEYS:
            t = arrays.get(k)
            if k in ("x", "y", "z", "ux", "uy", "uz"):
                check(f"{side}[{k}]", t, length, rbytes, True)
            elif k == "tau":
                check(f"{side}[tau]", t, length, 8, None)  # double, or the stored (hi, lo) float pair
            else:
                check(f"{side}[id]", t, length, 4, False)
    check("photon_counter", photon_counter, 3, 4, False)
    return errs


def step_emit_noalloc(tables: Tables, precision: int, electrons: dict, n: int, photons: dict, photon_counter,
                      params: StepParams, step: int, stream=None):
    """Allocation-free emission step on caller-owned device tensors (see qed_step_emit_noalloc):
    ``electrons``/``photons`` map x, y, z, ux, uy, uz, tau, id to device tensors.  Raises
    ValueError, before anything reaches the GPU, when an array is on the wrong device, not
    contiguous, too short or of the wrong element type (noalloc_arg_errors)."""
    errs = noalloc_arg_errors(precision, electrons, n, photons, photon_counter)
    if errs:
        raise ValueError("step_emit_noalloc: " + "; ".join(errs))
    keys = _SOA_KEYS
    es = Soa(*[electrons[k].data_ptr() for k in keys])
    ps = Soa(*[photons[k].data_ptr() for k in keys])
    _check_grid(params.field, precision)
    p = params.c(step)
    _check(lib().qed_step_emit_noalloc(tables._h, precision, C.byref(es), n, C.byref(ps), photons["x"].numel(),
                                       C.c_void_p(photon_counter.data_ptr()), C.byref(p), _stream_ptr(stream)))


class Batch:
    """Independent scenarios advanced together (qed_batch_*): one slot per scenario."""

    def __init__(self, tables: Tables, precision: int, slots: int, stream=None):
        self.tables, self.precision, self.slots = tables, precision, slots
        self._h = C.c_void_p()
        self._keep = {}
        _check(lib().qed_batch_create(tables._h, precision, slots, C.byref(default_allocator()), _stream_ptr(stream),
                                      C.byref(self._h)))

    def attach(self, slot: int, species, params: StepParams, first_step: int, n_steps: int, stream=None):
        sp = list(species) + [None] * (4 - len(species))
        _check_grid(params.field, self.precision)
        p = params.c(first_step)
        _check(lib().qed_batch_attach(self._h, slot, _sp_array(sp), C.byref(p), int(n_steps), _stream_ptr(stream)))
        self._keep[slot] = sp  # the species must outlive the slot

    def detach(self, slot: int, stream=None):
        _check(lib().qed_batch_detach(self._h, slot, _stream_ptr(stream)))
        self._keep.pop(slot, None)

    def run(self, n_steps: int, stream=None):
        _check(lib().qed_batch_run(self._h, int(n_steps), _stream_ptr(stream)))

    def remaining(self, stream=None) -> np.ndarray:
        out = np.zeros(self.slots, dtype=np.uint32)
        _check(lib().qed_batch_remaining(self._h, out.ctypes.data_as(C.POINTER(C.c_uint32)), _stream_ptr(stream)))
        return out

    def config(self, target_blocks: int, graph_steps: int):
        _check(lib().qed_batch_config(self._h, int(target_blocks), int(graph_steps)))

    def multistep(self, chunk: int):
        """Take each slot's event-free stretches of up to ``chunk`` steps in one pass (0: off)."""
        _check(lib().qed_batch_multistep(self._h, int(chunk)))

    def tune(self, trial_steps: int = 4, stream=None):
        tb, gs = C.c_int(), C.c_int()
        _check(lib().qed_batch_tune(self._h, int(trial_steps), C.byref(tb), C.byref(gs), _stream_ptr(stream)))
        return tb.value, gs.value

    def close(self):
        if self._h:
            lib().qed_batch_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def check(species, stream=None):
    sp = [s for s in species if s is not None]
    _check(lib().qed_check((C.c_void_p * len(sp))(*[s._h for s in sp]), len(sp), _stream_ptr(stream)))


def drain(drained: Species, stream=None) -> dict:
    n = drained.count(stream)
    dt = drained.real_dtype
    cols = [np.empty(n, dtype=dt) for _ in range(6)]
    tau = np.empty(n, dtype=np.float64)
    ids = np.empty(n, dtype=np.uint32)
    s = Soa(*[c.ctypes.data_as(C.c_void_p) for c in cols], tau.ctypes.data_as(C.c_void_p),
            ids.ctypes.data_as(C.c_void_p))
    got = C.c_size_t()
    _check(lib().qed_drain_new_particles(drained._h, C.byref(s), n, C.byref(got), _stream_ptr(stream)))
    m = int(got.value)
    return {"x": np.stack([c[:m] for c in cols[:3]], axis=1), "u": np.stack([c[:m] for c in cols[3:]], axis=1),
            "tau": tau[:m], "id": ids[:m]}


# ------------------------------------------------------------------------------ diagnostics
def eval_particles(tables: Tables, precision: int, kind: int, fld: Field, t: float, x, u, window_x0=0.0,
                   window_v=0.0, stream=None):
    """eta (or chi), gamma (or eps), rate and fields per particle, computed by the device functions."""
    torch = _torch()
    x = torch.as_tensor(x, dtype=torch.float64, device="cuda").contiguous()
    u = torch.as_tensor(u, dtype=torch.float64, device="cuda").contiguous()
    n = x.shape[0]
    cols = [x[:, c].contiguous() for c in range(3)] + [u[:, c].contiguous() for c in range(3)]
    oE = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    oB = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    op, oe, orate = (torch.empty(n, dtype=torch.float64, device="cuda") for _ in range(3))
    _check_grid(fld, precision)
    f = fld.c()
    _check(lib().qed_eval_particles(tables._h, precision, kind, C.byref(f), float(t), float(window_x0),
                                    float(window_v), n, *[_ptr(c) for c in cols], _ptr(oE), _ptr(oB), _ptr(op),
                                    _ptr(oe), _ptr(orate), _stream_ptr(stream)))
    torch.cuda.synchronize()
    return {"E": oE.cpu().numpy(), "B": oB.cpu().numpy(), "param": op.cpu().numpy(), "energy": oe.cpu().numpy(),
            "rate": orate.cpu().numpy()}


def sample(tables: Tables, precision: int, which: int, param, U, stream=None):
    """qed_sample: which = 0 xi(eta, U), 1 f(chi, U) (returns values, ok); which = 2 h(eta),
    3 T(chi) (U ignored; returns values, range flags)."""
    torch = _torch()
    p = torch.as_tensor(param, dtype=torch.float64, device="cuda").contiguous()
    u = torch.as_tensor(U, dtype=torch.float64, device="cuda").contiguous() if U is not None else None
    n = p.shape[0]
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    ok = torch.empty(n, dtype=torch.int32, device="cuda")
    _check(lib().qed_sample(tables._h, precision, which, n, _ptr(p), _ptr(u), _ptr(out), _ptr(ok),
                            _stream_ptr(stream)))
    torch.cuda.synchronize()
    flags = ok.cpu().numpy()
    return out.cpu().numpy(), (flags if which >= 2 else flags.astype(bool))


def philox(ctr, key, stream=None):
    torch = _torch()
    c = torch.as_tensor(np.asarray(ctr, dtype=np.uint64).view(np.int64), device="cuda").contiguous()
    n = c.numel() // 4
    out = torch.empty(4 * n, dtype=torch.int64, device="cuda")
    k = (C.c_uint64 * 2)(int(key[0]) & (2**64 - 1), int(key[1]) & (2**64 - 1))
    _check(lib().qed_philox(n, _ptr(c), k, _ptr(out), _stream_ptr(stream)))
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint64).reshape(n, 4)
