"""Failure detection without a GPU fault: the bounded mbarrier wait gives up and reports instead of
hanging, allocator failures and bad parameters are refused at the boundary, and the context stays
usable after each."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1311_5551_gb300 import build as qbuild  # noqa: E402
from paper_1311_5551_gb300 import qed, workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def tables():
    qbuild.build()
    return qed.Tables()


def small_run(tables, steps=5):
    w = W.uniform_b(n=500, seed=3)
    sp = [qed.Species(qed.ELECTRON, qed.MIXED, 1000, 1000), qed.Species(qed.POSITRON, qed.MIXED, 16, 16),
          qed.Species(qed.PHOTON, qed.MIXED, 4000, 1000)]
    sp[0].upload(w.x, w.u)
    sp[0].init_tau(w.seed)
    qed.run(tables, sp, qed.StepParams(dt=w.dt, seed=w.seed, field=qed.Field(B=w.field.B)), 0, steps)
    qed.check(sp)
    return sp


@pytest.mark.parametrize("polls", [1, 64, 4096])
def test_bounded_wait_gives_up_and_reports(tables, polls):
    # a completed barrier is waited for; one that nothing arrives at gives up after `polls`
    assert qed.selftest_wait(polls) == 3
    small_run(tables)  # the context is still usable


def test_allocator_failure_is_reported(tables):
    @C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
    def refuse(nbytes, stream, user):
        return None

    @C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
    def never(ptr, nbytes, stream, user):
        raise AssertionError("nothing was allocated")

    alloc = qed.Allocator(refuse, never, None)
    h = C.c_void_p()
    code = qed.lib().qed_species_alloc(qed.ELECTRON, qed.MIXED, 1000, 1000, C.byref(alloc), None, C.byref(h))
    assert code == qed.QED_ERR_OOM and not h.value
    assert "allocator returned NULL" in qed.lib().qed_last_error().decode()
    small_run(tables)


@pytest.mark.parametrize("bad", ["nan_field", "zero_dt", "species_order", "grid_without_array", "bad_shape"])
def test_bad_parameters_are_refused(tables, bad):
    w = W.uniform_b(n=100, seed=3)
    sp = [qed.Species(qed.ELECTRON, qed.MIXED, 200, 200), qed.Species(qed.POSITRON, qed.MIXED, 16, 16),
          qed.Species(qed.PHOTON, qed.MIXED, 400, 200)]
    sp[0].upload(w.x, w.u)
    p = qed.StepParams(dt=w.dt, seed=1, field=qed.Field(B=w.field.B))
    if bad == "nan_field":
        p.field = qed.Field(B=(0.0, 0.0, float("nan")))
    elif bad == "zero_dt":
        p.dt = 0.0
    elif bad == "species_order":
        sp = [sp[1], sp[0], sp[2]]
    elif bad == "grid_without_array":
        p.field = qed.Field(kind=qed.FIELD_GRID, shape=1)
    elif bad == "bad_shape":
        g = torch.zeros((6, 2, 2, 2), dtype=torch.float32, device="cuda")
        p.field = qed.Field(kind=qed.FIELD_GRID, grid=g, shape=3)
    before = sp[0].download() if bad != "species_order" else None
    with pytest.raises(qed.QedError):
        qed.run(tables, sp, p, 0, 3)
    if before is not None:  # refused before anything ran
        after = sp[0].download()
        assert np.array_equal(before["u"], after["u"]) and np.array_equal(before["x"], after["x"])
    small_run(tables)


def test_capacity_overflow_is_latched_and_reported(tables):
    # photons appended beyond the photon capacity: the step drops them, latches the error and
    # qed_check reports it; nothing is written out of bounds
    w = W.uniform_b(n=2000, cB=9e-3, seed=3)
    sp = [qed.Species(qed.ELECTRON, qed.MIXED, 4000, 4000), qed.Species(qed.POSITRON, qed.MIXED, 4000, 4000),
          qed.Species(qed.PHOTON, qed.MIXED, 64, 4000)]
    sp[0].upload(w.x, w.u)
    sp[0].init_tau(w.seed)
    qed.run(tables, sp, qed.StepParams(dt=w.dt * 50, seed=1, field=qed.Field(B=w.field.B)), 0, 4)
    with pytest.raises(qed.QedError) as e:
        qed.check(sp)
    assert "CAPACITY" in str(e.value)
    assert sp[2].count() <= 64
    small_run(tables)
