"""The allocation-free emission step against the regular path (GPU).

qed_step_emit_noalloc serves callers that cannot allocate device memory (a host code that owns
the whole device memory pool, or a loop that must keep its footprint fixed): it runs the same
kernels with their scratch in a fixed array inside the library.  This file is collected last so
that a run stopping at the first failure has already run every other test; it also passes when
run alone in a fresh process.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1311_5551_gb300 import build as qbuild  # noqa: E402
from paper_1311_5551_gb300 import qed, workloads as W  # noqa: E402

KEYS = ("x", "y", "z", "ux", "uy", "uz", "tau", "id")


def parse_checkpoint(buf, precision):
    """Arrays of a qed_species_save checkpoint (stored form)."""
    n = int(buf[16:24].view(np.uint64)[0])
    rt = np.float32 if precision == qed.MIXED else np.float64
    off, out = 64, {}
    for k in KEYS[:6]:
        out[k] = buf[off:off + n * rt().itemsize].view(rt)
        off += n * rt().itemsize
    out["tau"] = buf[off:off + 8 * n].view(np.float64)
    off += 8 * n
    out["id"] = buf[off:off + 4 * n].view(np.int32)
    return out


def device_arrays(host, cap=None):
    """Caller-owned device tensors (16-byte aligned) holding the given stored-form arrays."""
    out = {}
    for k in KEYS:
        a = host[k]
        t = torch.zeros(cap if cap else len(a), dtype=torch.from_numpy(a[:0].copy()).dtype, device="cuda")
        t[: len(a)] = torch.from_numpy(a.copy()).cuda()
        out[k] = t
    return out


@pytest.mark.parametrize("prec", [qed.FP64, qed.MIXED])
def test_noalloc_step_matches_regular_step(prec):
    qbuild.build()
    tables = qed.Tables()
    w = W.uniform_b(n=3001, n_steps=2)
    qp = qed.StepParams(dt=w.dt, seed=w.seed, field=qed.Field(**w.field.as_dict()), make_pairs=False,
                        drain_photons=True)
    # regular path: species objects allocated through the library
    e = qed.Species(qed.ELECTRON, prec, 4096, 4096)
    p = qed.Species(qed.POSITRON, prec, 64, 64)
    g = qed.Species(qed.PHOTON, prec, 64, 4096)
    d = qed.Species(qed.PHOTON, prec, 8192, 1)
    e.upload(w.x, w.u)
    e.init_tau(w.seed)
    start = parse_checkpoint(e.save(), prec)  # the same initial state for both paths
    # allocation-free path on caller-owned tensors, two calls in a row
    el = device_arrays(start)
    ph = device_arrays({k: v[:0] for k, v in start.items()}, cap=8192)
    counter = torch.zeros(3, dtype=torch.int32, device="cuda")
    for step in range(2):
        qed.run(tables, [e, p, g, d], qp, step)
        qed.step_emit_noalloc(tables, prec, el, w.n, ph, counter, qp, step)
        torch.cuda.synchronize()
        c = counter.cpu().numpy()
        assert c[2] == 0, "device error flags"
        ref_e = parse_checkpoint(e.save(), prec)
        ref_p = parse_checkpoint(d.save(), prec)
        assert c[0] == len(ref_p["id"]) and c[1] == d.count()
        tol = 1e-12 if prec == qed.FP64 else 1e-5
        for k in ("x", "y", "z", "ux", "uy", "uz"):
            np.testing.assert_allclose(el[k].cpu().numpy(), ref_e[k], rtol=tol, atol=tol)
            np.testing.assert_allclose(ph[k][: c[0]].cpu().numpy(), ref_p[k], rtol=tol, atol=tol)
        assert np.array_equal(ph["id"][: c[0]].cpu().numpy(), ref_p["id"])
        # tau in stored form: compare the values it represents
        def tau_of(a):
            if prec == qed.FP64:
                return a
            pr = a.view(np.float32).reshape(-1, 2).astype(np.float64)
            return pr[:, 0] + pr[:, 1]
        np.testing.assert_allclose(tau_of(el["tau"].cpu().numpy()), tau_of(ref_e["tau"]), rtol=tol, atol=tol)
    assert counter[0].item() > 0
    qed.check([e, p, g, d])


def _raw_call(tables, prec, el, n, ph, counter, qp, step):
    """qed_step_emit_noalloc straight through the C ABI (no binding-side checks)."""
    import ctypes as C

    es = qed.Soa(*[el[k].data_ptr() for k in KEYS])
    ps = qed.Soa(*[ph[k].data_ptr() for k in KEYS])
    p = qp.c(step)
    return qed.lib().qed_step_emit_noalloc(tables._h, prec, C.byref(es), n, C.byref(ps), ph["x"].numel(),
                                           C.c_void_p(counter.data_ptr()), C.byref(p),
                                           C.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_rejects_oversize_and_bad_dt():
    # the C entry point refuses these before it launches anything
    qbuild.build()
    tables = qed.Tables()
    z = {k: torch.zeros(16, dtype=torch.float64, device="cuda") for k in KEYS}
    z["id"] = torch.zeros(16, dtype=torch.int32, device="cuda")
    counter = torch.zeros(3, dtype=torch.int32, device="cuda")
    assert _raw_call(tables, qed.FP64, z, 65537, z, counter, qed.StepParams(dt=1.0), 0) == qed.QED_ERR_INVALID_ARG
    assert "65536" in qed.lib().qed_last_error().decode()
    for dt in (float("inf"), float("nan"), 0.0):
        assert _raw_call(tables, qed.FP64, z, 16, z, counter, qed.StepParams(dt=dt), 0) == qed.QED_ERR_INVALID_ARG
        assert "dt" in qed.lib().qed_last_error().decode()
    # the binding refuses an electron count beyond the caller's arrays before the C call
    with pytest.raises(ValueError):
        qed.step_emit_noalloc(tables, qed.FP64, z, 65537, z, counter, qed.StepParams(dt=1.0), 0)
    torch.cuda.synchronize()
    assert counter.sum().item() == 0  # nothing ran


def test_noalloc_call_after_a_failed_call():
    # a call that overflows the caller's photon capacity latches QED_ERR_CAPACITY in the counter
    # and drops that step's photons; the scratch it leaves behind must not leak into the next
    # call, which has to equal the regular path bit for bit (FP64)
    qbuild.build()
    tables = qed.Tables()
    prec = qed.FP64
    w = W.uniform_b(n=3001, n_steps=1)
    qp = qed.StepParams(dt=w.dt, seed=w.seed, field=qed.Field(**w.field.as_dict()), make_pairs=False,
                        drain_photons=True)
    e = qed.Species(qed.ELECTRON, prec, 4096, 4096)
    p = qed.Species(qed.POSITRON, prec, 64, 64)
    g = qed.Species(qed.PHOTON, prec, 64, 4096)
    d = qed.Species(qed.PHOTON, prec, 8192, 1)
    e.upload(w.x, w.u)
    e.init_tau(w.seed)
    start = parse_checkpoint(e.save(), prec)
    # first call: room for 4 photons only (about 140 are emitted)
    el = device_arrays(start)
    small = device_arrays({k: v[:0] for k, v in start.items()}, cap=4)
    counter = torch.zeros(3, dtype=torch.int32, device="cuda")
    qed.step_emit_noalloc(tables, prec, el, w.n, small, counter, qp, 0)
    torch.cuda.synchronize()
    c = counter.cpu().numpy()
    assert c[2] & (1 << qed.QED_ERR_CAPACITY), "the overflow is reported in the counter's error word"
    assert c[0] == 0, "no photon of the overflowing step is kept"
    # second call from the same initial state with enough room, against qed_run
    el = device_arrays(start)
    ph = device_arrays({k: v[:0] for k, v in start.items()}, cap=8192)
    counter.zero_()
    qed.step_emit_noalloc(tables, prec, el, w.n, ph, counter, qp, 0)
    qed.run(tables, [e, p, g, d], qp, 0)
    torch.cuda.synchronize()
    c = counter.cpu().numpy()
    assert c[2] == 0 and c[0] > 4
    ref_e = parse_checkpoint(e.save(), prec)
    ref_p = parse_checkpoint(d.save(), prec)
    assert c[0] == len(ref_p["id"])
    for k in KEYS:
        assert np.array_equal(el[k].cpu().numpy(), ref_e[k]), k
        assert np.array_equal(ph[k][: c[0]].cpu().numpy(), ref_p[k]), k
    qed.check([e, p, g, d])
