"""GPU parity of the grid field gather (the PIC interpolation of Sec. 3.2) against the oracle:
per-particle fields for both particle shapes (inside, at the edges and outside the grid), whole
runs in a grid field, and a grid-field scenario inside a batch."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle as o  # noqa: E402
from paper_1311_5551_gb300 import build as qbuild  # noqa: E402
from paper_1311_5551_gb300 import qed, workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def tables():
    qbuild.build()
    return qed.Tables()


def random_grid(n, seed, scale=1e-3):
    """Grid values representable in FP32, so both paths read the same numbers."""
    rng = np.random.default_rng(seed)
    return (rng.normal(size=(6, n[2], n[1], n[0])) * scale).astype(np.float32).astype(np.float64)


def dev_grid(g, prec):
    return torch.tensor(g, dtype=torch.float32 if prec == qed.MIXED else torch.float64, device="cuda").contiguous()


@pytest.mark.parametrize("prec", [qed.FP64, qed.MIXED])
@pytest.mark.parametrize("shape", [1, 2])
def test_grid_gather_parity(tables, prec, shape):
    N, org, sp = (13, 11, 9), (-20.0, 5.0, 100.0), (3.0, 2.5, 4.0)
    g = random_grid(N, 3 + shape)
    rng = np.random.default_rng(7)
    n = 3001
    # positions from 3 cells below the grid to 3 cells above it on every axis
    x = np.stack([rng.uniform(org[a] - 3 * sp[a], org[a] + (N[a] + 2) * sp[a], n) for a in range(3)], axis=1)
    x = x.astype(np.float32).astype(np.float64)
    u = np.tile([[100.0, 0.0, 0.0]], (n, 1))
    fq = qed.Field(kind=qed.FIELD_GRID, grid=dev_grid(g, prec), shape=shape, origin=org, spacing=sp)
    r = qed.eval_particles(tables, prec, qed.ELECTRON, fq, 0.0, x, u)
    fo = o.Field(kind=o.FIELD_GRID, grid=g, shape=shape, origin=org, spacing=sp)
    tol = (1e-12 if prec == qed.FP64 else 1e-5) * np.abs(g).max()
    outside = 0
    for i in range(n):
        E, B = o.field_eval(fo, 0.0, x[i])
        np.testing.assert_allclose(r["E"][i], E, rtol=0, atol=tol)
        np.testing.assert_allclose(r["B"][i], B, rtol=0, atol=tol)
        outside += not (np.any(E) or np.any(B))
    assert outside > 100  # the sample reaches past the grid


def grid_holding_test1(prec, pert=1e-4):
    """cB_z = 1e-3 (test problem 1) plus a random perturbation, on a grid covering the orbits."""
    n, sp = 16, 2.0e5
    g = random_grid((n, n, n), 11, scale=pert)
    g[5] += 1e-3
    g = g.astype(np.float32).astype(np.float64)
    org = (-sp * (n - 1) / 2,) * 3
    return g, org, (sp, sp, sp)


@pytest.mark.parametrize("prec", [qed.FP64, qed.MIXED])
def test_grid_run_against_oracle(tables, orc_tables, prec):
    w = W.uniform_b(n=2000, steps_per_gyro=1000.0, seed=8, make_pairs=True, drain_photons=False)
    g, org, sp = grid_holding_test1(prec)
    steps = 150
    oe = o.Species(w.n + 4)
    oe.set(w.x, w.u)
    oe.init_tau(o.ELECTRON, w.seed)
    op, og = o.Species(10_000), o.Species(50_000)
    fo = o.Field(kind=o.FIELD_GRID, grid=g, shape=2, origin=org, spacing=sp)
    osp = o.StepParams(dt=w.dt, seed=w.seed, make_pairs=True, field=fo)
    for k in range(steps):
        L = o.step(orc_tables, osp, k, oe, op, og)
    e = qed.Species(qed.ELECTRON, prec, 20_000, 20_000)
    p = qed.Species(qed.POSITRON, prec, 20_000, 20_000)
    ph = qed.Species(qed.PHOTON, prec, 100_000, 20_000)
    e.upload(w.x, w.u)
    e.init_tau(w.seed)
    fq = qed.Field(kind=qed.FIELD_GRID, grid=dev_grid(g, prec), shape=2, origin=org, spacing=sp)
    qed.run(tables, [e, p, ph], qed.StepParams(dt=w.dt, seed=w.seed, field=fq), 0, steps)
    qed.check([e, p, ph])
    led = qed.read_ledger([e, p, ph])
    assert L["n"][2] > 100
    if prec == qed.FP64:
        assert led["n"] == L["n"]
        d = e.download()
        assert np.allclose(d["u"], oe.u(), rtol=1e-9, atol=1e-9 * np.abs(oe.u()).max())
        assert np.allclose(d["x"], oe.x(), rtol=1e-9, atol=1e-9 * np.abs(oe.x()).max())
    else:
        assert led["n"][2] == pytest.approx(L["n"][2], rel=0.1)
        assert led["energy"][0] == pytest.approx(L["energy"][0], rel=0.01)


def test_grid_scenario_in_a_batch(tables):
    prec = qed.MIXED
    g, org, sp = grid_holding_test1(prec)
    fq = qed.Field(kind=qed.FIELD_GRID, grid=dev_grid(g, prec), shape=1, origin=org, spacing=sp)

    def make(k):
        w = W.uniform_b(n=3000 + 500 * k, steps_per_gyro=1000.0, seed=20 + k)
        s = [qed.Species(qed.ELECTRON, prec, 40_000, 40_000), qed.Species(qed.POSITRON, prec, 40_000, 40_000),
             qed.Species(qed.PHOTON, prec, 200_000, 40_000)]
        s[0].upload(w.x, w.u)
        s[0].init_tau(w.seed, k)
        fld = fq if k == 0 else qed.Field(B=w.field.B)
        return s, qed.StepParams(dt=w.dt, seed=w.seed, scenario=k, field=fld)

    ref, pr = make(0)
    qed.run(tables, ref, pr, 0, 60)
    b = qed.Batch(tables, prec, 2)
    mix = []
    for k in range(2):
        s, p = make(k)
        b.attach(k, s, p, 0, 60)
        mix.append(s)
    b.config(2 * 152, 8)
    b.run(60)
    assert np.all(b.remaining() == 0)
    for a, s in zip(ref, mix[0]):
        assert np.array_equal(a.save(), s.save())
