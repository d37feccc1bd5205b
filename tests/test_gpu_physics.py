"""Whole runs on the GPU against the oracle (statistics and the paper's tables).

Photon and electron spectra: two-sample Kolmogorov-Smirnov (p > 0.01) and means within 3 sigma
between the GPU (mixed precision) and the FP64 oracle run with independent seeds.  Test problem 3:
GPU energies per initial electron against the oracle's and against Table delta_energy_1.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle as o  # noqa: E402
from paper_1311_5551_gb300 import build as qbuild  # noqa: E402
from paper_1311_5551_gb300 import qed, workloads as W  # noqa: E402

from test_oracle_step import dt_over_dtqed_to_steps_per_gyro  # noqa: E402


@pytest.fixture(scope="module")
def tables():
    qbuild.build()
    return qed.Tables()


def gpu_uniform_b(tables, w, prec, pairs, drain, steps):
    n = w.n
    e = qed.Species(qed.ELECTRON, prec, 4 * n + 64, 4 * n + 64)
    p = qed.Species(qed.POSITRON, prec, 4 * n + 64, 4 * n + 64)
    g = qed.Species(qed.PHOTON, prec, 80 * n + 64, 4 * n + 64)
    d = qed.Species(qed.PHOTON, prec, 200 * n + 64, 1) if drain else None
    e.upload(w.x, w.u)
    e.init_tau(w.seed)
    qp = qed.StepParams(dt=w.dt, seed=w.seed, field=qed.Field(B=w.field.B), make_pairs=pairs, drain_photons=drain)
    sp = [e, p, g] + ([d] if drain else [])
    qed.run(tables, sp, qp, 0, steps)
    qed.check(sp)
    return sp


def test_spectra_ks_and_moments_test1(tables, orc_tables):
    stats = pytest.importorskip("scipy.stats")
    frac = 0.3
    spg = dt_over_dtqed_to_steps_per_gyro(frac)
    steps = 124  # ~1 fs
    wg = W.uniform_b(n=20000, steps_per_gyro=spg, seed=101)
    e, p, g, d = gpu_uniform_b(tables, wg, qed.MIXED, pairs=False, drain=True, steps=steps)
    gam_g = np.sqrt(1 + np.sum(e.download()["u"].astype(np.float64) ** 2, axis=1))
    eps_g = np.linalg.norm(qed.drain(d)["u"].astype(np.float64), axis=1)
    wo = W.uniform_b(n=10000, steps_per_gyro=spg, seed=202)
    oe = o.Species(wo.n + 4)
    oe.set(wo.x, wo.u)
    oe.init_tau(o.ELECTRON, wo.seed)
    op, og, od = o.Species(4), o.Species(4), o.Species(3_000_000)
    sp = o.StepParams(dt=wo.dt, seed=wo.seed, make_pairs=False, drain_photons=True, field=o.Field(B=wo.field.B))
    for k in range(steps):
        o.step(orc_tables, sp, k, oe, op, og, od)
    gam_o = oe.energy()
    eps_o = od.energy(photon=True)
    for a, b in ((gam_g, gam_o), (eps_g, eps_o)):
        assert stats.ks_2samp(a, b).pvalue > 0.01
        sig = math.sqrt(a.var() / len(a) + b.var() / len(b))
        assert abs(a.mean() - b.mean()) < 3 * sig
    # photons per electron
    assert len(eps_g) / wg.n == pytest.approx(len(eps_o) / wo.n, rel=0.03)


def oracle_test3_ledger(orc_tables, w, steps):
    e = o.Species(5 * w.n + 4)
    e.set(w.x, w.u)
    e.init_tau(o.ELECTRON, w.seed)
    p, g = o.Species(4 * w.n), o.Species(60 * w.n)
    sp = o.StepParams(dt=w.dt, seed=w.seed, make_pairs=True, field=o.Field(B=w.field.B))
    for k in range(steps):
        L = o.step(orc_tables, sp, k, e, p, g)
    return L


@pytest.mark.parametrize("prec", [qed.MIXED, qed.FP64])
def test_problem3_energies(tables, orc_tables, golden, prec):
    # test problem 3 (eta0 = 9, pairs on, photons kept) to t0 = 0.1 fs at dt = 0.3 dt_QED
    n = 10000
    w = W.uniform_b(n=n, cB=9e-3, steps_per_gyro=dt_over_dtqed_to_steps_per_gyro(0.3, 1000.0, 9e-3), seed=1,
                    make_pairs=True, drain_photons=False)
    steps = int(math.ceil(0.1e-15 / W.TIME_UNIT_S / w.dt))
    e, p, g = gpu_uniform_b(tables, w, prec, pairs=True, drain=False, steps=steps)
    led = qed.read_ledger([e, p, g])
    L = oracle_test3_ledger(orc_tables, w, steps)
    # same inputs and random streams as the oracle: FP64 follows it event for event; the FP32
    # trajectories drift after events, so the mixed path agrees to its statistical error
    tol = (1e-9, 1e-9, 1e-9) if prec == qed.FP64 else (0.01, 0.01, 0.05)
    for k, t in zip((0, 2, 1), tol):
        assert led["energy"][k] == pytest.approx(L["energy"][k], rel=t)
        if prec == qed.FP64:
            assert led["n"][k] == L["n"][k]
    # and the paper's table, within the statistical error of 1e4 electrons
    ref = golden["delta_energy_1"]["test3"]
    assert led["energy"][0] / n == pytest.approx(ref["electron"], rel=0.02)
    assert led["energy"][2] / n == pytest.approx(ref["photon"], rel=0.02)
    assert led["energy"][1] / n == pytest.approx(ref["positron"], rel=0.08)


def test_rotating_e_against_oracle(tables, orc_tables):
    # the rotating-field workload at small size, every photon kept, pairs on: FP64 follows the
    # oracle event for event (same Philox streams); the kept photons come out in the same order
    w = W.rotating_e(n=64, n_steps=1500, seed=3)
    f = w.field
    oe = o.Species(100_000)
    oe.set(w.x, w.u)
    oe.init_tau(o.ELECTRON, w.seed)
    op, og = o.Species(100_000), o.Species(400_000)
    osp = o.StepParams(dt=w.dt, seed=w.seed, make_pairs=True,
                       field=o.Field(kind=f.kind, E0=f.E0, omega=f.omega, phase0=f.phase0))
    for k in range(w.n_steps):
        L = o.step(orc_tables, osp, k, oe, op, og)
    for prec in (qed.FP64, qed.MIXED):
        e = qed.Species(qed.ELECTRON, prec, 100_000, 100_000)
        p = qed.Species(qed.POSITRON, prec, 100_000, 100_000)
        g = qed.Species(qed.PHOTON, prec, 400_000, 200_000)
        e.upload(w.x, w.u)
        e.init_tau(w.seed)
        qp = qed.StepParams(dt=w.dt, seed=w.seed, field=qed.Field(**f.as_dict()), make_pairs=True)
        qed.run(tables, [e, p, g], qp, 0, w.n_steps // 2)
        g.compact()
        qed.run(tables, [e, p, g], qp, w.n_steps // 2, w.n_steps - w.n_steps // 2)
        qed.check([e, p, g])
        led = qed.read_ledger([e, p, g])
        if prec == qed.FP64:
            assert led["n"] == L["n"]
            for k in range(3):
                assert led["energy"][k] == pytest.approx(L["energy"][k], rel=1e-9)
            d = g.download()
            assert np.array_equal(d["id"], og.get("id"))
            assert np.allclose(d["u"], og.u(), rtol=1e-9, atol=1e-9 * np.abs(og.u()).max())
        else:
            # FP32 trajectories: same statistics (photon number per electron within 5%)
            assert led["n"][2] == pytest.approx(L["n"][2], rel=0.05)
            assert led["energy"][0] == pytest.approx(L["energy"][0], rel=0.05)


@pytest.mark.parametrize("prec", [qed.FP64, qed.MIXED])
def test_problem2_against_oracle(tables, orc_tables, prec):
    # test problem 2 (CP wave, gamma0 = 4120, eta0 = 1) to t0 = 3 fs with photons kept and pairs on
    w = W.cp_head_on(n=5000)
    f = w.field
    oe = o.Species(40_000)
    oe.set(w.x, w.u)
    oe.init_tau(o.ELECTRON, w.seed)
    op, og = o.Species(40_000), o.Species(400_000)
    osp = o.StepParams(dt=w.dt, seed=w.seed, make_pairs=True, field=o.Field(kind=f.kind, E0=f.E0, omega=f.omega))
    for k in range(w.n_steps):
        L = o.step(orc_tables, osp, k, oe, op, og)
    e = qed.Species(qed.ELECTRON, prec, 40_000, 40_000)
    p = qed.Species(qed.POSITRON, prec, 40_000, 40_000)
    g = qed.Species(qed.PHOTON, prec, 400_000, 80_000)
    e.upload(w.x, w.u)
    e.init_tau(w.seed)
    qed.run(tables, [e, p, g], qed.StepParams(dt=w.dt, seed=w.seed, field=qed.Field(**f.as_dict())), 0, w.n_steps)
    qed.check([e, p, g])
    led = qed.read_ledger([e, p, g])
    if prec == qed.FP64:
        assert led["n"] == L["n"]
        for k in range(3):
            assert led["energy"][k] == pytest.approx(L["energy"][k], rel=1e-9, abs=1e-9 * L["energy"][0])
        d = e.download()
        assert np.allclose(d["u"], oe.u(), rtol=1e-9, atol=1e-9 * np.abs(oe.u()).max())
    else:
        assert led["energy"][0] == pytest.approx(L["energy"][0], rel=0.01)
        assert led["energy"][2] == pytest.approx(L["energy"][2], rel=0.01)
        assert led["n"][2] == pytest.approx(L["n"][2], rel=0.01)


def head_on_gpu_and_oracle(tables, n, n_steps, kw):
    """A head-on workload on the GPU (mixed precision, all steps) and an independent FP64 oracle
    sample of it (another draw of the electrons, other streams, eight chunks in parallel): the
    final energies of electrons, positrons and unconverted photons on each side."""
    import multiprocessing as mp

    import oracle_jobs

    w = W.head_on(n=n, n_steps=n_steps, seed=2, **kw)
    e = qed.Species(qed.ELECTRON, qed.MIXED, 8 * n + 64, 8 * n + 64)
    p = qed.Species(qed.POSITRON, qed.MIXED, 8 * n + 64, 8 * n + 64)
    g = qed.Species(qed.PHOTON, qed.MIXED, 1000 * n + 64, 16 * n + 64)
    xr = w.x.copy()
    xr[:, 0] -= w.window_x0
    e.upload(xr, w.u)
    e.init_tau(w.seed)
    qp = qed.StepParams(dt=w.dt, seed=w.seed, field=qed.Field(**w.field.as_dict()), window_x0=w.window_x0,
                        window_v=w.window_v)
    qed.run_multistep(tables, [e, p, g], qp, 0, w.n_steps, 64)
    qed.check([e, p, g])
    gd = g.download()
    alive = np.isfinite(gd["tau"])
    gpu = [np.sqrt(1 + np.sum(e.download()["u"].astype(np.float64) ** 2, axis=1)),
           np.sqrt(1 + np.sum(p.download()["u"].astype(np.float64) ** 2, axis=1)),
           np.linalg.norm(gd["u"][alive].astype(np.float64), axis=1)]
    chunks = [(n, k * n // 8, (k + 1) * n // 8, 7, w.n_steps, kw) for k in range(8)]
    with mp.get_context("spawn").Pool(8) as pool:
        parts = pool.map(oracle_jobs.head_on_chunk, chunks, chunksize=1)
    orc = [np.concatenate([q[c] for q in parts]) for c in range(3)]
    # the spread of a species' number over independent electron samples: from the eight chunks
    # (emission and pair numbers per electron are over-dispersed: cascades, energy-dependent
    # rates), scaled to the whole sample
    spread = [float(np.std([len(q[c]) for q in parts], ddof=1) * math.sqrt(len(parts))) for c in range(3)]
    return gpu, orc, spread


def same_distribution(stats, a, b, name, spread, min_count=500):
    """Two-sample KS (p > 0.01), mean energies within 3 sigma, numbers within 4 sigma of the
    difference of two independent samples (each with the spread the oracle's chunks show)."""
    assert len(a) > min_count and len(b) > min_count, (name, len(a), len(b))
    assert stats.ks_2samp(a, b).pvalue > 0.01, f"{name} spectrum"
    sig = math.sqrt(a.var() / len(a) + b.var() / len(b))
    assert abs(a.mean() - b.mean()) < 3 * sig, f"{name} mean energy"
    sig_n = math.sqrt(2.0) * max(spread, math.sqrt(len(b)))
    assert abs(len(a) - len(b)) < 4 * sig_n, f"{name} number: {len(a)} vs {len(b)} (sigma {sig_n:.0f})"


def test_head_on_spectra_ks_photons(tables, orc_tables):
    # the benchmark's head-on collision (a0 = 100, gamma0 = 2000, 30 fs, all 4000 steps) on 1e4
    # electrons: photon and electron spectra, GPU mixed precision against the FP64 oracle (its
    # pairs are too few there for a spectrum: about one per thousand electrons)
    stats = pytest.importorskip("scipy.stats")
    gpu, orc, spread = head_on_gpu_and_oracle(tables, 10000, 4000, {})
    same_distribution(stats, gpu[2], orc[2], "photon", spread[2])
    assert stats.ks_2samp(gpu[0], orc[0]).pvalue > 0.01  # electrons (initial and from pairs)


def test_head_on_spectra_ks_positrons_pair_rich(tables, orc_tables):
    # positrons where pairs are plentiful: the scan's strong corner (a0 = 400, gamma0 = 4000,
    # 30 fs), 2000 electrons through the whole collision
    stats = pytest.importorskip("scipy.stats")
    gpu, orc, spread = head_on_gpu_and_oracle(tables, 2000, 2400, {"a0": 400.0, "gamma_mean": 4000.0})
    same_distribution(stats, gpu[1], orc[1], "positron", spread[1])
    same_distribution(stats, gpu[2], orc[2], "photon", spread[2])
