"""Macroparticle weights and photon merging on the GPU against the oracle: the same groups, the
same survivors and (FP64) the same numbers; weights inherited by children; physical totals kept
by merging; checkpoints carry the weights; a cascade with merging stays bounded."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle as o  # noqa: E402
from paper_1311_5551_gb300 import build as qbuild  # noqa: E402
from paper_1311_5551_gb300 import qed, workloads as W  # noqa: E402

from test_oracle_merge import GRID, clustered  # noqa: E402


@pytest.fixture(scope="module")
def tables():
    qbuild.build()
    return qed.Tables()


def photon_inputs(seed, n_groups=40, f32=False):
    rng = np.random.default_rng(seed)
    x, k = clustered(rng, n_groups=n_groups, per=(2, 14))
    # sprinkle lone photons, photons outside the grid and a few identical copies
    x = np.concatenate([x, rng.uniform(-20, 60, (30, 3))])
    k = np.concatenate([k, rng.normal(size=(30, 3)) * 100])
    w = rng.uniform(0.5, 4.0, len(x))
    tau = rng.uniform(0.1, 3.0, len(x))
    if f32:
        x, k, w, tau = (a.astype(np.float32).astype(np.float64) for a in (x, k, w, tau))
    return x, k, w, tau


@pytest.mark.parametrize("prec", [qed.FP64, qed.MIXED])
def test_merge_matches_oracle(tables, prec):
    x, k, w, tau = photon_inputs(5, f32=prec == qed.MIXED)
    n = len(x)
    ids = np.arange(1000, 1000 + n, dtype=np.uint32)
    ref = o.Species(n + 4)
    ref.set(x, k, tau=tau, ids=ids, w=w)
    g_ref = ref.merge(**GRID, n_face=8, n_sub=4, min_group=3)
    g = qed.Species(qed.PHOTON, prec, n + 16, 16)
    g.upload(x, k, tau=tau, ids=ids, next_id=5000)
    g.set_weights(w)
    W0 = g.totals()
    got = g.merge(**GRID, n_face=8, n_sub=4, min_group=3)
    assert got == g_ref and got > 10
    d = g.download()
    assert np.array_equal(d["id"], ref.get("id"))
    if prec == qed.FP64:
        assert np.array_equal(d["x"], ref.x()) and np.array_equal(d["u"], ref.u())
        assert np.array_equal(g.weights(), ref.get("w")) and np.array_equal(d["tau"], ref.get("tau"))
    else:
        np.testing.assert_allclose(d["x"], ref.x(), rtol=1e-6, atol=1e-5)
        np.testing.assert_allclose(d["u"], ref.u(), rtol=1e-6, atol=1e-6 * np.abs(ref.u()).max())
        np.testing.assert_allclose(g.weights(), ref.get("w"), rtol=1e-6)
    W1 = g.totals()
    assert W1[0] == pytest.approx(W0[0], rel=1e-12 if prec == qed.FP64 else 1e-6)
    assert W1[1] == pytest.approx(W0[1], rel=1e-12 if prec == qed.FP64 else 1e-6)


def test_lepton_merge_matches_oracle(tables):
    x, k, w, tau = photon_inputs(8)
    k = k * 0.5
    n = len(x)
    ids = np.arange(n, dtype=np.uint32)
    ref = o.Species(n + 4)
    ref.set(x, k, tau=tau, ids=ids, w=w)
    g_ref = ref.merge(**GRID, n_face=8, n_sub=4, min_group=3, photon=False)
    e = qed.Species(qed.ELECTRON, qed.FP64, n + 16, 16)
    e.upload(x, k, tau=tau, ids=ids, next_id=n)
    e.set_weights(w)
    assert e.merge(**GRID, n_face=8, n_sub=4, min_group=3) == g_ref > 10
    d = e.download()
    assert np.array_equal(d["id"], ref.get("id")) and np.array_equal(d["u"], ref.u())
    assert np.array_equal(d["x"], ref.x()) and np.array_equal(e.weights(), ref.get("w"))
    gam = np.sqrt(1 + np.sum(d["u"] ** 2, axis=1))
    assert np.all(np.isfinite(gam))


def test_children_inherit_weight_and_checkpoint_keeps_it(tables, orc_tables):
    w = W.uniform_b(n=300, cB=9e-3, seed=3)
    e = qed.Species(qed.ELECTRON, qed.FP64, 2000, 2000)
    p = qed.Species(qed.POSITRON, qed.FP64, 2000, 2000)
    g = qed.Species(qed.PHOTON, qed.FP64, 4000, 2000)
    e.upload(w.x, w.u)
    e.set_weights(np.linspace(1.0, 4.0, 300))
    e.init_tau(3)
    qed.run(tables, [e, p, g], qed.StepParams(dt=w.dt * 20, seed=3, field=qed.Field(B=w.field.B), make_pairs=False),
            0, 2)
    # the oracle, event for event
    oe = o.Species(2000)
    oe.set(w.x, w.u, w=np.linspace(1.0, 4.0, 300))
    oe.init_tau(o.ELECTRON, 3)
    op, og = o.Species(2000), o.Species(4000)
    osp = o.StepParams(dt=w.dt * 20, seed=3, field=o.Field(B=w.field.B), make_pairs=False)
    for k in range(2):
        o.step(orc_tables, osp, k, oe, op, og)
    assert g.count() == og.n > 10
    assert np.array_equal(g.weights(), og.get("w"))
    buf = g.save()
    g2 = qed.Species(qed.PHOTON, qed.FP64, 4000, 2000)
    g2.restore(buf)
    assert np.array_equal(g2.weights(), g.weights())


def test_cascade_with_merging_stays_bounded(tables):
    # the rotating-field workload with the photons merged every 200 steps: the photon number stays
    # far below the unmerged run while the photons' weight, energy and momentum are what the
    # merges received
    prec = qed.MIXED
    w = W.rotating_e(n=2000, n_steps=1200, seed=3)
    f = w.field

    def fresh():
        sp = [qed.Species(qed.ELECTRON, prec, 20000, 20000), qed.Species(qed.POSITRON, prec, 20000, 20000),
              qed.Species(qed.PHOTON, prec, 400000, 40000)]
        sp[0].upload(w.x, w.u)
        sp[0].init_tau(w.seed)
        return sp, qed.StepParams(dt=w.dt, seed=w.seed, field=qed.Field(**f.as_dict()))

    sp, p = fresh()
    qed.run(tables, sp, p, 0, w.n_steps)
    n_plain = sp[2].count()
    sp, p = fresh()
    span = 2e7  # the photons stay within a few micrometres over the run
    for s0 in range(0, w.n_steps, 200):
        qed.run(tables, sp, p, s0, 200)
        before = sp[2].totals()
        sp[2].merge(origin=(-span,) * 3, cell=(span / 4,) * 3, n_cells=(8, 8, 8), n_face=6, n_sub=2, min_group=4)
        after = sp[2].totals()
        assert after[0] == pytest.approx(before[0], rel=1e-5)
        assert after[1] == pytest.approx(before[1], rel=1e-5)
        assert np.allclose(after[2], before[2], rtol=1e-4, atol=1e-5 * before[1])
    qed.check(sp)
    assert sp[2].count() < 0.5 * n_plain
    assert n_plain > 10000


def test_merge_scratch_comes_from_the_callers_allocator(tables):
    # the library allocates nothing on its own behalf: the merge's sort scratch (12 bytes per
    # photon, the count rounded up to a power of two, plus 256) and the weight arrays it needs
    # come from the allocator the species was created with; the scratch is given back before
    # the call returns, everything else when the species is freed
    log, live, freed = [], {}, []

    def on_alloc(ptr, nbytes):
        log.append((ptr, nbytes))
        live[ptr] = nbytes

    def on_free(ptr, nbytes):
        assert live.pop(ptr) == nbytes
        freed.append((ptr, nbytes))

    alloc = qed.torch_allocator(on_alloc, on_free)
    x, k, w, tau = photon_inputs(8, n_groups=300)
    n = len(x)
    g = qed.Species(qed.PHOTON, qed.FP64, n + 16, 16, allocator=alloc)
    g.upload(x, k, tau=tau)
    assert len(log) == 1 and len(live) == 1  # the species' own block only (no weight arrays yet)
    got = g.merge(**GRID, n_face=8, n_sub=4, min_group=3)
    assert got > 10
    scratch = 12 * (1 << (n - 1).bit_length()) + 256
    during = log[1:]
    assert [b for _, b in during].count(scratch) == 1, during
    ptr = next(p for p, b in during if b == scratch)
    assert freed == [(ptr, scratch)], "the merge releases its sort scratch, and nothing else"
    assert len(live) == len(log) - 1  # weights and the compaction's second set stay with the species
    g.close()
    assert not live, "every block is given back when the species is freed"
