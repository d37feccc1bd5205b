"""Batches of scenarios (GPU): a scenario's particles are the same alone, in a batch of one and
in a mix of uneven scenarios; its ledger agrees within rounding."""
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


def scenario(n, a0, g0, k, prec, steps=40):
    w = W.head_on(n=n, a0=a0, gamma_mean=g0, n_steps=steps, meet_step=steps // 2, fwhm_s=10e-15, seed=4,
                  rng=np.random.default_rng([4, k]))
    cap = 8 * n + 4096
    sp = [qed.Species(qed.ELECTRON, prec, cap, cap), qed.Species(qed.POSITRON, prec, cap, cap),
          qed.Species(qed.PHOTON, prec, 16 * cap, 2 * cap)]
    xr = w.x.copy()
    xr[:, 0] -= w.window_x0
    sp[0].upload(xr, w.u)
    sp[0].init_tau(w.seed, k)
    params = qed.StepParams(dt=w.dt, seed=w.seed, scenario=k, field=qed.Field(**w.field.as_dict()),
                            window_x0=w.window_x0, window_v=w.window_v)
    return w, sp, params


SIZES = [(1500, 300.0, 3000.0), (37, 150.0, 2500.0), (9000, 450.0, 3500.0), (1, 200.0, 1000.0), (4100, 80.0, 400.0)]


@pytest.mark.parametrize("prec", [qed.MIXED, qed.FP64])
def test_alone_and_in_the_mix(tables, prec):
    steps = 40
    # reference: scenario 0 through the single-scenario path
    w, sp, params = scenario(*SIZES[0], 0, prec, steps)
    qed.run(tables, sp, params, 0, steps)
    ref = [s.save() for s in sp]
    ref_led = qed.read_ledger(sp)
    # alone in a batch of one
    w, sp1, params = scenario(*SIZES[0], 0, prec, steps)
    b1 = qed.Batch(tables, prec, 1)
    b1.attach(0, sp1, params, 0, steps)
    b1.run(steps)
    assert b1.remaining()[0] == 0
    for a, s in zip(ref, sp1):
        assert np.array_equal(a, s.save())
    # in a mix of uneven scenarios, with more batch steps than it needs (it stops on its own)
    bm = qed.Batch(tables, prec, len(SIZES))
    mix = []
    for k, (n, a0, g0) in enumerate(SIZES):
        wk, spk, pk = scenario(n, a0, g0, k, prec, steps)
        bm.attach(k, spk, pk, 0, steps if k == 0 else steps + 7)
        mix.append(spk)
    bm.config(bm_blocks := 2 * 152, 8)
    bm.run(steps + 7)
    assert np.all(bm.remaining() == 0)
    for a, s in zip(ref, mix[0]):
        assert np.array_equal(a, s.save())
    # the ledger's block partials are grouped by the launch shape, which differs between the
    # single path and the batch: counts are exact, energy sums agree to the rounding of the
    # partials (compensated FP32 in the mixed path, FP64 in the FP64 path)
    led = qed.read_ledger(mix[0])
    rel = 1e-9 if prec == qed.MIXED else 1e-12
    for k in range(3):
        assert led["n"][k] == ref_led["n"][k]
        assert led["energy"][k] == pytest.approx(ref_led["energy"][k], rel=rel)
    assert mix[0][2].count() > 0
    qed.check([s for m in mix for s in m])
    del bm_blocks


def test_batch_autotune_and_graph(tables):
    prec = qed.MIXED
    bm = qed.Batch(tables, prec, 3)
    sps = []
    for k in range(3):
        w, sp, p = scenario(2000 * (k + 1), 300.0, 3000.0, k, prec, steps=200)
        bm.attach(k, sp, p, 0, 200)
        sps.append((sp, p))
    tb, gs = bm.tune(trial_steps=2)
    assert tb >= 1 and gs in (0, 8, 32)
    left = bm.remaining()
    bm.run(int(left.max()))
    assert np.all(bm.remaining() == 0)
    # the tuned, graph-replayed batch gives the same particles as the single path
    w, sp, p = scenario(2000, 300.0, 3000.0, 0, prec, steps=200)
    qed.run(tables, sp, p, 0, 200)
    for a, s in zip(sp, sps[0][0]):
        assert np.array_equal(a.save(), s.save())
