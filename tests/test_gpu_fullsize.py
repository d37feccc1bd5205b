"""Parity at the benchmark's full size and launch configuration: the head-on collision of 1e6
electrons over 4000 steps, multi-step runs (64-step stretches) as bench.py times them, on the
FP64 path.  Sampled electrons are recomputed one by one with the oracle (an electron's own
trajectory, emissions and recoils included, depends on nothing but its own state, the field and
its Philox stream), and the whole population is checked for what holds at any size."""
import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle as o  # noqa: E402
from paper_1311_5551_gb300 import build as qbuild  # noqa: E402
from paper_1311_5551_gb300 import qed, workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def full_run():
    qbuild.build()
    tables = qed.Tables()
    w = W.head_on(n=1_000_000, n_steps=4000, seed=2)
    n = w.n
    prec = qed.FP64
    sp = [qed.Species(qed.ELECTRON, prec, 2 * n + 4096, n + 4096), qed.Species(qed.POSITRON, prec, n + 4096, n + 4096),
          qed.Species(qed.PHOTON, prec, 80 * n + 4096, 2 * n + 4096)]
    xr = w.x.copy()
    xr[:, 0] -= w.window_x0
    sp[0].upload(xr, w.u)
    sp[0].init_tau(w.seed)
    p = qed.StepParams(dt=w.dt, seed=w.seed, field=qed.Field(**w.field.as_dict()), window_x0=w.window_x0,
                       window_v=w.window_v)
    qed.run_multistep(tables, sp, p, 0, w.n_steps, chunk=64)
    qed.check(sp)
    out = {"w": w, "e": sp[0].download(), "np": sp[1].count(), "ng": sp[2].count(),
           "work": qed.work_read_split(sp[0]), "gid": sp[2].download()["id"], "pid": sp[1].download()["id"]}
    for s in sp:
        s.close()
    return out


def test_sampled_electrons_match_oracle(full_run, orc_tables):
    w, e = full_run["w"], full_run["e"]
    rng = np.random.default_rng(17)
    sample = np.concatenate([[0, 1, w.n - 1], rng.choice(w.n, 29, replace=False)])
    t_end = w.n_steps * w.dt
    x_window = w.window_x0 + w.window_v * t_end
    fd = o.Field(**w.field.as_dict())
    emitted = 0
    for i in sample:
        s = o.Species(8)
        s.set(w.x[i:i + 1], w.u[i:i + 1], ids=np.array([i], dtype=np.uint32))
        s.init_tau(o.ELECTRON, w.seed)
        p, g, d = o.Species(4), o.Species(4), o.Species(8000)
        spar = o.StepParams(dt=w.dt, seed=w.seed, make_pairs=False, drain_photons=True, field=fd)
        for k in range(w.n_steps):
            o.step(orc_tables, spar, k, s, p, g, d)
        emitted += d.n
        assert e["id"][i] == i
        u_ref, x_ref = s.u()[0], s.x()[0]
        assert np.allclose(e["u"][i], u_ref, rtol=1e-9, atol=1e-9 * np.linalg.norm(u_ref))
        x_gpu = e["x"][i] + np.array([x_window, 0.0, 0.0])
        assert np.allclose(x_gpu, x_ref, rtol=1e-9, atol=1e-6)
        assert e["tau"][i] == pytest.approx(s.get("tau")[0], rel=1e-9, abs=1e-9)
    assert emitted > 10 * len(sample)  # the sampled electrons did emit during the collision


def test_population_properties(full_run):
    w, e = full_run["w"], full_run["e"]
    n_pairs = full_run["np"]
    # every pair adds one electron and one positron; the original electrons keep their slots
    assert len(e["id"]) == w.n + n_pairs
    assert np.array_equal(e["id"][: w.n], np.arange(w.n, dtype=np.uint32))
    # children ids are consecutive in order of creation, unique per species
    assert np.array_equal(e["id"][w.n:], np.arange(w.n, w.n + n_pairs, dtype=np.uint32))
    assert np.array_equal(full_run["pid"], np.arange(n_pairs, dtype=np.uint32))
    gid = full_run["gid"]
    assert len(np.unique(gid)) == len(gid) and full_run["ng"] > 2e7
    lep, ph, created, lep_multi, ph_multi = full_run["work"][:5]
    # every photon made is still held (converted ones as holes: no compaction in this run)
    assert created == full_run["ng"] + 2 * n_pairs and created > 2e7
    assert 0 < lep_multi < lep and 0 < ph_multi < ph
