"""Multi-step runs (GPU): event-free stretches taken in one pass over the particles give the same
particles, counts and work as the per-step path; the ledger's energies agree to the rounding of
their block partials."""
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


def head_on_species(prec, n=3000, steps=1200, a0=150.0, seed=9):
    # an 8 fs pulse crosses the bunch in ~330 steps around the meeting step: the steps well before
    # and after it have no events
    w = W.head_on(n=n, a0=a0, gamma_mean=2500.0, n_steps=steps, meet_step=steps // 2, fwhm_s=8e-15, seed=seed,
                  rng=np.random.default_rng(seed))
    cap = 30 * n + 4096
    sp = [qed.Species(qed.ELECTRON, prec, cap, cap), qed.Species(qed.POSITRON, prec, cap, cap),
          qed.Species(qed.PHOTON, prec, 40 * cap, 2 * cap)]
    xr = w.x.copy()
    xr[:, 0] -= w.window_x0
    sp[0].upload(xr, w.u)
    sp[0].init_tau(w.seed)
    p = qed.StepParams(dt=w.dt, seed=w.seed, field=qed.Field(**w.field.as_dict()), window_x0=w.window_x0,
                       window_v=w.window_v)
    return w, sp, p


def compare(ref, got, prec):
    for a, b in zip(ref, got):
        assert np.array_equal(a.save(), b.save())
    la, lb = qed.read_ledger(ref), qed.read_ledger(got)
    assert la["n"] == lb["n"]
    for k in range(3):
        assert lb["energy"][k] == pytest.approx(la["energy"][k], rel=1e-9 if prec == qed.MIXED else 1e-12)


@pytest.mark.parametrize("prec", [qed.MIXED, qed.FP64])
@pytest.mark.parametrize("chunk", [2, 7, 32, 64])
def test_head_on_multistep_matches_per_step(tables, prec, chunk):
    w, ref, p = head_on_species(prec)
    qed.run(tables, ref, p, 0, w.n_steps)
    qed.check(ref)
    wr = qed.work_read(ref[0], reset=True)
    w, got, p = head_on_species(prec)
    qed.run_multistep(tables, got, p, 0, w.n_steps, chunk=chunk)
    qed.check(got)
    wg = qed.work_read_split(got[0], reset=True)
    assert wg[:3] == wr
    # the stretches before and after the collision were taken in multi-step passes
    assert wg[3] + wg[4] > 0.25 * (wg[0] + wg[1])
    assert ref[2].count() > 1000  # the collision made photons
    compare(ref, got, prec)


def test_multistep_resumes_mid_run(tables):
    # multi-step from a step index other than 0, after per-step steps, on the same species
    prec = qed.MIXED
    w, ref, p = head_on_species(prec)
    qed.run(tables, ref, p, 0, w.n_steps)
    w, got, p = head_on_species(prec)
    qed.run(tables, got, p, 0, 37)
    qed.run_multistep(tables, got, p, 37, w.n_steps - 37, chunk=16)
    compare(ref, got, prec)


def test_no_events_runs_entirely_multistep(tables):
    # emission and pairs off: no step has events, every step is taken in multi-step passes
    prec = qed.MIXED
    w = W.uniform_b(n=5000, steps_per_gyro=1000.0, seed=4)
    runs = []
    for multi in (False, True):
        sp = [qed.Species(qed.ELECTRON, prec, 6000, 6000), qed.Species(qed.POSITRON, prec, 16, 16),
              qed.Species(qed.PHOTON, prec, 16, 6000)]
        sp[0].upload(w.x, w.u)
        sp[0].init_tau(w.seed)
        p = qed.StepParams(dt=w.dt, seed=w.seed, field=qed.Field(B=w.field.B), emit_photons=False, make_pairs=False)
        if multi:
            qed.run_multistep(tables, sp, p, 0, 100, chunk=32)
        else:
            qed.run(tables, sp, p, 0, 100)
        runs.append((sp, qed.work_read_split(sp[0], reset=True)))
    (ref, wr), (got, wg) = runs
    assert wg[3] == wg[0] == wr[0] == 100 * 5000
    compare(ref, got, prec)


def test_multistep_grid_field(tables):
    # a grid field (cB_z = 1e-3 on a 16^3 grid) with emission off: the grid-capable multi-step pass
    prec = qed.FP64
    w = W.uniform_b(n=2000, steps_per_gyro=1000.0, seed=6)
    n, spc = 16, 2.0e5
    g = torch.zeros((6, n, n, n), dtype=torch.float64, device="cuda")
    g[5] = 1e-3
    org = (-spc * (n - 1) / 2,) * 3
    fq = qed.Field(kind=qed.FIELD_GRID, grid=g, shape=2, origin=org, spacing=(spc, spc, spc))
    runs = []
    for multi in (False, True):
        sp = [qed.Species(qed.ELECTRON, prec, 3000, 3000), qed.Species(qed.POSITRON, prec, 16, 16),
              qed.Species(qed.PHOTON, prec, 16, 3000)]
        sp[0].upload(w.x, w.u)
        sp[0].init_tau(w.seed)
        p = qed.StepParams(dt=w.dt, seed=w.seed, field=fq, emit_photons=False, make_pairs=False)
        (qed.run_multistep(tables, sp, p, 0, 64, chunk=32) if multi else qed.run(tables, sp, p, 0, 64))
        runs.append(sp)
    compare(runs[0], runs[1], prec)


def test_multistep_rejects_bad_chunk(tables):
    w, sp, p = head_on_species(qed.MIXED, n=100, steps=10)
    with pytest.raises(qed.QedError):
        qed.run_multistep(tables, sp, p, 0, 10, chunk=1)
    with pytest.raises(qed.QedError):
        qed.run_multistep(tables, sp, p, 0, 10, chunk=65)


@pytest.mark.parametrize("graph_steps", [0, 8])
def test_batch_multistep_matches_single_runs(tables, graph_steps):
    # three head-on scenarios of different sizes, steps and meeting times in one batch with
    # multi-step passes: each slot ends with the particles of its own qed_run
    prec = qed.MIXED
    specs = [(2000, 900, 300, 11), (700, 1200, 900, 12), (3500, 600, 450, 13)]

    def make(n, steps, meet, seed, k):
        w = W.head_on(n=n, a0=150.0, gamma_mean=2500.0, n_steps=steps, meet_step=meet, fwhm_s=8e-15, seed=seed,
                      rng=np.random.default_rng(seed))
        cap = 30 * n + 4096
        sp = [qed.Species(qed.ELECTRON, prec, cap, cap), qed.Species(qed.POSITRON, prec, cap, cap),
              qed.Species(qed.PHOTON, prec, 40 * cap, 2 * cap)]
        xr = w.x.copy()
        xr[:, 0] -= w.window_x0
        sp[0].upload(xr, w.u)
        sp[0].init_tau(w.seed, k)
        p = qed.StepParams(dt=w.dt, seed=w.seed, scenario=k, field=qed.Field(**w.field.as_dict()),
                           window_x0=w.window_x0, window_v=w.window_v)
        return w, sp, p

    refs = []
    for k, spec in enumerate(specs):
        w, sp, p = make(*spec, k)
        qed.run(tables, sp, p, 0, w.n_steps)
        refs.append((sp, qed.work_read(sp[0], reset=True)))
    b = qed.Batch(tables, prec, len(specs))
    b.config(2 * 152, graph_steps)
    b.multistep(16)
    mix = []
    for k, spec in enumerate(specs):
        w, sp, p = make(*spec, k)
        b.attach(k, sp, p, 0, w.n_steps)
        mix.append(sp)
    rounds = 0
    while b.remaining().max() > 0:
        b.run(8)
        rounds += 8
        assert rounds < 1300
    assert rounds < 600  # the event-free stretches were taken several steps per batch step
    for (ref, wr), sp in zip(refs, mix):
        qed.check(sp)
        for a_, b_ in zip(ref, sp):
            assert np.array_equal(a_.save(), b_.save())
        ws = qed.work_read_split(sp[0], reset=True)
        assert ws[:3] == wr and ws[3] + ws[4] > 0
        la, lb = qed.read_ledger(ref), qed.read_ledger(sp)
        assert la["n"] == lb["n"]
