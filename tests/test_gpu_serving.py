"""Continuous batching on the GPU: scenarios join a running batch between rounds, into slots that
other scenarios have left, and each one's particles and ledger are exactly those it gets alone
(qed_run).  Both the batch API driven by hand and the serving loop are checked."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1311_5551_gb300 import build as qbuild  # noqa: E402
from paper_1311_5551_gb300 import qed, serving, workloads as W  # noqa: E402


@pytest.fixture(scope="module")
def tables():
    qbuild.build()
    return qed.Tables()


# (electrons, a0, gamma0, steps): uneven sizes, fields and lengths
REQS = [(1500, 300.0, 3000.0, 60), (37, 150.0, 2500.0, 45), (5000, 450.0, 3500.0, 80), (1, 200.0, 1000.0, 30),
        (2600, 80.0, 400.0, 70), (900, 400.0, 3900.0, 50)]


def request(k, prec):
    n, a0, g0, steps = REQS[k]
    w = W.head_on(n=n, a0=a0, gamma_mean=g0, n_steps=steps, meet_step=steps // 2, fwhm_s=10e-15, seed=5,
                  rng=np.random.default_rng([5, k]))
    sp = serving.make_species(qed, w, prec)
    xr = w.x.copy()
    xr[:, 0] -= w.window_x0
    sp[0].upload(xr, w.u)
    sp[0].init_tau(w.seed, k)
    p = qed.StepParams(dt=w.dt, seed=w.seed, scenario=k, field=qed.Field(**w.field.as_dict()),
                       window_x0=w.window_x0, window_v=w.window_v)
    return w, sp, p


def alone(tables, k, prec):
    w, sp, p = request(k, prec)
    qed.run(tables, sp, p, 0, w.n_steps)
    return [s.save() for s in sp], qed.read_ledger(sp)


@pytest.mark.parametrize("prec", [qed.MIXED, qed.FP64])
def test_requests_join_a_running_batch(tables, prec):
    # three slots; requests 0-2 start together, 3 joins after one round while 0-2 run, 4 and 5
    # take the slots that finished requests leave; every batch step is a graph replay or a
    # direct launch alike
    b = qed.Batch(tables, prec, 3)
    b.config(0, 8)  # default grid (one wave of the step kernel), 8-step graphs
    live, done, started_while_running = {}, {}, []
    queue = list(range(len(REQS)))
    rounds = 0
    while queue or live:
        free = [s for s in range(3) if s not in live]
        while free and queue:
            k = queue.pop(0)
            w, sp, p = request(k, prec)
            slot = free.pop(0)
            if live:
                started_while_running.append(k)
            b.attach(slot, sp, p, 0, w.n_steps)
            live[slot] = (k, sp)
        b.run(7 if rounds % 2 == 0 else 11)
        rounds += 1
        left = b.remaining()
        for slot in list(live):
            if left[slot] == 0:
                k, sp = live.pop(slot)
                done[k] = ([s.save() for s in sp], qed.read_ledger(sp))
                b.detach(slot)
    assert started_while_running, "some request joined while others were on the GPU"
    assert sorted(done) == list(range(len(REQS)))
    for k in range(len(REQS)):
        ref, ref_led = alone(tables, k, prec)
        got, led = done[k]
        for a, c in zip(ref, got):
            assert np.array_equal(a, c), f"request {k}: particles differ from its own run"
        # the batch's persistent grid gives a slot the ledger partials the single path gives it
        for key in ("n", "energy"):
            assert led[key] == ref_led[key], f"request {k}: ledger {key}"
        assert led["emitted_energy"] == ref_led["emitted_energy"]


def test_serving_loop_results_equal_alone(tables):
    # the serving loop itself: requests arriving over time (some while others run), admitted by
    # device-memory budget; each finished request equals its own run
    prec = qed.MIXED
    reqs = []
    for k in range(len(REQS)):
        n, a0, g0, steps = REQS[k]
        w = W.head_on(n=n, a0=a0, gamma_mean=g0, n_steps=steps, meet_step=steps // 2, fwhm_s=10e-15, seed=5,
                      rng=np.random.default_rng([5, k]))
        reqs.append((0.002 * k, w))
    saved = {}
    fin, st = serving.serve(qed, tables, reqs, prec, slots=2, chunk=5, max_wall=120.0,
                            on_finish=lambda r, sp: saved.__setitem__(r.rid, [s.save() for s in sp]))
    assert st["finished"] == len(REQS)
    assert any(r.admitted > min(o.admitted for o in fin if o.rid != r.rid) for r in fin)
    for r in fin:
        ref, ref_led = alone(tables, r.rid, prec)
        for a, c in zip(ref, saved[r.rid]):
            assert np.array_equal(a, c), f"request {r.rid}"
        assert r.result["ledger"]["energy"] == ref_led["energy"]
