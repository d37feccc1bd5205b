"""Host-side checks that need no GPU: the C-ABI library loads and exports every symbol declared in
include/qed.h, the input generators are seeded and shaped like the paper's workloads, and the
multi-rank aggregation of bench.py (gloo, world size 2)."""
import math
import os
import re
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    with open(os.path.join(ROOT, "include", "qed.h")) as f:
        hdr = f.read()
    return sorted(set(re.findall(r"^\s*(?:[\w\s\*]+?)\b(qed_\w+)\s*\(", hdr, re.M)))


def test_library_exports_every_declared_symbol():
    import ctypes

    from paper_1311_5551_gb300 import build

    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_symbols()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_abi():
    from paper_1311_5551_gb300 import qed

    assert set(declared_symbols()) == set(qed.EXPORTS)


def test_missing_library_fails_loudly(tmp_path):
    from paper_1311_5551_gb300 import qed

    saved = qed._lib
    qed._lib = None
    try:
        with pytest.raises(RuntimeError, match="not found"):
            qed.load_library(str(tmp_path / "nope.so"))
    finally:
        qed._lib = saved


def test_workloads_are_seeded_and_shaped():
    from paper_1311_5551_gb300 import workloads as W

    a = W.head_on(n=5000, seed=2)
    b = W.head_on(n=5000, seed=2)
    assert np.array_equal(a.x, b.x) and np.array_equal(a.u, b.u)
    g = np.sqrt(1 + np.sum(a.u**2, axis=1))
    assert abs(g.mean() / 2000 - 1) < 0.01 and abs(g.std() / 100 - 1) < 0.1
    assert np.all(a.u[:, 0] < 0)  # moving against the pulse
    ang = np.abs(a.u[:, 1] / a.u[:, 0])
    assert 0.5e-3 < np.median(ang) < 1e-3
    # a0 = 100 at 1 um: E0 = a0 omega (in units of E_s and m c^2/hbar)
    assert a.field.E0 == pytest.approx(100 * 2 * math.pi * W.LENGTH_UNIT_M / 1e-6)
    # sin^2 field envelope with 30 fs intensity FWHM: 82.5 fs full length
    assert a.field.phi_len / a.field.omega * W.TIME_UNIT_S == pytest.approx(82.5e-15, rel=1e-3)
    u = W.uniform_b(n=10)
    assert np.allclose(np.linalg.norm(u.u, axis=1) * u.field.B[2], 1.0, atol=1e-6)
    s = W.scan(n_scenarios=8, scale=1e-3)
    assert len(s) == 8 and all(w.n >= 1 for w in s)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import sys

    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ms, units = bench.aggregate_ranks(100.0 + 50.0 * rank, 1e6 * (rank + 1), world, "cpu")
    q.put((rank, ms, units))
    dist.destroy_process_group()


def test_bench_rank_aggregation_gloo():
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # slowest rank's time, units summed over the ranks
    assert out == [(0, 150.0, 3e6), (1, 150.0, 3e6)]


def test_serving_scheduler_fifo_budget_and_reuse():
    from paper_1311_5551_gb300.serving import Request, Scheduler, percentiles

    s = Scheduler(slots=2, budget_bytes=100)
    reqs = [Request(k, 0.1 * k, 10, 5, fp) for k, fp in enumerate([40, 50, 30, 20])]
    for r in reqs:
        s.arrive(r)
    got = s.admit(1.0)
    assert [r.rid for r in got] == [0, 1] and s.in_use == 90  # both slots taken
    assert s.admit(1.1) == []
    s.complete(got[0].slot, 2.0)  # frees 40: request 2 (30) fits, request 3 waits (FIFO)
    got2 = s.admit(2.0)
    assert [r.rid for r in got2] == [2] and s.in_use == 80
    s.complete(got[1].slot, 3.0)
    got3 = s.admit(3.0)
    assert [r.rid for r in got3] == [3] and s.in_use <= 100
    s.complete(got2[0].slot, 4.0)
    s.complete(got3[0].slot, 5.0)
    assert s.idle() and s.in_use == 0
    lat = sorted(r.latency for r in s.finished)
    assert lat == pytest.approx([2.0, 2.9, 3.8, 4.7])
    p50, p99 = percentiles(lat)
    assert 2.9 <= p50 <= 3.8 and p99 <= 4.7
    with pytest.raises(ValueError):
        big = Scheduler(slots=1, budget_bytes=10)
        big.arrive(Request(9, 0.0, 1, 1, 11))
        big.admit(0.0)


def test_serving_cancellation_frees_slot_and_budget():
    # a request withdrawn mid-flight gives its slot and memory back; a queued one leaves the queue
    from paper_1311_5551_gb300.serving import Request, Scheduler

    s = Scheduler(slots=2, budget_bytes=100)
    for k in range(4):
        s.arrive(Request(k, 0.0, 10, 100, 40))
    started = s.admit(0.0)
    assert [r.rid for r in started] == [0, 1] and s.in_use == 80
    assert s.cancel(1, 0.5).rid == 1 and s.in_use == 40 and 1 not in [r.rid for r in s.running.values()]
    assert s.cancel(3, 0.6).rid == 3 and [r.rid for r in s.pending] == [2]
    assert s.cancel(7, 0.7) is None
    assert [r.rid for r in s.admit(0.8)] == [2] and s.in_use == 80
    assert sorted(r.rid for r in s.cancelled) == [1, 3]
    done = s.complete(next(iter(s.running)), 1.0)
    assert done.rid in (0, 2) and s.in_use == 40
    assert s.cancel(done.rid, 1.1) is None  # already finished


def test_status_codes_match_the_header():
    import re

    from paper_1311_5551_gb300 import qed

    hdr = open(os.path.join(ROOT, "include", "qed.h")).read()
    body = re.search(r"typedef enum \{(.*?)\} qed_status;", hdr, re.S).group(1)
    codes = {name: int(v) for name, v in re.findall(r"(QED_\w+)\s*=\s*(\d+)", body)}
    names = sorted(codes, key=codes.get)
    assert [codes[n] for n in names] == list(range(len(names)))
    assert names == [qed.STATUS[k] for k in range(len(names))]
    assert qed.QED_ERR_OOM == names.index("QED_ERR_OOM") and qed.QED_ERR_TIMEOUT == names.index("QED_ERR_TIMEOUT")


def test_bench_energy_error_aggregation():
    import bench

    assert bench.energy_errors([]) is None
    pairs = [([1.0, 2.0, 0.0], [1.0, 2.002, 0.0]), ([1.01, 4.0, 3.0], [1.0, 4.0, 3.0])]
    e = bench.energy_errors(pairs)
    assert e["results"] == 2
    assert e["max_per_result"][0] == pytest.approx(0.01) and e["max_per_result"][1] == pytest.approx(0.001, rel=1e-3)
    assert e["ensemble"][0] == pytest.approx(0.01 / 2) and e["ensemble"][1] == pytest.approx(0.002 / 6.002)
    assert e["ensemble"][2] == 0.0 and e["max_per_result"][2] == 0.0
    assert bench.energy_errors([([0.5, 1.0, 1.0], [0.0, 1.0, 1.0])])["max_per_result"][0] == 0.5


def test_noalloc_binding_refuses_bad_arrays():
    # the allocation-free entry point sees raw pointers only: the binding must refuse every array
    # that would let the kernels read or write past the caller's tensors
    torch = pytest.importorskip("torch")
    from paper_1311_5551_gb300 import qed

    keys = ("x", "y", "z", "ux", "uy", "uz", "tau", "id")

    def arrays(n, real=torch.float64):
        a = {k: torch.zeros(n, dtype=real) for k in keys[:6]}
        a["tau"] = torch.zeros(n, dtype=torch.float64)
        a["id"] = torch.zeros(n, dtype=torch.int32)
        return a

    ok = lambda prec, e, n, p, c: qed.noalloc_arg_errors(prec, e, n, p, c, require_cuda=False)
    cnt = torch.zeros(3, dtype=torch.int32)
    assert ok(qed.FP64, arrays(100), 100, arrays(50), cnt) == []
    assert ok(qed.MIXED, arrays(100, torch.float32), 100, arrays(50, torch.float32), cnt) == []
    # an electron array shorter than n
    e = arrays(100)
    e["uy"] = torch.zeros(99, dtype=torch.float64)
    assert any("electrons[uy]" in m for m in ok(qed.FP64, e, 100, arrays(50), cnt))
    # a photon array shorter than the capacity that photons["x"] implies
    p = arrays(50)
    p["tau"] = torch.zeros(49, dtype=torch.float64)
    assert any("photons[tau]" in m for m in ok(qed.FP64, arrays(100), 100, p, cnt))
    p = arrays(50)
    p["id"] = torch.zeros(10, dtype=torch.int32)
    assert any("photons[id]" in m for m in ok(qed.FP64, arrays(100), 100, p, cnt))
    # float32 coordinates for the FP64 path, float64 for the mixed path
    assert ok(qed.FP64, arrays(100, torch.float32), 100, arrays(50), cnt)
    assert ok(qed.MIXED, arrays(100), 100, arrays(50, torch.float32), cnt)
    # 8-byte ids, 4-byte tau
    e = arrays(100)
    e["id"] = torch.zeros(100, dtype=torch.int64)
    assert any("electrons[id]" in m for m in ok(qed.FP64, e, 100, arrays(50), cnt))
    e = arrays(100)
    e["tau"] = torch.zeros(100, dtype=torch.float32)
    assert any("electrons[tau]" in m for m in ok(qed.FP64, e, 100, arrays(50), cnt))
    # a counter with fewer than 3 four-byte words, or of 8-byte words
    assert ok(qed.FP64, arrays(100), 100, arrays(50), torch.zeros(2, dtype=torch.int32))
    assert ok(qed.FP64, arrays(100), 100, arrays(50), torch.zeros(3, dtype=torch.int64))
    # non-contiguous, missing
    e = arrays(100)
    e["x"] = torch.zeros(200, dtype=torch.float64)[::2]
    assert any("contiguous" in m for m in ok(qed.FP64, e, 100, arrays(50), cnt))
    e = arrays(100)
    del e["z"]
    assert any("electrons[z] is missing" in m for m in ok(qed.FP64, e, 100, arrays(50), cnt))
    # host tensors are refused when CUDA tensors are required
    errs = qed.noalloc_arg_errors(qed.FP64, arrays(100), 100, arrays(50), cnt)
    assert any("current CUDA device" in m for m in errs)
    with pytest.raises(ValueError):
        qed.step_emit_noalloc(None, qed.FP64, arrays(100), 100, arrays(50), cnt, qed.StepParams(dt=1.0), 0)


def _reference_line(env_extra):
    import json
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--ref-sample", "4", "--cpu-cores", "2", "--time-steps", "150"],
                       capture_output=True, text=True, env=env, cwd=root, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    return [json.loads(ln) for ln in lines]


def test_reference_arm_line_on_host_cores():
    # the oracle timed on the host cores, one spawned process per core, one JSON line
    (out,) = _reference_line({"RANK": "0", "WORLD_SIZE": "1"})
    assert out["impl"] == "reference" and out["value"] > 0 and out["unit"] == "particle-steps/s"
    assert out["cpu_baseline"]["cores"] == min(2, os.cpu_count() or 1)
    assert out["cpu_baseline"]["kind"] == "oracle" and out["cpu_baseline"]["value"] == out["value"]
    assert out["e2e"] == {"value": out["value"], "unit": out["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    # under torchrun rank 0 alone runs and prints the reference line
    assert _reference_line({"RANK": "1", "WORLD_SIZE": "2"}) == []


def test_scan_recipe_ranges_and_laws():
    # the batched scan: 256 head-on scenarios, particle counts log-uniform in [1e3, 1e6] (times the
    # scale), a0 uniform in [10, 500], gamma0 in [200, 4000], pulse FWHM in [15, 60] fs; a subset
    # (`only`) draws the same scenarios as the whole scan
    from scipy import stats

    from paper_1311_5551_gb300 import workloads as W

    ws = W.scan(n_scenarios=256, scale=1e-2, n_steps=10)
    a0 = np.array([w.extra["a0"] for w in ws])
    g0 = np.array([w.extra["gamma_mean"] for w in ws])
    fw = np.array([w.extra["fwhm_s"] for w in ws])
    n = np.array([w.n for w in ws], dtype=np.float64)
    assert a0.min() >= 10 and a0.max() <= 500 and stats.kstest((a0 - 10) / 490, "uniform").pvalue > 0.01
    assert g0.min() >= 200 and g0.max() <= 4000 and stats.kstest((g0 - 200) / 3800, "uniform").pvalue > 0.01
    assert fw.min() >= 15e-15 and fw.max() <= 60e-15 and stats.kstest((fw - 15e-15) / 45e-15, "uniform").pvalue > 0.01
    assert n.min() >= 10 - 1 and n.max() <= 1e4 + 1
    assert stats.kstest((np.log(n) - math.log(10)) / math.log(1000), "uniform").pvalue > 0.01
    assert [w.extra["scenario"] for w in ws] == list(range(256))
    sub = W.scan(n_scenarios=256, scale=1e-2, n_steps=10, only=[7, 3])
    for w, k in zip(sub, (7, 3)):
        assert w.extra["scenario"] == k and np.array_equal(w.x, ws[k].x) and np.array_equal(w.u, ws[k].u)


def test_request_stream_recipe():
    # the serving stream: Poisson arrivals at 200 requests/s over 60 s, particle counts
    # log-uniform in [1e3, 2e6], a0 uniform in [10, 500], gamma0 in [200, 4000], 2000-8000 steps
    from scipy import stats

    from paper_1311_5551_gb300 import workloads as W

    reqs = W.request_specs(rate_hz=200.0, duration_s=60.0)
    t = np.array([r[0] for r in reqs])
    assert abs(len(reqs) - 12000) < 4 * math.sqrt(12000)
    assert np.all(np.diff(t) > 0) and t[-1] <= 60.0
    assert stats.kstest(np.diff(t) * 200.0, "expon").pvalue > 0.01
    n = np.array([r[1].n for r in reqs], dtype=np.float64)
    steps = np.array([r[1].n_steps for r in reqs])
    a0 = np.array([r[1].a0 for r in reqs])
    g0 = np.array([r[1].gamma0 for r in reqs])
    assert n.min() >= 1e3 - 1 and n.max() <= 2e6 + 1
    assert stats.kstest((np.log(n) - math.log(1e3)) / math.log(2e3), "uniform").pvalue > 0.01
    assert steps.min() >= 2000 and steps.max() <= 8000
    assert a0.min() >= 10 and a0.max() <= 500 and g0.min() >= 200 and g0.max() <= 4000
    # a request is built only when asked for, and the same request is built the same way twice
    w1, w2 = reqs[5][1].workload(), reqs[5][1].workload()
    assert w1.n == reqs[5][1].n and np.array_equal(w1.x, w2.x) and w1.extra["scenario"] == 5


def test_rotating_field_recipe():
    # the cascade: 1e4 electrons at rest in E = 1e-3 E_s rotating at the frequency of
    # lambda = 0.8 um, B = 0, dt = lambda / (200 c)
    from paper_1311_5551_gb300 import workloads as W

    w = W.rotating_e()
    assert w.n == 10_000 and np.all(w.u == 0.0)
    assert w.field.E0 == 1e-3 and np.allclose(w.field.B, 0.0)
    period = 2 * math.pi / w.field.omega  # lambda / c in the time unit
    assert w.dt == pytest.approx(period / 200.0, rel=1e-12)
    assert w.field.omega == pytest.approx(2 * math.pi * 299792458.0 / 0.8e-6 * W.TIME_UNIT_S, rel=1e-9)
