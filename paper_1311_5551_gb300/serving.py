"""Continuous batching of collision requests on one GPU.

Requests (one head-on collision each) arrive over time.  A request is admitted into a free slot of
a qed_batch when its device-memory footprint fits the budget; admitted requests advance together,
``chunk`` batch steps per round, and new requests join between rounds while others are running.
A finished request is drained (its ledger is its result), its slot and memory are freed, and its
latency (completion - arrival) is recorded.

``Scheduler`` is the host-side policy (no GPU); ``serve`` drives the GPU through the C ABI.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    arrival: float           # seconds from the start of the run
    n: int                   # electrons
    steps: int
    footprint: int           # device bytes while admitted
    payload: object = None   # the workload
    admitted: float = math.nan
    done: float = math.nan
    slot: int = -1
    result: dict = field(default_factory=dict)

    @property
    def latency(self):
        return self.done - self.arrival


class Scheduler:
    """FIFO admission into free slots under a device-memory budget."""

    def __init__(self, slots: int, budget_bytes: int):
        self.free = list(range(slots))[::-1]
        self.budget = budget_bytes
        self.in_use = 0
        self.pending: collections.deque[Request] = collections.deque()
        self.running: dict[int, Request] = {}
        self.finished: list[Request] = []
        self.cancelled: list[Request] = []

    def arrive(self, r: Request):
        self.pending.append(r)

    def admit(self, now: float) -> list[Request]:
        """Requests to start now, in arrival order; stops at the first that does not fit (FIFO)."""
        out = []
        while self.pending and self.free:
            r = self.pending[0]
            if r.footprint > self.budget:
                raise ValueError(f"request {r.rid} needs {r.footprint} bytes, more than the whole budget")
            if self.in_use + r.footprint > self.budget:
                break
            self.pending.popleft()
            r.slot = self.free.pop()
            r.admitted = now
            self.in_use += r.footprint
            self.running[r.slot] = r
            out.append(r)
        return out

    def complete(self, slot: int, now: float) -> Request:
        r = self.running.pop(slot)
        r.done = now
        self.in_use -= r.footprint
        self.free.append(slot)
        self.finished.append(r)
        return r

    def cancel(self, rid: int, now: float) -> Request | None:
        """Withdraw request rid: a queued one leaves the queue; a running one gives its slot and its
        memory back (the caller detaches the slot).  Returns the request, or None if it is unknown
        or already finished."""
        for r in self.pending:
            if r.rid == rid:
                self.pending.remove(r)
                r.done = now
                self.cancelled.append(r)
                return r
        for slot, r in list(self.running.items()):
            if r.rid == rid:
                self.running.pop(slot)
                self.in_use -= r.footprint
                self.free.append(slot)
                r.done = now
                self.cancelled.append(r)
                return r
        return None

    def idle(self) -> bool:
        return not self.pending and not self.running


def percentiles(lat):
    if not len(lat):
        return None, None
    a = np.sort(np.asarray(lat))
    return float(np.percentile(a, 50)), float(np.percentile(a, 99))


def capacities(n: int, a0: float, gamma0: float = 2000.0, fwhm_s: float = 30e-15) -> tuple[int, int, int]:
    """Slots (electrons, positrons, photons) for a head-on collision of n electrons that keeps
    every particle it makes.

    Upper estimates with about 2x margin over FP64 oracle runs of whole collisions at the corners
    of the parameter ranges used here (a0 <= 500, gamma0 <= 4000, 15-60 fs, lambda = 1 um), where
    the worst case (a0 = 500, gamma0 = 4000, 60 fs) ended with 4.8 electrons, 3.8 positrons and
    540 photons per initial electron.  Photon numbers grow like a0 times the crossing time (the
    emission rate is proportional to the field); pairs grow with chi ~ gamma0 a0."""
    dur = 0.5 + 0.5 * fwhm_s / 30e-15
    pairs = 2.5 * (gamma0 * a0 / 1e6) ** 1.2 * dur
    e_cap = int(n * (1.0 + pairs)) + 4096
    p_cap = int(n * pairs) + 4096
    g_cap = int(n * (a0 * dur * (0.5 + 0.5 * gamma0 / 2000.0) + 16)) + 4096
    return e_cap, p_cap, g_cap


def formula_capacities(w) -> tuple[int, int, int]:
    """capacities() for a head-on workload."""
    return capacities(w.n, w.extra.get("a0", 100.0), w.extra.get("gamma_mean", 2000.0), w.extra.get("fwhm_s", 30e-15))


def make_species(qed, w, precision, caps=None):
    """Electron, positron and photon stores for a head-on workload; the append region of each
    species holds the children of one step (at most one per parent: a photon per lepton, a pair
    per photon, and never more pairs than positrons in all).  ``caps`` = (electrons, positrons,
    photons), by default the upper estimates of capacities()."""
    e_cap, p_cap, g_cap = caps if caps is not None else formula_capacities(w)
    return [qed.Species(qed.ELECTRON, precision, e_cap, p_cap), qed.Species(qed.POSITRON, precision, p_cap, p_cap),
            qed.Species(qed.PHOTON, precision, g_cap, e_cap + p_cap)]


def footprint(w, precision_bytes: int, caps=None) -> int:
    """Device bytes of make_species' stores: arrays and append regions (3 coordinates, 3 momenta,
    8-byte tau, id and, in the append region, the parent index)."""
    e_cap, p_cap, g_cap = caps if caps is not None else formula_capacities(w)
    per = 6 * precision_bytes + 8 + 4
    return (e_cap + p_cap + g_cap) * per + (2 * p_cap + e_cap + p_cap) * (per + 4)


def pilot_capacities(qed, tables, workloads, precision, sample: int = 1024, stream=None):
    """Capacities (electrons, positrons, photons) for each workload from a pilot run on the GPU.

    The first ``sample`` electrons of every workload (all of them when it has fewer) run all its
    steps, the pilots of all workloads together in one batch, each under the workload's own
    Philox key.  A species only grows during a run (converted photons stay as holes), so the
    particles it holds at the end are its peak.  A workload no larger than the sample is its own
    pilot and gets its counts exactly; a larger one gets the pilot's count per initial electron
    times its size, with a margin for the pilot's sampling error (2/sqrt(sample) relative, which
    allows a per-electron spread of half the mean at 4 standard errors, plus 8 Poisson standard
    deviations of the scaled count); positrons (pairs are rare) take 4 Poisson deviations of the
    pilot's own count on top.  Returns ([(e, p, g)] per workload, pilot stats)."""
    t0 = time.perf_counter()
    batch = qed.Batch(tables, precision, len(workloads))
    pil = []
    for k, w in enumerate(workloads):
        m = min(w.n, sample)
        sp = make_species(qed, w, precision, capacities(m, w.extra.get("a0", 100.0), w.extra.get("gamma_mean", 2000.0),
                                                        w.extra.get("fwhm_s", 30e-15)))
        xr = w.x[:m].copy()
        xr[:, 0] -= w.window_x0
        sp[0].upload(xr, w.u[:m], stream=stream)
        sp[0].init_tau(w.seed, w.extra.get("scenario", k), stream=stream)
        p = qed.StepParams(dt=w.dt, seed=w.seed, scenario=w.extra.get("scenario", k), field=qed.Field(**w.field.as_dict()),
                           window_x0=w.window_x0, window_v=w.window_v)
        batch.attach(k, sp, p, 0, w.n_steps, stream=stream)
        pil.append((m, sp))
    batch.run(max(w.n_steps for w in workloads), stream=stream)
    qed.check([s for _, sp in pil for s in sp], stream=stream)
    caps, units = [], 0
    for w, (m, sp) in zip(workloads, pil):
        ce, cp, cg = (s.count(stream=stream) for s in sp)
        units += sum(qed.work_read(sp[0], stream=stream)[:2])
        if w.n <= m:
            caps.append((ce + 64, cp + 64, cg + 64))
        else:
            f = w.n / m
            g = f * cg
            g_cap = int(math.ceil(g * (1.0 + 2.0 / math.sqrt(m)) + 8.0 * math.sqrt(g + 1.0))) + 4096
            p_cap = int(math.ceil(f * (cp + 4.0 * math.sqrt(cp) + 8.0))) + 4096
            caps.append((w.n + p_cap, p_cap, g_cap))
        for s in sp:
            s.close()
    batch.close()
    return caps, {"sample_electrons": sample, "pilot_particle_steps": units, "wall_s": time.perf_counter() - t0}


def serve(qed, tables, requests, precision, slots: int = 64, budget_bytes: int = 200 << 30, chunk: int = 50,
          max_wall: float = 120.0, admit_until: float | None = None, multistep: int = 0, on_finish=None):
    """Serve (arrival_s, Workload) requests; returns the finished Requests and run statistics.
    ``chunk`` batch steps run per round; with ``multistep`` > 0 a batch step also takes each slot's
    event-free stretch of up to that many steps.  ``on_finish(request, species)``, if given, sees
    each finished request's species before they are released."""
    prec_bytes = 4 if precision == qed.MIXED else 8
    batch = qed.Batch(tables, precision, slots)
    if multistep:
        batch.multistep(multistep)
    sched = Scheduler(slots, budget_bytes)
    future = collections.deque()
    for k, (t, w) in enumerate(requests):
        # a request spec is built into its workload only when it is admitted
        caps = formula_capacities(w) if not hasattr(w, "workload") else capacities(w.n, w.a0, w.gamma0, 30e-15)
        future.append(Request(k, t, w.n, w.n_steps, footprint(w, prec_bytes, caps), w))
    species = {}
    served_units = 0
    t0 = time.perf_counter()
    rounds = 0
    while True:
        now = time.perf_counter() - t0
        if now > max_wall:
            break
        while future and future[0].arrival <= now and (admit_until is None or future[0].arrival <= admit_until):
            sched.arrive(future.popleft())
        if admit_until is not None:
            while future and future[0].arrival > admit_until:
                future.popleft()  # arrivals after the window are not part of the run
        for r in sched.admit(now):
            w = r.payload.workload() if hasattr(r.payload, "workload") else r.payload
            sp = make_species(qed, w, precision)
            xr = w.x.copy()
            xr[:, 0] -= w.window_x0
            sp[0].upload(xr, w.u)
            sp[0].init_tau(w.seed, r.rid)
            p = qed.StepParams(dt=w.dt, seed=w.seed, scenario=r.rid, field=qed.Field(**w.field.as_dict()),
                               window_x0=w.window_x0, window_v=w.window_v)
            batch.attach(r.slot, sp, p, 0, w.n_steps)
            qed.work_read(sp[0], reset=True)
            species[r.slot] = sp
        if not sched.running:
            if sched.idle() and not future:
                break
            time.sleep(0.0005)
            continue
        batch.run(chunk)
        rounds += 1
        left = batch.remaining()
        now = time.perf_counter() - t0
        for slot in list(sched.running):
            if left[slot] == 0:
                sp = species.pop(slot)
                led = qed.read_ledger(sp)
                lep, ph, created = qed.work_read(sp[0])
                r = sched.complete(slot, now)
                r.result = {"ledger": led, "particle_steps": lep + ph, "created": created}
                served_units += lep + ph
                if on_finish is not None:
                    on_finish(r, sp)
                batch.detach(slot)
                for s in sp:
                    s.close()
    wall = time.perf_counter() - t0
    # work done on requests still running when the run stopped (a request waiting in the queue
    # has done none)
    partial_units = 0
    for slot, sp in species.items():
        lep, ph, _ = qed.work_read(sp[0])
        partial_units += lep + ph
        batch.detach(slot)
        for s in sp:
            s.close()
    fin = sched.finished
    p50, p99 = percentiles([r.latency for r in fin])
    # requests still queued or running when the run stopped have waited at least this long:
    # with them the percentiles are lower bounds of the true ones
    unfinished = list(sched.pending) + list(sched.running.values())
    lb50, lb99 = percentiles([r.latency for r in fin] + [wall - r.arrival for r in unfinished])
    stats = {"finished": len(fin), "arrived": len(fin) + len(unfinished),
             "still_running": len(sched.running), "queued": len(sched.pending), "wall_s": wall,
             "served_particle_steps_per_s": served_units / wall if wall > 0 else 0.0,
             "served_particle_steps": served_units,
             "processed_particle_steps_per_s": (served_units + partial_units) / wall if wall > 0 else 0.0,
             "latency_p50_s": p50, "latency_p99_s": p99,
             "latency_p50_lower_bound_s": lb50, "latency_p99_lower_bound_s": lb99,
             "rounds": rounds, "chunk_steps": chunk, "slots": slots}
    batch.close()
    return fin, stats
