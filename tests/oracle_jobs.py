"""Oracle runs that tests hand to a process pool (spawned: no CUDA state is inherited).  Imports
neither torch nor the CUDA library."""
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def head_on_chunk(job):
    """Electrons [lo, hi) of a head-on workload run alone on the oracle for all its steps: the
    final energies of electrons, positrons and (unconverted) photons."""
    n_total, lo, hi, seed, n_steps, kw = job
    import oracle as o
    from paper_1311_5551_gb300 import workloads as W

    w = W.head_on(n=n_total, n_steps=n_steps, seed=seed, **kw)
    path = os.path.join(ROOT, "oracle", "_build", "tables_default.npz")
    tables = o.Tables.load(path)
    m = hi - lo
    e, p, g = o.Species(8 * m + 64), o.Species(8 * m + 64), o.Species(1200 * m + 64)
    e.set(w.x[lo:hi], w.u[lo:hi])
    e.init_tau(o.ELECTRON, w.seed, lo)  # each chunk its own stream (scenario = first electron)
    sp = o.StepParams(dt=w.dt, seed=w.seed, scenario=lo, field=o.Field(**w.field.as_dict()))
    for k in range(w.n_steps):
        o.step(tables, sp, k, e, p, g)
    alive = np.isfinite(g.get("tau"))
    return e.energy(), p.energy(), g.energy(photon=True)[alive]
