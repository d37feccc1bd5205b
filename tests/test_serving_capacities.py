"""The per-scenario capacities that the batched scan and the serving loop allocate are upper
bounds: FP64 oracle runs of whole head-on collisions at the corners of the scan's parameter ranges
never hold more particles than the per-electron part of the estimate.  CPU only."""
import numpy as np
import pytest

import oracle as o
from paper_1311_5551_gb300 import serving
from paper_1311_5551_gb300 import workloads as W

SLACK = 4096  # the fixed part of every capacity


@pytest.mark.parametrize("a0,gamma0,fwhm_s", [(500.0, 4000.0, 60e-15), (500.0, 200.0, 15e-15),
                                              (10.0, 4000.0, 60e-15), (250.0, 2000.0, 30e-15)])
def test_capacities_bound_oracle_collisions(orc_tables, a0, gamma0, fwhm_s):
    n = 48
    w = W.head_on(n=n, gamma_mean=gamma0, a0=a0, fwhm_s=fwhm_s, n_steps=4000, rng=np.random.default_rng(7))
    e_cap, p_cap, g_cap = serving.capacities(n, a0, gamma0, fwhm_s)
    e, p, g = o.Species(e_cap), o.Species(p_cap), o.Species(g_cap)
    e.set(w.x, w.u)
    e.init_tau(o.ELECTRON, w.seed)
    sp = o.StepParams(dt=w.dt, seed=w.seed, field=o.Field(**w.field.as_dict()))
    peak = np.zeros(3, dtype=np.int64)
    for k in range(w.n_steps):
        o.step(orc_tables, sp, k, e, p, g)
        peak = np.maximum(peak, [e.n, p.n, g.n])
    assert peak[0] <= e_cap - SLACK and peak[1] <= p_cap - SLACK and peak[2] <= g_cap - SLACK
    assert peak[2] > 0  # the collision happened: photons were emitted
