"""Pins of the oracle's grid field gather (the PIC interpolation of Sec. 3.2) against what the
particle shapes fix exactly: linear fields are reproduced by both shapes, the second moments of
the weights give closed forms for quadratic fields, missing nodes outside the grid drop out, and a
grid holding a uniform field reproduces the uniform-field run.  CPU only."""
import math

import numpy as np
import pytest

import oracle as o
from paper_1311_5551_gb300 import workloads as W

N = (7, 6, 5)            # nodes along x, y, z
ORIGIN = (-1.5, 2.0, 0.25)
SPACING = (0.5, 0.75, 1.25)


def node_pos(c, i, j, k):
    """Position of node (i, j, k) of component c (0..2: E, 3..5: cB), Yee-staggered."""
    idx = [i, j, k]
    out = []
    for a in range(3):
        st = (a == c) if c < 3 else (a != c - 3)
        out.append(ORIGIN[a] + (idx[a] + (0.5 if st else 0.0)) * SPACING[a])
    return out


def grid_of(fn):
    g = np.zeros((6, N[2], N[1], N[0]))
    for c in range(6):
        for k in range(N[2]):
            for j in range(N[1]):
                for i in range(N[0]):
                    g[c, k, j, i] = fn(c, *node_pos(c, i, j, k))
    return g


def interior_points(rng, m, margin=2.0):
    lo = [ORIGIN[a] + margin * SPACING[a] for a in range(3)]
    hi = [ORIGIN[a] + (N[a] - 1 - margin) * SPACING[a] for a in range(3)]
    return rng.uniform(lo, hi, size=(m, 3))


def field(grid, shape):
    return o.Field(kind=o.FIELD_GRID, grid=grid, shape=shape, origin=ORIGIN, spacing=SPACING)


@pytest.mark.parametrize("shape", [1, 2])
def test_linear_fields_are_reproduced(shape):
    rng = np.random.default_rng(1)
    A = rng.normal(size=6)
    Bm = rng.normal(size=(6, 3))
    fd = field(grid_of(lambda c, x, y, z: A[c] + Bm[c] @ np.array([x, y, z])), shape)
    for x in interior_points(rng, 40):
        E, B = o.field_eval(fd, 0.0, x)
        got = np.concatenate([E, B])
        want = A + Bm @ x
        assert np.allclose(got, want, rtol=0, atol=1e-12 * (1 + np.abs(want).max()))


@pytest.mark.parametrize("shape", [1, 2])
def test_quadratic_field_second_moment(shape):
    # f = s^2 with s the continuous node index of the component along its axis: cloud-in-cell gives
    # s^2 + w(1 - w) (w the fractional part), the triangular-shaped cloud s^2 + 1/4
    rng = np.random.default_rng(2)
    for c in (0, 4):  # Ex (staggered along x) and cBy (staggered along x and z)
        def fn(cc, x, y, z, c=c):
            if cc != c:
                return 0.0
            st = 0.5 if (c == 0 or c == 4) else 0.0
            s = (x - ORIGIN[0]) / SPACING[0] - st
            return s * s
        fd = field(grid_of(fn), shape)
        for x in interior_points(rng, 20):
            E, B = o.field_eval(fd, 0.0, x)
            v = np.concatenate([E, B])[c]
            s = (x[0] - ORIGIN[0]) / SPACING[0] - 0.5
            w = s - math.floor(s)
            want = s * s + (w * (1 - w) if shape == 1 else 0.25)
            assert v == pytest.approx(want, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("shape", [1, 2])
def test_missing_nodes_outside_the_grid(shape):
    fd = field(np.ones((6, N[2], N[1], N[0])), shape)
    # far outside: nothing
    for x in ([100.0, 3.0, 2.0], [-100.0, 3.0, 2.0], [0.0, -50.0, 2.0]):
        E, B = o.field_eval(fd, 0.0, x)
        assert not np.any(E) and not np.any(B)
    # Ey (unstaggered along x) a quarter cell below node 0 along x, deep inside along y and z:
    # node -1 does not exist, so cloud-in-cell keeps node 0's weight 3/4 and the triangular cloud
    # keeps node 0's 3/4 - d^2 and node 1's (1/2)(3/2 - (1 + d))^2, with d = 1/4
    y = ORIGIN[1] + 3.0 * SPACING[1]
    z = ORIGIN[2] + 2.0 * SPACING[2]
    x = ORIGIN[0] - 0.25 * SPACING[0]
    E, _ = o.field_eval(fd, 0.0, [x, y, z])
    d = 0.25
    want = (1 - d) if shape == 1 else (0.75 - d * d) + 0.5 * (1.5 - (1 + d)) ** 2
    assert E[1] == pytest.approx(want, rel=1e-14)


def test_uniform_grid_reproduces_uniform_field_run(orc_tables):
    # test problem 1 geometry on a grid holding cB = 1e-3 everywhere: same run as the analytic field
    w = W.uniform_b(n=300, steps_per_gyro=1000.0, seed=5)
    rad = 1000.0 / 1e-3  # gyro-radius gamma/cB
    n, sp = 12, 2.5 * rad / 10
    g = np.zeros((6, n, n, n))
    g[5] = 1e-3
    org = (-sp * (n - 1) / 2,) * 3
    fg = o.Field(kind=o.FIELD_GRID, grid=g, shape=2, origin=org, spacing=(sp, sp, sp))
    runs = []
    for fd in (o.Field(B=w.field.B), fg):
        e = o.Species(w.n + 4)
        e.set(w.x, w.u)
        e.init_tau(o.ELECTRON, w.seed)
        p, ph = o.Species(4), o.Species(4)
        spar = o.StepParams(dt=w.dt, seed=w.seed, make_pairs=False, drain_photons=True, field=fd)
        for k in range(200):
            L = o.step(orc_tables, spar, k, e, p, ph)
        runs.append((L, e.u()))
    (La, ua), (Lb, ub) = runs
    assert La["n"] == Lb["n"] and La["drained_n"] == Lb["drained_n"]
    assert Lb["energy"][0] == pytest.approx(La["energy"][0], rel=1e-12)
    assert np.allclose(ua, ub, rtol=1e-12, atol=1e-9)
