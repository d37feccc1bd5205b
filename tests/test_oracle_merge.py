"""Pins of the oracle's macroparticle merging (Sec. 3.1 names merging as the remedy for growing
populations and leaves it unimplemented) and of weight inheritance: what the merge must conserve
(weight, momentum, energy of every group, exactly up to rounding), what it must leave alone, and
which photons survive.  CPU only."""
import numpy as np
import pytest

import oracle as o

GRID = dict(origin=(0.0, 0.0, 0.0), cell=(10.0, 10.0, 10.0), n_cells=(4, 4, 4))


def photons(x, k, w=None, ids=None):
    s = o.Species(len(x) + 8)
    s.set(np.asarray(x, float), np.asarray(k, float), tau=np.linspace(0.5, 2.0, len(x)), ids=ids, w=w)
    return s


def clustered(rng, n_groups=20, per=(3, 12)):
    """Photons in tight clusters of position and momentum (each cluster inside one bin)."""
    xs, ks = [], []
    for g in range(n_groups):
        c = rng.uniform(1, 39, 3)
        c = np.floor(c / 10) * 10 + 5  # centre of a cell
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        e = 2.0 ** rng.integers(2, 12) * 1.3  # inside one energy sub-bin
        for _ in range(rng.integers(*per)):
            xs.append(c + rng.uniform(-1, 1, 3))
            kk = d + rng.normal(scale=1e-3, size=3)
            ks.append(kk / np.linalg.norm(kk) * e * (1 + rng.uniform(-1e-3, 1e-3)))
    return np.array(xs), np.array(ks)


def test_merge_conserves_weight_momentum_energy():
    rng = np.random.default_rng(1)
    x, k = clustered(rng)
    w = rng.uniform(0.5, 3.0, len(x))
    s = photons(x, k, w)
    W0, E0, P0 = s.totals(photon=True)
    n0 = s.n
    g = s.merge(**GRID, n_face=8, n_sub=4, min_group=3)
    W1, E1, P1 = s.totals(photon=True)
    assert g > 10 and s.n < n0
    assert W1 == pytest.approx(W0, rel=1e-13)
    assert E1 == pytest.approx(E0, rel=1e-12)
    assert np.allclose(P1, P0, rtol=1e-12, atol=1e-12 * E0)


def test_merged_pair_shape():
    # every merged group becomes two photons of weight W/2, energy E/W each, symmetric about P/W
    rng = np.random.default_rng(2)
    x, k = clustered(rng, n_groups=1, per=(9, 10))
    w = rng.uniform(0.5, 2.0, len(x))
    s = photons(x, k, w)
    W, E, P = s.totals(photon=True)
    assert s.merge(**GRID, min_group=3) == 1 and s.n == 2
    kk = s.u()
    assert np.allclose(s.get("w"), W / 2, rtol=1e-14)
    assert np.allclose(np.linalg.norm(kk, axis=1), E / W, rtol=1e-12)
    assert np.allclose(kk.sum(axis=0) / 2, P / W, rtol=1e-12, atol=1e-12 * E)
    d = kk[0] - P / W
    assert abs(d @ P) < 1e-9 * np.linalg.norm(d) * np.linalg.norm(P) + 1e-12
    assert np.allclose(s.x()[0], (w[:, None] * x).sum(0) / W) and np.allclose(s.x()[1], s.x()[0])


def test_survivors_and_order():
    # the two lowest-index photons of a group survive with their ids and optical depths; the
    # photons of other groups keep their order
    rng = np.random.default_rng(3)
    x, k = clustered(rng, n_groups=1, per=(6, 7))
    lone_x = np.array([[35.0, 35.0, 35.0], [5.0, 35.0, 5.0]])
    lone_k = np.array([[0.0, 0.0, 50.0], [-70.0, 1.0, 0.0]])
    xs = np.concatenate([lone_x[:1], x, lone_x[1:]])
    ks = np.concatenate([lone_k[:1], k, lone_k[1:]])
    s = photons(xs, ks, ids=np.arange(100, 100 + len(xs), dtype=np.uint32))
    tau0 = s.get("tau")
    assert s.merge(**GRID, min_group=3) == 1
    assert list(s.get("id")) == [100, 101, 102, 100 + len(xs) - 1]
    assert np.array_equal(s.get("tau")[[0, 1, 2, 3]], tau0[[0, 1, 2, len(xs) - 1]])
    assert np.array_equal(s.u()[[0, 3]], ks[[0, -1]])


def test_small_groups_outside_and_distinct_bins_are_untouched():
    rng = np.random.default_rng(4)
    x, k = clustered(rng, n_groups=6, per=(2, 3))  # groups of 2 < min_group
    far = np.array([[-5.0, 5.0, 5.0], [5.0, 45.0, 5.0], [5.0, 5.0, 41.0]])  # outside the grid
    xs = np.concatenate([x, far, far, far])
    ks = np.concatenate([k, k[:3], k[:3] * 1.0, k[:3]])
    s = photons(xs, ks)
    before = (s.x().copy(), s.u().copy(), s.get("w").copy())
    assert s.merge(**GRID, min_group=3) == 0
    assert np.array_equal(s.x(), before[0]) and np.array_equal(s.u(), before[1])
    assert np.array_equal(s.get("w"), before[2])
    # one photon per cell, all alike otherwise: never merged across cells
    cells = np.array([[5.0 + 10 * i, 5.0, 5.0] for i in range(4)] * 3)
    s = photons(cells, np.tile([[10.0, 0.1, 0.0]], (12, 1)))
    assert s.merge(**GRID, min_group=3) == 4 and s.n == 8  # 4 cells x 3 alike -> 4 x 2


def test_identical_photons_merge_without_spread():
    # photons identical up to weight: the merged pair has no transverse spread
    s = photons(np.tile([[12.0, 13.0, 14.0]], (5, 1)), np.tile([[3.0, -4.0, 12.0]], (5, 1)), w=[1, 2, 3, 4, 5])
    assert s.merge(**GRID, min_group=3) == 1
    assert np.allclose(s.u(), [[3.0, -4.0, 12.0]] * 2, rtol=1e-14) and np.allclose(s.get("w"), 7.5)


def test_children_inherit_weight(orc_tables):
    # one emission: the photon carries its parent's weight
    from paper_1311_5551_gb300 import workloads as W

    w = W.uniform_b(n=200, cB=9e-3, seed=3)
    e = o.Species(1000)
    e.set(w.x, w.u, w=np.full(200, 3.5))
    e.init_tau(o.ELECTRON, 3)
    p, g = o.Species(1000), o.Species(1000)
    sp = o.StepParams(dt=w.dt * 20, seed=3, make_pairs=False, field=o.Field(B=w.field.B))
    o.step(orc_tables, sp, 0, e, p, g)
    assert g.n > 10 and np.all(g.get("w") == 3.5)


def test_lepton_merge_conserves_and_keeps_mass_shell():
    # electrons: the merged pair carries the group's weight, momentum and energy, each member on
    # the mass shell gamma^2 = 1 + |u|^2 with gamma = E/W
    rng = np.random.default_rng(6)
    x, k = clustered(rng, n_groups=15, per=(3, 10))
    k = k * 0.7  # momenta of e+- (u), same clustering
    w = rng.uniform(0.5, 3.0, len(x))
    s = photons(x, k, w)
    W0, E0, P0 = s.totals(photon=False)
    g = s.merge(**GRID, min_group=3, photon=False)
    W1, E1, P1 = s.totals(photon=False)
    assert g > 5
    assert W1 == pytest.approx(W0, rel=1e-13) and E1 == pytest.approx(E0, rel=1e-12)
    assert np.allclose(P1, P0, rtol=1e-12, atol=1e-12 * E0)
    # a single group: both members have gamma = E/W
    x1, k1 = clustered(np.random.default_rng(7), n_groups=1, per=(6, 7))
    s = photons(x1, k1 * 0.3, w=np.arange(1.0, 7.0))
    W, E, _ = s.totals(photon=False)
    assert s.merge(**GRID, min_group=3, photon=False) == 1
    gam = np.sqrt(1 + np.sum(s.u() ** 2, axis=1))
    assert np.allclose(gam, E / W, rtol=1e-12)
