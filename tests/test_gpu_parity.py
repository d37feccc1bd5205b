"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by element.

Tolerances: FP64 path 1e-12 relative on eta, chi, rates and look-ups; FP32 (mixed) path 1e-5
relative.  Quantities that pass through independently built tables (library quadrature vs
oracle quadrature, which agree to ~1e-14) use the same bars.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle as o  # noqa: E402
from paper_1311_5551_gb300 import qed, workloads as W  # noqa: E402
from paper_1311_5551_gb300 import build as qbuild  # noqa: E402

RTOL = {qed.FP64: 1e-12, qed.MIXED: 1e-5}


@pytest.fixture(scope="module")
def lib_tables():
    qbuild.build()
    return qed.Tables()


@pytest.fixture(scope="module")
def same_tables(orc_tables):
    """The oracle's table values loaded into the library (isolates the look-up arithmetic)."""
    qbuild.build()
    return qed.Tables(arrays=orc_tables.a)


def to_orc_field(f: W.FieldSpec):
    return o.Field(**f.as_dict())


def to_qed_field(f: W.FieldSpec):
    return qed.Field(**f.as_dict())


# ------------------------------------------------------------------ tables and generator
def test_library_tables_match_oracle(lib_tables, orc_tables):
    a = lib_tables.export()
    b = orc_tables.a
    np.testing.assert_allclose(a["ln_h"], b["ln_h"], rtol=1e-13, atol=0)
    np.testing.assert_allclose(a["g"], b["g"], rtol=1e-13)
    np.testing.assert_allclose(a["zeta_lo"], b["zeta_lo"], rtol=1e-13)
    np.testing.assert_allclose(a["zeta_hi"], b["zeta_hi"], rtol=1e-13)
    np.testing.assert_allclose(a["P"], b["P"], rtol=0, atol=1e-13)
    m = b["Q"] > 1e-12
    np.testing.assert_allclose(a["Q"][m], b["Q"][m], rtol=1e-11)
    np.testing.assert_allclose(a["ln_T"], b["ln_T"], rtol=1e-13)
    np.testing.assert_allclose(a["Pf"], b["Pf"], rtol=0, atol=1e-12)


def test_philox_device_matches_oracle():
    qbuild.build()
    rng = np.random.default_rng(5)
    ctr = rng.integers(0, 2**63, size=(513, 4), dtype=np.int64).astype(np.uint64) * 2 + 1
    key = [int(rng.integers(0, 2**62)), 77]
    dev = qed.philox(ctr.ravel(), key)
    for i in range(0, 513, 37):
        assert [int(v) for v in dev[i]] == o.philox4x64([int(c) for c in ctr[i]], key)


# ------------------------------------------------------------------ per-particle look-ups
def random_particles(n, seed, kind):
    rng = np.random.default_rng(seed)
    x = np.zeros((n, 3))
    x[:, 0] = rng.uniform(-3e6, 3e6, n)
    mag = 10 ** rng.uniform(0.5, 3.7, n)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return x, d * mag[:, None]


FIELDS = {
    "uniform": W.FieldSpec(W.FIELD_UNIFORM, E=(1e-4, -2e-4, 5e-5), B=(3e-4, 1e-3, -2e-4)),
    "rotating": W.FieldSpec(W.FIELD_ROTATING_E, E0=1e-3, omega=3.03e-6, phase0=0.3),
    "plane_lp": W.FieldSpec(W.FIELD_PLANE_LP, E0=2.4e-4, omega=2.4263e-6, phi_start=-60.0, phi_len=226.0),
    "plane_cp": W.FieldSpec(W.FIELD_PLANE_CP, E0=1.2e-4, omega=2.4263e-6, phi_start=-40.0, phi_len=0.0),
}


@pytest.mark.parametrize("prec", [qed.FP64, qed.MIXED])
@pytest.mark.parametrize("fname", list(FIELDS))
@pytest.mark.parametrize("kind", [qed.ELECTRON, qed.PHOTON])
def test_eval_particles_parity(same_tables, orc_tables, prec, fname, kind):
    fs = FIELDS[fname]
    n = 4099  # several blocks and a ragged tail
    x, u = random_particles(n, 11 + kind, kind)
    if prec == qed.MIXED:  # the mixed path sees float inputs: compare on those values
        x = x.astype(np.float32).astype(np.float64)
        u = u.astype(np.float32).astype(np.float64)
    t = 1.7e7
    r = qed.eval_particles(same_tables, prec, kind, to_qed_field(fs), t, x, u)
    ofd = to_orc_field(fs)
    tol = RTOL[prec]
    fe = fs.E0 if fs.E0 else max(np.abs(fs.E).max(), np.abs(fs.B).max())
    chi_min = orc_tables.params.chi_min
    for i in range(0, n, 7):
        E, B = o.field_eval(ofd, t, x[i])
        # fields: absolute error against the amplitude (FP32 phase rounding for the mixed path)
        np.testing.assert_allclose(r["E"][i], E, rtol=0, atol=4 * tol * fe)
        np.testing.assert_allclose(r["B"][i], B, rtol=0, atol=4 * tol * fe)
        if kind == qed.PHOTON:
            eps = np.linalg.norm(u[i])
            p = o.chi_of(u[i], eps, E, B)
            rate = orc_tables.rate_pair(p, eps) if p > 0 else 0.0
            terms = [np.cross(u[i], E) @ np.cross(u[i], E), 2 * eps * abs(E @ np.cross(u[i], B)),
                     np.cross(u[i], B) @ np.cross(u[i], B)]
            sq = 4 * p * p
        else:
            eps = math.sqrt(1 + u[i] @ u[i])
            p = o.eta_of(u[i], eps, E, B)
            rate = orc_tables.rate_photon(p, eps) if p > 0 else 0.0
            terms = [E @ E, np.cross(u[i], E) @ np.cross(u[i], E), 2 * eps * abs(E @ np.cross(u[i], B)),
                     np.cross(u[i], B) @ np.cross(u[i], B)]
            sq = p * p
        # the invariant is a sum of terms that can cancel: scale the bar by its condition number
        kappa = max(1.0, sum(terms) / sq) if sq > 0 else 1.0
        assert r["energy"][i] == pytest.approx(eps, rel=tol)
        p_abs = 4 * tol * fe * eps
        assert r["param"][i] == pytest.approx(p, rel=4 * tol * kappa, abs=p_abs)
        if p <= 0:
            assert r["rate"][i] == 0.0
            continue
        # the parameter's error propagates through d ln(lambda)/d ln(p): about 1 for eta (h varies
        # slowly) and 1 + 4/(3 chi) for chi (T ~ exp(-4/(3 chi)) at small chi, App. B)
        rel_p = max(4 * tol * kappa, p_abs / p)
        gain = 1.0 if kind == qed.ELECTRON else 1.0 + 4.0 / (3.0 * p)
        if kind == qed.PHOTON and abs(p / chi_min - 1) < rel_p:
            continue  # at the lower edge of the T table the zero cut-off may go either way
        # FP32 flushes rates below ~1e-37 (units m c^2/hbar) to zero: over any run (< 1e12 time
        # units) such a rate converts a photon with probability < 1e-25
        floor = 1e-37 if prec == qed.MIXED else 0.0
        assert r["rate"][i] == pytest.approx(rate, rel=rel_p * gain + tol, abs=floor)


def same_inputs(prec, *arrays):
    """The inputs as the path sees them: the mixed path takes the parameter and the uniform U as
    floats (the step hands it the correctly rounded float of its 53-bit U), so the oracle is
    given those same values; the FP64 path takes doubles."""
    if prec == qed.MIXED:
        return [a.astype(np.float32).astype(np.float64) for a in arrays]
    return list(arrays)


@pytest.mark.parametrize("prec", [qed.FP64, qed.MIXED])
def test_sample_xi_parity(same_tables, orc_tables, prec):
    # identical (eta, U) and identical table values: the FP32 inverse CDF is held to 1e-5 (the
    # bulk is near 3e-7: table values, U and the xi nodes each rounded once to FP32)
    rng = np.random.default_rng(3)
    n = 20000
    eta, U = same_inputs(prec, 10 ** rng.uniform(-4.5, 2.0, n), rng.random(n))  # below and in the table
    out, ok = qed.sample(same_tables, prec, 0, eta, U)
    tol = RTOL[prec]
    checked = 0
    for i in range(0, n, 5):
        ref = orc_tables.sample_xi(eta[i], U[i])
        if ref is None:
            # below the cut-off; the FP32 path may decide either way within rounding of the cut
            if prec == qed.FP64:
                assert not ok[i]
            continue
        if not ok[i]:
            assert prec == qed.MIXED
            continue
        assert out[i] == pytest.approx(ref, rel=tol)
        checked += 1
    assert checked > 3500


@pytest.mark.parametrize("prec", [qed.FP64, qed.MIXED])
def test_sample_f_parity(same_tables, orc_tables, prec):
    rng = np.random.default_rng(4)
    n = 20000
    chi, U = same_inputs(prec, 10 ** rng.uniform(-2.5, 2.5, n), rng.random(n))
    out, ok = qed.sample(same_tables, prec, 1, chi, U)
    tol = RTOL[prec]
    for i in range(0, n, 5):
        ref = orc_tables.sample_f(chi[i], U[i])
        assert out[i] == pytest.approx(ref, rel=tol, abs=1e-15)


@pytest.mark.parametrize("prec", [qed.FP64, qed.MIXED])
def test_rate_lookup_parity(same_tables, orc_tables, prec):
    # h(eta) and T(chi) for identical parameters and table values (the look-up alone, apart from
    # the error of eta or chi that the step's own parity tests carry).  h: 1e-5 (FP32), 1e-12
    # (FP64).  T in FP32: 1e-5 plus what FP32 cannot avoid, the error of ln chi (the fast FP32
    # logarithm, |d ln chi| <= 2^-20) carried by d ln T / d ln chi (about 4/(3 chi) at small chi,
    # App. B), and the FP32 rounding of the interpolated ln T (2^-22 |ln T|); values FP32 cannot
    # hold (below 1e-37) may flush to zero
    rng = np.random.default_rng(6)
    n = 20000
    eta = same_inputs(prec, 10 ** rng.uniform(-4.5, 2.3, n))[0]
    hv, hflag = qed.sample(same_tables, prec, 2, eta, None)
    tol = RTOL[prec]
    for i in range(0, n, 3):
        assert hv[i] == pytest.approx(orc_tables.h(eta[i]), rel=tol)
        assert hflag[i] == (-1 if eta[i] < orc_tables.params.eta_min else (1 if eta[i] > orc_tables.params.eta_max
                                                                            else 0))
    chi = same_inputs(prec, 10 ** rng.uniform(-2.3, 2.3, n))[0]
    tv, tflag = qed.sample(same_tables, prec, 3, chi, None)
    lnT = orc_tables.a["ln_T"]
    lc0, lc1 = math.log(orc_tables.params.chi_min), math.log(orc_tables.params.chi_max)
    d = (lc1 - lc0) / (len(lnT) - 1)
    for i in range(0, n, 3):
        ref = orc_tables.T(chi[i])
        if ref == 0.0:
            assert tv[i] == 0.0
            continue
        bar = tol
        if prec == qed.MIXED:
            c = min(max(int((math.log(chi[i]) - lc0) / d), 0), len(lnT) - 2)
            slope = abs(lnT[c + 1] - lnT[c]) / d
            bar = tol + 2.0 ** -20 * slope + 2.0 ** -22 * abs(math.log(ref))
        assert tv[i] == pytest.approx(ref, rel=bar, abs=1e-37 if prec == qed.MIXED else 0.0)
        assert tflag[i] == (1 if chi[i] > orc_tables.params.chi_max else 0)


# ------------------------------------------------------------------ whole steps
def make_gpu_species(w: W.Workload, prec, cap=None, app=None, drain=False):
    n = w.n
    cap = cap or max(4 * n, 4096)
    app = app or max(n, 4096)
    e = qed.Species(qed.ELECTRON, prec, cap, app)
    p = qed.Species(qed.POSITRON, prec, cap, app)
    g = qed.Species(qed.PHOTON, prec, 8 * cap, 2 * app)
    d = qed.Species(qed.PHOTON, prec, 64 * cap, 1) if drain else None
    xr = w.x.copy()
    xr[:, 0] -= w.window_x0
    e.upload(xr, w.u)
    e.init_tau(w.seed)
    return e, p, g, d


def make_orc_species(w: W.Workload, drain=False):
    e = o.Species(4 * max(w.n, 1024) + 4)
    e.set(w.x, w.u)
    e.init_tau(o.ELECTRON, w.seed)
    p = o.Species(4 * max(w.n, 1024) + 4)
    g = o.Species(32 * max(w.n, 1024))
    d = o.Species(256 * max(w.n, 1024)) if drain else None
    return e, p, g, d


def qparams(w: W.Workload, drain=False):
    return qed.StepParams(dt=w.dt, seed=w.seed, field=to_qed_field(w.field), emit_photons=w.emit_photons,
                          make_pairs=w.make_pairs, drain_photons=drain, window_x0=w.window_x0, window_v=w.window_v)


def oparams(w: W.Workload, drain=False):
    return o.StepParams(dt=w.dt, seed=w.seed, field=to_orc_field(w.field), emit_photons=w.emit_photons,
                        make_pairs=w.make_pairs, drain_photons=drain)


def abs_x(dl, w, step):
    x = dl["x"].astype(np.float64).copy()
    x[:, 0] += w.window_x0 + w.window_v * (step * w.dt)
    return x


def compare_species(gd, os_, w, step, rtol, what):
    assert len(gd["id"]) == os_.n, f"{what}: count {len(gd['id'])} vs {os_.n} at step {step}"
    if os_.n == 0:
        return
    assert np.array_equal(gd["id"], os_.get("id")), f"{what}: ids differ at step {step}"
    u_o = os_.u()
    scale = np.maximum(np.linalg.norm(u_o, axis=1, keepdims=True), 1.0)
    np.testing.assert_allclose(gd["u"] / scale, u_o / scale, rtol=0, atol=rtol, err_msg=f"{what} u step {step}")
    xg = abs_x(gd, w, step)
    xo = os_.x()
    xs = max(1.0, float(np.abs(xo).max()))
    np.testing.assert_allclose(xg / xs, xo / xs, rtol=0, atol=rtol, err_msg=f"{what} x step {step}")
    alive = np.isfinite(gd["tau"])
    np.testing.assert_allclose(gd["tau"][alive], os_.get("tau")[alive], rtol=rtol, atol=rtol,
                               err_msg=f"{what} tau step {step}")


def test_fp64_uniform_b_full_trajectories(lib_tables, orc_tables):
    # test problem 1 set-up with photons drained: every electron and every emitted photon match
    w = W.uniform_b(n=2083, n_steps=40)
    e, p, g, d = make_gpu_species(w, qed.FP64, drain=True)
    oe, op, og, od = make_orc_species(w, drain=True)
    qp, opp = qparams(w, drain=True), oparams(w, drain=True)
    emitted = 0
    for step in range(w.n_steps):
        qed.run(lib_tables, [e, p, g, d], qp, step)
        L = o.step(orc_tables, opp, step, oe, op, og, od)
        gl = qed.read_ledger([e, p, g, d])
        assert gl["emitted_n"] == L["emitted_n"] and gl["dropped_n"] == L["dropped_n"]
        assert gl["energy"][0] == pytest.approx(L["energy"][0], rel=1e-12)
        assert gl["emit_defect"] == pytest.approx(L["emit_defect"], rel=1e-8, abs=1e-12)
        emitted += L["emitted_n"]
        if step % 8 == 7 or step == w.n_steps - 1:
            compare_species(e.download(), oe, w, step + 1, 1e-12, "electrons")
    assert emitted > 1000
    dr = qed.drain(d)
    assert np.array_equal(dr["id"], od.get("id"))
    np.testing.assert_allclose(dr["u"], od.u(), rtol=1e-12)
    qed.check([e, p, g, d])


@pytest.mark.parametrize("prec", [qed.FP64, qed.MIXED])
def test_head_on_with_pairs_and_window(lib_tables, orc_tables, prec):
    # head-on collision through the peak of a strong pulse so that pairs appear within a few
    # dozen steps; the GPU stores positions relative to the moving window
    w = W.head_on(n=3001, a0=400.0, gamma_mean=4000.0, n_steps=60, meet_step=30, fwhm_s=8e-15, seed=9)
    if prec == qed.MIXED:
        w.x[:, 0] = (w.x[:, 0] - w.window_x0).astype(np.float32).astype(np.float64) + w.window_x0
        w.u = w.u.astype(np.float32).astype(np.float64)
    e, p, g, _ = make_gpu_species(w, prec)
    oe, op, og, _ = make_orc_species(w)
    qp, opp = qparams(w), oparams(w)
    first_event = {}
    pairs = 0
    prev_tau = oe.get("tau")[: w.n].copy()
    prev_gpu_tau = e.download()["tau"][: w.n].copy()
    photons_aligned, photon_checks, aligned_steps = True, 0, 0
    seen = 0  # photons with smaller ids were compared at their creation (ids follow creation)

    def amplitude_slope(xph, kph, t):
        """|d ln|E| / d phi| of the LP pulse at the emission of photons now at xph moving along
        kph (the emitter was at x - dt khat when the step's fields were taken, at time t)."""
        f = w.field
        xn = xph[:, 0] - w.dt * kph[:, 0] / np.linalg.norm(kph, axis=1)
        phi = f.omega * (t - xn) - f.phi_start
        a = np.pi * phi / f.phi_len
        return np.abs(np.tan(phi)) + 2.0 * (np.pi / f.phi_len) * np.abs(1.0 / np.tan(a))
    for step in range(w.n_steps):
        qed.run(lib_tables, [e, p, g], qp, step)
        L = o.step(orc_tables, opp, step, oe, op, og)
        pairs += L["pairs_n"]
        if prec == qed.FP64:
            gl = qed.read_ledger([e, p, g])
            assert gl["emitted_n"] == L["emitted_n"] and gl["pairs_n"] == L["pairs_n"], f"step {step}"
            for k in range(3):
                assert gl["n"][k] == L["n"][k]
                assert gl["energy"][k] == pytest.approx(L["energy"][k], rel=1e-11)
            if step % 10 == 9:
                compare_species(e.download(), oe, w, step + 1, 1e-11, "electrons")
                compare_species(p.download(), op, w, step + 1, 1e-11, "positrons")
                gd = g.download()
                keep = np.isfinite(gd["tau"])  # converted photons stay as holes on the GPU
                gd = {k: v[keep] for k, v in gd.items()}
                compare_species(gd, og, w, step + 1, 1e-11, "photons")
        else:
            # mixed: each electron particle by particle up to its first event (the oracle's
            # optical depth jumps up when it is redrawn); both sides must take the same decision
            gd = e.download()
            ou, ot = oe.u()[: w.n], oe.get("tau")[: w.n]
            for i in range(0, w.n, 3):
                if i in first_event:
                    continue
                if ot[i] > prev_tau[i]:
                    first_event[i] = step
                    continue
                assert gd["tau"][i] <= prev_gpu_tau[i] or abs(ot[i]) < 1e-4, f"event decision differs, {i}"
                err = np.abs(gd["u"][i] - ou[i]).max() / max(1.0, np.abs(ou[i]).max())
                assert err < 1e-5 * math.sqrt(step + 1), f"electron {i} step {step}: {err}"
                assert gd["tau"][i] == pytest.approx(ot[i], rel=1e-5, abs=1e-5 * (step + 1))
            prev_tau, prev_gpu_tau = ot.copy(), gd["tau"][: w.n].copy()
            # photons, particle by particle, as long as both sides created the same photons (a
            # rounding-level difference at one emitter's threshold renumbers all later photons):
            # momentum at creation, then the optical depth the pair rate wears down, until each
            # one converts (tau = +inf on both sides)
            if photons_aligned:
                gp = g.download()
                keep = np.isfinite(gp["tau"])  # converted photons stay as holes on the GPU
                gp = {k: v[keep] for k, v in gp.items()}
                if len(gp["id"]) != og.n or not np.array_equal(gp["id"], og.get("id")):
                    photons_aligned = False
                elif og.n:
                    ku, kt = og.u(), og.get("tau")
                    # momentum, once, at creation: k = xi gamma uhat, and xi follows eta, which the
                    # FP32 path evaluates from the field amplitude |E| = E0 env |cos phi|: its
                    # relative error is the FP32 phase error (below 1e-5 rad here: phases of a few
                    # hundred radians) times |d ln|E|/d phi|, large near a zero of the carrier or
                    # the envelope, on top of 1e-5 per step of the emitter's own drift
                    new = og.get("id") >= seen
                    if new.any():
                        errk = np.abs(gp["u"][new] - ku[new]).max(axis=1) / np.linalg.norm(ku[new], axis=1)
                        bar = 2e-5 * math.sqrt(step + 1) + 1e-5 * amplitude_slope(og.x()[new], ku[new], step * w.dt)
                        bad = np.flatnonzero(errk > bar)
                        assert len(bad) == 0, f"photon momenta, step {step}: {errk[bad][:5]} vs {bar[bad][:5]}"
                        seen = int(og.get("id").max()) + 1
                    np.testing.assert_allclose(gp["tau"], kt, rtol=1e-5, atol=1e-5 * (step + 1),
                                               err_msg=f"photon optical depths, step {step}")
                    photon_checks += og.n
                    aligned_steps += 1
    if prec == qed.MIXED:
        assert aligned_steps >= 20 and photon_checks > 2000, (aligned_steps, photon_checks)
    if prec == qed.FP64:
        assert pairs > 0
        # stable compaction removes the converted photons and keeps the survivors' order
        n_before = g.count()
        g.compact()
        assert g.count() == og.n < n_before
        compare_species(g.download(), og, w, w.n_steps, 1e-11, "photons after compaction")
        # stepping continues on the compacted arrays exactly like the oracle
        for step in range(w.n_steps, w.n_steps + 5):
            qed.run(lib_tables, [e, p, g], qp, step)
            o.step(orc_tables, opp, step, oe, op, og)
        gd = g.download()
        keep = np.isfinite(gd["tau"])
        compare_species({k: v[keep] for k, v in gd.items()}, og, w, w.n_steps + 5, 1e-11, "photons")
        compare_species(e.download(), oe, w, w.n_steps + 5, 1e-11, "electrons")
    qed.check([e, p, g])


@pytest.mark.parametrize("prec", [qed.FP64, qed.MIXED])
def test_resume_bit_identical_gpu(lib_tables, prec):
    # counter-based streams keyed by (seed, id, step): a run stopped, checkpointed into fresh
    # species and resumed equals the uninterrupted run bit for bit
    w = W.head_on(n=2500, a0=300.0, gamma_mean=3000.0, n_steps=30, meet_step=15, fwhm_s=8e-15, seed=12)
    qp = qparams(w)
    e, p, g, _ = make_gpu_species(w, prec)
    qed.run(lib_tables, [e, p, g], qp, 0, w.n_steps)
    straight = [s.save() for s in (e, p, g)]
    e, p, g, _ = make_gpu_species(w, prec)
    qed.run(lib_tables, [e, p, g], qp, 0, 13)
    ck = [s.save() for s in (e, p, g)]
    fresh = [qed.Species(k, prec, s.capacity, s.append_capacity) for k, s in
             ((qed.ELECTRON, e), (qed.POSITRON, p), (qed.PHOTON, g))]
    for s, c in zip(fresh, ck):
        s.restore(c)
    qed.run(lib_tables, fresh, qp, 13, w.n_steps - 13)
    resumed = [s.save() for s in fresh]
    assert fresh[2].count() > 0
    for a, b in zip(straight, resumed):
        assert np.array_equal(a, b)


def test_capacity_overflow_is_reported_not_fatal(lib_tables):
    w = W.uniform_b(n=5000, n_steps=5)
    e = qed.Species(qed.ELECTRON, qed.MIXED, 6000, 64)
    p = qed.Species(qed.POSITRON, qed.MIXED, 64, 64)
    g = qed.Species(qed.PHOTON, qed.MIXED, 1000, 8)  # far too small an append region
    e.upload(w.x, w.u)
    e.init_tau(1)
    qp = qparams(w)
    qp.make_pairs = False
    qed.run(lib_tables, [e, p, g], qp, 0, 3)
    with pytest.raises(qed.QedError) as ex:
        qed.check([e, p, g])
    assert ex.value.code == 3
    # the species stay usable
    qed.run(lib_tables, [e, p, g], qp, 3, 1)
    assert e.count() == 5000


@pytest.mark.parametrize("n", [0, 1, 31, 33])
def test_edge_sizes(lib_tables, n):
    w = W.uniform_b(n=max(n, 1), n_steps=3)
    e = qed.Species(qed.ELECTRON, qed.FP64, 64, 64)
    p = qed.Species(qed.POSITRON, qed.FP64, 64, 64)
    g = qed.Species(qed.PHOTON, qed.FP64, 256, 64)
    if n:
        e.upload(w.x[:n], w.u[:n], tau=np.zeros(n))  # tau = 0: every particle emits at once
    qed.run(lib_tables, [e, p, g], qparams(w), 0, 1)
    led = qed.read_ledger([e, p, g])
    assert led["emitted_n"] + led["dropped_n"] == n
    assert g.count() == led["emitted_n"]
    ids = g.download()["id"]
    assert np.array_equal(ids, np.arange(len(ids)))
    qed.check([e, p, g])
