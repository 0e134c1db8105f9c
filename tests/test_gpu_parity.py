"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Bars: bit-exact for cell coordinates, neighbour counts and neighbour sets;
1e-11 (normwise: max |gpu - oracle| / max |oracle| per field) after one Heun
step and for the right-hand side; 1e-8 over a full evolution.
"""
import numpy as np
import pytest

import gubser_viscous as VG
from oracle import oracle as O
from paper_2511_22852_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_STEP = 1e-11
TOL_EVOL = 1e-8


@pytest.fixture(scope="module")
def Bd():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_22852_gb300 import binding, build_lib
    build_lib.build()
    return binding


def relerr(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    den = np.max(np.abs(b)) if b.size else 1.0
    if den == 0.0:
        return float(np.max(np.abs(a))) if a.size else 0.0
    return float(np.max(np.abs(a - b)) / den)


def state_errors(g, run):
    st = g.read(("X", "U", "S", "BV", "PV"))
    y = run.y
    return {"x": relerr(st["X"], y[0:2]), "u": relerr(st["U"], y[2:4]), "S": relerr(st["S"], y[4]),
            "Bv": relerr(st["BV"], y[5]), "Pv": relerr(st["PV"], y[6:9])}


def _with_partons(ev, extent, dim, h=0.5, charges=0.0):
    """The event with seeded parton sources formed from just before its first stage to 8 steps in
    (charges > 0: each parton a light quark or antiquark carrying its (B, S, Q) times charges)."""
    ev.partons = I.parton_sources(12, (ev.tau0 - 0.5 * ev.dtau, ev.tau0 + 8 * ev.dtau), extent, dim,
                                  E_GeV=(0.1, 0.3), norm=0.42, h=h)
    if charges > 0.0:
        ev.partons.charges = I.parton_quark_charges(12, 13, charges)
    return ev


def _with_stop(ev, T_GeV):
    """The event with the stop temperature: particles colder than T_GeV stream freely."""
    ev.transport.T_stop_GeV = T_GeV
    return ev


def _with_dnmr(ev):
    """The event with the DNMR equations of motion (14-moment coefficients)."""
    ev.transport.dnmr = I.DNMR_14_MOMENT
    return ev


CASES = {
    "gubser": lambda: I.gubser_ideal_2p1(),
    "bsq_small": lambda: I.viscous_bsq_2p1(n_target=3000, R=3.0, n_hot=20),
    "blob_causal": lambda: I.smooth_blob_2p1(half_width=2.0, eos=I.CAUSAL_EOS),
    "bjorken": lambda: I.bjorken_lattice_2p1(n_side=21),
    "gubser_viscous": lambda: VG.gubser_viscous_2p1(VG.GubserODE(eta_over_s=0.2)),
    "bsq_small_dnmr": lambda: _with_dnmr(I.viscous_bsq_2p1(n_target=3000, R=3.0, n_hot=20)),
    "bsq_small_partons": lambda: _with_partons(I.viscous_bsq_2p1(n_target=3000, R=3.0, n_hot=20), 1.5, 2),
    "bsq_small_stop": lambda: _with_stop(I.viscous_bsq_2p1(n_target=3000, R=3.0, n_hot=20), 0.2),
}
def _blob3_jets():
    ev = I.smooth_blob_3d(milne=False, flow=0.3, eos=I.CAUSAL_EOS)
    ev.jets = I.jet_tracks(n_tracks=3, R=1.0, t0=ev.tau0, z_half=0.5, seed=7)
    return ev


CASES3 = {
    "blob3_milne": lambda: I.smooth_blob_3d(milne=True, flow=0.3),
    "blob3_cart": lambda: I.smooth_blob_3d(milne=False, flow=0.3, eos=I.CAUSAL_EOS),
    "bjorken3": lambda: I.bjorken_lattice_3p1(),
    "box_jet": lambda: I.uniform_box_3d(
        jets=I.JetTracks(tracks=np.array([[-0.6, 0.1, -0.05, 1.0, 0.0, 0.0, 1.0, 5.0 / I.HBARC]]), sigma=0.3)),
    "blob3_cart_jets": _blob3_jets,
    "gubser_shifted3": lambda: I.gubser_shifted_3p1(t0=2.0),
    "blob3_milne_dnmr": lambda: _with_dnmr(I.smooth_blob_3d(milne=True, flow=0.3)),
    "box_partons": lambda: _with_partons(I.uniform_box_3d(), 0.4, 3, h=0.3),
    "blob3_milne_partons": lambda: _with_partons(I.smooth_blob_3d(milne=True, flow=0.3), 0.3, 3),
}


def state_errors3(g, run):
    st = g.read(("X", "U", "S", "BV", "PV"))
    y = run.y
    return {"x": relerr(st["X"], y[0:3]), "u": relerr(st["U"], y[3:6]), "S": relerr(st["S"], y[6]),
            "Bv": relerr(st["BV"], y[7]), "Pv": relerr(st["PV"], y[8:13])}


@pytest.mark.parametrize("case", list(CASES3))
def test_3d_cells_neighbours_densities(Bd, case):
    ev = CASES3[case]()
    g = Bd.GpuEvent(ev, use_graph=False)
    f = g.read(("CELL", "NNB", "SIGMA_STAR", "S_DENS", "T", "P"))
    cc, _ = O.cell_coords(ev.x, ev.h)
    assert np.array_equal(f["CELL"], cc)
    pa, pb = g.neighbors()
    oa, ob = O.neighbors(ev.x, ev.h, "cells")
    assert np.array_equal(pa, oa) and np.array_equal(pb, ob)
    assert np.array_equal(f["NNB"], np.bincount(oa, minlength=ev.n))
    run = O.OracleRun.start(ev)
    aux, st = run.observe()
    assert relerr(f["SIGMA_STAR"], aux[O.AUX["sigstar"]]) < 1e-13
    assert relerr(f["S_DENS"], aux[O.AUX["s"]]) < 1e-13
    assert relerr(f["T"], aux[O.AUX["T"]]) < 1e-12 and relerr(f["P"], aux[O.AUX["p"]]) < 1e-12
    g.free()


@pytest.mark.parametrize("case", list(CASES3))
def test_3d_rates(Bd, case):
    ev = CASES3[case]()
    g = Bd.GpuEvent(ev, use_graph=False)
    r, grad = g.rates()
    run = O.OracleRun.start(ev)
    dydt, aux, ograd, st, wr = run.stage()
    for k in range(13):
        if not np.any(dydt[k]) and not np.any(r[k]):
            continue
        assert relerr(r[k], dydt[k]) < TOL_STEP, (k, relerr(r[k], dydt[k]))
    assert relerr(grad[0:9], ograd[0:9]) < TOL_STEP and relerr(grad[9:12], ograd[9:12]) < TOL_STEP
    g.free()


@pytest.mark.parametrize("case", list(CASES3))
def test_3d_step_and_evolution(Bd, case):
    ev = CASES3[case]()
    g = Bd.GpuEvent(ev, use_graph=True)
    g.step(1, sync=True)
    run = O.OracleRun.start(ev)
    run.step(1)
    errs = state_errors3(g, run)
    assert all(v < TOL_STEP for v in errs.values()), errs
    g.step(9, sync=True)
    run.step(9)
    errs = state_errors3(g, run)
    assert all(v < TOL_EVOL for v in errs.values()), errs
    t, ot = g.totals(), run.totals()
    assert abs(t["E"] / ot["E"] - 1) < TOL_EVOL
    g.free()


def test_3d_full_size_milne_event_one_step(Bd):
    """The 3+1D hyperbolic viscous BSQ event (about 10^6 particles), one Heun step."""
    ev = I.viscous_bsq_3p1()
    assert ev.n > 900000
    g = Bd.GpuEvent(ev, use_graph=True)
    g.step(1, sync=True)
    run = O.OracleRun.start(ev)
    run.step(1)
    errs = state_errors3(g, run)
    assert all(v < TOL_STEP for v in errs.values()), errs
    g.free()


@pytest.mark.parametrize("case", list(CASES))
def test_cells_and_neighbours_bit_exact(Bd, case):
    ev = CASES[case]()
    g = Bd.GpuEvent(ev, use_graph=False)
    f = g.read(("CELL", "NNB"))
    cc, _ = O.cell_coords(ev.x, ev.h)
    assert np.array_equal(f["CELL"], cc)
    pa, pb = g.neighbors()
    oa, ob = O.neighbors(ev.x, ev.h, "cells")
    assert np.array_equal(pa, oa) and np.array_equal(pb, ob)
    assert np.array_equal(f["NNB"], np.bincount(oa, minlength=ev.n))
    g.free()


def test_neighbours_random_and_boundary_points(Bd):
    for n, seed in [(700, 31), (1, 32), (2, 33)]:
        ev = I.bjorken_lattice_2p1(n_side=3, viscous=False)
        x = I.random_points(n, 2, 1.7, seed)
        ev.x, ev.u = x, np.zeros((2, n))
        ev.S, ev.Nq, ev.Bv, ev.Pv = np.ones(n), np.zeros((3, n)), np.zeros(n), np.zeros((3, n))
        g = Bd.GpuEvent(ev, use_graph=False)
        pa, pb = g.neighbors()
        oa, ob = O.neighbors(x, ev.h, "brute")
        assert np.array_equal(pa, oa) and np.array_equal(pb, ob)
        g.free()
    # particles exactly on cell faces and pairs exactly at r = 2h (dyadic coordinates)
    h = 0.3125
    two_h = 2 * h
    pts = np.array([(0.0, 0.0), (two_h, 0.0), (0.0, two_h), (2 * two_h, two_h), (0.25, 0.375),
                    (0.25 + two_h, 0.375), (1.0, 1.0), (1.375, 1.5), (1.0, 1.0)]).T.copy()
    ev = I.bjorken_lattice_2p1(n_side=3, viscous=False, h=h)
    n = pts.shape[1]
    ev.x, ev.u = pts, np.zeros((2, n))
    ev.S, ev.Nq, ev.Bv, ev.Pv = np.ones(n), np.zeros((3, n)), np.zeros(n), np.zeros((3, n))
    g = Bd.GpuEvent(ev, use_graph=False)
    pa, pb = g.neighbors()
    oa, ob = O.neighbors(pts, h, "brute")
    assert np.array_equal(pa, oa) and np.array_equal(pb, ob)
    g.free()


@pytest.mark.parametrize("case", list(CASES))
def test_densities_and_eos(Bd, case):
    ev = CASES[case]()
    g = Bd.GpuEvent(ev, use_graph=False)
    f = g.read(("SIGMA_STAR", "S_DENS", "N_DENS", "T", "MU", "P", "E", "STATUS"))
    run = O.OracleRun.start(ev)
    aux, st = run.observe()
    A = O.AUX
    assert relerr(f["SIGMA_STAR"], aux[A["sigstar"]]) < 1e-13
    assert relerr(f["S_DENS"], aux[A["s"]]) < 1e-13
    if np.any(aux[A["nB"]]):
        assert relerr(f["N_DENS"], aux[A["nB"]:A["nQ"] + 1]) < 1e-13
    assert relerr(f["T"], aux[A["T"]]) < 1e-12
    assert relerr(f["P"], aux[A["p"]]) < 1e-12
    assert relerr(f["E"], aux[A["e"]]) < 1e-12
    if np.any(aux[A["muB"]]):
        assert relerr(f["MU"], aux[A["muB"]:A["muQ"] + 1]) < 1e-10
    # same EoS branch (table / closed form) for every particle
    branch = Bd.PST_FALLBACK | Bd.PST_OUT_OF_TABLE | Bd.PST_NOCONV
    assert np.array_equal(f["STATUS"] & branch, st & branch)
    g.free()


@pytest.mark.parametrize("case", list(CASES))
def test_rates(Bd, case):
    ev = CASES[case]()
    if case == "bsq_small":  # start from a flowing, viscous state
        run0 = O.OracleRun.start(ev)
        run0.step(20)
        ev.x, ev.u, ev.S = run0.y[0:2].copy(), run0.y[2:4].copy(), run0.y[4].copy()
        ev.Bv, ev.Pv, ev.tau0 = run0.y[5].copy(), run0.y[6:9].copy(), run0.tau
    g = Bd.GpuEvent(ev, use_graph=False)
    r, grad = g.rates()
    run = O.OracleRun.start(ev)
    dydt, aux, ograd, st, wr = run.stage()
    names = ["x", "y", "ux", "uy", "S", "Bv", "Pxx", "Pxy", "Pyy"]
    for k, nm in enumerate(names):
        if not np.any(dydt[k]) and not np.any(r[k]):
            continue
        assert relerr(r[k], dydt[k]) < TOL_STEP, (nm, relerr(r[k], dydt[k]))
    assert relerr(grad[0:4], ograd[0:4]) < TOL_STEP
    assert relerr(grad[4:6], ograd[4:6]) < TOL_STEP
    g.free()


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("graph", [False, True])
def test_one_heun_step(Bd, case, graph):
    ev = CASES[case]()
    g = Bd.GpuEvent(ev, use_graph=graph)
    g.step(1, sync=True)
    run = O.OracleRun.start(ev)
    run.step(1)
    errs = state_errors(g, run)
    assert all(v < TOL_STEP for v in errs.values()), errs
    t = g.totals()
    assert abs(t["tau"] - run.tau) < 1e-14 and t["steps"] == 1
    g.free()


def test_graph_and_stream_launches_are_bitwise_identical(Bd):
    ev = CASES["bsq_small"]()
    a = Bd.GpuEvent(ev, use_graph=True)
    b = Bd.GpuEvent(ev, use_graph=False)
    a.step(5)
    b.step(5)
    fa, fb = a.read(), b.read()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k
    a.free()
    b.free()


@pytest.mark.parametrize("case,nsteps", [("gubser", 60), ("bsq_small", 150), ("blob_causal", 100),
                                        ("bsq_small_dnmr", 100), ("bsq_small_partons", 20), ("bsq_small_stop", 100)])
def test_evolution(Bd, case, nsteps):
    ev = CASES[case]()
    g = Bd.GpuEvent(ev, use_graph=True)
    g.step(nsteps, sync=True)
    run = O.OracleRun.start(ev)
    run.step(nsteps)
    errs = state_errors(g, run)
    assert all(v < TOL_EVOL for v in errs.values()), errs
    t = g.totals()
    ot = run.totals()
    assert abs(t["E"] / ot["E"] - 1) < TOL_EVOL and abs(t["work"] / max(ot["work"], 1e-300) - 1) < TOL_EVOL
    g.free()


def test_full_size_viscous_bsq_one_step(Bd):
    """The 40k-particle viscous BSQ event in the launch configuration the benchmark times."""
    ev = I.viscous_bsq_2p1()
    assert 39000 < ev.n < 41000
    g = Bd.GpuEvent(ev, use_graph=True)
    g.step(1, sync=True)
    run = O.OracleRun.start(ev)
    run.step(1)
    errs = state_errors(g, run)
    assert all(v < TOL_STEP for v in errs.values()), errs
    f = g.read(("T", "STATUS"))
    aux, st = run.observe()
    assert relerr(f["T"], aux[O.AUX["T"]]) < 1e-12
    g.free()


def test_ideal_invariants_bitwise(Bd):
    ev = I.gubser_ideal_2p1()
    g = Bd.GpuEvent(ev)
    t0 = g.totals()
    g.step(30, sync=True)
    f = g.read(("S", "NQ"))
    assert np.array_equal(f["S"], ev.S) and np.array_equal(f["NQ"], ev.Nq)
    ev2 = I.viscous_bsq_2p1(n_target=3000, R=3.0, n_hot=20)
    g2 = Bd.GpuEvent(ev2)
    t0 = g2.totals()
    g2.step(40, sync=True)
    t1 = g2.totals()
    assert np.array_equal(t0["N"], t1["N"])  # charge totals bitwise constant
    assert t1["S"] > t0["S"]  # second law
    g.free()
    g2.free()


def test_resume_from_read_state_is_bitwise(Bd):
    ev = CASES["bsq_small"]()
    a = Bd.GpuEvent(ev)
    a.step(10, sync=True)
    ref = a.read()
    b = Bd.GpuEvent(ev)
    b.step(5, sync=True)
    mid = b.read(("X", "U", "S", "NQ", "BV", "PV", "GUESS"))
    tau_mid = b.totals()["tau"]
    assert np.all(mid["GUESS"][0] > 0)  # every particle's EoS came from the table
    ev2 = CASES["bsq_small"]()
    ev2.x, ev2.u, ev2.S, ev2.Bv, ev2.Pv, ev2.tau0 = mid["X"], mid["U"], mid["S"], mid["BV"], mid["PV"], tau_mid
    c = Bd.GpuEvent(ev2)
    c.write_state(guess=mid["GUESS"])  # the EoS warm start is part of the evolved state
    c.step(5, sync=True)
    out = c.read()
    for k in ref:
        assert np.array_equal(out[k], ref[k]), k
    # write_state into an existing event gives the same
    b.write_state(x=mid["X"], u=mid["U"], S=mid["S"], Bv=mid["BV"], Pv=mid["PV"], guess=mid["GUESS"])
    b.step(5, sync=True)
    for k, v in b.read().items():
        assert np.array_equal(v, ref[k]), k
    for e in (a, b, c):
        e.free()


def test_warm_start_matches_oracle_over_steps(Bd):
    """The carried EoS warm start: after several steps the GPU guess equals the oracle's."""
    ev = CASES["bsq_small"]()
    g = Bd.GpuEvent(ev)
    g.step(3, sync=True)
    run = O.OracleRun.start(ev)
    run.step(3)
    gs = g.read(("GUESS",))["GUESS"]
    assert np.array_equal(gs[0] > 0, run.guess[0] > 0)
    assert relerr(gs, run.guess) < TOL_STEP
    g.free()


def test_eos_stall_at_table_edge_ends_fast(Bd):
    """A warm start inside the table whose root lies below the table's lowest T: the clamped
    Newton walks to the edge and stalls there; the failed line search ends it (a few
    iterations plus 9 trials, where running on took 30 x 9), and the closed form takes over,
    flagged out-of-table -- as in the oracle."""
    ev = CASES["bsq_small"]()
    hot = Bd.GpuEvent(ev)
    hot.step(1, sync=True)
    gs = hot.read(("GUESS",))["GUESS"]
    hot.free()
    assert np.all(gs[0] > 0)
    ev2 = CASES["bsq_small"]()
    # s -> 1e-5 s puts every particle below T = 0.05 GeV (s ~ f(T) T^3, f from 2.8 down to 0.3)
    ev2.S = ev2.S * 1e-5
    ev2.Nq = ev2.Nq * 1e-5
    g = Bd.GpuEvent(ev2)
    g.write_state(guess=gs)
    t0 = g.totals()
    g.step(1, sync=True)
    t1 = g.totals()
    assert t1["eos_work"][0] - t0["eos_work"][0] <= 50 * ev2.n
    run = O.OracleRun.start(ev2)
    run.guess[:] = gs
    run.step(1)
    aux, st = run.observe()
    f = g.read(("X", "U", "S", "T", "STATUS"))
    assert np.array_equal(f["STATUS"] & Bd.PST_OUT_OF_TABLE, st.astype(np.uint32) & Bd.PST_OUT_OF_TABLE)
    assert np.all(f["STATUS"] & Bd.PST_OUT_OF_TABLE)
    assert relerr(f["X"], run.y[:2]) < TOL_STEP and relerr(f["U"], run.y[2:4]) < TOL_STEP
    assert relerr(f["T"], aux[O.AUX["T"]]) < TOL_STEP
    g.free()


def test_edge_cases_and_errors(Bd):
    # empty event: every call succeeds
    ev = I.bjorken_lattice_2p1(n_side=3, viscous=False)
    ev0 = I.bjorken_lattice_2p1(n_side=3, viscous=False)
    n = 0
    ev0.x, ev0.u, ev0.S = np.zeros((2, n)), np.zeros((2, n)), np.zeros(n)
    ev0.Nq, ev0.Bv, ev0.Pv = np.zeros((3, n)), np.zeros(n), np.zeros((3, n))
    g0 = Bd.GpuEvent(ev0)
    g0.step(3, sync=True)
    assert g0.read()["S"].size == 0
    assert g0.totals()["steps"] == 0
    g0.free()
    # a single particle: its own neighbour only; runs
    ev1 = I.bjorken_lattice_2p1(n_side=1, viscous=False)
    g1 = Bd.GpuEvent(ev1)
    g1.step(2, sync=True)
    assert g1.read(("NNB",))["NNB"][0] == 1
    g1.free()
    # non-finite position
    bad = I.bjorken_lattice_2p1(n_side=3, viscous=False)
    bad.x[0, 4] = np.nan
    with pytest.raises(Bd.SphError) as e:
        Bd.GpuEvent(bad)
    assert e.value.code == Bd.SPH_ERR_NONFINITE
    # invalid arguments
    g = Bd.GpuEvent(ev)
    with pytest.raises(Bd.SphError) as e:
        Bd.sph_step(g.h, -1, 0)
    assert e.value.code == Bd.SPH_ERR_ARG
    g.free()
    bad2 = I.bjorken_lattice_2p1(n_side=3, viscous=False)
    bad2.dtau = 0.0
    with pytest.raises(Bd.SphError) as e:
        Bd.GpuEvent(bad2)
    assert e.value.code == Bd.SPH_ERR_ARG


def test_infeasible_charges_are_flagged(Bd):
    """Coherent n_q = 0.1 s: no EoS solution for hot particles -- flagged, no hang, the particles
    frozen, and fatal when the caller's policy says so."""
    ev = I.viscous_bsq_2p1(n_target=1500, R=2.2, n_hot=12, charge_frac=0.1, coherent_charges=True)
    g = Bd.GpuEvent(ev)
    f = g.read(("STATUS",))
    run = O.OracleRun.start(ev)
    aux, st = run.observe()
    assert np.any(st & O.ST_NOCONV)
    assert np.array_equal(f["STATUS"] & Bd.PST_NOCONV, st & O.ST_NOCONV)
    # the step runs; frozen particles keep their state; the result matches the oracle
    g.step(2, sync=True)
    run.step(2)
    s = g.read(("S", "U"))
    assert np.all(np.isfinite(s["S"])) and np.all(np.isfinite(s["U"]))
    assert relerr(s["S"], run.y[4]) < TOL_STEP and relerr(s["U"], run.y[2:4]) < TOL_STEP
    g.free()
    g = Bd.GpuEvent(ev, fatal_mask=Bd.PST_NOCONV)
    with pytest.raises(Bd.SphError) as e:
        g.step(1, sync=True)
    assert e.value.code == Bd.SPH_ERR_EOS_NOCONV
    g.free()


def test_backup_eos_takes_the_infeasible_particles(Bd):
    """With the conformal-diagonal backup on, the particles neither the table nor the closed form
    inverts get the backup's solution (flagged BACKUP, not NOCONV) and evolve; every field follows
    the oracle over the steps, T and mu included."""
    ev = I.viscous_bsq_2p1(n_target=1500, R=2.2, n_hot=12, charge_frac=0.1, coherent_charges=True)
    ev.eos_backup = (0.165, 0.45)
    g = Bd.GpuEvent(ev)
    f = g.read(("STATUS", "T", "MU"))
    run = O.OracleRun.start(ev)
    aux, st = run.observe()
    assert np.any(st & O.ST_BACKUP) and not np.any(st & O.ST_NOCONV)
    assert np.array_equal(f["STATUS"] & Bd.PST_BACKUP, st & O.ST_BACKUP)
    assert relerr(f["T"], aux[O.AUX["T"]]) < TOL_STEP and relerr(f["MU"], aux[O.AUX["muB"]:O.AUX["muQ"] + 1]) < TOL_STEP
    g.step(1, sync=True)
    run.step(1)
    errs = state_errors(g, run)
    assert all(v < TOL_STEP for v in errs.values()), errs
    g.step(9, sync=True)
    run.step(9)
    errs = state_errors(g, run)
    assert all(v < TOL_EVOL for v in errs.values()), errs
    g.free()


TOL_MIXED = 1e-5  # the mixed-precision form against the FP64 oracle (T, mu, densities)


def oracle_nnb_at(ev, X):
    """The oracle's neighbour counts (exact FP64 test r < 2h, self pair included) with the
    particles at positions X (the rest of the state is irrelevant to them).  The mixed form's
    positions differ from the FP64 evolution's by ~1e-7 relative, so a pair that sits at the
    kernel support (lattice spacings that divide 2h) may legitimately flip between the two
    evolutions; its decisions must be exact for its own positions."""
    r = O.OracleRun.start(ev)
    r.y[0:X.shape[0]] = X
    aux, _ = r.observe()
    return aux[O.AUX["nnb"]].astype(np.int32)


@pytest.mark.parametrize("case,nsteps", [("bsq_small", 50), ("gubser", 60), ("blob_causal", 40)])
def test_mixed_precision_against_fp64_oracle(Bd, case, nsteps):
    """SPH_MIXED: FP32 neighbour passes, FP64 EoS/EoM -- within 1e-5 of the FP64 oracle on T, mu
    and the densities after many steps; neighbour counts exactly those of the FP64 test."""
    ev = CASES[case]()
    g = Bd.GpuEvent(ev, precision=Bd.SPH_MIXED)
    run = O.OracleRun.start(ev)
    aux0, _ = run.observe()
    assert np.array_equal(g.read(("NNB",))["NNB"], aux0[O.AUX["nnb"]].astype(np.int32))
    g.step(nsteps, sync=True)
    run.step(nsteps)
    f = g.read(("X", "T", "MU", "S_DENS", "N_DENS", "NNB"))
    aux, _ = run.observe()
    A = O.AUX
    assert np.array_equal(f["NNB"], oracle_nnb_at(ev, f["X"]))
    assert relerr(f["T"], aux[A["T"]]) < TOL_MIXED
    assert relerr(f["S_DENS"], aux[A["s"]]) < TOL_MIXED
    if np.any(aux[A["nB"]]):
        assert relerr(f["N_DENS"], aux[A["nB"]:A["nQ"] + 1]) < TOL_MIXED
        assert relerr(f["MU"], aux[A["muB"]:A["muQ"] + 1]) < TOL_MIXED
    g.free()


def test_mixed_precision_full_size_event(Bd):
    ev = I.viscous_bsq_2p1()
    g = Bd.GpuEvent(ev, precision=Bd.SPH_MIXED)
    g.step(10, sync=True)
    run = O.OracleRun.start(ev)
    run.step(10)
    f = g.read(("T", "MU", "S_DENS"))
    aux, _ = run.observe()
    A = O.AUX
    assert relerr(f["T"], aux[A["T"]]) < TOL_MIXED and relerr(f["S_DENS"], aux[A["s"]]) < TOL_MIXED
    assert relerr(f["MU"], aux[A["muB"]:A["muQ"] + 1]) < TOL_MIXED
    g.free()


@pytest.mark.parametrize("case", [c for c in CASES3 if not c.startswith("box")])
def test_mixed_precision_3d_against_fp64_oracle(Bd, case):
    """SPH_MIXED in 3+1D: FP32 27-cell neighbour passes, FP64 EoS/EoM -- within 1e-5 of the FP64
    oracle after 10 steps, neighbour counts exact.  The uniform boxes are left out: their
    spacing divides 2h, so pairs start exactly at the kernel support, and the mixed evolution's
    ~1e-7 position differences from the FP64 one legitimately flip some of them."""
    ev = CASES3[case]()
    g = Bd.GpuEvent(ev, precision=Bd.SPH_MIXED)
    run = O.OracleRun.start(ev)
    g.step(10, sync=True)
    run.step(10)
    f = g.read(("X", "U", "T", "MU", "S_DENS", "N_DENS", "NNB"))
    aux, _ = run.observe()
    A = O.AUX
    assert np.array_equal(f["NNB"], oracle_nnb_at(ev, f["X"]))
    assert relerr(f["X"], run.y[0:3]) < TOL_MIXED and relerr(f["U"], run.y[3:6]) < TOL_MIXED
    assert relerr(f["T"], aux[A["T"]]) < TOL_MIXED
    assert relerr(f["S_DENS"], aux[A["s"]]) < TOL_MIXED
    if np.any(aux[A["nB"]]):
        assert relerr(f["N_DENS"], aux[A["nB"]:A["nQ"] + 1]) < TOL_MIXED
        assert relerr(f["MU"], aux[A["muB"]:A["muQ"] + 1]) < TOL_MIXED
    g.free()


def test_mixed_precision_3d_full_size_event(Bd):
    """The 3+1D hyperbolic viscous BSQ event (about 10^6 particles) in the mixed form, one step."""
    ev = I.viscous_bsq_3p1()
    g = Bd.GpuEvent(ev, precision=Bd.SPH_MIXED)
    g.step(1, sync=True)
    run = O.OracleRun.start(ev)
    run.step(1)
    f = g.read(("X", "U", "T", "S_DENS", "NNB"))
    aux, _ = run.observe()
    A = O.AUX
    assert np.array_equal(f["NNB"], oracle_nnb_at(ev, f["X"]))
    assert relerr(f["U"], run.y[3:6]) < TOL_MIXED and relerr(f["T"], aux[A["T"]]) < TOL_MIXED
    assert relerr(f["S_DENS"], aux[A["s"]]) < TOL_MIXED
    assert g.totals()["shell_tests"] >= 0
    g.free()


def _fo_compare(recs, ids, orecs, oids):
    assert np.array_equal(ids, oids)
    # ordering in both: (tau, id); state and thermodynamics columns to the step tolerance
    for c in list(range(0, 15)):
        assert relerr(recs[:, c], orecs[:, c]) < TOL_STEP, c
    # the normal and the element: well conditioned away from light-like normals
    nn = np.abs(orecs[:, 15] ** 2 - orecs[:, 16] ** 2 - orecs[:, 17] ** 2)
    ok = np.abs(orecs[:, 15]) > 0  # every element
    N = recs[:, 15:18] / np.linalg.norm(recs[:, 15:18], axis=1)[:, None]
    ON = orecs[:, 15:18] / np.linalg.norm(orecs[:, 15:18], axis=1)[:, None]
    assert np.max(np.abs(N - ON)[ok]) < 1e-9
    good = nn > 1e-3
    assert relerr(recs[good, 19], orecs[good, 19]) < 1e-8


@pytest.mark.parametrize("case", ["gubser", "gubser_viscous", "blob_causal"])
def test_freezeout_surface_matches_oracle(Bd, case):
    """Freeze-out surface elements at constant e: the same particles cross in the same steps,
    with the oracle's normals and element sizes."""
    ev = CASES[case]()
    run = O.OracleRun.start(ev)
    aux0, _ = run.observe()
    e0 = aux0[O.AUX["e"]]
    # a surface that sweeps through the fluid as it cools, in the middle of a clear gap between
    # particles' values (mirror particles of a symmetric lattice differ by rounding only, and a
    # particle within rounding of e_fo would cross or not by rounding)
    se = np.sort(e0)
    k = int(0.6 * len(se))
    while se[k + 1] - se[k] < 1e-6 * se[k]:
        k += 1
    e_fo = 0.5 * float(se[k] + se[k + 1])
    nsteps = 40
    orecs, oids = run.evolve_freezeout(nsteps, e_fo)
    assert len(oids) > 20
    g = Bd.GpuEvent(ev)
    g.freezeout_setup(e_fo, 100000)
    g.step(nsteps + 1, sync=True)  # crossings of step k are found by step k + 1's first stage
    recs, ids = g.read_freezeout()
    _fo_compare(recs, ids, orecs, oids)
    g.free()


# charge scales: full quark charges would push particles of the small BSQ event's cold edge out
# of the EoS's reach (no solution: frozen particles, whose set a rounding difference can change);
# a tenth of a quark's charge per parton keeps every particle solvable
CHARGED = {
    "bsq_small_partons_q": (lambda: _with_partons(I.viscous_bsq_2p1(n_target=3000, R=3.0, n_hot=20), 1.5, 2,
                                                  charges=0.1), state_errors),
    "box_partons_q": (lambda: _with_partons(I.uniform_box_3d(), 0.4, 3, h=0.3, charges=1.0), state_errors3),
    "blob3_milne_partons_q": (lambda: _with_partons(I.smooth_blob_3d(milne=True, flow=0.3), 0.3, 3, charges=1.0),
                              state_errors3),
}


@pytest.mark.parametrize("case", list(CHARGED))
def test_parton_charge_sources(Bd, case):
    """Charge sources of the partons (I_q): the particles' charges evolve (dN_q/dx0 = sqrt(-g)
    I_q/sigma*, Heun) with the entropy and enthalpy couplings; charges, state and thermodynamics
    match the oracle over 10 steps to the evolution tolerance, and the deposit is visible."""
    make, errs = CHARGED[case]
    ev = make()
    g = Bd.GpuEvent(ev)
    run = O.OracleRun.start(ev)
    N0 = run.Nq.sum(axis=1).copy()
    g.step(10, sync=True)
    run.step(10)
    assert np.abs(run.Nq.sum(axis=1) - N0).max() > 1e-2 * np.abs(ev.partons.charges).sum()  # charge deposited
    assert not run.status_or & 4  # every particle solvable (no frozen particles)
    f = g.read(("NQ", "T", "S_DENS"))
    aux, _ = run.observe()
    assert relerr(f["NQ"], run.Nq) < TOL_EVOL
    for k, e in errs(g, run).items():
        assert e < TOL_EVOL, (k, e)
    assert relerr(f["T"], aux[O.AUX["T"]]) < TOL_EVOL and relerr(f["S_DENS"], aux[O.AUX["s"]]) < TOL_EVOL
    g.free()


def test_3d_viscous_gubser_matches_oracle(Bd):
    """The boost-invariant shear-viscous Gubser flow on a 3+1D Milne lattice (the oracle's 3D
    off-diagonal shear pin, 28,577 particles): the FP64 GPU step matches the oracle after one step
    (1e-11) and over 10 steps (1e-8), shear components pi^{xx}, pi^{xy}, pi^{yy} and the zero
    eta components included."""
    ev = VG.gubser_viscous_3p1(VG.GubserODE(eta_over_s=0.2), n_side=41, half_width=4.0, eta_half=1.6)
    g = Bd.GpuEvent(ev)
    run = O.OracleRun.start(ev)
    g.step(1, sync=True)
    run.step(1)
    for k, e in state_errors3(g, run).items():
        assert e < TOL_STEP, (k, e)
    g.step(9, sync=True)
    run.step(9)
    for k, e in state_errors3(g, run).items():
        assert e < TOL_EVOL, (k, e)
    f = g.read(("T",))
    aux, _ = run.observe()
    assert relerr(f["T"], aux[O.AUX["T"]]) < TOL_EVOL
    g.free()


def _gap_e_fo(e0, quantile=0.6):
    """A surface value in the middle of a clear gap between particles' initial values, so that no
    particle sits within rounding of it."""
    se = np.sort(e0)
    k = int(quantile * len(se))
    while se[k + 1] - se[k] < 1e-6 * se[k]:
        k += 1
    return 0.5 * float(se[k] + se[k + 1])


@pytest.mark.parametrize("case", ["gubser_shifted3", "blob3_milne", "blob3_cart"])
def test_freezeout_surface_3d_matches_oracle(Bd, case):
    """3+1D freeze-out elements (Milne: eta_s and u^eta components, n_eta normalised with
    g^{eta eta} = -1/tau^2; Cartesian): the same particles cross in the same steps, with the
    oracle's four-component normals and element sizes."""
    ev = CASES3[case]()
    run = O.OracleRun.start(ev)
    aux0, _ = run.observe()
    e_fo = _gap_e_fo(aux0[O.AUX["e"]])
    nsteps = 20
    orecs, oids = run.evolve_freezeout(nsteps, e_fo)
    assert len(oids) > 100
    g = Bd.GpuEvent(ev)
    g.freezeout_setup(e_fo, 100000)
    g.step(nsteps + 1, sync=True)  # crossings of step k are found by step k + 1's first stage
    recs, ids = g.read_freezeout()
    g.free()
    assert np.array_equal(ids, oids)
    for c in range(0, 15):  # tau, x^1..3, u^0..3, T, mu, e, p, s
        assert relerr(recs[:, c], orecs[:, c]) < TOL_STEP, c
    assert np.abs(orecs[:, 3]).max() > 0 and np.abs(orecs[:, 7]).max() > 0  # third axis exercised
    N = recs[:, 15:19] / np.linalg.norm(recs[:, 15:19], axis=1)[:, None]
    ON = orecs[:, 15:19] / np.linalg.norm(orecs[:, 15:19], axis=1)[:, None]
    assert np.max(np.abs(N - ON)) < 1e-9
    assert relerr(recs[:, 19], orecs[:, 19]) < 1e-8
    assert relerr(recs[:, 20:24], orecs[:, 20:24]) < 1e-8


def test_stress_event_fp64_and_mixed(Bd):
    """The stress configuration at full size (about 8 10^6 particles, Cartesian 3+1D, 10 jet
    tracks, 128 x 64^3 table), one Heun step in each form: the same neighbour counts, T and u
    within 1e-5 of each other, and no particle without an EoS solution."""
    ev = I.stress_cartesian_3d()
    assert ev.n > 7_000_000
    out = {}
    for prec in (Bd.SPH_FP64, Bd.SPH_MIXED):
        g = Bd.GpuEvent(ev, precision=prec)
        g.step(1, sync=True)
        out[prec] = g.read(("U", "T", "NNB", "STATUS"))
        g.free()
    a, b = out[Bd.SPH_FP64], out[Bd.SPH_MIXED]
    assert np.array_equal(a["NNB"], b["NNB"])
    assert relerr(b["T"], a["T"]) < TOL_MIXED and relerr(b["U"], a["U"]) < TOL_MIXED
    bad = Bd.PST_NOCONV | Bd.PST_NONFINITE
    assert not np.any(a["STATUS"] & bad) and not np.any(b["STATUS"] & bad)
    assert np.max(np.abs(a["U"])) > 0  # the jets and pressure gradients moved the fluid


def test_offline_inverter_matches_oracle(Bd):
    """SPH_EOS_OFFLINE: the inverted table built on the device by the online root finder, then
    interpolated -- the oracle's offline inverter on the same grid, to the step and evolution
    tolerances; and the mode takes effect (the results differ from the online inversion)."""
    ev = I.smooth_blob_2p1(half_width=2.0, eos=I.CAUSAL_EOS)
    ev.inverse = I.InverseGrid(per_decade=90, nx=17, xmax=0.12)
    g = Bd.GpuEvent(ev)
    run = O.OracleRun.start(ev)
    aux, _ = run.observe()
    f = g.read(("T", "MU", "P"))
    A = O.AUX
    assert relerr(f["T"], aux[A["T"]]) < TOL_STEP and relerr(f["P"], aux[A["p"]]) < TOL_STEP
    assert relerr(f["MU"], aux[A["muB"]:A["muQ"] + 1]) < TOL_STEP
    online = O.OracleRun.start(I.smooth_blob_2p1(half_width=2.0, eos=I.CAUSAL_EOS)).observe()[0]
    assert relerr(f["T"], online[A["T"]]) > 1e-6
    g.step(1, sync=True)
    run.step(1)
    st = g.read(("X", "U", "S", "BV", "PV"))
    assert relerr(st["U"], run.y[2:4]) < TOL_STEP and relerr(st["S"], run.y[4]) < TOL_STEP
    g.step(9, sync=True)
    run.step(9)
    st = g.read(("X", "U", "S", "BV", "PV"))
    assert relerr(st["U"], run.y[2:4]) < TOL_EVOL and relerr(st["PV"], run.y[6:9]) < TOL_EVOL
    g.free()
    ev2 = I.smooth_blob_2p1(half_width=2.0, eos=I.CAUSAL_EOS)
    g2 = Bd.GpuEvent(ev2)
    with pytest.raises(Bd.SphError) as e:
        Bd.sph_set_eos_mode(g2.h, Bd.SPH_EOS_OFFLINE)
    assert e.value.code == Bd.SPH_ERR_STATE
    g2.free()


def test_wait_limit_reports_timeout(Bd, monkeypatch):
    """Failure detection without a GPU fault: a host wait limit far below the step's duration
    makes a synchronous step return SPH_ERR_TIMEOUT (the device finishes its work normally; the
    handle stays usable and is freed after its stream drains)."""
    monkeypatch.setenv("SPH_WAIT_LIMIT_S", "0.000001")
    ev = I.viscous_bsq_2p1()
    g = Bd.GpuEvent(ev)
    with pytest.raises(Bd.SphError) as e:
        g.step(20, sync=True)
    assert e.value.code == Bd.SPH_ERR_TIMEOUT
    g.free()
    monkeypatch.delenv("SPH_WAIT_LIMIT_S")
    g2 = Bd.GpuEvent(ev)  # the default limit: the same call completes
    g2.step(2, sync=True)
    assert g2.totals()["steps"] == 2
    g2.free()


def test_pair_lists_match_per_particle_passes(Bd, monkeypatch):
    """Plain 2D: the neighbour passes over half-pair lists (the kernel of each pair evaluated once
    and added to both particles) and the per-particle passes (SPH_PAIR_LISTS=0) form the same sums
    in another order: states agree to rounding, pair counts exactly, and both follow the oracle."""
    ev = CASES["bsq_small"]()
    g = Bd.GpuEvent(ev)
    g.step(5, sync=True)
    monkeypatch.setenv("SPH_PAIR_LISTS", "0")
    g0 = Bd.GpuEvent(ev)
    g0.step(5, sync=True)
    names = ("X", "U", "S", "BV", "PV", "T", "SIGMA_STAR")
    a, b = g.read(names), g0.read(names)
    for k in names:
        assert relerr(a[k], b[k]) < 1e-13, (k, relerr(a[k], b[k]))
    t, t0 = g.totals(), g0.totals()
    assert t["pair_overflows"] == 0 and t0["pair_overflows"] == 0
    assert t["kernel_launches"] == 5 * 38 and t0["kernel_launches"] == 5 * 26  # 19 and 13 per stage
    # the lists were sized by one read-out evaluation (its pairs are counted): compare one step
    g.step(1, sync=True)
    g0.step(1, sync=True)
    assert g.totals()["pairs"] - t["pairs"] == g0.totals()["pairs"] - t0["pairs"] > 0
    run = O.OracleRun.start(ev)
    run.step(6)
    errs = state_errors(g, run)
    assert all(v < TOL_EVOL for v in errs.values()), errs
    g.free()
    g0.free()


def test_pair_list_overflow_falls_back_then_grows(Bd, monkeypatch):
    """Lists allocated far too small (64 entries against ~330,000 needed): the stage runs the
    per-particle passes (the result still follows the oracle), the overflow is counted, and the
    allocation grows before the next step, after which the stages run on the lists."""
    monkeypatch.setenv("SPH_PAIR_TOTAL", "64")
    ev = CASES["bsq_small"]()
    g = Bd.GpuEvent(ev)
    run = O.OracleRun.start(ev)
    g.step(1, sync=True)
    run.step(1)
    assert g.totals()["pair_overflows"] >= 2  # both stages (and the read-out evaluation of totals)
    errs = state_errors(g, run)
    assert all(v < TOL_STEP for v in errs.values()), errs
    seen = []
    for _ in range(4):
        g.step(1, sync=True)
        seen.append(g.totals()["pair_overflows"])
    run.step(4)
    assert seen[-1] == seen[-2] == seen[-3], seen  # the grown lists fit
    errs = state_errors(g, run)
    assert all(v < TOL_EVOL for v in errs.values()), errs
    g.free()


def test_pair_list_rows_resize_on_the_device(Bd, monkeypatch):
    """Rows with no margin over the previous stage's neighbour counts: a particle whose count
    grew overflows its row, the stage runs the per-particle passes and records the new counts,
    which size the next stage's rows -- no host involvement; every stage follows the oracle."""
    monkeypatch.setenv("SPH_PAIR_MARGIN", "0")
    ev = CASES["bsq_small"]()
    g = Bd.GpuEvent(ev)
    g.step(10, sync=True)
    run = O.OracleRun.start(ev)
    run.step(10)
    errs = state_errors(g, run)
    assert all(v < TOL_EVOL for v in errs.values()), errs
    t = g.totals()
    assert t["pair_overflows"] <= 21  # at most every stage and the read-out
    g.free()


def test_pair_lists_3d_match_per_particle_passes(Bd, monkeypatch):
    """Plain 3D: the half-pair-list passes against the per-particle passes (SPH_PAIR_LISTS=0):
    the same sums in another order -- states within rounding, equal pair counts per step, and
    both on the oracle."""
    ev = CASES3["blob3_milne"]()
    g = Bd.GpuEvent(ev)
    g.step(4, sync=True)
    monkeypatch.setenv("SPH_PAIR_LISTS", "0")
    g0 = Bd.GpuEvent(ev)
    g0.step(4, sync=True)
    names = ("X", "U", "S", "BV", "PV", "T", "SIGMA_STAR")
    a, b = g.read(names), g0.read(names)
    for k in names:
        assert relerr(a[k], b[k]) < 1e-13, (k, relerr(a[k], b[k]))
    t, t0 = g.totals(), g0.totals()
    assert t["pair_overflows"] == 0
    g.step(1, sync=True)
    g0.step(1, sync=True)
    assert g.totals()["pairs"] - t["pairs"] == g0.totals()["pairs"] - t0["pairs"] > 0
    run = O.OracleRun.start(ev)
    run.step(5)
    errs = state_errors3(g, run)
    assert all(v < TOL_EVOL for v in errs.values()), errs
    g.free()
    g0.free()


def test_pair_lists_3d_overflow_falls_back_then_grows(Bd, monkeypatch):
    """3D lists allocated far too small: per-particle passes for the stage (the step still
    matches the oracle), then the allocation grows and the stages run on the lists."""
    monkeypatch.setenv("SPH_PAIR_TOTAL", "64")
    ev = CASES3["blob3_milne"]()
    g = Bd.GpuEvent(ev)
    run = O.OracleRun.start(ev)
    g.step(1, sync=True)
    run.step(1)
    assert g.totals()["pair_overflows"] >= 2
    errs = state_errors3(g, run)
    assert all(v < TOL_STEP for v in errs.values()), errs
    seen = []
    for _ in range(3):
        g.step(1, sync=True)
        seen.append(g.totals()["pair_overflows"])
    assert seen[-1] == seen[-2], seen
    g.free()


def _diffusing(ev, kap=None, tauJT=(0.2, 0.2, 0.2)):
    """The event with BSQ diffusion (the paper's full matrix unless kap is given)."""
    ev.diffusion = I.Diffusion(kappaT2=kap if kap is not None else I.KAPPA_BSQ, tauJT=tauJT)
    return ev


DIFF_CASES = {
    "bsq_small_diff": lambda: _diffusing(I.viscous_bsq_2p1(n_target=3000, R=3.0, n_hot=20)),
    "diffusion_box_moving": lambda: I.diffusion_box_2d(v=0.7, half_widths=(3.0, 1.5),
                                                      kappaT2=((0.05, 0.02, 0.0), (-0.01, 0.14, 0.015), (0.0, 0.03, 0.09))),
    "blob_causal_diff": lambda: _diffusing(I.smooth_blob_2p1(half_width=2.0, eos=I.CAUSAL_EOS)),
}


def _diff_state(g, run, dim=2):
    st = g.read(("X", "U", "S", "BV", "PV", "JV", "NQ"))
    y = run.y
    k = 2 * dim
    return {"x": relerr(st["X"], y[0:dim]), "u": relerr(st["U"], y[dim:k]), "S": relerr(st["S"], y[k]),
            "Bv": relerr(st["BV"], y[k + 1]), "Pv": relerr(st["PV"], y[k + 2:k + 5]), "J": relerr(st["JV"], y[9:15]),
            "Nq": relerr(st["NQ"], run.Nq)}


@pytest.mark.parametrize("case", list(DIFF_CASES))
def test_diffusion_step_and_evolution(Bd, case):
    """BSQ diffusion (2+1D, plain FP64): the densities with the currents' J^0, the inversion, the
    currents' relaxation and the lab-charge fluxes match the oracle: 1e-11 after one Heun step,
    1e-8 over 40; the lab charges' totals stay constant."""
    ev = DIFF_CASES[case]()
    g = Bd.GpuEvent(ev, use_graph=True)
    run = O.OracleRun.start(ev)
    f = g.read(("N_DENS", "T", "MU"))
    aux, _ = run.observe()
    assert relerr(f["N_DENS"], aux[O.AUX["nB"]:O.AUX["nQ"] + 1]) < TOL_STEP
    g.step(1, sync=True)
    run.step(1)
    errs = _diff_state(g, run)
    assert all(v < TOL_STEP for v in errs.values()), errs
    g.step(39, sync=True)
    run.step(39)
    errs = _diff_state(g, run)
    assert all(v < TOL_EVOL for v in errs.values()), errs
    jv = g.read(("JV",))["JV"]
    assert np.max(np.abs(jv)) > 0.0
    t = g.totals()
    N0 = np.array([np.sum(ev.Nq[q]) for q in range(3)])
    assert np.allclose(t["N"], N0, rtol=1e-12, atol=1e-12 * np.max(np.abs(ev.Nq)) * ev.n)
    g.free()


def test_diffusion_mixed_form_against_oracle(Bd):
    """The mixed single-event form (FP32 neighbour sums) with diffusion: within 1e-5 over 40 steps."""
    ev = DIFF_CASES["bsq_small_diff"]()
    g = Bd.GpuEvent(ev, use_graph=True, precision=Bd.SPH_MIXED)
    g.step(40, sync=True)
    run = O.OracleRun.start(ev)
    run.step(40)
    errs = _diff_state(g, run)
    assert all(v < TOL_MIXED for v in errs.values()), errs
    g.free()


def test_diffusion_pair_list_overflow_uses_the_cell_pass(Bd, monkeypatch):
    """Pair lists far too small: the stages whose lists overflowed take the diffusion sums from
    the cell pass (distances and kernel gradients evaluated again), the others from the lists;
    both follow the oracle."""
    monkeypatch.setenv("SPH_PAIR_TOTAL", "64")
    ev = DIFF_CASES["bsq_small_diff"]()
    g = Bd.GpuEvent(ev)
    run = O.OracleRun.start(ev)
    g.step(1, sync=True)
    run.step(1)
    assert g.totals()["pair_overflows"] >= 2
    errs = _diff_state(g, run)
    assert all(v < TOL_STEP for v in errs.values()), errs
    g.step(9, sync=True)
    run.step(9)
    errs = _diff_state(g, run)
    assert all(v < TOL_EVOL for v in errs.values()), errs
    g.free()


def test_diffusion_rejected_where_not_built(Bd):
    """3+1D events and the serving form run without diffusion currents: asking for them is an error."""
    ev3 = _diffusing(I.smooth_blob_3d(milne=True, flow=0.3))
    with pytest.raises(Bd.SphError):
        Bd.GpuEvent(ev3)
    ev = DIFF_CASES["bsq_small_diff"]()
    srv = Bd.GpuServer(ev.eos, ev.table, max_events=2, max_particles=1 << 13)
    with pytest.raises(Bd.SphError):
        srv.submit(ev, 1)
    srv.free()
