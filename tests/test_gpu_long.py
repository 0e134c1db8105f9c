"""Long and large parity runs of the CUDA path against the FP64 oracle (GPU).

- The 40k-particle viscous BSQ event over its whole evolution, tau 0.6 -> 8 fm/c (1480 Heun
  steps), in the launch configuration of the benchmark's FP64 arm: the state within 1e-8
  normwise, T and s per particle, and the per-particle EoS branch (table, closed form) the
  same on both sides except where a particle sits on a branch boundary.
- The stress configuration's path (Cartesian 3+1D, h = 0.15 fm, the 128 x 64^3 EoS table, ten
  jet tracks) on a cut-down event of the same generator (a 1.2 fm disc, |z| <= 0.8 fm, the same
  0.0577 fm spacing): one step at 1e-11, ten at 1e-8, the mixed form at 1e-5, and the counts
  of particles outside the table or on the closed form equal to the oracle's.
- The serving form: two events of different size served together for 300 steps, each within
  1e-5 of the oracle on T, mu, s, n_q and the state, with the neighbour counts exact.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2511_22852_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL_STEP = 1e-11
TOL_EVOL = 1e-8
TOL_MIXED = 1e-5
BRANCH = 1 | 2  # FALLBACK | OUT_OF_TABLE: the closed-form branch of the inversion


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
    return float(np.max(np.abs(a - b)) / den) if den > 0 else float(np.max(np.abs(a)))


def state_errors(st, y, dim):
    npi = 3 if dim == 2 else 5
    k = 2 * dim
    return {"x": relerr(st["X"], y[0:dim]), "u": relerr(st["U"], y[dim:k]), "S": relerr(st["S"], y[k]),
            "Bv": relerr(st["BV"], y[k + 1]), "Pv": relerr(st["PV"], y[k + 2:k + 2 + npi])}


def test_full_size_event_whole_evolution(Bd):
    ev = I.viscous_bsq_2p1()
    assert ev.nsteps == 1480 and 39000 < ev.n < 41000
    g = Bd.GpuEvent(ev, use_graph=True)
    g.step(ev.nsteps, sync=True)
    f = g.read(("X", "U", "S", "BV", "PV", "T", "S_DENS", "STATUS"))
    tg = g.totals()
    g.free()
    run = O.OracleRun.start(ev)
    run.step(ev.nsteps)
    aux, st = run.observe()
    errs = state_errors(f, run.y, 2)
    assert all(v < TOL_EVOL for v in errs.values()), errs
    # per-particle: the EoS branch, and T and s relative to themselves where the branch agrees
    bg, bo = f["STATUS"] & BRANCH, st & BRANCH
    flips = int(np.count_nonzero(bg != bo))
    assert flips <= ev.n // 1000, f"{flips} particles on different EoS branches"
    same = bg == bo
    T_ref, s_ref = aux[O.AUX["T"]], aux[O.AUX["s"]]
    t_rel = float(np.max(np.abs(f["T"][same] / T_ref[same] - 1.0)))
    s_rel = float(np.max(np.abs(f["S_DENS"][same] / s_ref[same] - 1.0)))
    assert t_rel < TOL_EVOL and s_rel < TOL_EVOL, (t_rel, s_rel, flips)
    ot = run.totals()
    assert abs(tg["E"] / ot["E"] - 1.0) < TOL_EVOL and abs(tg["work"] / ot["work"] - 1.0) < TOL_EVOL


@pytest.fixture(scope="module")
def stress_small():
    """The stress generator on a 1.2 fm disc, |z| <= 0.8 fm at the full event's spacing (the
    n_target that gives 0.0577 fm), with its 128 x 64^3 table and ten tracks in the disc."""
    ev = I.stress_cartesian_3d(n_target=int(round(np.pi * 1.2 ** 2 * 1.6 / 0.0577 ** 3)), R=1.2, z_max=0.8)
    assert abs(ev.meta["dx"] - 0.0577) < 2e-4 and ev.table.nT == 128
    assert len(ev.jets.tracks) == 10
    return ev


def test_stress_path_matches_oracle(Bd, stress_small):
    ev = stress_small
    run = O.OracleRun.start(ev)
    run.step(1)
    g = Bd.GpuEvent(ev, use_graph=True)
    g.step(1, sync=True)
    errs = state_errors(g.read(("X", "U", "S", "BV", "PV")), run.y, 3)
    assert all(v < TOL_STEP for v in errs.values()), errs
    run.step(9)
    g.step(9, sync=True)
    f = g.read(("X", "U", "S", "BV", "PV", "T", "STATUS", "NNB"))
    g.free()
    errs = state_errors(f, run.y, 3)
    assert all(v < TOL_EVOL for v in errs.values()), errs
    aux, st = run.observe()
    assert relerr(f["T"], aux[O.AUX["T"]]) < TOL_EVOL
    assert np.array_equal(f["NNB"], aux[O.AUX["nnb"]].astype(np.int32))
    for bit in (1, 2, 4):  # FALLBACK, OUT_OF_TABLE, NOCONV counted, not only OR-ed
        assert np.count_nonzero(f["STATUS"] & bit) == np.count_nonzero(st & bit), bit
    assert np.max(np.abs(f["U"])) > 0.0
    gm = Bd.GpuEvent(ev, use_graph=True, precision=Bd.SPH_MIXED)
    gm.step(10, sync=True)
    fm = gm.read(("X", "U", "T", "NNB"))
    gm.free()
    assert relerr(fm["T"], aux[O.AUX["T"]]) < TOL_MIXED and relerr(fm["U"], run.y[3:6]) < TOL_MIXED
    assert np.array_equal(fm["NNB"], f["NNB"])


def test_serving_two_events_300_steps(Bd):
    evs = [I.viscous_bsq_2p1(n_target=n, R=7.0 * np.sqrt(n / 40000.0), seed_hot=1000 + k, seed_charge=500000 + k)
           for k, n in enumerate((5000, 20000))]
    srv = Bd.GpuServer(evs[0].eos, evs[0].table, max_events=4, max_particles=1 << 16)
    tk = [srv.submit(ev, 300) for ev in evs]
    srv.drain(600.0)
    outs = [srv.collect(t) for t in tk]
    srv.free()
    A = O.AUX
    for ev, out in zip(evs, outs):
        run = O.OracleRun.start(ev)
        run.step(300)
        aux, _ = run.observe()
        assert np.array_equal(out["NNB"], aux[A["nnb"]].astype(np.int32))
        assert relerr(out["X"], run.y[:2]) < TOL_MIXED and relerr(out["U"], run.y[2:4]) < TOL_MIXED
        assert relerr(out["S"], run.y[4]) < TOL_MIXED
        assert relerr(out["BV"], run.y[5]) < TOL_MIXED and relerr(out["PV"], run.y[6:9]) < TOL_MIXED
        assert relerr(out["T"], aux[A["T"]]) < TOL_MIXED
        assert relerr(out["MU"], aux[A["muB"]:A["muQ"] + 1]) < TOL_MIXED
        assert relerr(out["S_DENS"], aux[A["s"]]) < TOL_MIXED
        assert relerr(out["N_DENS"], aux[A["nB"]:A["nQ"] + 1]) < TOL_MIXED
        assert float(np.max(np.abs(out["T"] / aux[A["T"]] - 1.0))) < TOL_MIXED
