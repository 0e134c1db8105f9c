"""The serving form on the GPU: continuously batched 2+1D events in one segmented arena.

* every event's results match the FP64 oracle to 1e-5 (normwise) on T, mu, the rest-frame
  densities and the evolved state, with neighbour counts exact;
* an event's results are bitwise the same alone and in a batch with other events, whatever
  its arena position and admission time (batch invariance);
* events submitted while others run are admitted as slots and arena ranges free up;
* argument errors and states of the ticket protocol.
"""
import numpy as np
import pytest

import gubser_viscous as VG
from oracle import oracle as O
from paper_2511_22852_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def Bd():
    from paper_2511_22852_gb300 import binding, build_lib
    build_lib.build()
    return binding


def relerr(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    den = np.max(np.abs(b)) if b.size else 1.0
    return float(np.max(np.abs(a - b)) / den) if den > 0 else float(np.max(np.abs(a)))


def bsq(n, seed=1, R=None, hot=None):
    R = R if R is not None else float(np.sqrt(n / 40000.0) * 7.0)
    return I.viscous_bsq_2p1(n_target=n, R=R, n_hot=hot or max(5, n // 200), seed_hot=seed, seed_charge=seed + 1)


def serve_alone(Bd, ev, nsteps, **kw):
    s = Bd.GpuServer(ev.eos, ev.table, **kw)
    t = s.submit(ev, nsteps)
    s.drain(120.0)
    st, lat = s.poll(t)
    assert st == Bd.SPH_TICKET_DONE and lat > 0
    out = s.collect(t)
    s.free()
    return out


def check_against_oracle(out, ev, nsteps):
    run = O.OracleRun.start(ev)
    run.step(nsteps)
    aux, st = run.observe()
    A = O.AUX
    assert abs(out["totals"]["tau"] - run.tau) < 1e-12
    assert np.array_equal(out["NNB"], aux[A["nnb"]].astype(np.int32))
    assert relerr(out["X"], run.y[:2]) < TOL and relerr(out["U"], run.y[2:4]) < TOL
    assert relerr(out["S"], run.y[4]) < TOL
    assert relerr(out["T"], aux[A["T"]]) < TOL
    assert relerr(out["S_DENS"], aux[A["s"]]) < TOL
    if np.any(aux[A["nB"]]):
        assert relerr(out["N_DENS"], aux[A["nB"]:A["nQ"] + 1]) < TOL
        assert relerr(out["MU"], aux[A["muB"]:A["muQ"] + 1]) < TOL
    if ev.transport.viscous:
        assert relerr(out["BV"], run.y[5]) < TOL
        assert relerr(out["PV"], run.y[6:9]) < TOL
    assert np.array_equal(out["NQ"], run.Nq)  # charges travel with their particles exactly
    return run


def _stopped(ev, T_GeV):
    ev.transport.T_stop_GeV = T_GeV
    return ev


@pytest.mark.parametrize("case,nsteps", [("bsq", 20), ("gubser", 30), ("blob_causal", 20), ("bjorken", 10),
                                        ("gubser_viscous", 30), ("bsq_stop", 40)])
def test_server_event_matches_fp64_oracle(Bd, case, nsteps):
    ev = {"bsq": lambda: bsq(3000), "bsq_stop": lambda: _stopped(bsq(3000), 0.2), "gubser": lambda: I.gubser_ideal_2p1(),
          "blob_causal": lambda: I.smooth_blob_2p1(half_width=2.0, eos=I.CAUSAL_EOS),
          "bjorken": lambda: I.bjorken_lattice_2p1(n_side=21),
          "gubser_viscous": lambda: VG.gubser_viscous_2p1(VG.GubserODE(eta_over_s=0.2))}[case]()
    out = serve_alone(Bd, ev, nsteps, max_events=4, max_particles=1 << 16)
    run = check_against_oracle(out, ev, nsteps)
    tt = out["totals"]
    assert tt["steps"] == nsteps
    assert np.array_equal(tt["N"], np.array([np.sum(run.Nq[q]) for q in range(3)])) or \
        np.allclose(tt["N"], [np.sum(run.Nq[q]) for q in range(3)], rtol=1e-14, atol=1e-300)


def test_server_observe_only_event(Bd):
    """nsteps = 0: the fields at the initial state."""
    ev = bsq(2000, seed=5)
    out = serve_alone(Bd, ev, 0, max_events=2, max_particles=1 << 14)
    check_against_oracle(out, ev, 0)


def test_batch_invariance_bitwise(Bd):
    """The same event alone, and admitted into a running batch of other events at another arena
    position: bitwise equal results (every sum of an event runs over its own particles in a
    fixed order)."""
    target = bsq(4000, seed=11)
    alone = serve_alone(Bd, target, 12, max_events=8, max_particles=1 << 16)
    s = Bd.GpuServer(target.eos, target.table, max_events=8, max_particles=1 << 16)
    others = [bsq(1500, seed=21), bsq(6000, seed=31), bsq(700, seed=41)]
    tk = [s.submit(others[0], 20), s.submit(others[1], 7)]
    s.pump(3)  # the batch is running when the target arrives
    t = s.submit(target, 12)
    tk.append(s.submit(others[2], 30))
    s.drain(120.0)
    mixed = s.collect(t)
    for k in tk:
        s.collect(k)
    s.free()
    for k in ("X", "U", "S", "BV", "PV", "T", "MU", "S_DENS", "N_DENS", "NNB"):
        assert np.array_equal(alone[k], mixed[k]), k
    for k in ("tau", "E", "S", "work", "pairs"):
        assert alone["totals"][k] == mixed["totals"][k], k


def test_continuous_admission_and_reuse(Bd):
    """Two slots, an arena for about two events: five events submitted at once run two at a
    time, each admitted when a slot and a range free up; every result equals its lone run."""
    evs = [bsq(1000 + 300 * k, seed=100 + k) for k in range(5)]
    steps = [6, 3, 9, 4, 5]
    s = Bd.GpuServer(evs[0].eos, evs[0].table, max_events=2, max_particles=4096)
    tickets = [s.submit(e, k) for e, k in zip(evs, steps)]
    assert s.stats()["queued"] == 5
    max_running = 0
    for _ in range(200):
        r = s.pump(1)
        max_running = max(max_running, r)
        st = s.stats()
        assert st["slots_in_use"] <= 2 and st["arena_in_use"] <= st["arena_capacity"]
        if all(s.poll(t)[0] == Bd.SPH_TICKET_DONE for t in tickets):
            break
    s.drain(60.0)
    assert max_running == 2
    lat = [s.poll(t)[1] for t in tickets]
    assert all(v > 0 for v in lat)
    res = [s.collect(t) for t in tickets]
    s.free()
    for e, k, r in zip(evs, steps, res):
        a = serve_alone(Bd, e, k, max_events=2, max_particles=4096)
        for f in ("X", "U", "T", "MU", "NNB"):
            assert np.array_equal(a[f], r[f]), f


def test_server_errors(Bd):
    ev = bsq(1000)
    s = Bd.GpuServer(ev.eos, ev.table, max_events=2, max_particles=1024)
    big = bsq(3000)
    with pytest.raises(Bd.SphError) as e:
        s.submit(big, 1)
    assert e.value.code == Bd.SPH_ERR_OOM
    ev3 = I.smooth_blob_3d(milne=True, flow=0.3)
    with pytest.raises(Bd.SphError) as e:
        s.submit(ev3, 1)
    assert e.value.code == Bd.SPH_ERR_ARG
    with pytest.raises(Bd.SphError) as e:
        s.submit(ev, -1)
    assert e.value.code == Bd.SPH_ERR_ARG
    t = s.submit(ev, 2)
    assert s.poll(t)[0] == Bd.SPH_TICKET_QUEUED
    with pytest.raises(Bd.SphError) as e:
        s.collect(t)
    assert e.value.code == Bd.SPH_ERR_STATE
    s.n_of[t] = ev.n
    with pytest.raises(Bd.SphError) as e:
        s.poll(t + 1000)
    assert e.value.code == Bd.SPH_ERR_ARG
    s.drain(60.0)
    assert s.poll(t)[0] == Bd.SPH_TICKET_DONE
    s.collect(t)
    with pytest.raises(Bd.SphError) as e:
        s.poll(t)  # released
    assert e.value.code == Bd.SPH_ERR_ARG
    s.free()
    with pytest.raises(Bd.SphError):
        Bd.GpuServer(ev.eos, ev.table, max_events=0)


def test_autotuner_keeps_results_and_counters(Bd):
    """The autotuner times the tiled passes on the running batch and picks a launch shape; the
    events still match the oracle, and the counters its trial runs touched are restored (the
    neighbour-pair count equals that of an untuned run)."""
    evs = [bsq(3000, seed=61), bsq(5000, seed=62)]
    s = Bd.GpuServer(evs[0].eos, evs[0].table, max_events=4, max_particles=1 << 16)
    with pytest.raises(Bd.SphError) as e:
        s.autotune(1)
    assert e.value.code == Bd.SPH_ERR_STATE
    tk = [s.submit(ev, 12) for ev in evs]
    s.pump(2)
    tt, lw = s.autotune(2, lanes=True)
    assert tt in (64, 96, 128, 192, 256) and lw in (2, 4, 8)
    s.drain(120.0)
    out = [s.collect(t) for t in tk]
    s.free()
    check_against_oracle(out[0], evs[0], 12)
    plain = serve_alone(Bd, evs[1], 12, max_events=4, max_particles=1 << 16)
    assert out[1]["totals"]["pairs"] == plain["totals"]["pairs"]
    assert np.array_equal(out[1]["NNB"], plain["NNB"])


def test_server_wait_limit_reports_timeout(Bd, monkeypatch):
    """The server's bounded waits: a wait limit far below a batch step's duration makes the pump
    return SPH_ERR_TIMEOUT instead of blocking; the server is then freed cleanly."""
    monkeypatch.setenv("SPH_WAIT_LIMIT_S", "0.000001")
    ev = bsq(40000)
    s = Bd.GpuServer(ev.eos, ev.table, max_events=2, max_particles=1 << 17, max_inflight=1)
    s.submit(ev, 20)
    with pytest.raises(Bd.SphError) as e:
        for _ in range(10):
            s.pump(1)
    assert e.value.code == Bd.SPH_ERR_TIMEOUT
    s.free()


def test_nonfinite_event_ends_early_without_touching_others(Bd):
    """An event whose rates overflow (a shear stress of 1e305 on every particle) is ended within
    a few batch steps: its ticket completes with the non-finite status bit and fewer steps than
    requested, the server counts one failed event, and the healthy event served beside it is
    bitwise what it is alone."""
    healthy = bsq(3000, seed=81)
    alone = serve_alone(Bd, healthy, 40, max_events=4, max_particles=1 << 15)
    bad = bsq(1500, seed=82)
    bad.Pv = np.full_like(bad.Pv, 1e305)
    s = Bd.GpuServer(healthy.eos, healthy.table, max_events=4, max_particles=1 << 15)
    tb = s.submit(bad, 200)
    th = s.submit(healthy, 40)
    s.drain(120.0)
    st = s.stats()
    assert st["failed"] == 1
    ob = s.collect(tb, names=("X", "T", "STATUS"))
    oh = s.collect(th)
    s.free()
    assert ob["totals"]["status_or"] & 8
    assert 1 <= ob["totals"]["steps"] <= 6, ob["totals"]["steps"]
    assert oh["totals"]["status_or"] & 8 == 0 and oh["totals"]["steps"] == 40
    for k in ("X", "U", "S", "BV", "PV", "T", "MU", "S_DENS", "N_DENS", "NNB"):
        assert np.array_equal(alone[k], oh[k]), k


def test_fixed_shape_runs_match_oracle_and_are_batch_invariant(Bd):
    """Every lane split, set by hand, gives the oracle's results within the form's tolerance and,
    for a fixed shape, the same bits alone and in a batch; shapes outside the lists are refused."""
    ev = bsq(2500, seed=91)
    other = bsq(4000, seed=92)
    s = Bd.GpuServer(ev.eos, ev.table, max_events=4, max_particles=1 << 15)
    for bad in ((100, 4), (128, 3), (0, 0)):
        with pytest.raises(Bd.SphError) as e:
            s.set_shape(*bad)
        assert e.value.code == Bd.SPH_ERR_ARG
    s.free()
    for tt, lw in ((64, 2), (192, 8)):
        a = Bd.GpuServer(ev.eos, ev.table, max_events=4, max_particles=1 << 15)
        a.set_shape(tt, lw)
        t = a.submit(ev, 10)
        a.drain(60.0)
        lone = a.collect(t)
        a.free()
        check_against_oracle(lone, ev, 10)
        b = Bd.GpuServer(ev.eos, ev.table, max_events=4, max_particles=1 << 15)
        b.set_shape(tt, lw)
        to = b.submit(other, 14)
        b.pump(2)
        t = b.submit(ev, 10)
        b.drain(60.0)
        mixed = b.collect(t)
        b.collect(to)
        b.free()
        for k in ("X", "U", "T", "MU", "NNB"):
            assert np.array_equal(lone[k], mixed[k]), (tt, lw, k)


def test_overlapped_groups_give_the_same_bits(Bd):
    """The two-group schedule (one group's EoS and equations of motion beside the other's
    neighbour passes) computes exactly what the one-group schedule does: every event's results
    bitwise equal."""
    evs = [bsq(3000, seed=101), bsq(5000, seed=102), bsq(2000, seed=103)]
    outs = {}
    for groups in (1, 2):
        s = Bd.GpuServer(evs[0].eos, evs[0].table, max_events=4, max_particles=1 << 15, groups=groups)
        tk = [s.submit(ev, 15) for ev in evs]
        s.drain(60.0)
        outs[groups] = [s.collect(t) for t in tk]
        s.free()
    for a, b in zip(outs[1], outs[2]):
        for k in ("X", "U", "S", "BV", "PV", "T", "MU", "S_DENS", "N_DENS", "NNB"):
            assert np.array_equal(a[k], b[k]), k
        for k in ("tau", "E", "work", "pairs"):
            assert a["totals"][k] == b["totals"][k], k
