"""Energy-momentum source terms of jet tracks in the oracle (eqs. conservation_source,
e_conservation, momentum_conservation with I^nu != 0; CPU only).

A uniform ideal fluid at rest in a Cartesian box is crossed by a straight track depositing
dE/dx into a Gaussian around its position.  The total momentum P^i = sum_a T^{0i}_a / sigma*_a
and energy E = sum_a T^{00}_a / sigma*_a change by the deposited momentum and energy
int dt sum_a I^nu(x_a) / sigma*_a, to the accuracy with which this SPH form conserves them: the
kernel-sum sigma* and the velocity-gradient continuity equation agree only to discretisation
error, which leaves 0.4 % (momentum) and 0.3 % (energy) of the deposit here, independent of
dtau (checked at dtau/2 and dtau/4).  Without the deposit, the imbalance would be 100 %.  The
deposit is integrated here from this file's own statement of the track profile.
"""
import math

import numpy as np

from oracle import oracle as O
from paper_2511_22852_gb300 import inputs as I


def deposit(tracks, sigma, t, x):
    """I^nu at positions x [3][N] and time t: sum over tracks of dE/dx G_sigma (1, n)."""
    I4 = np.zeros((4, x.shape[1]))
    for tr in tracks:
        if t < tr[6]:
            continue
        c = x - (tr[0:3] + tr[3:6] * (t - tr[6]))[:, None]
        g = tr[7] * np.exp(-np.sum(c * c, axis=0) / (2 * sigma ** 2)) / ((2 * math.pi) ** 1.5 * sigma ** 3)
        I4[0] += g
        I4[1:] += g[None, :] * tr[3:6, None]
    return I4


def totals(run, aux):
    A = O.AUX
    u = run.y[3:6]
    g = aux[A["u0"]]
    w = aux[A["e"]] + aux[A["p"]]
    sig = aux[A["sigstar"]]
    P = np.sum(w * g * u / sig, axis=1)
    E = np.sum((w * g * g - aux[A["p"]]) / sig)
    return E, P


def test_track_deposits_its_energy_and_momentum():
    track = np.array([[-0.6, 0.1, -0.05, 1.0, 0.0, 0.0, 1.0, 5.0 / I.HBARC]])
    jets = I.JetTracks(tracks=track, sigma=0.3)
    ev = I.uniform_box_3d(jets=jets, nsteps=12)
    run = O.OracleRun.start(ev)
    aux, _ = run.observe()
    E0, P0 = totals(run, aux)
    assert np.all(np.abs(P0) < 1e-12 * E0)
    D = np.zeros(4)
    rate_prev = np.sum(deposit(track, 0.3, run.tau, run.y[0:3]) / aux[O.AUX["sigstar"]], axis=1)
    for _ in range(ev.nsteps):
        run.step(1)
        aux, _ = run.observe()
        rate = np.sum(deposit(track, 0.3, run.tau, run.y[0:3]) / aux[O.AUX["sigstar"]], axis=1)
        D += 0.5 * ev.dtau * (rate_prev + rate)
        rate_prev = rate
    E1, P1 = totals(run, aux)
    assert D[0] > 1e-3 * E0  # a resolvable deposit
    assert abs((P1[0] - P0[0]) / D[1] - 1) < 0.01
    assert np.all(np.abs(P1[1:] - P0[1:]) < 1e-3 * D[0]) and np.all(np.abs(D[2:]) < 1e-12 * D[0])
    assert abs((E1 - E0) / D[0] - 1) < 0.01
    # the track's energy went into heat: entropy rises, only there
    assert run.status_or == 0


def test_partons_deposit_their_four_momentum():
    """Dynamical-initialisation sources (Sec. "Dynamical initialization"): partons formed during
    the run, each smeared over the step in which it forms.  Once every parton's window has
    closed, the fluid's total momentum and energy have grown by N sum_j p_j^mu, to the SPH
    conservation accuracy of the source coupling (as for the jet tracks: 0.6 % here).  Partons
    of 0.1-0.3 GeV deposit ~2 % of the local energy within the kernel support per step; the
    SPH energy responds nonlinearly to much stronger deposits (1-3 GeV partons on h = 0.3 fm:
    +5.9 %, independent of dtau; +1.6 % on h = 0.5 fm), a discretisation effect of the
    smoothed densities, not of the source term."""
    ev = I.uniform_box_3d(nsteps=14)
    src = I.parton_sources(6, (ev.tau0 + 0.5 * ev.dtau, ev.tau0 + 10 * ev.dtau), 0.4, 3, E_GeV=(0.1, 0.3),
                           norm=0.42, h=0.3)
    ev.partons = src
    run = O.OracleRun.start(ev)
    aux, _ = run.observe()
    E0, P0 = totals(run, aux)
    run.step(ev.nsteps)
    aux, _ = run.observe()
    E1, P1 = totals(run, aux)
    dep = src.norm * src.partons[:, 4:].sum(axis=0)
    assert dep[0] > 0.003 * E0  # a resolvable deposit (the box alone drifts by ~1e-5 of E0)
    assert abs((E1 - E0) / dep[0] - 1) < 0.01
    assert np.all(np.abs((P1 - P0) - dep[1:]) < 0.01 * np.abs(dep[1:]).max())
    assert run.status_or == 0


def test_partons_outside_the_run_deposit_nothing():
    """The formation-time window (x^0 - dtau, x^0] of each stage: partons formed before the
    first stage's window or after the last stage leave the evolution bitwise unchanged."""
    ev = I.uniform_box_3d(nsteps=6)
    src = I.parton_sources(3, (ev.tau0 + 0.5 * ev.dtau, ev.tau0 + 3 * ev.dtau), 0.4, 3, norm=0.42, h=0.3)
    ev.partons = src
    a = O.OracleRun.start(ev)
    a.step(ev.nsteps)
    extra = src.partons[:2].copy()
    extra[0, 0] = ev.tau0 - 1.5 * ev.dtau    # before the window of the first stage
    extra[1, 0] = ev.tau0 + 20 * ev.dtau     # after the run
    ev.partons = I.PartonSources(np.concatenate([src.partons, extra]), norm=src.norm, h=src.h)
    b = O.OracleRun.start(ev)
    b.step(ev.nsteps)
    assert np.array_equal(a.y, b.y)


def test_partons_in_milne_coordinates():
    """The parton source in Milne coordinates (2+1D, tau0 = 0.6 fm, so sqrt(-g) = tau matters):
    the fluid's transverse momentum P^i = sum_a tau T^{tau i} / sigma*_a grows by N sum_j p_j^i,
    to 1.3 % (the pressure forces conserve it exactly; the rest is the partition of unity
    sum_a W(r_a - r_j) / sigma*_a of the source as the deposit moves the particles off the
    lattice).  A source missing its 1/sqrt(-g) would be off by 67 %."""
    ev = I.bjorken_lattice_2p1(T0_GeV=0.3, n_side=41, nsteps=14)
    ev.transport = I.Transport(viscous=False)
    src = I.parton_sources(5, (ev.tau0 + 0.5 * ev.dtau, ev.tau0 + 10 * ev.dtau), 0.6, 2, E_GeV=(0.1, 0.3),
                           norm=0.42, h=0.5)
    ev.partons = src
    A = O.AUX

    def px(run, aux):
        u = run.y[2:4]
        w = aux[A["e"]] + aux[A["p"]]
        return run.tau * np.sum(w * aux[A["u0"]] * u / aux[A["sigstar"]], axis=1)

    run = O.OracleRun.start(ev)
    aux, _ = run.observe()
    P0 = px(run, aux)
    run.step(ev.nsteps)
    aux, _ = run.observe()
    dep = src.norm * src.partons[:, 5:7].sum(axis=0)
    assert np.all(np.abs((px(run, aux) - P0) - dep) < 0.02 * np.abs(dep).max())
    assert run.status_or == 0


def test_parton_charges_are_deposited():
    """Charge sources (eq. charge_conservation with I_q != 0): each parton's (B, S, Q) smeared
    like its four-momentum.  The particles' charges grow by dN_q/dx0 = sqrt(-g) I_q / sigma* (the
    lab charge of a particle's volume 1/sigma*), so once every window has closed the fluid's
    total charge has grown by N sum_j q_j, to the partition of unity sum_a W(r_a - r_j) /
    sigma*_a of the source on the lattice: 2.8e-4 of the deposit in a Cartesian box, 1.3e-5 in
    Milne 2+1D at tau0 = 0.6 fm (where the 1/sqrt(-g) of the source and the sqrt(-g) of the rate
    cancel; without the latter the total would be off by 40 %)."""
    ev = I.uniform_box_3d(nsteps=14)
    src = I.parton_sources(6, (ev.tau0 + 0.5 * ev.dtau, ev.tau0 + 10 * ev.dtau), 0.4, 3, E_GeV=(0.1, 0.3),
                           norm=0.42, h=0.3)
    src.charges = I.parton_quark_charges(6, 11)
    ev.partons = src
    run = O.OracleRun.start(ev)
    N0 = run.Nq.sum(axis=1).copy()
    run.step(ev.nsteps)
    dep = src.norm * src.charges.sum(axis=0)
    assert np.abs(dep).max() > 0.5
    assert np.all(np.abs(run.Nq.sum(axis=1) - N0 - dep) < 2e-3 * np.abs(dep).max())
    assert run.status_or == 0

    ev = I.bjorken_lattice_2p1(T0_GeV=0.3, n_side=41, nsteps=14)
    ev.transport = I.Transport(viscous=False)
    src = I.parton_sources(5, (ev.tau0 + 0.5 * ev.dtau, ev.tau0 + 10 * ev.dtau), 0.6, 2, E_GeV=(0.1, 0.3),
                           norm=0.42, h=0.5)
    src.charges = I.parton_quark_charges(5, 12)
    ev.partons = src
    run = O.OracleRun.start(ev)
    N0 = run.Nq.sum(axis=1).copy()
    run.step(ev.nsteps)
    dep = src.norm * src.charges.sum(axis=0)
    assert np.abs(dep).max() > 0.5
    assert np.all(np.abs(run.Nq.sum(axis=1) - N0 - dep) < 1e-4 * np.abs(dep).max())
    assert run.status_or == 0


def test_charge_deposit_changes_entropy_by_minus_mu_over_T():
    """The entropy equation's charge term (eq. dsdnrewr: R^S_q = -mu_q / T): baryon number
    deposited into a static uniform fluid at mu_B = 0.1 GeV, T = 0.3 GeV by sources that carry no
    energy or momentum changes the total entropy by -(mu_B / T) Delta N_B to first order in the
    deposit (T ds = de - mu dn at fixed e): measured 0.2 % off for deposits that raise the local
    baryon density by a few per cent (1.9 % at three times the charge: the second-order drift of
    mu/T); without the term the entropy would not change."""
    ev = I.uniform_box_3d(nsteps=14)
    n = ev.x.shape[1]
    T, mu = np.full(n, 0.3 / I.HBARC), np.zeros((3, n))
    mu[0] = 0.1 / I.HBARC
    _, s, nq = I._analytic_p_s_n(I.CAUSAL_EOS, T, mu)
    vol = ev.meta["dx"] ** 3
    ev.S, ev.Nq = s * vol, nq * vol
    src = I.parton_sources(6, (ev.tau0 + 0.5 * ev.dtau, ev.tau0 + 10 * ev.dtau), 0.4, 3, norm=0.42, h=0.3)
    src.partons[:, 4:] = 0.0  # no energy or momentum
    src.charges = np.zeros((6, 3))
    src.charges[:, 0] = 0.003
    ev.partons = src
    run = O.OracleRun.start(ev)
    aux, _ = run.observe()
    mu_over_T = float(np.mean(aux[O.AUX["muB"]] / aux[O.AUX["T"]]))
    S0, N0 = run.y[6].sum(), run.Nq[0].sum()
    run.step(ev.nsteps)
    dS, dN = run.y[6].sum() - S0, run.Nq[0].sum() - N0
    assert abs(dN / (src.norm * src.charges[:, 0].sum()) - 1.0) < 1e-3
    assert abs(dS / (-mu_over_T * dN) - 1.0) < 0.01
    assert run.status_or == 0


def test_charge_deposit_into_moving_fluid_keeps_energy_and_momentum():
    """A charge-only source (I^nu = 0, I_q != 0) leaves the energy-momentum tensor conserved: in a
    uniform box moving with u^x = 0.5 at mu_B = 0.1 GeV the totals E = sum T^{00}/sigma* and P^x
    = sum T^{0x}/sigma* change exactly as without the deposit (3e-10 of P, 2e-10 of E measured),
    although the deposit changes the local pressure and drives flow.  It needs the enthalpy rate
    of the momentum equation to carry dn_q = N_q dsigma + sigma dN_q: without sigma dN_q the
    totals drift by 5e-6 and 1.3e-6."""
    A = O.AUX
    ev = I.uniform_box_3d(nsteps=14)
    n = ev.x.shape[1]
    T, mu = np.full(n, 0.3 / I.HBARC), np.zeros((3, n))
    mu[0] = 0.1 / I.HBARC
    _, s, nq = I._analytic_p_s_n(I.CAUSAL_EOS, T, mu)
    ux = 0.5
    vol = ev.meta["dx"] ** 3 * np.sqrt(1.0 + ux * ux)  # lab-frame content of a lattice cell
    ev.u = np.zeros((3, n))
    ev.u[0] = ux
    ev.S, ev.Nq = s * vol, nq * vol

    def totals(run):
        aux, _ = run.observe()
        w = aux[A["e"]] + aux[A["p"]]
        P = np.sum(w * aux[A["u0"]] * run.y[3:6] / aux[A["sigstar"]], axis=1)
        E = np.sum((w * aux[A["u0"]] ** 2 - aux[A["p"]]) / aux[A["sigstar"]])
        return P, E

    out = []
    for q in (0.0, 0.003):
        src = I.parton_sources(6, (ev.tau0 + 0.5 * ev.dtau, ev.tau0 + 10 * ev.dtau), 0.4, 3, norm=0.42, h=0.3)
        src.partons[:, 4:] = 0.0
        src.charges = np.zeros((6, 3))
        src.charges[:, 0] = q
        ev.partons = src
        run = O.OracleRun.start(ev)
        P0, E0 = totals(run)
        N0 = run.Nq[0].sum()
        run.step(ev.nsteps)
        P1, E1 = totals(run)
        out.append((P1 - P0, E1 - E0, run.Nq[0].sum() - N0))
        assert run.status_or == 0
    (dP0, dE0, _), (dP1, dE1, dN1) = out
    assert dN1 > 0.99 * 0.42 * 6 * 0.003  # the deposit happened
    assert np.all(np.abs(dP1 - dP0) < 1e-8 * abs(P0[0])) and abs(dE1 - dE0) < 1e-8 * E0
