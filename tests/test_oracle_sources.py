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
