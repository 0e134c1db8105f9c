"""Pins of the oracle's equation of state and its inversion (CPU only).

Pinned against thermodynamic identities (s = dp/dT, n = dp/dmu by finite
differences), exact reproduction of table node values, round trips
(T, mu) -> (s, n) -> (T, mu) (Sec. "EoS inverter"), the closed form of the
conformal EoS, and finite differences of p(s, n) for the EoS derivatives.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2511_22852_gb300 import inputs as I


@pytest.fixture(scope="module")
def bsq():
    ev = I.viscous_bsq_2p1(n_target=200, R=2.0, n_hot=3)
    P, keep = O.make_params(ev)
    return ev, P, keep


def test_analytic_thermodynamic_identities(bsq):
    ev, P, _ = bsq
    rng = np.random.default_rng(3)
    for _ in range(30):
        T = rng.uniform(0.2, 4.0)
        mu = rng.uniform(-0.5, 0.5, 3) * T
        p, sn, H = O.eos_analytic(P, T, mu)
        e = 1e-6 * T
        dpdT = (O.eos_analytic(P, T + e, mu)[0] - O.eos_analytic(P, T - e, mu)[0]) / (2 * e)
        assert abs(dpdT - sn[0]) < 1e-6 * abs(sn[0])
        for q in range(3):
            d = np.zeros(3)
            d[q] = e
            dpdm = (O.eos_analytic(P, T, mu + d)[0] - O.eos_analytic(P, T, mu - d)[0]) / (2 * e)
            assert abs(dpdm - sn[1 + q]) < 1e-6 * abs(sn[0])
        # H is the Jacobian of (s, n)
        Hfd = np.zeros((4, 4))
        x0 = np.array([T, *mu])
        for k in range(4):
            d = np.zeros(4)
            d[k] = e
            Hfd[:, k] = (O.eos_analytic(P, *(lambda z: (z[0], z[1:]))(x0 + d))[1]
                         - O.eos_analytic(P, *(lambda z: (z[0], z[1:]))(x0 - d))[1]) / (2 * e)
        assert np.allclose(Hfd, H, rtol=1e-5, atol=1e-6 * abs(H[0, 0]))


def test_table_nodes_and_jacobian(bsq):
    ev, P, _ = bsq
    t = ev.table
    rng = np.random.default_rng(4)
    for _ in range(20):
        i = rng.integers(0, t.nT)
        j = rng.integers(0, t.nmu[0], 3)
        x = np.array([t.T0 + i * t.dT, *(t.mu0[q] + j[q] * t.dmu[q] for q in range(3))])
        p, sn, _ = O.eos_table(P, x)
        ref = [t.s[i, j[0], j[1], j[2]], t.nB[i, j[0], j[1], j[2]], t.nS[i, j[0], j[1], j[2]],
               t.nQ[i, j[0], j[1], j[2]]]
        assert abs(p - t.p[i, j[0], j[1], j[2]]) <= 1e-13 * abs(p)
        assert np.allclose(sn, ref, rtol=1e-13, atol=1e-13 * abs(ref[0]))
    # Jacobian against finite differences inside one cell
    x = np.array([t.T0 + 10.37 * t.dT, *(t.mu0[q] + (14.41 + q) * t.dmu[q] for q in range(3))])
    _, sn, J = O.eos_table(P, x)
    for k in range(4):
        d = np.zeros(4)
        d[k] = 1e-4 * (t.dT if k == 0 else t.dmu[k - 1])
        fd = (O.eos_table(P, x + d)[1] - O.eos_table(P, x - d)[1]) / (2 * d[k])
        assert np.allclose(fd, J[:, k], rtol=1e-8, atol=1e-10 * abs(J[0, 0]))


def test_table_inversion_round_trip(bsq):
    ev, P, _ = bsq
    t = ev.table
    rng = np.random.default_rng(5)
    for _ in range(40):
        T = t.T0 + rng.uniform(2, t.nT - 3) * t.dT
        mu = rng.uniform(-0.3, 0.3, 3) * T
        mu = np.clip(mu, t.mu0[0] + 2 * t.dmu[0], -t.mu0[0] - 2 * t.dmu[0])
        p, sn, _ = O.eos_table(P, np.array([T, *mu]))
        out, st = O.eos_invert(P, sn[0], sn[1:])
        assert st & (O.ST_NOCONV | O.ST_FALLBACK | O.ST_OUT_OF_TABLE) == 0
        assert abs(out[0] - T) < 1e-10 * T
        assert np.all(np.abs(out[1:4] - mu) < 1e-10 * T)
        assert abs(out[4] - p) < 1e-10 * abs(p)
        # Gibbs-Duhem: e + p = T s + mu.n
        assert abs(out[5] + out[4] - (out[0] * sn[0] + np.dot(out[1:4], sn[1:]))) < 1e-12 * abs(out[5])


def test_analytic_inversion_round_trip(bsq):
    ev, P, _ = bsq
    Pn, _ = O.make_params(ev)
    Pn.has_table = 0
    rng = np.random.default_rng(6)
    for _ in range(40):
        T = rng.uniform(0.05, 5.0)
        mu = rng.uniform(-0.4, 0.4, 3) * T
        _, sn, _ = O.eos_analytic(Pn, T, mu)
        out, st = O.eos_invert(Pn, sn[0], sn[1:])
        assert st & O.ST_NOCONV == 0
        assert abs(out[0] - T) < 1e-12 * T
        assert np.all(np.abs(out[1:4] - mu) < 1e-11 * T)


def test_conformal_closed_form():
    ev = I.gubser_ideal_2p1(n_side=3)
    P, _ = O.make_params(ev)
    a0 = I.GUBSER_FSTAR / 3.0
    for s in [1e-3, 0.5, 17.0, 3000.0]:
        out, st = O.eos_invert(P, s, [0, 0, 0])
        T = (s / (4 * a0)) ** (1 / 3)
        assert st == 0
        assert abs(out[0] - T) < 2e-15 * T * 4
        assert abs(out[5] - 3 * out[4]) < 1e-13 * out[5]  # eps = 3 p
        assert abs(out[10] - 1 / 3) < 1e-14  # c_s^2 = 1/3
        assert abs(out[6] - T / 3) < 1e-14 * T  # dp/ds = T/3


def test_eos_derivatives_by_finite_difference(bsq):
    """(p_s, p_n) = dp/d(s, n) at fixed other densities, by finite differences of the inversion.

    Closed-form EoS: p itself.  Table: p and s are interpolated independently, so the
    identity dp = s dT + n.dmu holds only for w = e + p = T s + mu.n along the interpolant,
    whose derivatives must be T + p_s and mu_q + p_nq."""
    ev, P, _ = bsq
    Pa, _ = O.make_params(ev)
    Pa.cs2_cap = 1e30
    Pa.has_table = 0
    Pt, _ = O.make_params(ev)
    Pt.cs2_cap = 1e30
    inv = lambda PP, z: O.eos_invert(PP, z[0], z[1:])
    for Tg in [0.25, 0.4, 0.12]:
        T = Tg / I.HBARC
        mu = np.array([0.05, -0.03, 0.02]) * T
        _, sn, _ = O.eos_analytic(Pa, T, mu)
        out, st = inv(Pa, sn)
        for k in range(4):
            d = np.zeros(4)
            d[k] = 1e-6 * sn[0]
            fd = (inv(Pa, sn + d)[0][4] - inv(Pa, sn - d)[0][4]) / (2 * d[k])
            assert abs(fd - out[6 + k]) < 1e-6 * abs(out[6])
        _, sn, _ = O.eos_table(Pt, np.array([T, *mu]))
        out, st = inv(Pt, sn)
        w = lambda o, z: o[0] * z[0] + np.dot(o[1:4], z[1:])
        for k in range(4):
            d = np.zeros(4)
            d[k] = 1e-7 * sn[0]
            fd = (w(inv(Pt, sn + d)[0], sn + d) - w(inv(Pt, sn - d)[0], sn - d)) / (2 * d[k])
            ref = out[0] + out[6] if k == 0 else out[k] + out[6 + k]
            assert abs(fd - ref) < 1e-6 * abs(out[0])


def test_infeasible_charges_flagged_not_nan(bsq):
    """The literal +-10 % charge fraction has no solution for hot particles: flagged, finite."""
    ev, P, _ = bsq
    T = 0.5 / I.HBARC
    _, sn, _ = O.eos_analytic(P, T, np.zeros(3))
    s = sn[0]
    out, st = O.eos_invert(P, s, [0.1 * s, 0.1 * s, -0.1 * s])
    assert st & O.ST_NOCONV
    assert np.all(np.isfinite(out))


def test_acausal_band_is_capped(bsq):
    ev, P, _ = bsq
    T = 0.175 / I.HBARC
    _, sn, _ = O.eos_analytic(P, T, np.zeros(3))
    out, st = O.eos_invert(P, sn[0], [0, 0, 0])
    assert st & O.ST_CS2_CAPPED and abs(out[10] - 1.0) < 1e-15
    T = 0.3 / I.HBARC
    _, sn, _ = O.eos_analytic(P, T, np.zeros(3))
    out, st = O.eos_invert(P, sn[0], [0, 0, 0])
    assert not st & O.ST_CS2_CAPPED and 0.3 < out[10] < 0.6


def test_warm_started_inversion_reaches_the_same_root(bsq):
    """Newton from the previous stage's solution (the warm-start reading) converges to the root the cold
    start (closed form, then table) finds; a guess outside the table falls back to the cold path."""
    import ctypes as C
    ev, P, _ = bsq
    t = ev.table
    rng = np.random.default_rng(9)
    for _ in range(30):
        T = t.T0 + rng.uniform(3, t.nT - 4) * t.dT
        mu = rng.uniform(-0.2, 0.2, 3) * T
        p, sn, _ = O.eos_table(P, np.array([T, *mu]))
        cold, st = O.eos_invert(P, sn[0], sn[1:])
        guess = np.array([T * (1 + rng.uniform(-0.02, 0.02)), *(mu + rng.uniform(-0.02, 0.02, 3) * T)])
        for gs in [guess, np.array([t.T0 * 0.5, 0, 0, 0]), np.zeros(4)]:
            out = np.zeros(11)
            used = C.c_int(0)
            nn = np.ascontiguousarray(sn[1:])
            st2 = O.lib().oc_eos_invert_ws(C.byref(P), float(sn[0]), nn.ctypes.data_as(C.c_void_p),
                                           gs.ctypes.data_as(C.c_void_p), out.ctypes.data_as(C.c_void_p),
                                           C.byref(used))
            assert used.value == 1 and st2 == st
            assert np.all(np.abs(out[:4] - cold[:4]) <= 1e-13 * T)
            assert abs(out[4] / cold[4] - 1) < 1e-13


@pytest.fixture(scope="module")
def bsq_backup():
    ev = I.viscous_bsq_2p1(n_target=200, R=2.0, n_hot=3)
    ev.eos_backup = (0.165, 0.45)
    P, keep = O.make_params(ev)
    return ev, P, keep


def _p_cd(P, T, mu):
    """The conformal-diagonal pressure of Sec. "Equation of state" (backup EoS), T_0 = 1/fm."""
    return P.cd_A0 * (T ** 4 + sum((mu[q] / P.cd_mu0[q]) ** 4 for q in range(3)))


def test_backup_eos_matches_the_closed_form_at_T_scale(bsq_backup):
    """The backup's constants satisfy the paper's matching conditions: its pressure equals the
    closed form's at (T_scale, 0) and at (T_scale, mu_q = mu_max) for each charge."""
    ev, P, _ = bsq_backup
    Ts, mm = 0.165 / I.HBARC, 0.45 / I.HBARC
    p0, _, _ = O.eos_analytic(P, Ts, np.zeros(3))
    assert abs(_p_cd(P, Ts, np.zeros(3)) / p0 - 1) < 1e-13
    for q in range(3):
        mu = np.zeros(3)
        mu[q] = mm
        pq, _, _ = O.eos_analytic(P, Ts, mu)
        assert abs(_p_cd(P, Ts, mu) / pq - 1) < 1e-13


def test_backup_eos_inverts_what_the_closed_form_cannot(bsq_backup):
    """Infeasible charges (the literal +-10 % fraction at 0.5 GeV): the closed form has no
    solution, the conformal-diagonal backup does -- thermodynamically consistent: its pressure's
    derivatives at the returned (T, mu) reproduce (s, n), e = 3p, and (p_s, p_n) match finite
    differences of the inversion."""
    ev, P, _ = bsq_backup
    T = 0.5 / I.HBARC
    _, sn, _ = O.eos_analytic(P, T, np.zeros(3))
    s = sn[0]
    n = np.array([0.1 * s, 0.1 * s, -0.1 * s])
    out, st = O.eos_invert(P, s, n)
    assert st == O.ST_BACKUP
    Tb, mu = out[0], out[1:4]
    d = 1e-6
    dpdT = (_p_cd(P, Tb * (1 + d), mu) - _p_cd(P, Tb * (1 - d), mu)) / (2 * d * Tb)
    assert abs(dpdT / s - 1) < 1e-8
    for q in range(3):
        m1, m2 = mu.copy(), mu.copy()
        m1[q] *= 1 + d
        m2[q] *= 1 - d
        dpdm = (_p_cd(P, Tb, m1) - _p_cd(P, Tb, m2)) / (2 * d * mu[q])
        assert abs(dpdm / n[q] - 1) < 1e-8
    assert abs(out[4] / _p_cd(P, Tb, mu) - 1) < 1e-13 and abs(out[5] / (3 * out[4]) - 1) < 1e-13
    o2, _ = O.eos_invert(P, s * (1 + d), n)
    assert abs((o2[4] - out[4]) / (s * d) / out[6] - 1) < 1e-5
    for q in range(3):
        n2 = n.copy()
        n2[q] *= 1 + d
        o2, _ = O.eos_invert(P, s, n2)
        assert abs((o2[4] - out[4]) / (n[q] * d) / out[7 + q] - 1) < 1e-5
    assert abs(out[10] - 1.0 / 3.0) < 1e-15


def test_newton_polish_stays_within_the_stopping_rule(bsq):
    """The table Newton's polishing step (one Newton step past the first iterate that meets the
    tolerance, kept when its point meets the tolerance too) only chooses between points the
    stopping rule of Sec. "EoS inverter" accepts.  So with and without it the inversion agrees
    within the image of the tolerance: T to 1e-12 relative (s ~ T^3), each mu_q within
    tol s / (chi_q T^2) (n_q = chi_q T^2 mu_q in the closed form the table samples), p within
    s dT + n.dmu of those differences;
    and the evolved state of a viscous event after 20 Heun steps to 1e-12 normwise."""
    ev, P, _ = bsq
    Pn, _ = O.make_params(ev, newton_polish=False)
    t = ev.table
    tol = P.newton_tol
    rng = np.random.default_rng(21)
    for _ in range(400):
        T = t.T0 + rng.uniform(1, t.nT - 2) * t.dT
        mu = np.clip(rng.uniform(-0.3, 0.3, 3) * T, t.mu0[0] + t.dmu[0], -t.mu0[0] - t.dmu[0])
        _, sn, _ = O.eos_table(P, np.array([T, *mu]))
        a, sa = O.eos_invert(P, sn[0], sn[1:])
        b, sb = O.eos_invert(Pn, sn[0], sn[1:])
        assert sa == sb
        assert abs(a[0] - b[0]) <= 1e-12 * a[0]
        for q in range(3):
            assert abs(a[1 + q] - b[1 + q]) <= 2.0 * tol * sn[0] / (ev.eos.chi[q] * a[0] ** 2)
        # dp = s dT + n.dmu (Gibbs-Duhem) to first order
        dp = sn[0] * abs(a[0] - b[0]) + float(np.dot(np.abs(sn[1:]), np.abs(a[1:4] - b[1:4])))
        assert abs(a[4] - b[4]) <= 2.0 * dp + 1e-14 * abs(a[4])
    small = I.viscous_bsq_2p1(n_target=1200, R=2.0, n_hot=8)
    ys = []
    for pol in (True, False):
        r = O.OracleRun.start(small, newton_polish=pol)
        r.step(20)
        ys.append(r.y.copy())
    for k in range(ys[0].shape[0]):
        scale = max(np.max(np.abs(ys[0][k])), 1e-300)
        assert np.max(np.abs(ys[0][k] - ys[1][k])) <= 1e-12 * scale
