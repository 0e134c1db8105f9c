"""Pins of the oracle's BSQ diffusion (CPU only).

Small charge waves, alpha_q = mu_q / T = a_q cos(k x) with different amplitudes for B, S and Q,
ride on a uniform fluid at T = 0.3 GeV and zero chemical potentials (Cartesian 2D box, spacing
0.1 fm, h = 0.3 fm, lambda = 4 fm), at rest and moving with v = 0.7 along x; the diffusion
matrix kappa_{qq'}/T^2 is deliberately not symmetric (so a transposed matrix is seen), with the
paper's relaxation times tau_q = 0.2 / T.  To first order the charge densities and the currents
follow the linearised equations of Sec. "Equations of motion" (eqs. charge_conservation,
min_dif_rel) solved exactly in ``diffusion_linear`` (sympy, from the covariant equations; at rest
it is the telegraph equation).  The particles starting within one wavelength of the centre are
fitted with cos + sin + const at t = 0.5 .. 2 fm: the charge densities within 7 % of each one's
largest amplitude, the currents within 8 % of the largest current (measured at rest 3-5 % and
2-3 %, moving 1.6-2.7 % and 3-4 %; the SPH discretisation error at kh = 0.47).  In the moving
fluid the pin sees J^0 in the rest-frame density, the flux J^i - v^i J^0 of the lab charge, the
projection of the gradient (its D alpha part) and of D J, and the order of kappa's indices.

Also: the lab charges are conserved exactly up to rounding (the pairwise antisymmetric flux
divergence) in a viscous BSQ event with the paper's full matrix.
"""
import numpy as np
import pytest

import diffusion_linear as L
from oracle import oracle as O
from paper_2511_22852_gb300 import inputs as I

KAP = ((0.05, 0.02, 0.0), (-0.01, 0.14, 0.015), (0.0, 0.03, 0.09))
TIMES = (0.5, 1.0, 1.5, 2.0)
TOL_N, TOL_J = 0.07, 0.08


def _fit(xs, f, k):
    """Complex amplitude Z with f = Re[Z exp(i k x)] + const (least squares)."""
    A = np.stack([np.cos(k * xs), np.sin(k * xs), np.ones_like(xs)], 1)
    c, *_ = np.linalg.lstsq(A, f, rcond=None)
    return c[0] - 1j * c[1]


def wave_errors(v):
    ev = I.diffusion_box_2d(v=v, kappaT2=KAP)
    m = ev.meta
    k, T0 = m["k"], m["T0"]
    kappa = np.array(KAP) * T0 ** 2
    tau = np.array(ev.diffusion.tauJT) / T0
    win = (np.abs(ev.x[0]) <= np.pi / k) & (np.abs(ev.x[1]) <= 0.6)
    nrow = [O.AUX[c] for c in ("nB", "nS", "nQ")]
    jrow = [9 + 2 * q for q in range(3)]  # J^x_q / sigma: after the 9 state rows of 2D, q major
    run = O.OracleRun.start(ev)
    aux, _ = run.observe()
    Y0 = np.array([_fit(run.y[0][win], aux[nrow[q]][win], k) for q in range(3)] + [0.0] * 3, dtype=complex)
    meas, lin = [], []
    t = 0.0
    for tt in TIMES:
        run.step(int(round((tt - t) / ev.dtau)))
        t = tt
        aux, _ = run.observe()
        xs, sig = run.y[0][win], aux[O.AUX["sigma"]][win]
        meas.append([_fit(xs, aux[nrow[q]][win], k) for q in range(3)] +
                    [_fit(xs, sig * run.y[jrow[q]][win], k) for q in range(3)])
        lin.append(L.amplitudes(Y0, tt, v=v, T0=T0, chi=ev.eos.chi, kappa=kappa, tau=tau, k=k))
    meas, lin = np.array(meas), np.array(lin)
    err_n = [float(np.max(np.abs(meas[:, q] - lin[:, q])) / np.max(np.abs(lin[:, q]))) for q in range(3)]
    err_j = float(np.max(np.abs(meas[:, 3:] - lin[:, 3:])) / np.max(np.abs(lin[:, 3:])))
    return err_n, err_j


@pytest.mark.parametrize("v", [0.0, 0.7])
def test_charge_waves_against_linear_diffusion(v):
    err_n, err_j = wave_errors(v)
    assert max(err_n) < TOL_N, err_n
    assert err_j < TOL_J, err_j


def test_lab_charge_conserved_exactly():
    ev = I.viscous_bsq_2p1(n_target=1500, R=2.2, n_hot=12)
    ev.diffusion = I.Diffusion(kappaT2=I.KAPPA_BSQ)
    run = O.OracleRun.start(ev)
    N0 = run.Nq.sum(axis=1)
    run.step(20)
    assert np.max(np.abs(run.y[9:])) > 0.0  # currents developed
    assert np.all(np.abs(run.Nq.sum(axis=1) - N0) <= 1e-13 * np.abs(run.Nq).sum(axis=1))
    assert np.max(np.abs(run.Nq - ev.Nq)) > 1e-6 * np.max(np.abs(ev.Nq))  # charge moved between particles
