"""Pin of the oracle's bulk-viscous channel with flow (CPU only).

A small sound wave rides on a uniform conformal fluid moving at v = 0.7 along x in a Cartesian
2D box, with bulk viscosity zeta/s = 0.2 (and a negligible shear viscosity, whose relaxation
time sets tau_Pi).  To first order the amplitudes of exp(i k x) in the energy density, u^x and
the bulk pressure Pi follow the linearised Israel-Stewart equations of the paper's Sec.
"Equations of motion" (eqs. min_bul_rel, min_she_rel with d_mu T^{mu nu} = 0) in the moving
frame, solved exactly in ``bulk_sound_linear`` (a sympy linearisation of the covariant
equations, independent of the oracle's code).  In the moving frame the bulk pressure enters the
momentum equation through its gradient and through the enthalpy rate u^i d(e + p + Pi)/dt, and
its relaxation through the comoving derivative u^mu d_mu = gamma (d_t + v d_x).

The oracle's particles (those starting within one wavelength of the centre) are fitted with
a cos + sin + constant in x at t = 0.5 .. 2 fm, before the rarefactions from the box edges
arrive; the measured amplitudes must follow the linear solution within the SPH discretisation
error at this resolution (kh = 0.47): u^x within 5 % and Pi within 10 % of the largest
amplitude of each over the window (measured 2.2 % and 6.8 %; an ideal fluid of the same
resolution errs by 3.0 % on u^x).  The bulk viscosity moves u^x by 29 % of its amplitude, so
the pin sees the channel: dropping the bulk rate from the enthalpy rate of the momentum
equation gives 13 % and 22 %, dropping Pi from the stress 22 % and 20 %.  The initial energy
amplitude is taken from the oracle's own smoothed densities at t = 0 (the kernel sum lowers
the lattice's amplitude by 3.5 %).
"""
import numpy as np
import pytest

import bulk_sound_linear as L
from oracle import oracle as O
from paper_2511_22852_gb300 import inputs as I

TIMES = (0.5, 1.0, 1.5, 2.0)
TOL_U, TOL_PI = 0.05, 0.10


def _fit(xs, f, k):
    """Complex amplitude Z with f = Re[Z exp(i k x)] + const (least squares)."""
    A = np.stack([np.cos(k * xs), np.sin(k * xs), np.ones_like(xs)], 1)
    c, *_ = np.linalg.lstsq(A, f, rcond=None)
    return c[0] - 1j * c[1]


def wave_errors(v=0.7, zeta_over_s=0.2):
    """Normwise errors of the oracle's u^x and Pi amplitudes against the linear solution, and
    the linear solutions' amplitudes (for the size of the bulk effect)."""
    ev = I.boosted_sound_wave_2d(v=v, zeta_over_s=zeta_over_s, half_widths=(6.0, 3.4))
    m = ev.meta
    k, T0, a0 = m["k"], m["T0"], ev.eos.a0
    e0, w0, s0 = 3 * a0 * T0 ** 4, 4 * a0 * T0 ** 4, 4 * a0 * T0 ** 3
    tr = ev.transport
    eta, zeta = tr.eta_over_s * s0, tr.zeta_peak * s0
    tau_pi = tr.tau_pi_coef * eta / w0
    lin_kw = dict(v=v, w0=w0, cs2=1.0 / 3.0, zeta=zeta, eta=eta, tau_Pi=tr.tau_Pi_ratio * tau_pi, tau_pi=tau_pi, k=k)
    gam = 1.0 / np.sqrt(1.0 - v * v)
    win = (np.abs(ev.x[0]) <= np.pi / k) & (np.abs(ev.x[1]) <= 0.6)
    run = O.OracleRun.start(ev)
    aux, _ = run.observe()
    Y0 = [_fit(run.y[0][win], aux[O.AUX["e"]][win] - e0, k), 0.0, 0.0, 0.0]
    meas, lin = [], []
    t = 0.0
    for tt in TIMES:
        run.step(int(round((tt - t) / ev.dtau)))
        t = tt
        aux, _ = run.observe()
        xs = run.y[0][win]
        meas.append([_fit(xs, run.y[2][win] - gam * v, k), _fit(xs, aux[O.AUX["Pi"]][win], k)])
        lin.append(L.amplitudes(Y0, tt, **lin_kw)[[1, 2]])
    meas, lin = np.array(meas), np.array(lin)
    err = [float(np.max(np.abs(meas[:, j] - lin[:, j])) / max(np.max(np.abs(lin[:, j])), 1e-300)) for j in range(2)]
    return err, lin


@pytest.mark.slow
def test_bulk_sound_wave_in_moving_fluid():
    err, lin = wave_errors()
    assert err[0] < TOL_U, f"u^x amplitude off the linear IS solution by {err[0]:.3f}"
    assert err[1] < TOL_PI, f"Pi amplitude off the linear IS solution by {err[1]:.3f}"
