"""Semi-analytic viscous Gubser flow (conformal EoS e = 11 T^4, shear viscosity, no charges):
the reference solution of the viscous physics pin.

The paper's Gubser benchmark (Sec. "Code validation", EoS2 with zero chemical potentials)
reduces Israel-Stewart hydrodynamics on Gubser flow to two ODEs in the de Sitter time rho:

    dT/drho  = T (pibar - 2)/3 tanh(rho),
    dpibar/drho = 4/(3 C) tanh(rho) - pibar / tauR - (4/3) pibar^2 tanh(rho),   tauR = C (eta/s)/T,

with T the Weyl-rescaled temperature (T_Milne = T(rho)/tau, fm^-1) and pibar the Weyl-rescaled
pi^eta_eta over (e + p).  The minimal Israel-Stewart equation with its -(4/3) tau_pi pi theta
term and tau_pi = 5 eta/(e + p) gives exactly these with C = 5.  In Milne coordinates
tau^2 pi^{eta eta} = pibar (e + p) at every point, and the transverse shear follows from the two
equal de Sitter eigenvalues -pibar (e + p)/2 along the theta and phi directions.
"""
import math

import numpy as np
from scipy.integrate import solve_ivp

from paper_2511_22852_gb300 import inputs as I

FSTAR = I.GUBSER_FSTAR


def rho_of(tau, r, q=1.0):
    return np.arcsinh((q * q * (tau * tau - r * r) - 1.0) / (2.0 * q * tau))


def gubser_u(tau, r, q=1.0):
    den = np.sqrt(1.0 + 2.0 * q * q * (tau * tau + r * r) + q ** 4 * (tau * tau - r * r) ** 2)
    return (1.0 + q * q * (tau * tau + r * r)) / den, 2.0 * q * q * r * tau / den


class GubserODE:
    """T(rho), pibar(rho) from rho_start (pibar = 0 there) to rho_end, dense output."""

    def __init__(self, eta_over_s, T_at_0=0.4 / I.HBARC, rho_start=-5.0, rho_end=2.0, C=5.0):
        self.C, self.eta_over_s = C, eta_over_s
        T_start = T_at_0 / math.cosh(rho_start) ** (2.0 / 3.0)

        def rhs(rho, Y):
            T, pb = Y
            th = math.tanh(rho)
            tauR = C * eta_over_s / T
            return [T * (pb - 2.0) / 3.0 * th, 4.0 / (3.0 * C) * th - pb / tauR - 4.0 / 3.0 * pb * pb * th]

        self.sol = solve_ivp(rhs, (rho_start, rho_end), [T_start, 0.0], rtol=1e-11, atol=1e-13, dense_output=True,
                             method="DOP853")

    def T(self, rho):
        return self.sol.sol(rho)[0]

    def pibar(self, rho):
        return self.sol.sol(rho)[1]


def gubser_viscous_2p1(ode: GubserODE, n_side=51, half_width=5.0, h=0.5, tau0=1.0, dtau=0.01, nsteps=60):
    """Lattice event on one trajectory of the ODEs: T, u and pi^{ij} of viscous Gubser flow at tau0."""
    g = np.linspace(-half_width, half_width, n_side)
    dx = g[1] - g[0]
    X, Y = np.meshgrid(g, g, indexing="ij")
    x, y = X.ravel().copy(), Y.ravel().copy()
    n = x.size
    r = np.sqrt(x * x + y * y)
    phi = np.arctan2(y, x)
    rho0 = rho_of(tau0, r)
    T = ode.T(rho0) / tau0
    utau, ur = gubser_u(tau0, r)
    c, s_ = np.cos(phi), np.sin(phi)
    ux, uy = ur * c, ur * s_
    e = FSTAR * T ** 4
    w = 4.0 / 3.0 * e          # e + p
    s = w / T                  # mu = 0
    half = 0.5 * ode.pibar(rho0) * w
    pxx = -half * (utau * utau * c * c + s_ * s_)
    pxy = -half * (utau * utau - 1.0) * c * s_
    pyy = -half * (utau * utau * s_ * s_ + c * c)
    vol = utau * tau0 * dx * dx  # 1/sigma of a lattice particle
    eos = I.AnalyticEoS(a0=FSTAR / 3.0)
    return I.Event(name="gubser_viscous_2p1", dim=2, milne=True, h=h, tau0=tau0, dtau=dtau, nsteps=nsteps,
                   x=np.stack([x, y]), u=np.stack([ux, uy]), S=s * vol, Nq=np.zeros((3, n)),
                   Bv=np.zeros(n), Pv=np.stack([pxx, pxy, pyy]) * vol, eos=eos, table=None,
                   transport=I.Transport(viscous=True, eta_over_s=ode.eta_over_s, zeta_peak=0.0,
                                         tau_pi_coef=ode.C, tau_Pi_ratio=1.0),
                   meta={"dx": dx})


def gubser_viscous_3p1(ode: GubserODE, n_side=51, half_width=5.0, eta_half=1.5, deta=0.2, h=0.5, tau0=1.0,
                       dtau=0.01, nsteps=60):
    """The same boost-invariant flow on a 3+1D Milne lattice: the transverse lattice of
    gubser_viscous_2p1 repeated on eta layers |eta| <= eta_half (spacing deta), u^eta = 0, shear
    stored as (xx, xy, x eta, yy, y eta) / sigma with the eta components zero."""
    ev2 = gubser_viscous_2p1(ode, n_side=n_side, half_width=half_width, h=h, tau0=tau0, dtau=dtau, nsteps=nsteps)
    etas = deta * np.arange(-round(eta_half / deta), round(eta_half / deta) + 1)
    m, n2 = etas.size, ev2.x.shape[1]
    x = np.concatenate([np.stack([ev2.x[0], ev2.x[1], np.full(n2, e)]) for e in etas], axis=1)
    u = np.concatenate([np.stack([ev2.u[0], ev2.u[1], np.zeros(n2)]) for _ in etas], axis=1)
    # per particle 1/sigma gains the eta spacing; the stored shear is pi / sigma
    S = np.tile(ev2.S, m) * deta
    P2 = ev2.Pv * deta
    z = np.zeros(n2)
    Pv = np.tile(np.stack([P2[0], P2[1], z, P2[2], z]), (1, m))
    return I.Event(name="gubser_viscous_3p1", dim=3, milne=True, h=h, tau0=tau0, dtau=dtau, nsteps=nsteps,
                   x=x, u=u, S=S, Nq=np.zeros((3, n2 * m)), Bv=np.zeros(n2 * m), Pv=Pv, eos=ev2.eos, table=None,
                   transport=ev2.transport, meta={"dx": ev2.meta["dx"], "deta": deta})
