"""Linearised BSQ charge diffusion in a uniformly moving fluid: the reference solution of the
diffusion pins.

Background: a uniform fluid at temperature T0 with zero chemical potentials, moving with
velocity v along x in Cartesian coordinates, u = gamma (1, v, 0, 0).  Its EoS gives
n_q = chi_q T^2 mu_q, so alpha_q = mu_q / T = n_q / (chi_q T0^3) at fixed T, and the pressure
is unchanged to first order in the charges: the flow and T are not perturbed.  Perturbations
f(t, x) = F(t) exp(i k x) of the charge densities (E_q) and the currents' x components (B_q;
J^0 follows from u_mu J^mu = 0, J^y = J^z = 0) obey, to first order, the equations of Sec.
"Equations of motion" of the paper (metric (+,-,-,-)):

    d_mu (n_q u^mu + J^mu_q) = 0                                  (eq. charge_conservation),
    tau_q Delta^mu_nu D J^nu_q + J^mu_q = kappa_{qq'} nabla^<mu> alpha_{q'}   (eq. min_dif_rel),

with nabla^<mu> = Delta^{mu nu} d_nu, D = u^mu d_mu, constant kappa_{qq'} and tau_q (the sign of
the current's source makes charge flow down the gradient of mu / T).  The six equations are
assembled with sympy from these covariant expressions at the numeric parameters and solved for
the time derivatives: dY/dt = M Y, Y(t) = expm(M t) Y(0).  At rest and for one charge this is
the telegraph equation tau E'' + E' + kappa k^2 / (chi T0^3) E = 0.
"""
import numpy as np
import sympy as sp
from scipy.linalg import expm


def rate_matrix(v, T0, chi, kappa, tau, k):
    """M of dY/dt = M Y for Y = (E_B, E_S, E_Q, B_B, B_S, B_Q) (complex amplitudes of exp(i k x));
    kappa[q][q'] and tau[q] absolute (fm^-2, fm), T0 in fm^-1."""
    I = sp.I
    rat = lambda a: sp.nsimplify(float(a), rational=True)
    v_, T_, k_ = rat(v), rat(T0), rat(k)
    g_ = 1 / sp.sqrt(1 - v_ ** 2)
    g = sp.diag(1, -1, -1, -1)
    u = sp.Matrix([g_, g_ * v_, 0, 0])
    E = sp.symbols("E0:3")
    B = sp.symbols("B0:3")
    dE = sp.symbols("dE0:3")
    dB = sp.symbols("dB0:3")

    def d_(mu, amp, damp):  # partial derivative of a plane-wave amplitude: d_t -> damp, d_x -> i k amp
        return damp if mu == 0 else (I * k_ * amp if mu == 1 else 0)

    def current(b):  # J^mu with J^x = b, J^y = J^z = 0 and u_mu J^mu = 0
        J = sp.Matrix([0, b, 0, 0])
        J[0] = -sum(g[i, i] * u[i] * J[i] for i in range(1, 4)) / (g[0, 0] * u[0])
        return J

    eqs = []
    for q in range(3):
        J, Jt = current(B[q]), current(dB[q])
        # d_mu N^mu with N^mu = n u^mu + J^mu (the background n and u are uniform)
        eqs.append(sum(u[m] * d_(m, E[q], dE[q]) + d_(m, J[m], Jt[m]) for m in range(4)))
        # the x component of tau Delta^x_nu D J^nu + J^x - kappa Delta^{x nu} d_nu alpha
        DJ = [sum(u[m] * d_(m, J[nu], Jt[nu]) for m in range(4)) for nu in range(4)]
        proj = sum(((1 if nu == 1 else 0) - u[1] * g[nu, nu] * u[nu]) * DJ[nu] for nu in range(4))
        src = 0
        for q2 in range(3):
            alpha, dalpha = E[q2] / (rat(chi[q2]) * T_ ** 3), dE[q2] / (rat(chi[q2]) * T_ ** 3)
            src += rat(kappa[q][q2]) * sum((g[1, nu] - u[1] * u[nu]) * d_(nu, alpha, dalpha) for nu in range(4))
        eqs.append(rat(tau[q]) * proj + J[1] - src)
    A, _ = sp.linear_eq_to_matrix([sp.expand(e) for e in eqs], list(dE) + list(dB) + list(E) + list(B))
    A = np.array(A.evalf(), dtype=complex)
    return -np.linalg.solve(A[:, :6], A[:, 6:])


def amplitudes(Y0, t, **kw):
    """Y(t) = expm(M t) Y0."""
    return expm(rate_matrix(**kw) * t) @ np.asarray(Y0, dtype=complex)
