"""Linearised Israel-Stewart sound wave in a uniformly moving fluid: the reference solution of
the bulk-viscosity pin with flow.

Background: a uniform fluid (energy density e0, p = c_s^2 e, w0 = e0 + p0) moving with
velocity v along x in Cartesian coordinates, u = gamma (1, v, 0, 0), no charges.  Perturbations
of the form f(t, x) = F(t) exp(i k x) in the energy density (E), the contravariant velocity u^x
(U; u^0 follows from u.u = 1 as v U), the bulk pressure Pi (B) and the shear stress of a
compression along x (Q: pi^{mu nu} = Q Xi^{mu nu}, Xi the boost of diag(0, 1, -1/2, -1/2),
the only shear structure such a wave excites) obey, to first order, the equations of
Sec. "Equations of motion" of the paper (metric mostly minus):

    d_mu T^{mu nu} = 0,  T^{mu nu} = (e + p + Pi) u^mu u^nu - (p + Pi) g^{mu nu} + pi^{mu nu},
    tau_Pi D Pi + Pi = -zeta theta                                        (eq. min_bul_rel),
    tau_pi Delta^{mu nu}_{alpha beta} D pi^{alpha beta} + pi^{mu nu} = 2 eta sigma^{mu nu}
                                                                          (eq. min_she_rel;
    the -(4/3) tau_pi pi theta term is second order).

The four equations are linear in (E, U, B, Q) and their time derivatives; they are assembled
here with sympy from the covariant expressions above (and nothing else) at the numeric
parameters, and solved for the time derivatives, giving dY/dt = M Y with a constant complex
matrix M.  The amplitudes at time t are expm(M t) Y(0).  With v = 0 and zeta = eta = 0 this is the ideal
sound wave, E'' = -c_s^2 k^2 E.
"""
import numpy as np
import sympy as sp
from scipy.linalg import expm


def _equations(v, w0, cs2, zeta, eta, tau_Pi, tau_pi, k):
    """The four linearised equations at numeric parameters, as sympy expressions linear in the
    amplitudes Y = (E, U, B, Q) and their time derivatives dY; returns (eqs, Y, dY, shear check)."""
    E, U, B, Q, dE, dU, dB, dQ = sp.symbols("E U B Q dE dU dB dQ")
    I = sp.I
    v, w0, cs2, zeta, eta, tPi, tpi, k = [sp.nsimplify(float(a), rational=True) for a in
                                           (v, w0, cs2, zeta, eta, tau_Pi, tau_pi, k)]
    g_ = 1 / sp.sqrt(1 - v ** 2)
    g = sp.diag(1, -1, -1, -1)
    u = sp.Matrix([g_, g_ * v, 0, 0])
    du = sp.Matrix([v * U, U, 0, 0])  # u^0 du^0 = u^x du^x
    ddu_t = sp.Matrix([v * dU, dU, 0, 0])

    def d_(mu, amp, damp):  # partial derivative of a plane-wave amplitude: d_t -> damp, d_x -> i k amp
        return damp if mu == 0 else (I * k * amp if mu == 1 else 0)

    Xi = sp.zeros(4, 4)
    Xi[0, 0], Xi[0, 1], Xi[1, 0], Xi[1, 1] = g_ ** 2 * v ** 2, g_ ** 2 * v, g_ ** 2 * v, g_ ** 2
    Xi[2, 2] = Xi[3, 3] = -sp.Rational(1, 2)
    # perturbation of T^{mu nu} and its time derivative
    dw, dP = (1 + cs2) * E + B, cs2 * E + B
    dw_t, dP_t = (1 + cs2) * dE + dB, cs2 * dE + dB

    def dT(mu, nu, t):
        if t:
            return dw_t * u[mu] * u[nu] + w0 * (ddu_t[mu] * u[nu] + u[mu] * ddu_t[nu]) - dP_t * g[mu, nu] + dQ * Xi[mu, nu]
        return dw * u[mu] * u[nu] + w0 * (du[mu] * u[nu] + u[mu] * du[nu]) - dP * g[mu, nu] + Q * Xi[mu, nu]

    eqs = [dT(0, nu, True) + I * k * dT(1, nu, False) for nu in (0, 1)]  # d_t T^{0 nu} + d_x T^{x nu}
    theta = v * dU + I * k * U  # d_t du^0 + d_x du^x

    def D(amp, damp):  # u^lambda d_lambda
        return g_ * (damp + I * k * v * amp)

    eqs.append(tPi * D(B, dB) + B + zeta * theta)
    # sigma^{mu nu} = (nabla^mu u^nu + nabla^nu u^mu)/2 - (u^mu Du^nu + u^nu Du^mu)/2 - Delta^{mu nu} theta/3
    nab = sp.zeros(4, 4)  # nabla^mu du^nu = g^{mu alpha} d_alpha du^nu
    for mu in range(4):
        for nu in range(4):
            nab[mu, nu] = g[mu, mu] * d_(mu, du[nu], ddu_t[nu])
    Du = sp.Matrix([D(du[nu], ddu_t[nu]) for nu in range(4)])
    sig = sp.zeros(4, 4)
    for mu in range(4):
        for nu in range(4):
            Delta = g[mu, nu] - u[mu] * u[nu]
            sig[mu, nu] = (nab[mu, nu] + nab[nu, mu]) / 2 - (u[mu] * Du[nu] + u[nu] * Du[mu]) / 2 - Delta * theta / 3

    def con(A, C):  # A^{mu nu} C_{mu nu}
        return sum(A[m, n] * g[m, m] * g[n, n] * C[m, n] for m in range(4) for n in range(4))

    XX = con(Xi, Xi)
    sx = con(sig, Xi)
    eqs.append(tpi * D(Q, dQ) + Q - 2 * eta * sx / XX)
    check = sig - (sx / XX) * Xi  # zero when sigma is along Xi
    return eqs, (E, U, B, Q), (dE, dU, dB, dQ), check


def rate_matrix(v, w0, cs2, zeta, eta, tau_Pi, tau_pi, k):
    """M of dY/dt = M Y for Y = (E, U, B, Q) (complex amplitudes of exp(i k x))."""
    eqs, Y, dY, check = _equations(v, w0, cs2, zeta, eta, tau_Pi, tau_pi, k)
    # sigma of a 1D wave lies along Xi at first order, so the shear equation projects onto it
    rnd = {Y[1]: sp.Rational(3, 7), Y[0]: 0, Y[2]: 0, Y[3]: 0, dY[1]: sp.Rational(-5, 11)}
    assert max(abs(complex(c.subs(rnd))) for c in check) < 1e-12, "shear of a 1D wave is not along Xi"
    A, rhs = sp.linear_eq_to_matrix([sp.expand(e) for e in eqs], list(dY) + list(Y))
    A = np.array(A.evalf(), dtype=complex)
    # eqs: A_d dY + A_y Y = 0
    return -np.linalg.solve(A[:, :4], A[:, 4:])


def amplitudes(Y0, t, **kw):
    """Y(t) = expm(M t) Y0."""
    return expm(rate_matrix(**kw) * t) @ np.asarray(Y0, dtype=complex)
