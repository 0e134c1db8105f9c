"""Seeded synthetic inputs for the SPH particle step.

This module only *synthesises inputs*: particle lattices, hotspot entropy
profiles, random charge fractions, the Gubser initial state and the node values
of a tabulated equation of state.  It holds none of the arithmetic of the step
itself (no kernel sums, no EoS inversion, no equations of motion), so the CUDA
path and the CPU oracle can both consume what it produces without sharing any
of the method's code.

Units everywhere: lengths and times in fm, temperatures and chemical potentials
in fm^-1, entropy and charge densities in fm^-3, energy densities and pressures
in fm^-4 (hbar*c = 0.1973269804 GeV fm converts GeV <-> fm^-1).

Workloads (shapes follow the paper's test setups, Sec. "Code validation" and
Sec. "Convergence Tests"):
  * ``gubser_ideal_2p1``      -- ideal conformal 2+1D Gubser flow, 51x51 lattice.
  * ``viscous_bsq_2p1``       -- 2+1D viscous BSQ event: 200 Gaussian hotspots in a
                                 7 fm disc, ~40k particles, synthetic 4D EoS table.
  * ``synthetic_eos_table``   -- node values of p, s, n_B, n_S, n_Q on a regular
                                 (T, mu_B, mu_S, mu_Q) grid (the paper's online-inverter
                                 input, Sec. "Equation of state").
  * ``bjorken_lattice_2p1``   -- uniform lattice (longitudinal Bjorken flow test).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

HBARC = 0.1973269804  # GeV fm

# ---------------------------------------------------------------------------
# counter-based generator (SplitMix64), so every input is reproducible bit for
# bit on any machine and numpy version
# ---------------------------------------------------------------------------
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n outputs of SplitMix64 started at counter ``offset`` for ``seed``."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed) + k * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


# ---------------------------------------------------------------------------
# parameter records
# ---------------------------------------------------------------------------
@dataclass
class AnalyticEoS:
    """p(T, mu) = T^4 [a0 + a1 (1 + tanh((T - Tc)/w))/2] + T^2 sum_q chi_q mu_q^2 / 2.

    Tc and w are in GeV (the tanh argument is evaluated in GeV); T, mu in fm^-1.
    a1 = 0 and chi = 0 give the conformal EoS p = eps/3 with eps = 3 a0 T^4.
    """
    a0: float
    a1: float = 0.0
    Tc_GeV: float = 0.155
    w_GeV: float = 0.02
    chi: tuple = (0.0, 0.0, 0.0)


@dataclass
class EoSTable:
    """Regular (T, mu_B, mu_S, mu_Q) grid, axis values in fm^-1, row-major with mu_Q fastest."""
    T0: float
    dT: float
    nT: int
    mu0: tuple
    dmu: tuple
    nmu: tuple
    p: np.ndarray
    s: np.ndarray
    nB: np.ndarray
    nS: np.ndarray
    nQ: np.ndarray


@dataclass
class Transport:
    viscous: bool = False
    eta_over_s: float = 0.0
    zeta_peak: float = 0.0        # peak of zeta/s
    zeta_T_GeV: float = 0.155     # temperature of the peak
    zeta_w_GeV: float = 0.02      # Gaussian standard deviation
    tau_pi_coef: float = 5.0      # tau_pi = coef * eta / (eps + p)
    tau_Pi_ratio: float = 1.0     # tau_Pi = ratio * tau_pi
    cs2_cap: float = 1.0          # causal cap on c_s^2 in the acceleration system
    # temperature (GeV) below which a particle leaves the fluid and streams freely (0: off)
    T_stop_GeV: float = 0.0
    # None: minimal Israel-Stewart; else DNMR with the coefficient ratios (delta_PiPi / tau_Pi,
    # lambda_Pipi / (tau_Pi (1/3 - c_s^2)), delta_pipi / tau_pi, tau_pipi / tau_pi,
    # lambda_piPi / tau_pi, phi_7 p), e.g. DNMR_14_MOMENT
    dnmr: tuple | None = None


# DNMR coefficient ratios of the 14-moment approximation for a massless Boltzmann gas
DNMR_14_MOMENT = (2.0 / 3.0, 8.0 / 5.0, 4.0 / 3.0, 10.0 / 7.0, 6.0 / 5.0, 9.0 / 70.0)


@dataclass
class Diffusion:
    """BSQ diffusion (minimal Israel-Stewart): constant kappa_{qq'}/T^2 (3 x 3, row q = B, S, Q)
    and relaxation times tau_q = tauJT[q] / T; Jv (3 dim x N, charge major, or None for zero):
    the initial J^i_q / sigma."""
    kappaT2: tuple
    tauJT: tuple = (0.2, 0.2, 0.2)
    Jv: np.ndarray | None = None


# the full BSQ matrix of the paper's diffusion study (Sec. "BSQ Diffusion and the Beam Energy Scan")
KAPPA_BSQ = ((0.0482, -0.0482, 0.0), (-0.0482, 0.1447, 0.0147), (0.0, 0.0147, 0.0880))


@dataclass
class JetTracks:
    """Straight jet tracks moving at the speed of light, each depositing energy dE/dx per unit
    path length (spread over a Gaussian of width sigma) into the fluid: rows
    (x0, y0, z0, n_x, n_y, n_z, t0, dE/dx [fm^-2]) in Cartesian coordinates."""
    tracks: np.ndarray
    sigma: float


@dataclass
class PartonSources:
    """Dynamical-initialisation sources: partons [N][8] = formation time, position (x, y,
    z or eta), four-momentum p^mu (contravariant, fm^-1, the event's coordinates); each is
    smeared with the SPH kernel of width h over the step in which it forms, scaled by norm."""
    partons: np.ndarray
    norm: float = 1.0
    h: float = 1.4
    # [N][3] charges (B, S, Q) of the partons, smeared like their four-momenta (None: no charge
    # sources, the particles' charges stay constant)
    charges: np.ndarray | None = None


@dataclass
class InverseGrid:
    """Grid of the offline-inverted EoS table: s on log decades 10^decade_lo .. 10^(decade_lo +
    decades) with per_decade uniform nodes per decade (s = 10^d (1 + 9 j / per_decade)), and the
    charge ratios n_q / s on nx uniform nodes in [-xmax, xmax]."""
    per_decade: int = 90
    decade_lo: int = -3
    decades: int = 6
    nx: int = 17
    xmax: float = 0.04


@dataclass
class Event:
    """One event: SoA particle arrays plus run parameters."""
    name: str
    dim: int
    milne: bool
    h: float
    tau0: float
    dtau: float
    nsteps: int
    x: np.ndarray            # [dim][N] positions (fm; eta is dimensionless)
    u: np.ndarray            # [dim][N] contravariant spatial u^i
    S: np.ndarray            # [N] entropy per particle
    Nq: np.ndarray           # [3][N] B, S, Q charge per particle
    Bv: np.ndarray           # [N]  Pi / sigma
    Pv: np.ndarray           # [npi][N] pi^{ij} / sigma (xx, xy, yy for dim 2)
    eos: AnalyticEoS
    table: EoSTable | None
    transport: Transport
    meta: dict = field(default_factory=dict)
    jets: JetTracks | None = None
    inverse: InverseGrid | None = None  # set: the EoS is inverted by the offline table
    partons: PartonSources | None = None  # dynamical-initialisation sources
    # backup EoS (conformal diagonal) where neither the table nor the closed form inverts:
    # (T_scale, mu_max) in GeV, or None for none
    eos_backup: tuple | None = None
    diffusion: Diffusion | None = None  # BSQ diffusion currents

    @property
    def n(self) -> int:
        return int(self.S.shape[0])


# ---------------------------------------------------------------------------
# forward closed-form EoS, used here only to synthesise inputs (table nodes,
# initial entropy amplitudes).  The step's own EoS code lives elsewhere.
# ---------------------------------------------------------------------------
def _analytic_p_s_n(eos: AnalyticEoS, T: np.ndarray, mu: np.ndarray):
    T = np.asarray(T, dtype=np.float64)
    x = T * HBARC
    arg = (x - eos.Tc_GeV) / eos.w_GeV
    th = np.tanh(arg)
    f = eos.a0 + eos.a1 * (1.0 + th) / 2.0
    fp = eos.a1 / 2.0 * (1.0 - th * th) * HBARC / eos.w_GeV
    chi = np.asarray(eos.chi, dtype=np.float64).reshape(3, *([1] * T.ndim))
    mu = np.asarray(mu, dtype=np.float64)
    sum_chi_mu2 = np.sum(chi * mu * mu, axis=0)
    p = T ** 4 * f + T * T * sum_chi_mu2 / 2.0
    s = 4.0 * T ** 3 * f + T ** 4 * fp + T * sum_chi_mu2
    n = chi * T * T * mu
    return p, s, n


def synthetic_eos_table(eos: AnalyticEoS, nT=64, nmu=32, T_GeV=(0.05, 0.8), mu_GeV=0.45) -> EoSTable:
    """Tabulate the closed-form EoS on the grid T in [0.05, 0.8] GeV, mu in [-0.45, 0.45] GeV."""
    T0 = T_GeV[0] / HBARC
    dT = (T_GeV[1] - T_GeV[0]) / (nT - 1) / HBARC
    m0 = -mu_GeV / HBARC
    dm = 2.0 * mu_GeV / (nmu - 1) / HBARC
    T = T0 + dT * np.arange(nT)
    mu = m0 + dm * np.arange(nmu)
    TT, MB, MS, MQ = np.meshgrid(T, mu, mu, mu, indexing="ij")
    p, s, n = _analytic_p_s_n(eos, TT, np.stack([MB, MS, MQ]))
    c = np.ascontiguousarray
    return EoSTable(T0=T0, dT=dT, nT=nT, mu0=(m0, m0, m0), dmu=(dm, dm, dm), nmu=(nmu, nmu, nmu),
                    p=c(p), s=c(s), nB=c(n[0]), nS=c(n[1]), nQ=c(n[2]))


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
BJ_EOS = AnalyticEoS(a0=0.3, a1=2.5, Tc_GeV=0.155, w_GeV=0.02, chi=(0.3, 0.5, 0.4))
# the same family with a 0.04 GeV crossover: c_s^2 <= 0.41 everywhere (causal), used by the
# energy-balance test where the c_s^2 cap must not engage
CAUSAL_EOS = AnalyticEoS(a0=0.3, a1=2.5, Tc_GeV=0.155, w_GeV=0.04, chi=(0.3, 0.5, 0.4))
GUBSER_FSTAR = 11.0


def gubser_T_u(tau, x, y, q=1.0, T0_GeV=0.4, tau0=1.0):
    """Ideal Gubser flow (H0 = 0): T in fm^-1 and (u^tau, u^x, u^y), with T(tau0, r=0) = T0."""
    r2 = x * x + y * y
    r = np.sqrt(r2)

    def cosh_rho(t, rr2):
        sh = (q * q * (t * t - rr2) - 1.0) / (2.0 * q * t)
        return np.sqrt(1.0 + sh * sh)

    T = (T0_GeV / HBARC) * (tau0 / tau) * (cosh_rho(tau0, 0.0) / cosh_rho(tau, r2)) ** (2.0 / 3.0)
    den = np.sqrt(1.0 + 2.0 * q * q * (tau * tau + r2) + q ** 4 * (tau * tau - r2) ** 2)
    utau = (1.0 + q * q * (tau * tau + r2)) / den
    ur = 2.0 * q * q * r * tau / den
    with np.errstate(invalid="ignore", divide="ignore"):
        ux = np.where(r > 0, ur * x / np.where(r > 0, r, 1.0), 0.0)
        uy = np.where(r > 0, ur * y / np.where(r > 0, r, 1.0), 0.0)
    return T, utau, ux, uy


def gubser_ideal_2p1(n_side=51, half_width=5.0, h=0.5, tau0=1.0, dtau=0.01, nsteps=60) -> Event:
    """Config: ideal conformal 2+1D boost-invariant Gubser flow (q = 1/fm, T0 = 0.4 GeV at tau0 = 1 fm)."""
    g = np.linspace(-half_width, half_width, n_side)
    dx = g[1] - g[0]
    X, Y = np.meshgrid(g, g, indexing="ij")
    x, y = X.ravel().copy(), Y.ravel().copy()
    T, utau, ux, uy = gubser_T_u(tau0, x, y)
    eos = AnalyticEoS(a0=GUBSER_FSTAR / 3.0)
    _, s, _ = _analytic_p_s_n(eos, T, np.zeros((3, x.size)))
    S = s * utau * tau0 * dx * dx
    n = x.size
    return Event(name="gubser_ideal_2p1", dim=2, milne=True, h=h, tau0=tau0, dtau=dtau, nsteps=nsteps,
                 x=np.stack([x, y]), u=np.stack([ux, uy]), S=S, Nq=np.zeros((3, n)),
                 Bv=np.zeros(n), Pv=np.zeros((3, n)), eos=eos, table=None,
                 transport=Transport(viscous=False), meta={"dx": dx})


def gubser_shifted_T_u(tau, x, y, eta, t0=0.5, q=1.0, T0_GeV=0.4):
    """Ideal Gubser flow shifted in Minkowski time, t -> t + t0 (Sec. "Code validation", eqs.
    tau_prime, shifted_viscous_Gubser_T/_ur/_utau/_ueta with H0 = 0): T(tau', r) in fm^-1 and the
    contravariant (u^tau, u^x, u^y, u^eta) in Milne coordinates (tau, x, y, eta)."""
    ch, sh = np.cosh(eta), np.sinh(eta)
    taup = np.sqrt(tau * tau + 2.0 * t0 * tau * ch + t0 * t0)
    T, utp, ux, uy = gubser_T_u(taup, x, y, q=q, T0_GeV=T0_GeV)
    utau = utp * (tau + t0 * ch) / taup
    ueta = -utp * t0 * sh / (tau * taup)
    return T, utau, ux, uy, ueta


def gubser_shifted_3p1(half_widths=(2.4, 2.4, 1.5), spacings=(0.2, 0.2, 0.1), h=0.4, tau0=1.0, t0=0.5,
                       dtau=0.01, nsteps=20) -> Event:
    """Config: ideal conformal 3+1D Milne flow with rapidity dependence, the Gubser solution
    shifted by t0 in Minkowski time (q = 1/fm; T = 0.4 GeV at tau' = 1 fm, r = 0), on a box
    lattice in (x, y, eta)."""
    x = lattice_3d(half_widths, spacings)
    n = x.shape[1]
    T, utau, ux, uy, ueta = gubser_shifted_T_u(tau0, x[0], x[1], x[2], t0=t0)
    eos = AnalyticEoS(a0=GUBSER_FSTAR / 3.0)
    _, s, _ = _analytic_p_s_n(eos, T, np.zeros((3, n)))
    S = s * utau * tau0 * spacings[0] * spacings[1] * spacings[2]
    return Event(name="gubser_shifted_3p1", dim=3, milne=True, h=h, tau0=tau0, dtau=dtau, nsteps=nsteps,
                 x=x, u=np.stack([ux, uy, ueta]), S=S, Nq=np.zeros((3, n)), Bv=np.zeros(n),
                 Pv=np.zeros((5, n)), eos=eos, table=None, transport=Transport(viscous=False),
                 meta={"spacings": spacings, "t0": t0})


def disc_lattice(R: float, n_target: int):
    """Square lattice with spacing sqrt(pi R^2 / n_target), points with x^2 + y^2 <= R^2."""
    dx = math.sqrt(math.pi * R * R / n_target)
    m = int(math.ceil(R / dx)) + 1
    g = dx * np.arange(-m, m + 1)
    X, Y = np.meshgrid(g, g, indexing="ij")
    keep = (X * X + Y * Y) <= R * R
    return X[keep].copy(), Y[keep].copy(), dx


def viscous_bsq_2p1(n_target=40000, R=7.0, n_hot=200, sigma_hot=0.4, T_max_GeV=0.5,
                    charge_frac=0.1, tau0=0.6, dtau=0.005, tau_end=8.0, h=0.3,
                    seed_hot=1, seed_charge=2, with_table=True, table_shape=(64, 32),
                    coherent_charges=False) -> Event:
    """Config: viscous 2+1D BSQ single event (eta/s = 0.08, Gaussian zeta/s, synthetic 4D EoS table).

    Entropy: sum of ``n_hot`` Gaussian hotspots (sigma 0.4 fm) with centres uniform in the disc,
    scaled so that max s = s(T_max, mu = 0).  Charges n_q = eps_q s with eps_q ~ U(-charge_frac,
    charge_frac) per particle and charge.  ``coherent_charges``: eps_q = +charge_frac everywhere
    (the kernel sums then keep n/s = charge_frac, which has no EoS solution for hot particles
    at 0.1 -- the failure-path case).
    """
    x, y, dx = disc_lattice(R, n_target)
    u = uniform01(seed_hot, 2 * n_hot)
    rc = R * np.sqrt(u[:n_hot])
    ph = 2.0 * math.pi * u[n_hot:]
    cx, cy = rc * np.cos(ph), rc * np.sin(ph)
    s_raw = np.zeros_like(x)
    for k in range(n_hot):
        s_raw += np.exp(-((x - cx[k]) ** 2 + (y - cy[k]) ** 2) / (2.0 * sigma_hot ** 2))
    _, s_max, _ = _analytic_p_s_n(BJ_EOS, np.array(T_max_GeV / HBARC), np.zeros(3))
    s = s_raw * (float(s_max) / s_raw.max())
    n = x.size
    if coherent_charges:
        eps = np.full((3, n), charge_frac)
    else:
        eps = charge_frac * (2.0 * uniform01(seed_charge, 3 * n).reshape(3, n) - 1.0)
    nq = eps * s[None, :]
    vol = tau0 * dx * dx
    table = synthetic_eos_table(BJ_EOS, nT=table_shape[0], nmu=table_shape[1]) if with_table else None
    nsteps = int(round((tau_end - tau0) / dtau))
    return Event(name="viscous_bsq_2p1", dim=2, milne=True, h=h, tau0=tau0, dtau=dtau, nsteps=nsteps,
                 x=np.stack([x, y]), u=np.zeros((2, n)), S=s * vol, Nq=nq * vol,
                 Bv=np.zeros(n), Pv=np.zeros((3, n)), eos=BJ_EOS, table=table,
                 transport=Transport(viscous=True, eta_over_s=0.08, zeta_peak=0.05,
                                     zeta_T_GeV=0.155, zeta_w_GeV=0.02),
                 meta={"dx": dx, "hotspots": np.stack([cx, cy])})


def bjorken_lattice_2p1(T0_GeV=0.16, n_side=41, dx=0.1, h=0.3, tau0=0.6, dtau=0.005, nsteps=100,
                        viscous=True, with_table=False) -> Event:
    """Uniform-temperature square lattice at rest: interior particles follow longitudinal
    (Bjorken) boost-invariant flow until the edge rarefaction arrives."""
    g = dx * (np.arange(n_side) - (n_side - 1) / 2.0)
    X, Y = np.meshgrid(g, g, indexing="ij")
    x, y = X.ravel().copy(), Y.ravel().copy()
    n = x.size
    _, s, _ = _analytic_p_s_n(BJ_EOS, np.full(n, T0_GeV / HBARC), np.zeros((3, n)))
    table = synthetic_eos_table(BJ_EOS) if with_table else None
    return Event(name="bjorken_lattice_2p1", dim=2, milne=True, h=h, tau0=tau0, dtau=dtau, nsteps=nsteps,
                 x=np.stack([x, y]), u=np.zeros((2, n)), S=s * tau0 * dx * dx, Nq=np.zeros((3, n)),
                 Bv=np.zeros(n), Pv=np.zeros((3, n)), eos=BJ_EOS, table=table,
                 transport=Transport(viscous=viscous, eta_over_s=0.08 if viscous else 0.0,
                                     zeta_peak=0.05 if viscous else 0.0),
                 meta={"dx": dx})


def random_points(n: int, dim: int, extent: float, seed: int) -> np.ndarray:
    """[dim][n] uniform points in [-extent, extent]^dim (neighbour-search tests)."""
    return (2.0 * uniform01(seed, dim * n).reshape(dim, n) - 1.0) * extent


def smooth_blob_2p1(half_width=4.0, dx=0.1, h=0.3, T_peak_GeV=0.45, T_floor_GeV=0.06, sigma=1.2,
                    ecc=0.25, charge_frac=0.01, tau0=0.6, dtau=0.005, nsteps=200, viscous=True,
                    with_table=True, seed_charge=7, eos: AnalyticEoS = None) -> Event:
    """Smooth elliptic Gaussian temperature profile on a square lattice that reaches a cold floor
    well inside the lattice edge (no free surface at high pressure): the energy-balance test case."""
    g = dx * np.arange(-int(round(half_width / dx)), int(round(half_width / dx)) + 1)
    X, Y = np.meshgrid(g, g, indexing="ij")
    x, y = X.ravel().copy(), Y.ravel().copy()
    n = x.size
    eos = BJ_EOS if eos is None else eos
    prof = np.exp(-(x * x / (1.0 + ecc) + y * y / (1.0 - ecc)) / (2.0 * sigma * sigma))
    T = (T_floor_GeV + (T_peak_GeV - T_floor_GeV) * prof) / HBARC
    _, s, _ = _analytic_p_s_n(eos, T, np.zeros((3, n)))
    eps = charge_frac * (2.0 * uniform01(seed_charge, 3 * n).reshape(3, n) - 1.0)
    vol = tau0 * dx * dx
    table = synthetic_eos_table(eos) if with_table else None
    return Event(name="smooth_blob_2p1", dim=2, milne=True, h=h, tau0=tau0, dtau=dtau, nsteps=nsteps,
                 x=np.stack([x, y]), u=np.zeros((2, n)), S=s * vol, Nq=eps * s[None, :] * vol,
                 Bv=np.zeros(n), Pv=np.zeros((3, n)), eos=eos, table=table,
                 transport=Transport(viscous=viscous, eta_over_s=0.08 if viscous else 0.0,
                                     zeta_peak=0.05 if viscous else 0.0),
                 meta={"dx": dx})


def lattice_3d(half_widths, spacings):
    """[3][N] points of a box lattice centred on the origin (x, y, and eta or z)."""
    axes = [d * (np.arange(int(round(2 * hw / d)) + 1) - int(round(2 * hw / d)) / 2.0)
            for hw, d in zip(half_widths, spacings)]
    G = np.meshgrid(*axes, indexing="ij")
    return np.stack([g.ravel() for g in G]).copy()


def bjorken_lattice_3p1(T0_GeV=0.16, half_widths=(0.8, 0.8, 0.4), spacings=(0.1, 0.1, 0.05), h=0.3,
                        tau0=0.6, dtau=0.005, nsteps=40, viscous=True) -> Event:
    """Uniform temperature at rest on a 3D Milne lattice (x, y, eta): interior particles follow
    longitudinal Bjorken flow until the edge rarefaction arrives."""
    x = lattice_3d(half_widths, spacings)
    n = x.shape[1]
    _, s, _ = _analytic_p_s_n(BJ_EOS, np.full(n, T0_GeV / HBARC), np.zeros((3, n)))
    vol = tau0 * spacings[0] * spacings[1] * spacings[2]
    return Event(name="bjorken_lattice_3p1", dim=3, milne=True, h=h, tau0=tau0, dtau=dtau, nsteps=nsteps,
                 x=x, u=np.zeros((3, n)), S=s * vol, Nq=np.zeros((3, n)), Bv=np.zeros(n), Pv=np.zeros((5, n)),
                 eos=BJ_EOS, table=None,
                 transport=Transport(viscous=viscous, eta_over_s=0.08 if viscous else 0.0,
                                     zeta_peak=0.05 if viscous else 0.0),
                 meta={"spacings": spacings})


def smooth_blob_3d(milne=True, half_widths=(1.6, 1.6, 1.2), spacings=(0.16, 0.16, 0.12), h=0.3,
                   T_peak_GeV=0.4, T_floor_GeV=0.07, sigma=(0.8, 0.6, 0.5), charge_frac=0.1, tau0=0.6,
                   dtau=0.005, nsteps=20, viscous=True, with_table=True, eos: AnalyticEoS = None, seed_charge=11,
                   flow=0.0) -> Event:
    """Smooth anisotropic Gaussian temperature profile on a 3D lattice, Milne (x, y, eta) or
    Cartesian (x, y, z), optional initial radial flow u^i = flow * x^i (transverse) to exercise
    the acceleration and shear terms."""
    eos = BJ_EOS if eos is None else eos
    x = lattice_3d(half_widths, spacings)
    n = x.shape[1]
    prof = np.exp(-sum(x[d] ** 2 / (2.0 * sigma[d] ** 2) for d in range(3)))
    T = (T_floor_GeV + (T_peak_GeV - T_floor_GeV) * prof) / HBARC
    _, s, _ = _analytic_p_s_n(eos, T, np.zeros((3, n)))
    eps = charge_frac * (2.0 * uniform01(seed_charge, 3 * n).reshape(3, n) - 1.0)
    u = np.zeros((3, n))
    u[0], u[1] = flow * x[0], flow * x[1]
    gamma = np.sqrt(1.0 + u[0] ** 2 + u[1] ** 2)
    vol = (tau0 if milne else 1.0) * spacings[0] * spacings[1] * spacings[2]
    table = synthetic_eos_table(eos) if with_table else None
    return Event(name="smooth_blob_3d", dim=3, milne=milne, h=h, tau0=tau0, dtau=dtau, nsteps=nsteps,
                 x=x, u=u, S=s * gamma * vol, Nq=eps * (s * gamma * vol)[None, :], Bv=np.zeros(n),
                 Pv=np.zeros((5, n)), eos=eos, table=table,
                 transport=Transport(viscous=viscous, eta_over_s=0.08 if viscous else 0.0,
                                     zeta_peak=0.05 if viscous else 0.0),
                 meta={"spacings": spacings})


def viscous_bsq_3p1(dx=0.124, deta=0.1, R=7.0, n_hot=200, sigma_hot=0.4, eta_sigma=1.5, eta_max=5.0,
                    T_max_GeV=0.5, charge_frac=0.1, tau0=0.6, dtau=0.005, h=0.3, seed_hot=1, seed_charge=2,
                    with_table=True) -> Event:
    """Config: 3+1D hyperbolic (tau, x, y, eta_s) viscous BSQ event: the transverse hotspot
    profile of the 2+1D event times exp(-eta^2/(2 sigma_eta^2)) for |eta| <= eta_max, on a
    lattice dx = dy = 0.124 fm, d_eta = 0.1 (about 10^6 particles at the defaults)."""
    m = int(math.ceil(R / dx)) + 1
    g = dx * np.arange(-m, m + 1)
    X, Y = np.meshgrid(g, g, indexing="ij")
    keep = (X * X + Y * Y) <= R * R
    xt, yt = X[keep], Y[keep]
    ke = int(round(eta_max / deta))
    etas = deta * np.arange(-ke, ke + 1)
    u = uniform01(seed_hot, 2 * n_hot)
    rc = R * np.sqrt(u[:n_hot])
    ph = 2.0 * math.pi * u[n_hot:]
    cx, cy = rc * np.cos(ph), rc * np.sin(ph)
    s_t = np.zeros_like(xt)
    for k in range(n_hot):
        s_t += np.exp(-((xt - cx[k]) ** 2 + (yt - cy[k]) ** 2) / (2.0 * sigma_hot ** 2))
    _, s_max, _ = _analytic_p_s_n(BJ_EOS, np.array(T_max_GeV / HBARC), np.zeros(3))
    s_t *= float(s_max) / s_t.max()
    x = np.repeat(xt[None, :], etas.size, axis=0).ravel()
    y = np.repeat(yt[None, :], etas.size, axis=0).ravel()
    eta = np.repeat(etas[:, None], xt.size, axis=1).ravel()
    s = np.repeat(s_t[None, :], etas.size, axis=0).ravel() * np.exp(-eta ** 2 / (2.0 * eta_sigma ** 2))
    n = x.size
    eps = charge_frac * (2.0 * uniform01(seed_charge, 3 * n).reshape(3, n) - 1.0)
    vol = tau0 * dx * dx * deta
    table = synthetic_eos_table(BJ_EOS) if with_table else None
    return Event(name="viscous_bsq_3p1", dim=3, milne=True, h=h, tau0=tau0, dtau=dtau, nsteps=20,
                 x=np.stack([x, y, eta]), u=np.zeros((3, n)), S=s * vol, Nq=eps * (s * vol)[None, :],
                 Bv=np.zeros(n), Pv=np.zeros((5, n)), eos=BJ_EOS, table=table,
                 transport=Transport(viscous=True, eta_over_s=0.08, zeta_peak=0.05, zeta_T_GeV=0.155,
                                     zeta_w_GeV=0.02),
                 meta={"dx": dx, "deta": deta})


def jet_tracks(n_tracks=10, R=7.0, dEdx_GeV_per_fm=5.0, sigma=0.3, t0=0.0, z_half=0.0, seed=5) -> JetTracks:
    """Seeded straight tracks: origins uniform in the disc of radius R (z uniform in +-z_half),
    isotropic directions, all starting at t0, depositing dEdx (GeV/fm, stored in fm^-2)."""
    u = uniform01(seed, 5 * n_tracks).reshape(5, n_tracks)
    rr = R * np.sqrt(u[0])
    ph = 2.0 * math.pi * u[1]
    z0 = z_half * (2.0 * u[2] - 1.0)
    cth = 2.0 * u[3] - 1.0
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    ps = 2.0 * math.pi * u[4]
    tr = np.stack([rr * np.cos(ph), rr * np.sin(ph), z0, sth * np.cos(ps), sth * np.sin(ps), cth,
                   np.full(n_tracks, float(t0)), np.full(n_tracks, dEdx_GeV_per_fm / HBARC)], axis=1)
    return JetTracks(tracks=np.ascontiguousarray(tr), sigma=float(sigma))


def uniform_box_3d(T_GeV=0.3, half_widths=(1.2, 1.2, 1.2), spacing=0.12, h=0.3, t0=1.0, dtau=0.005,
                   nsteps=10, viscous=False, jets: JetTracks | None = None) -> Event:
    """A uniform fluid at rest in a Cartesian box (the test medium of the source terms)."""
    x = lattice_3d(half_widths, (spacing, spacing, spacing))
    n = x.shape[1]
    _, s, _ = _analytic_p_s_n(CAUSAL_EOS, np.full(n, T_GeV / HBARC), np.zeros((3, n)))
    return Event(name="uniform_box_3d", dim=3, milne=False, h=h, tau0=t0, dtau=dtau, nsteps=nsteps, x=x,
                 u=np.zeros((3, n)), S=s * spacing ** 3, Nq=np.zeros((3, n)), Bv=np.zeros(n),
                 Pv=np.zeros((5, n)), eos=CAUSAL_EOS, table=None,
                 transport=Transport(viscous=viscous, eta_over_s=0.08 if viscous else 0.0),
                 meta={"dx": spacing}, jets=jets)


def boosted_sound_wave_2d(T_GeV=0.3, v=0.5, amp=1e-3, wavelength=4.0, half_widths=(5.6, 3.4), spacing=0.1,
                          h=0.3, t0=0.0, dtau=0.01, nsteps=300, zeta_over_s=0.2, eta_over_s=1e-4,
                          tau_pi_coef=5000.0, tau_Pi_ratio=1.0) -> Event:
    """A uniform conformal fluid (e = 11 T^4, no charges) moving with velocity v along x in a
    Cartesian 2D box, carrying a small sound wave: e(x) = e0 (1 + amp cos(2 pi x / wavelength)),
    u^i = (gamma v, 0), Pi = pi = 0 at t0.  Bulk viscosity zeta/s constant (a Gaussian of
    essentially infinite width), a small shear viscosity whose relaxation time
    tau_pi = tau_pi_coef eta/(e + p) sets tau_Pi = tau_Pi_ratio tau_pi."""
    eos = AnalyticEoS(a0=GUBSER_FSTAR / 3.0)
    gx = spacing * (np.arange(int(round(2 * half_widths[0] / spacing)) + 1) - round(half_widths[0] / spacing))
    gy = spacing * (np.arange(int(round(2 * half_widths[1] / spacing)) + 1) - round(half_widths[1] / spacing))
    X, Y = np.meshgrid(gx, gy, indexing="ij")
    x, y = X.ravel().copy(), Y.ravel().copy()
    n = x.size
    k = 2.0 * math.pi / wavelength
    T = (T_GeV / HBARC) * (1.0 + amp * np.cos(k * x)) ** 0.25
    _, s, _ = _analytic_p_s_n(eos, T, np.zeros((3, n)))
    gam = 1.0 / math.sqrt(1.0 - v * v)
    u = np.zeros((2, n))
    u[0] = gam * v
    return Event(name="boosted_sound_wave_2d", dim=2, milne=False, h=h, tau0=t0, dtau=dtau, nsteps=nsteps,
                 x=np.stack([x, y]), u=u, S=s * gam * spacing * spacing, Nq=np.zeros((3, n)), Bv=np.zeros(n),
                 Pv=np.zeros((3, n)), eos=eos, table=None,
                 transport=Transport(viscous=True, eta_over_s=eta_over_s, zeta_peak=zeta_over_s,
                                     zeta_T_GeV=T_GeV, zeta_w_GeV=1.0e6, tau_pi_coef=tau_pi_coef,
                                     tau_Pi_ratio=tau_Pi_ratio),
                 meta={"dx": spacing, "k": k, "v": v, "T0": T_GeV / HBARC, "amp": amp})


def diffusion_box_2d(T_GeV=0.3, v=0.0, amps=(1e-3, -7e-4, 5e-4), wavelength=4.0, half_widths=(6.0, 3.4),
                     spacing=0.1, h=0.3, t0=0.0, dtau=0.01, nsteps=200, kappaT2=None, tauJT=(0.2, 0.2, 0.2)) -> Event:
    """A uniform fluid at zero chemical potentials (e = 11 T^4 plus the charges' chi_q T^2 mu_q^2 / 2,
    chi = (0.3, 0.5, 0.4)) moving with velocity v along x in a Cartesian 2D box, carrying small
    charge waves n_q = chi_q T^3 amps[q] cos(2 pi x / wavelength) (alpha_q = mu_q / T = amps[q]
    cos(...)), ideal apart from BSQ diffusion with constant kappaT2 (3 x 3) and tau_q = tauJT[q] / T,
    J = 0 at t0."""
    eos = AnalyticEoS(a0=GUBSER_FSTAR / 3.0, chi=(0.3, 0.5, 0.4))
    gx = spacing * (np.arange(int(round(2 * half_widths[0] / spacing)) + 1) - round(half_widths[0] / spacing))
    gy = spacing * (np.arange(int(round(2 * half_widths[1] / spacing)) + 1) - round(half_widths[1] / spacing))
    X, Y = np.meshgrid(gx, gy, indexing="ij")
    x, y = X.ravel().copy(), Y.ravel().copy()
    n = x.size
    k = 2.0 * math.pi / wavelength
    T = T_GeV / HBARC
    mu = np.stack([T * amps[q] * np.cos(k * x) for q in range(3)])
    _, s, nq = _analytic_p_s_n(eos, np.full(n, T), mu)
    gam = 1.0 / math.sqrt(1.0 - v * v)
    u = np.zeros((2, n))
    u[0] = gam * v
    vol = gam * spacing * spacing
    kap = KAPPA_BSQ if kappaT2 is None else kappaT2
    return Event(name="diffusion_box_2d", dim=2, milne=False, h=h, tau0=t0, dtau=dtau, nsteps=nsteps,
                 x=np.stack([x, y]), u=u, S=s * vol, Nq=nq * vol, Bv=np.zeros(n), Pv=np.zeros((3, n)), eos=eos,
                 table=None, transport=Transport(viscous=False),
                 meta={"dx": spacing, "k": k, "v": v, "T0": T, "amps": amps},
                 diffusion=Diffusion(kappaT2=kap, tauJT=tauJT))


def stress_cartesian_3d(n_target=8_000_000, R=7.0, z_sigma=1.5, z_max=5.0, h=0.15, n_hot=200, sigma_hot=0.4,
                        T_max_GeV=0.5, charge_frac=0.1, t0=0.6, dtau=0.005, n_tracks=10, seed_hot=1,
                        seed_charge=2, seed_tracks=5, table_shape=(128, 64), with_table=True) -> Event:
    """Config: 3+1D Cartesian (t, x, y, z) viscous BSQ event with jet tracks -- the transverse
    hotspot profile of the 2+1D event times exp(-z^2/(2 z_sigma^2)) for |z| <= z_max on a cubic
    lattice whose spacing gives about n_target particles (0.0577 fm for 8 10^6), h = 0.15 fm
    (about 600 neighbours, as in the 3+1D Milne event), 10 seeded tracks (origins in the disc,
    |z0| <= 1 fm, isotropic directions) depositing 5 GeV/fm into Gaussians of width 0.3 fm from
    t0, and a 128 x 64^3 EoS table."""
    dx = (math.pi * R * R * 2.0 * z_max / n_target) ** (1.0 / 3.0)
    m = int(math.ceil(R / dx)) + 1
    g = dx * np.arange(-m, m + 1)
    X, Y = np.meshgrid(g, g, indexing="ij")
    keep = (X * X + Y * Y) <= R * R
    xt, yt = X[keep], Y[keep]
    kz = int(math.floor(z_max / dx))
    zs = dx * np.arange(-kz, kz + 1)
    u = uniform01(seed_hot, 2 * n_hot)
    rc = R * np.sqrt(u[:n_hot])
    ph = 2.0 * math.pi * u[n_hot:]
    cx, cy = rc * np.cos(ph), rc * np.sin(ph)
    s_t = np.zeros_like(xt)
    for k in range(n_hot):
        s_t += np.exp(-((xt - cx[k]) ** 2 + (yt - cy[k]) ** 2) / (2.0 * sigma_hot ** 2))
    _, s_max, _ = _analytic_p_s_n(BJ_EOS, np.array(T_max_GeV / HBARC), np.zeros(3))
    s_t *= float(s_max) / s_t.max()
    nt, nz = xt.size, zs.size
    x = np.tile(xt, nz)
    y = np.tile(yt, nz)
    z = np.repeat(zs, nt)
    s = np.tile(s_t, nz) * np.exp(-z ** 2 / (2.0 * z_sigma ** 2))
    n = x.size
    eps = charge_frac * (2.0 * uniform01(seed_charge, 3 * n).reshape(3, n) - 1.0)
    vol = dx ** 3
    table = synthetic_eos_table(BJ_EOS, nT=table_shape[0], nmu=table_shape[1]) if with_table else None
    return Event(name="stress_cartesian_3d", dim=3, milne=False, h=h, tau0=t0, dtau=dtau, nsteps=5,
                 x=np.stack([x, y, z]), u=np.zeros((3, n)), S=s * vol, Nq=eps * (s * vol)[None, :],
                 Bv=np.zeros(n), Pv=np.zeros((5, n)), eos=BJ_EOS, table=table,
                 transport=Transport(viscous=True, eta_over_s=0.08, zeta_peak=0.05, zeta_T_GeV=0.155,
                                     zeta_w_GeV=0.02),
                 meta={"dx": dx},
                 jets=jet_tracks(n_tracks=n_tracks, R=R, t0=t0, z_half=1.0, seed=seed_tracks))


def parton_sources(n: int, t_range, half_extent, dim: int, E_GeV=(1.0, 3.0), norm=0.42, h=1.4, seed=6):
    """n seeded partons with formation times uniform in t_range, positions uniform in a centred
    cube of half-width half_extent (dim axes), massless four-momenta with energies uniform in
    E_GeV and isotropic directions in the event's dimensions."""
    u = uniform01(seed, 6 * n).reshape(6, n)
    t = t_range[0] + (t_range[1] - t_range[0]) * u[0]
    x = np.zeros((3, n))
    for d in range(dim):
        x[d] = half_extent * (2.0 * u[1 + d] - 1.0)
    E = (E_GeV[0] + (E_GeV[1] - E_GeV[0]) * u[4]) / HBARC
    phi = 2.0 * np.pi * u[5]
    if dim == 3:
        ct = 2.0 * u[3] - 1.0
        st = np.sqrt(1.0 - ct * ct)
        nvec = np.stack([st * np.cos(phi), st * np.sin(phi), ct])
    else:
        nvec = np.stack([np.cos(phi), np.sin(phi), np.zeros(n)])
    p = np.concatenate([E[None, :], E[None, :] * nvec])
    partons = np.concatenate([t[None, :], x, p]).T.copy()
    return PartonSources(partons=partons, norm=norm, h=h)


# (B, S, Q) of the light quarks u, d, s and their antiquarks
QUARK_CHARGES = np.array([[1 / 3, 0, 2 / 3], [1 / 3, 0, -1 / 3], [1 / 3, -1, -1 / 3],
                          [-1 / 3, 0, -2 / 3], [-1 / 3, 0, 1 / 3], [-1 / 3, 1, 1 / 3]])


def parton_quark_charges(n: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """[n][3] seeded parton charges: each parton a light quark or antiquark (uniform choice of
    the six), its (B, S, Q) times scale."""
    u = uniform01(seed, n)
    return scale * QUARK_CHARGES[np.minimum((u * 6).astype(int), 5)]
