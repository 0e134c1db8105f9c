"""ctypes front end of the FP64 CPU oracle (``sph_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()`` (to
check the CUDA path) and by the cpu_baseline / reference leg of bench.py.  The
product package never imports it.

``build()`` compiles the C file with gcc (-O2 -ffp-contract=off -fopenmp) into
``oracle/_build/libsph_oracle.so``; it is rebuilt when the source is newer.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libsph_oracle.so")

NAUX = 18
FO_NREC = 24  # freeze-out record: tau, x^1..3, u^0..3, T, mu x3, e, p, s, n_0..3, |dsigma|, dsigma_0..3
AUX = {name: i for i, name in enumerate(
    ["sigstar", "s", "nB", "nS", "nQ", "T", "muB", "muS", "muQ", "p", "e", "cs2", "theta", "Pi",
     "u0", "nnb", "sigma", "status"])}
ST_FALLBACK, ST_OUT_OF_TABLE, ST_NOCONV, ST_NONFINITE, ST_CS2_CAPPED, ST_SOLVE_FAIL = 1, 2, 4, 8, 16, 32
ST_BACKUP = 64


def build(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-ffp-contract=off", "-fopenmp",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


HBARC_GEV_FM = 0.1973269804  # hbar c in GeV fm


class Params(C.Structure):
    _fields_ = [
        ("dim", C.c_int), ("milne", C.c_int), ("viscous", C.c_int), ("has_table", C.c_int),
        ("h", C.c_double),
        ("a0", C.c_double), ("a1", C.c_double), ("Tc_GeV", C.c_double), ("w_GeV", C.c_double),
        ("chi", C.c_double * 3),
        ("nT", C.c_int), ("nmu", C.c_int * 3),
        ("T0", C.c_double), ("dT", C.c_double), ("mu0", C.c_double * 3), ("dmu", C.c_double * 3),
        ("tp", C.c_void_p), ("ts", C.c_void_p), ("tnB", C.c_void_p), ("tnS", C.c_void_p), ("tnQ", C.c_void_p),
        ("eta_over_s", C.c_double), ("zeta_peak", C.c_double), ("zeta_T_GeV", C.c_double),
        ("zeta_w_GeV", C.c_double), ("tau_pi_coef", C.c_double), ("tau_Pi_ratio", C.c_double),
        ("cs2_cap", C.c_double),
        ("newton_tol", C.c_double), ("newton_maxit", C.c_int), ("newton_no_polish", C.c_int),
        ("ntrack", C.c_int), ("pad2", C.c_int), ("tracks", C.c_void_p), ("track_sigma", C.c_double),
        ("inv", C.c_void_p), ("inv_p10", C.c_void_p), ("inv_K", C.c_int), ("inv_nd", C.c_int), ("inv_nx", C.c_int),
        ("pad3", C.c_int), ("inv_xmax", C.c_double),
        ("eom_model", C.c_int), ("pad4", C.c_int), ("dnmr", C.c_double * 6),
        ("nparton", C.c_int), ("pad5", C.c_int), ("partons", C.c_void_p),
        ("parton_norm", C.c_double), ("parton_h", C.c_double), ("parton_dt", C.c_double),
        ("backup", C.c_int), ("pad6", C.c_int), ("cd_A0", C.c_double), ("cd_mu0", C.c_double * 3),
        ("parton_q", C.c_void_p),
        ("T_stop_GeV", C.c_double),
        ("diffusion", C.c_int), ("pad8", C.c_int), ("kappaT2", C.c_double * 9), ("tauJT", C.c_double * 3),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        # SPH_ORACLE_LIB: a deliberately mutated build, loaded by the mutation tests to show
        # that the pins fail when a mistake is planted in the oracle
        override = os.environ.get("SPH_ORACLE_LIB")
        _lib = C.CDLL(override if override else build())
        d, i, l, p, u64 = C.c_double, C.c_int, C.c_long, C.c_void_p, C.c_uint64
        P = C.POINTER(Params)
        sig = {
            "oc_W": (d, [d, d, i]), "oc_dWdr": (d, [d, d, i]),
            "oc_cell_coords": (None, [l, i, p, d, p, p]),
            "oc_morton": (u64, [i, p]),
            "oc_sort_by_cell": (None, [l, i, p, d, p, p, p]),
            "oc_neighbors_brute": (l, [l, i, p, d, l, p, p]),
            "oc_neighbors_cells": (l, [l, i, p, d, l, p, p]),
            "oc_eos_analytic": (None, [P, d, p, p, p, p]),
            "oc_eos_invert_analytic": (i, [P, d, p, p, p]),
            "oc_eos_table": (None, [P, p, p, p, p]),
            "oc_eos_invert": (C.c_uint, [P, d, p, p]),
            "oc_eos_invert_ws": (C.c_uint, [P, d, p, p, p, p]),
            "oc_stage": (i, [P, l, d, p, p, p, p, p, p, p, p, p, p]),
            "oc_observe": (None, [P, l, d, p, p, p, p, p]),
            "oc_heun": (i, [P, l, p, d, i, p, p, p, p, p, p, p, p]),
            "oc_totals": (None, [P, l, d, p, p, p, p]),
            "oc_pi_pairs": (i, [i, p]),
            "oc_pi_full": (None, [i, i, d, p, p, p]),
            "oc_freezeout": (l, [P, l, d, d, p, p, p, d, l, p, p]),
            "oc_inverse_lookup": (i, [P, d, p, p]),
            "oc_inverse_build": (None, [P, p]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------
def make_params(ev, newton_tol=1e-12, newton_maxit=30, newton_polish=True) -> tuple[Params, list]:
    """Params for an inputs.Event; returns (params, keep-alive list of table arrays)."""
    P = Params()
    P.dim, P.milne, P.viscous = ev.dim, int(ev.milne), int(ev.transport.viscous)
    P.h = ev.h
    e = ev.eos
    P.a0, P.a1, P.Tc_GeV, P.w_GeV = e.a0, e.a1, e.Tc_GeV, e.w_GeV
    for q in range(3):
        P.chi[q] = e.chi[q]
    keep = []
    if ev.table is not None:
        t = ev.table
        P.has_table = 1
        P.nT = t.nT
        for q in range(3):
            P.nmu[q] = t.nmu[q]
            P.mu0[q] = t.mu0[q]
            P.dmu[q] = t.dmu[q]
        P.T0, P.dT = t.T0, t.dT
        arrs = [_f64(t.p), _f64(t.s), _f64(t.nB), _f64(t.nS), _f64(t.nQ)]
        keep += arrs
        P.tp, P.ts, P.tnB, P.tnS, P.tnQ = [a.ctypes.data for a in arrs]
    tr = ev.transport
    P.eta_over_s, P.zeta_peak, P.zeta_T_GeV, P.zeta_w_GeV = tr.eta_over_s, tr.zeta_peak, tr.zeta_T_GeV, tr.zeta_w_GeV
    P.tau_pi_coef, P.tau_Pi_ratio, P.cs2_cap = tr.tau_pi_coef, tr.tau_Pi_ratio, tr.cs2_cap
    dn = getattr(tr, "dnmr", None)
    if dn is not None:
        P.eom_model = 1
        for k in range(6):
            P.dnmr[k] = float(dn[k])
    P.newton_tol, P.newton_maxit = newton_tol, newton_maxit
    P.newton_no_polish = 0 if newton_polish else 1
    P.T_stop_GeV = float(getattr(tr, "T_stop_GeV", 0.0) or 0.0)
    df = getattr(ev, "diffusion", None)
    if df is not None:
        P.diffusion = 1
        kap = np.asarray(df.kappaT2, dtype=np.float64).reshape(9)
        for k in range(9):
            P.kappaT2[k] = float(kap[k])
        for q in range(3):
            P.tauJT[q] = float(df.tauJT[q])
    inv = getattr(ev, "inverse", None)
    if inv is not None:
        table, p10 = inverse_table(P, inv)
        keep += [table, p10]
        P.inv, P.inv_p10 = table.ctypes.data, p10.ctypes.data
        P.inv_K, P.inv_nd, P.inv_nx, P.inv_xmax = inv.per_decade, inv.decades, inv.nx, inv.xmax
    jets = getattr(ev, "jets", None)
    if jets is not None and len(jets.tracks):
        if ev.milne:
            raise ValueError("jet sources are defined in Cartesian coordinates")
        tr = _f64(jets.tracks).reshape(-1, 8)
        keep.append(tr)
        P.ntrack, P.tracks, P.track_sigma = tr.shape[0], tr.ctypes.data, float(jets.sigma)
    bk = getattr(ev, "eos_backup", None)
    if bk is not None:
        # conformal-diagonal backup (Sec. "Equation of state", backup EoS), matched to the closed
        # form at T_scale: A0 = p(T_scale, 0) / T_scale^4, mu_q0 = mu_max (A0 / (p(T_scale,
        # mu_q = mu_max) - p(T_scale, 0)))^(1/4) with T_0 = 1/fm
        Ts, mumax = bk[0] / HBARC_GEV_FM, bk[1] / HBARC_GEV_FM
        A0 = e.a0 + e.a1 * (1.0 + math.tanh((bk[0] - e.Tc_GeV) / e.w_GeV)) / 2.0
        P.backup, P.cd_A0 = 1, A0
        for q in range(3):
            dp = e.chi[q] * Ts * Ts * mumax * mumax / 2.0
            P.cd_mu0[q] = mumax * (A0 / dp) ** 0.25 if dp > 0.0 else mumax
    src = getattr(ev, "partons", None)
    if src is not None and len(src.partons):
        pt = _f64(src.partons).reshape(-1, 8)
        keep.append(pt)
        P.nparton, P.partons = pt.shape[0], pt.ctypes.data
        P.parton_norm, P.parton_h, P.parton_dt = float(src.norm), float(src.h), float(ev.dtau)
        if getattr(src, "charges", None) is not None:
            qc = _f64(src.charges).reshape(-1, 3)
            assert qc.shape[0] == pt.shape[0]
            keep.append(qc)
            P.parton_q = qc.ctypes.data
    return P, keep


_inverse_cache = {}


def inverse_table(P: Params, grid):
    """The oracle's inverted EoS table on grid (inputs.InverseGrid): (T, mu_B, mu_S, mu_Q) at every
    node of the log-decade s axis times the charge-ratio axes, from the online root finder."""
    key = (P.tp, P.has_table, grid.per_decade, grid.decade_lo, grid.decades, grid.nx, grid.xmax)
    if key in _inverse_cache:
        return _inverse_cache[key]
    p10 = np.array([10.0 ** (grid.decade_lo + d) for d in range(grid.decades + 1)])
    ns = grid.per_decade * grid.decades + 1
    table = np.zeros((ns, grid.nx, grid.nx, grid.nx, 4))
    Q = Params()
    C.pointer(Q)[0] = P  # a copy without the inverse table: the build inverts online
    Q.inv, Q.inv_p10 = None, p10.ctypes.data
    Q.inv_K, Q.inv_nd, Q.inv_nx, Q.inv_xmax = grid.per_decade, grid.decades, grid.nx, grid.xmax
    lib().oc_inverse_build(C.byref(Q), _ptr(table))
    _inverse_cache[key] = (table, p10)
    return table, p10


def npi(dim: int) -> int:
    return 3 if dim == 2 else 5


def nv(dim: int) -> int:
    return 2 * dim + 2 + npi(dim)


def pack_state(ev) -> np.ndarray:
    """y[nv][N]: x^i, u^i, S, Pi/sigma, pi^{ij}/sigma, and with diffusion J^i_q/sigma (charge major)."""
    rows = [ev.x, ev.u, ev.S[None], ev.Bv[None], ev.Pv]
    df = getattr(ev, "diffusion", None)
    if df is not None:
        jv = df.Jv if df.Jv is not None else np.zeros((3 * ev.dim, ev.n))
        rows.append(np.asarray(jv, dtype=np.float64).reshape(3 * ev.dim, ev.n))
    return np.ascontiguousarray(np.vstack(rows), dtype=np.float64)


def W(r, h, dim):
    return lib().oc_W(float(r), float(h), int(dim))


def dWdr(r, h, dim):
    return lib().oc_dWdr(float(r), float(h), int(dim))


def cell_coords(x: np.ndarray, h: float):
    x = _f64(x)
    dim, n = x.shape
    cc = np.zeros((dim, n), dtype=np.int32)
    xmin = np.zeros(3)
    lib().oc_cell_coords(n, dim, _ptr(x), h, _ptr(cc), _ptr(xmin))
    return cc, xmin[:dim]


def sort_by_cell(x: np.ndarray, h: float):
    """(cell coords [dim][N] int32, Morton keys uint64, permutation sorting by (key, id))."""
    x = _f64(x)
    dim, n = x.shape
    cc = np.zeros((dim, n), dtype=np.int32)
    keys = np.zeros(n, dtype=np.uint64)
    perm = np.zeros(n, dtype=np.int64)
    lib().oc_sort_by_cell(n, dim, _ptr(x), h, _ptr(cc), _ptr(keys), _ptr(perm))
    return cc, keys, perm


def neighbors(x: np.ndarray, h: float, method: str = "cells"):
    """Sorted (a, b) pairs with r_ab < 2h (self pairs included)."""
    x = _f64(x)
    dim, n = x.shape
    fn = lib().oc_neighbors_cells if method == "cells" else lib().oc_neighbors_brute
    cnt = fn(n, dim, _ptr(x), h, 0, None, None)
    pa = np.zeros(max(cnt, 1), dtype=np.int32)
    pb = np.zeros(max(cnt, 1), dtype=np.int32)
    fn(n, dim, _ptr(x), h, cnt, _ptr(pa), _ptr(pb))
    return pa[:cnt], pb[:cnt]


def eos_invert(P: Params, s: float, n3):
    out = np.zeros(11)
    n3 = _f64(n3)
    st = lib().oc_eos_invert(C.byref(P), float(s), _ptr(n3), _ptr(out))
    return out, int(st)


def eos_analytic(P: Params, T: float, mu3):
    mu3 = _f64(mu3)
    p = np.zeros(1)
    sn = np.zeros(4)
    H = np.zeros(16)
    lib().oc_eos_analytic(C.byref(P), float(T), _ptr(mu3), _ptr(p), _ptr(sn), _ptr(H))
    return p[0], sn, H.reshape(4, 4)


def eos_table(P: Params, x4):
    x4 = _f64(x4)
    p = np.zeros(1)
    sn = np.zeros(4)
    J = np.zeros(16)
    lib().oc_eos_table(C.byref(P), _ptr(x4), _ptr(p), _ptr(sn), _ptr(J))
    return p[0], sn, J.reshape(4, 4)


@dataclass
class OracleRun:
    """Holds an evolving state; ``step`` advances Heun steps, ``observe`` fills aux."""
    ev: object
    P: Params
    keep: list
    y: np.ndarray
    Nq: np.ndarray
    tau: float
    work: float = 0.0
    status_or: int = 0
    guess: np.ndarray = None  # [4][N] warm start of the EoS Newton (previous table solution, T = 0: none)

    @classmethod
    def start(cls, ev, **kw):
        P, keep = make_params(ev, **kw)
        # Nq is integrated in place under charge sources: the run owns a copy
        return cls(ev=ev, P=P, keep=keep, y=pack_state(ev), Nq=_f64(ev.Nq).copy(), tau=float(ev.tau0),
                   guess=np.zeros((4, ev.n)))

    @property
    def n(self):
        return self.y.shape[1]

    def step(self, nsteps: int):
        n, dim = self.n, self.P.dim
        aux = np.zeros((NAUX, n))
        grad = np.zeros((dim * dim + dim, n))
        st = np.zeros(n, dtype=np.uint32)
        tau = C.c_double(self.tau)
        work = C.c_double(self.work)
        stor = C.c_uint(0)
        lib().oc_heun(C.byref(self.P), n, C.byref(tau), float(self.ev.dtau), int(nsteps), _ptr(self.y),
                      _ptr(self.Nq), _ptr(aux), _ptr(grad), _ptr(st), C.byref(stor), C.byref(work), _ptr(self.guess))
        self.tau, self.work = tau.value, work.value
        self.status_or |= stor.value
        return aux

    def stage(self, y=None, tau=None):
        """One right-hand-side evaluation: (dydt, aux, grad, status, work_rate), warm-started from
        the current guess (which is not updated)."""
        y = self.y if y is None else _f64(y)
        tau = self.tau if tau is None else tau
        n, dim = self.n, self.P.dim
        dydt = np.zeros_like(y)
        aux = np.zeros((NAUX, n))
        grad = np.zeros((dim * dim + dim, n))
        st = np.zeros(n, dtype=np.uint32)
        wr = C.c_double(0.0)
        gout = np.zeros((4, n))
        dNq = np.zeros((3, n))
        lib().oc_stage(C.byref(self.P), n, float(tau), _ptr(y), _ptr(self.Nq), _ptr(dydt), _ptr(aux), _ptr(grad),
                       _ptr(st), C.byref(wr), _ptr(self.guess), _ptr(gout), _ptr(dNq))
        self.last_dNq = dNq  # the charge rates (zero without charge sources)
        return dydt, aux, grad, st, wr.value

    def observe(self):
        """Densities and EoS at the current state (warm-started from the guess, which is not updated)."""
        n = self.n
        aux = np.zeros((NAUX, n))
        st = np.zeros(n, dtype=np.uint32)
        lib().oc_observe(C.byref(self.P), n, float(self.tau), _ptr(self.y), _ptr(self.Nq), _ptr(aux), _ptr(st),
                         _ptr(self.guess))
        return aux, st

    def evolve_freezeout(self, nsteps: int, e_fo: float):
        """nsteps Heun steps, recording the freeze-out surface elements at e_fo: before each step
        (and after the last) the state is observed and particles whose e fell through e_fo since
        the previous observation yield one element each (records of FO_NREC doubles, particle
        indices).  The first observation only records e."""
        dtau = float(self.ev.dtau)
        eprev = np.full(self.n, np.nan)
        recs, ids = [], []
        for k in range(nsteps + 1):
            aux, _ = self.observe()
            if k > 0:
                out = np.zeros((self.n, FO_NREC))
                idx = np.zeros(self.n, dtype=np.int64)
                cnt = lib().oc_freezeout(C.byref(self.P), self.n, float(self.tau), dtau, _ptr(self.y), _ptr(aux),
                                         _ptr(eprev), float(e_fo), self.n, _ptr(out), _ptr(idx))
                recs.append(out[:cnt].copy())
                ids.append(idx[:cnt].copy())
            eprev = aux[AUX["e"]].copy()
            if k < nsteps:
                self.step(1)
        return np.concatenate(recs) if recs else np.zeros((0, FO_NREC)), \
            np.concatenate(ids) if ids else np.zeros(0, dtype=np.int64)

    def totals(self, aux=None):
        if aux is None:
            aux, _ = self.observe()
        tot = np.zeros(5)
        lib().oc_totals(C.byref(self.P), self.n, float(self.tau), _ptr(self.y), _ptr(self.Nq), _ptr(aux), _ptr(tot))
        return {"E": tot[0], "S": tot[1], "N": tot[2:5].copy(), "work": self.work}
