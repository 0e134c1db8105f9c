"""The offline EoS inverter of the oracle (Sec. "Equation of state": the EoS converted once onto a
grid in (s, n) with s on logarithmic decades, then interpolated instead of root-found; CPU only).

* At the grid nodes the interpolant returns the online root finder's solution (the table's
  construction), and the forward EoS there reproduces (s, n) to the root finder's tolerance.
* Off the nodes the interpolant converges to the online inversion when the grid is refined:
  at least first order in T (the online inverse of the piecewise-quadrilinear forward table has
  kinks along the forward grid's node lines) and second order in mu (smooth in the ratios).
"""
import ctypes as C

import numpy as np

from oracle import oracle as O
from paper_2511_22852_gb300 import inputs as I


def _event(K, nx):
    ev = I.smooth_blob_2p1(half_width=2.0, eos=I.CAUSAL_EOS)
    ev.inverse = I.InverseGrid(per_decade=K, nx=nx, xmax=0.12)
    return ev


def test_nodes_reproduce_the_online_inversion():
    ev = _event(90, 17)
    P, keep = O.make_params(ev)
    rng = np.random.default_rng(3)
    g = ev.inverse
    dx = 2 * g.xmax / (g.nx - 1)
    checked = 0
    for _ in range(300):
        i = int(rng.integers(g.per_decade * 2, g.per_decade * 5))  # s from 0.1 to 100 fm^-3
        j = rng.integers(0, g.nx, 3)
        s = 10.0 ** (g.decade_lo + i // g.per_decade) * (1 + 9 * (i % g.per_decade) / g.per_decade)
        n3 = (-g.xmax + j * dx) * s
        x = np.zeros(4)
        r = O.lib().oc_inverse_lookup(C.byref(P), s, n3.ctypes.data_as(C.c_void_p), x.ctypes.data_as(C.c_void_p))
        if r != 0:
            continue
        out = np.zeros(11)
        P.inv = None
        st = O.lib().oc_eos_invert(C.byref(P), s, n3.ctypes.data_as(C.c_void_p), out.ctypes.data_as(C.c_void_p))
        P.inv = keep[-2].ctypes.data
        assert np.allclose(x, out[:4], rtol=1e-13, atol=1e-15)
        if st & (O.ST_OUT_OF_TABLE | O.ST_FALLBACK):
            continue  # the closed form solved this node: the forward table is not its EoS
        # forward table at the node's solution gives back (s, n)
        sn = np.zeros(4)
        O.lib().oc_eos_table(C.byref(P), x.ctypes.data_as(C.c_void_p), None, sn.ctypes.data_as(C.c_void_p), None)
        assert abs(sn[0] / s - 1) < 1e-11 and np.all(np.abs(sn[1:] - n3) < 1e-11 * s)
        checked += 1
    assert checked > 60


def test_interpolant_converges_to_the_online_inversion():
    ref = I.smooth_blob_2p1(half_width=2.0, eos=I.CAUSAL_EOS)
    aux_on, _ = O.OracleRun.start(ref).observe()
    A = O.AUX
    eT, emu = [], []
    for K, nx in [(45, 9), (90, 17), (180, 33)]:
        aux, _ = O.OracleRun.start(_event(K, nx)).observe()
        eT.append(np.max(np.abs(aux[A["T"]] / aux_on[A["T"]] - 1)))
        emu.append(np.max(np.abs(aux[A["muB"]] - aux_on[A["muB"]])) / np.max(np.abs(aux_on[A["muB"]])))
    assert eT[0] < 5e-3 and emu[0] < 5e-2
    for k in range(2):
        assert eT[k + 1] < 0.6 * eT[k]      # at least first order
        assert emu[k + 1] < 0.35 * emu[k]   # second order
