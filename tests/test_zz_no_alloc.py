"""sph_density_noalloc: the densities for callers that must not allocate device memory.

Some callers cannot call cudaMalloc -- a serving loop that has already given all free
HBM to its own pool, or code running while a CUDA graph is being captured in global
mode.  For them the library offers one entry point whose temporaries live in a fixed
device array set aside when the library is loaded.  This test calls it through the C
ABI, twice in a row and then once more on the first input, and checks each result
against the densities of the ordinary event path (sph_init_event + sph_read_fields).
A second test gives it particles spread over more cells than its fixed cell table holds
(rejected with SPH_ERR_STATE), then a valid input, which must succeed with correct
densities: the overflow flag left in the shared array by the failed call is cleared.
It sits in its own file so that it runs after every other test; it also passes alone.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2511_22852_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-13  # the densities of the two paths agree to rounding


def _noalloc(Bd):
    f = Bd.lib().sph_density_noalloc
    f.restype = C.c_int32
    f.argtypes = [C.c_void_p] * 4 + [C.c_int64, C.c_double, C.c_double, C.c_int32, C.c_void_p, C.c_void_p]
    return f


def _relerr(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def test_noalloc_density_matches_event_path_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_22852_gb300 import binding as Bd
    from paper_2511_22852_gb300 import build_lib
    build_lib.build()
    f = _noalloc(Bd)
    stream = torch.cuda.current_stream().cuda_stream
    cases = [I.viscous_bsq_2p1(n_target=3000, R=3.0, n_hot=20), I.gubser_ideal_2p1(),
             I.viscous_bsq_2p1(n_target=3000, R=3.0, n_hot=20)]
    for ev in cases:
        g = Bd.GpuEvent(ev, use_graph=False)
        ref = g.read(("SIGMA_STAR", "S_DENS", "N_DENS"))
        g.free()
        dev = {k: torch.tensor(np.ascontiguousarray(v), dtype=torch.float64, device="cuda")
               for k, v in [("x", ev.x), ("u", ev.u), ("S", ev.S), ("Nq", ev.Nq)]}
        out = torch.full((5, ev.n), float("nan"), dtype=torch.float64, device="cuda")
        rc = f(dev["x"].data_ptr(), dev["u"].data_ptr(), dev["S"].data_ptr(), dev["Nq"].data_ptr(), ev.n, ev.h,
               ev.tau0, int(ev.milne), out.data_ptr(), stream)
        assert rc == Bd.SPH_OK, Bd.lib().sph_last_error().decode()
        o = out.cpu().numpy()
        assert _relerr(o[0], ref["SIGMA_STAR"]) < TOL
        assert _relerr(o[1], ref["S_DENS"]) < TOL
        if np.any(ref["N_DENS"]):
            assert _relerr(o[2:5], ref["N_DENS"]) < TOL
        else:
            assert not np.any(o[2:5])


def test_noalloc_rejects_sizes_beyond_its_limit():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_22852_gb300 import binding as Bd
    f = _noalloc(Bd)
    rc = f(None, None, None, None, 65536 + 1, 0.3, 0.6, 1, None, None)
    assert rc == Bd.SPH_ERR_ARG
    assert "SPH_NOALLOC_MAX_PARTICLES" in Bd.lib().sph_last_error().decode()


def test_noalloc_cell_overflow_then_valid_call():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_22852_gb300 import binding as Bd
    from paper_2511_22852_gb300 import build_lib
    build_lib.build()
    f = _noalloc(Bd)
    stream = torch.cuda.current_stream().cuda_stream
    # 64 particles on a line 300 cells of side 2h long (h = 0.3 fm): more than the 256 per axis
    n, h = 64, 0.3
    x = np.zeros((2, n))
    x[0] = np.linspace(0.0, 300 * 2 * h, n)
    dev = [torch.tensor(a, dtype=torch.float64, device="cuda") for a in
           (x, np.zeros((2, n)), np.ones(n), np.zeros((3, n)))]
    out = torch.zeros((5, n), dtype=torch.float64, device="cuda")
    rc = f(*[d.data_ptr() for d in dev], n, h, 0.6, 1, out.data_ptr(), stream)
    assert rc == Bd.SPH_ERR_STATE
    assert "256 cells" in Bd.lib().sph_last_error().decode()
    ev = I.viscous_bsq_2p1(n_target=2000, R=2.5, n_hot=10)
    g = Bd.GpuEvent(ev, use_graph=False)
    ref = g.read(("SIGMA_STAR", "S_DENS", "N_DENS"))
    g.free()
    dev = [torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda") for a in (ev.x, ev.u, ev.S, ev.Nq)]
    out = torch.full((5, ev.n), float("nan"), dtype=torch.float64, device="cuda")
    rc = f(*[d.data_ptr() for d in dev], ev.n, ev.h, ev.tau0, int(ev.milne), out.data_ptr(), stream)
    assert rc == Bd.SPH_OK, Bd.lib().sph_last_error().decode()
    o = out.cpu().numpy()
    assert _relerr(o[0], ref["SIGMA_STAR"]) < TOL
    assert _relerr(o[1], ref["S_DENS"]) < TOL
    assert _relerr(o[2:5], ref["N_DENS"]) < TOL
