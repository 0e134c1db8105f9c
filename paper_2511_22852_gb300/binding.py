"""Thin ctypes binding of the C ABI in ``include/sph_gb300.h``.

The names are the C names (``sph_set_eos_table``, ``sph_init_event``,
``sph_step``, ``sph_read_fields``, ...); this module only marshals arguments.
Every step of the SPH path runs in the CUDA library: if the library is not
built (``__graft_entry__.build()`` or ``python -m paper_2511_22852_gb300.build_lib``),
loading fails with an error -- there is no CPU fallback.

``GpuEvent`` wraps one event built from ``inputs.Event`` for tests and the
benchmark.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build_lib

# ---------------------------------------------------------------------------
SPH_OK, SPH_ERR_ARG, SPH_ERR_OOM, SPH_ERR_CUDA, SPH_ERR_EOS_RANGE, SPH_ERR_EOS_NOCONV, SPH_ERR_NONFINITE, \
    SPH_ERR_TIMEOUT, SPH_ERR_STATE = range(9)
STATUS_NAMES = ["SPH_OK", "SPH_ERR_ARG", "SPH_ERR_OOM", "SPH_ERR_CUDA", "SPH_ERR_EOS_RANGE", "SPH_ERR_EOS_NOCONV",
                "SPH_ERR_NONFINITE", "SPH_ERR_TIMEOUT", "SPH_ERR_STATE"]
PST_FALLBACK, PST_OUT_OF_TABLE, PST_NOCONV, PST_NONFINITE, PST_CS2_CAPPED, PST_SOLVE_FAIL = 1, 2, 4, 8, 16, 32
PST_BACKUP = 64
SPH_SYNC = 1
SPH_FP64, SPH_MIXED = 0, 1

F = {name: 1 << i for i, name in enumerate(
    ["X", "U", "S", "NQ", "BV", "PV", "SIGMA_STAR", "S_DENS", "N_DENS", "T", "MU", "P", "E", "PI_BULK", "STATUS",
     "NNB", "CELL", "GUESS", "JV"])}

EXPORTS = ["sph_set_eos_table", "sph_free_eos", "sph_init_event", "sph_free_event", "sph_step", "sph_read_fields",
           "sph_write_state", "sph_last_error", "sph_debug_neighbors", "sph_debug_rates", "sph_kernel_times",
           "sph_server_create", "sph_server_free", "sph_submit", "sph_server_pump", "sph_poll", "sph_collect",
           "sph_server_stats_get", "sph_server_drain", "sph_freezeout_setup", "sph_read_freezeout",
           "sph_set_jets", "sph_server_autotune", "sph_server_set_shape", "sph_eos_build_inverse", "sph_set_eos_mode",
           "sph_set_viscous_eom", "sph_set_partons", "sph_set_eos_backup", "sph_server_profile",
           "sph_server_kernel_times", "sph_measure_fma_peak"]
SPH_EOS_ONLINE, SPH_EOS_OFFLINE = 0, 1
SPH_FO_NREC = 24
SPH_TICKET_QUEUED, SPH_TICKET_RUNNING, SPH_TICKET_DONE = 0, 1, 2


class SphError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES[code] if 0 <= code < len(STATUS_NAMES) else code}: {msg}")
        self.code = code


class EosDesc(C.Structure):
    _fields_ = [("a0", C.c_double), ("a1", C.c_double), ("Tc_GeV", C.c_double), ("w_GeV", C.c_double),
                ("chi", C.c_double * 3), ("has_table", C.c_int32), ("nT", C.c_int32), ("nmu", C.c_int32 * 3),
                ("newton_maxit", C.c_int32), ("T0", C.c_double), ("dT", C.c_double), ("mu0", C.c_double * 3),
                ("dmu", C.c_double * 3), ("p", C.c_void_p), ("s", C.c_void_p), ("nB", C.c_void_p),
                ("nS", C.c_void_p), ("nQ", C.c_void_p), ("newton_tol", C.c_double)]


class EventDesc(C.Structure):
    _fields_ = [("dim", C.c_int32), ("milne", C.c_int32), ("viscous", C.c_int32), ("on_device", C.c_int32),
                ("n", C.c_int64), ("h", C.c_double), ("tau0", C.c_double), ("dtau", C.c_double),
                ("x", C.c_void_p), ("u", C.c_void_p), ("S", C.c_void_p), ("Nq", C.c_void_p), ("Bv", C.c_void_p),
                ("Pv", C.c_void_p), ("eta_over_s", C.c_double), ("zeta_peak", C.c_double),
                ("zeta_T_GeV", C.c_double), ("zeta_w_GeV", C.c_double), ("tau_pi_coef", C.c_double),
                ("tau_Pi_ratio", C.c_double), ("cs2_cap", C.c_double), ("fatal_mask", C.c_uint32),
                ("use_graph", C.c_int32), ("stream", C.c_void_p), ("profile", C.c_int32), ("precision", C.c_int32),
                ("T_stop_GeV", C.c_double), ("kappaT2", C.c_void_p), ("tauJT", C.c_void_p), ("Jv", C.c_void_p)]


class FieldBufs(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ["x", "u", "S", "Nq", "Bv", "Pv", "sigstar", "s", "nq", "T", "mu", "p",
                                          "e", "Pi", "status", "nnb", "cell", "guess"]] + [("on_device", C.c_int32),
                                                                                          ("Jv", C.c_void_p)]


class Totals(C.Structure):
    _fields_ = [("tau", C.c_double), ("E", C.c_double), ("S", C.c_double), ("N", C.c_double * 3),
                ("work", C.c_double), ("status_or", C.c_uint32), ("pair_overflows", C.c_int32), ("steps", C.c_int64),
                ("pairs", C.c_int64), ("kernel_launches", C.c_int64), ("eos_work", C.c_int64 * 3),
                ("shell_tests", C.c_int64)]


class ServerDesc(C.Structure):
    _fields_ = [("max_events", C.c_int32), ("max_inflight", C.c_int32), ("max_particles", C.c_int64),
                ("hbm_fraction", C.c_double), ("pinned_bytes", C.c_int64), ("stream", C.c_void_p),
                ("polish", C.c_int32), ("groups", C.c_int32), ("newton_tol", C.c_double)]


class ServerStats(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ["queued", "running", "done", "batch_steps", "particle_steps",
                                         "arena_capacity", "arena_in_use", "kernel_launches"]] + \
               [("slots_in_use", C.c_int32), ("max_events", C.c_int32), ("device_ms", C.c_double),
                ("steps_timed", C.c_int64), ("failed", C.c_int64)]


_lib = None


def library_path() -> str:
    return build_lib.LIB


def lib():
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library not built ({path}); run __graft_entry__.build()")
        _lib = C.CDLL(path)
        vp, i32, i64, u32 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32
        sig = {
            "sph_set_eos_table": (i32, [C.POINTER(vp), C.POINTER(EosDesc)]),
            "sph_free_eos": (None, [vp]),
            "sph_init_event": (i32, [C.POINTER(vp), C.POINTER(EventDesc), vp]),
            "sph_free_event": (None, [vp]),
            "sph_step": (i32, [vp, i32, u32]),
            "sph_read_fields": (i32, [vp, C.c_uint64, C.POINTER(FieldBufs), C.POINTER(Totals)]),
            "sph_write_state": (i32, [vp, C.c_uint64, C.POINTER(FieldBufs)]),
            "sph_last_error": (C.c_char_p, []),
            "sph_debug_neighbors": (i32, [vp, i64, vp, vp, C.POINTER(i64)]),
            "sph_debug_rates": (i32, [vp, vp, vp]),
            "sph_kernel_times": (i32, [vp, i32, vp, vp, vp, C.POINTER(i32)]),
            "sph_server_create": (i32, [C.POINTER(vp), C.POINTER(ServerDesc), vp]),
            "sph_server_free": (None, [vp]),
            "sph_submit": (i32, [vp, C.POINTER(EventDesc), i32, C.POINTER(i64)]),
            "sph_server_pump": (i32, [vp, i32, C.POINTER(i32)]),
            "sph_poll": (i32, [vp, i64, C.POINTER(i32), C.POINTER(C.c_double)]),
            "sph_collect": (i32, [vp, i64, C.c_uint64, C.POINTER(FieldBufs), C.POINTER(Totals)]),
            "sph_server_stats_get": (i32, [vp, C.POINTER(ServerStats)]),
            "sph_server_drain": (i32, [vp, C.c_double]),
            "sph_freezeout_setup": (i32, [vp, C.c_double, i64]),
            "sph_set_jets": (i32, [vp, i64, vp, C.c_double]),
            "sph_set_viscous_eom": (i32, [vp, i32, vp]),
            "sph_set_partons": (i32, [vp, i64, vp, vp, C.c_double, C.c_double]),
            "sph_set_eos_backup": (i32, [vp, i32, C.c_double, C.c_double]),
            "sph_server_autotune": (i32, [vp, i32, C.POINTER(i32), C.POINTER(i32)]),
            "sph_server_set_shape": (i32, [vp, i32, i32]),
            "sph_server_profile": (i32, [vp, i32]),
            "sph_measure_fma_peak": (i32, [i32, i32, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
            "sph_server_kernel_times": (i32, [vp, i32, vp, vp, vp, C.POINTER(i32)]),
            "sph_eos_build_inverse": (i32, [vp, i32, i32, i32, i32, C.c_double]),
            "sph_set_eos_mode": (i32, [vp, i32]),
            "sph_read_freezeout": (i32, [vp, i64, vp, vp, C.POINTER(i64)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


def _check(code):
    if code != SPH_OK:
        raise SphError(code, lib().sph_last_error().decode())


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return int(a.data_ptr())  # torch tensor


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------
# the C entry points under their own names
def sph_set_eos_table(desc: EosDesc):
    h = C.c_void_p()
    _check(lib().sph_set_eos_table(C.byref(h), C.byref(desc)))
    return h


def sph_free_eos(h):
    lib().sph_free_eos(h)


def sph_init_event(desc: EventDesc, eos):
    h = C.c_void_p()
    _check(lib().sph_init_event(C.byref(h), C.byref(desc), eos))
    return h


def sph_free_event(h):
    lib().sph_free_event(h)


def sph_step(h, nsteps: int, flags: int = 0):
    _check(lib().sph_step(h, int(nsteps), int(flags)))


def sph_read_fields(h, mask: int, bufs: FieldBufs | None, tot: Totals | None):
    _check(lib().sph_read_fields(h, C.c_uint64(mask), C.byref(bufs) if bufs is not None else None,
                                 C.byref(tot) if tot is not None else None))


def sph_write_state(h, mask: int, bufs: FieldBufs):
    _check(lib().sph_write_state(h, C.c_uint64(mask), C.byref(bufs)))


def sph_debug_neighbors(h, cap: int, pa, pb):
    cnt = C.c_int64(0)
    _check(lib().sph_debug_neighbors(h, int(cap), _ptr(pa), _ptr(pb), C.byref(cnt)))
    return cnt.value


def sph_debug_rates(h, rates, grad):
    _check(lib().sph_debug_rates(h, _ptr(rates), _ptr(grad)))


def sph_kernel_times(h):
    """{group: (milliseconds, launches)} of an event created with profile = 1."""
    names = C.create_string_buffer(32 * 16)
    ms = np.zeros(16)
    nl = np.zeros(16, dtype=np.int64)
    cnt = C.c_int32(0)
    _check(lib().sph_kernel_times(h, 16, names, ms.ctypes.data, nl.ctypes.data, C.byref(cnt)))
    raw = names.raw
    return {raw[32 * k:32 * k + 32].split(b"\0")[0].decode(): (float(ms[k]), int(nl[k])) for k in range(cnt.value)}


def sph_server_kernel_times(h):
    """{group: (milliseconds, stages timed)} of the server's sampled batch steps."""
    names = C.create_string_buffer(32 * 16)
    ms = np.zeros(16)
    nl = np.zeros(16, dtype=np.int64)
    cnt = C.c_int32(0)
    _check(lib().sph_server_kernel_times(h, 16, names, ms.ctypes.data, nl.ctypes.data, C.byref(cnt)))
    raw = names.raw
    return {raw[32 * k:32 * k + 32].split(b"\0")[0].decode(): (float(ms[k]), int(nl[k])) for k in range(cnt.value)}


def sph_measure_fma_peak(fp64: bool, reps: int = 5):
    """(GFLOP/s, best launch ms) of the device's FP64 or FP32 multiply-add chains."""
    g, ms = C.c_double(0.0), C.c_double(0.0)
    _check(lib().sph_measure_fma_peak(int(bool(fp64)), int(reps), C.byref(g), C.byref(ms)))
    return g.value, ms.value


def sph_eos_build_inverse(eos, grid):
    """Builds the offline inverter of an EoS handle on grid (inputs.InverseGrid)."""
    _check(lib().sph_eos_build_inverse(eos, int(grid.per_decade), int(grid.decade_lo), int(grid.decades),
                                       int(grid.nx), float(grid.xmax)))


def sph_set_eos_mode(h, mode: int):
    _check(lib().sph_set_eos_mode(h, int(mode)))


def sph_set_jets(h, tracks, sigma: float):
    tr = _f64(tracks).reshape(-1, 8) if tracks is not None else np.zeros((0, 8))
    _check(lib().sph_set_jets(h, int(tr.shape[0]), _ptr(tr) if tr.size else None, float(sigma)))


SPH_EOM_MIN_IS, SPH_EOM_DNMR = 0, 1


def sph_set_viscous_eom(h, model: int, coeffs=None):
    c = _f64(coeffs) if coeffs is not None else None
    _check(lib().sph_set_viscous_eom(h, int(model), _ptr(c) if c is not None else None))


def sph_set_partons(h, partons, norm: float, h_src: float, charges=None):
    pt = _f64(partons).reshape(-1, 8) if partons is not None else np.zeros((0, 8))
    qc = None if charges is None else np.ascontiguousarray(charges, dtype=np.float64).reshape(-1, 3)
    if qc is not None and qc.shape[0] != pt.shape[0]:
        raise ValueError("one (B, S, Q) row per parton")
    _check(lib().sph_set_partons(h, int(pt.shape[0]), _ptr(pt) if pt.size else None,
                                 _ptr(qc) if qc is not None and qc.size else None, float(norm), float(h_src)))


def sph_set_eos_backup(h, enable: bool, T_scale_GeV: float = 0.165, mu_max_GeV: float = 0.45):
    _check(lib().sph_set_eos_backup(h, int(bool(enable)), float(T_scale_GeV), float(mu_max_GeV)))


def sph_freezeout_setup(h, e_fo: float, capacity: int):
    _check(lib().sph_freezeout_setup(h, float(e_fo), int(capacity)))


def sph_read_freezeout(h, cap: int, elems, ids) -> int:
    cnt = C.c_int64(0)
    _check(lib().sph_read_freezeout(h, int(cap), _ptr(elems), _ptr(ids), C.byref(cnt)))
    return cnt.value


def sph_server_create(desc: ServerDesc, eos):
    h = C.c_void_p()
    _check(lib().sph_server_create(C.byref(h), C.byref(desc), eos))
    return h


def sph_server_free(h):
    lib().sph_server_free(h)


def sph_submit(h, desc: EventDesc, nsteps: int) -> int:
    t = C.c_int64(0)
    _check(lib().sph_submit(h, C.byref(desc), int(nsteps), C.byref(t)))
    return t.value


def sph_server_pump(h, max_steps: int) -> int:
    r = C.c_int32(0)
    _check(lib().sph_server_pump(h, int(max_steps), C.byref(r)))
    return r.value


def sph_poll(h, ticket: int):
    st, lat = C.c_int32(0), C.c_double(0.0)
    _check(lib().sph_poll(h, int(ticket), C.byref(st), C.byref(lat)))
    return st.value, lat.value


def sph_collect(h, ticket: int, mask: int, bufs: FieldBufs | None, tot: Totals | None):
    _check(lib().sph_collect(h, int(ticket), C.c_uint64(mask), C.byref(bufs) if bufs is not None else None,
                             C.byref(tot) if tot is not None else None))


def sph_server_stats_get(h) -> dict:
    o = ServerStats()
    _check(lib().sph_server_stats_get(h, C.byref(o)))
    return {k: getattr(o, k) for k, _ in ServerStats._fields_}


def sph_server_drain(h, timeout_s: float = 0.0):
    _check(lib().sph_server_drain(h, float(timeout_s)))


# ---------------------------------------------------------------------------
def eos_desc(eos, table=None, newton_tol=1e-12, newton_maxit=30):
    """(EosDesc, keep-alive list) from inputs.AnalyticEoS / inputs.EoSTable."""
    d = EosDesc()
    d.a0, d.a1, d.Tc_GeV, d.w_GeV = eos.a0, eos.a1, eos.Tc_GeV, eos.w_GeV
    for q in range(3):
        d.chi[q] = eos.chi[q]
    d.newton_tol, d.newton_maxit = newton_tol, newton_maxit
    keep = []
    if table is not None:
        d.has_table = 1
        d.nT, d.T0, d.dT = table.nT, table.T0, table.dT
        for q in range(3):
            d.nmu[q], d.mu0[q], d.dmu[q] = table.nmu[q], table.mu0[q], table.dmu[q]
        arrs = [_f64(table.p), _f64(table.s), _f64(table.nB), _f64(table.nS), _f64(table.nQ)]
        keep += arrs
        d.p, d.s, d.nB, d.nS, d.nQ = [a.ctypes.data for a in arrs]
    return d, keep


def event_desc(ev):
    """(EventDesc, keep-alive list) of an ``inputs.Event`` (host arrays)."""
    d = EventDesc()
    d.dim, d.milne, d.viscous, d.on_device = ev.dim, int(ev.milne), int(ev.transport.viscous), 0
    d.n, d.h, d.tau0, d.dtau = ev.n, ev.h, ev.tau0, ev.dtau
    keep = [_f64(ev.x), _f64(ev.u), _f64(ev.S), _f64(ev.Nq), _f64(ev.Bv), _f64(ev.Pv)]
    d.x, d.u, d.S, d.Nq, d.Bv, d.Pv = [a.ctypes.data if a.size else None for a in keep]
    tr = ev.transport
    d.eta_over_s, d.zeta_peak, d.zeta_T_GeV, d.zeta_w_GeV = tr.eta_over_s, tr.zeta_peak, tr.zeta_T_GeV, tr.zeta_w_GeV
    d.tau_pi_coef, d.tau_Pi_ratio, d.cs2_cap = tr.tau_pi_coef, tr.tau_Pi_ratio, tr.cs2_cap
    d.T_stop_GeV = float(getattr(tr, "T_stop_GeV", 0.0) or 0.0)
    df = getattr(ev, "diffusion", None)
    if df is not None:
        kap = _f64(np.asarray(df.kappaT2, dtype=np.float64).reshape(9))
        tj = _f64(np.asarray(df.tauJT, dtype=np.float64).reshape(3))
        keep += [kap, tj]
        d.kappaT2, d.tauJT = kap.ctypes.data, tj.ctypes.data
        if df.Jv is not None:
            jv = _f64(np.asarray(df.Jv, dtype=np.float64).reshape(6, ev.n))
            keep.append(jv)
            d.Jv = jv.ctypes.data
    return d, keep


_FIELD_SHAPES = {"X": (2, "x"), "U": (2, "u"), "S": (1, "S"), "NQ": (3, "Nq"), "BV": (1, "Bv"), "PV": (3, "Pv"),
                 "SIGMA_STAR": (1, "sigstar"), "S_DENS": (1, "s"), "N_DENS": (3, "nq"), "T": (1, "T"),
                 "MU": (3, "mu"), "P": (1, "p"), "E": (1, "e"), "PI_BULK": (1, "Pi"), "STATUS": (1, "status"),
                 "NNB": (1, "nnb")}


class GpuServer:
    """The serving form: events submitted from ``inputs.Event`` objects, batched on the GPU."""

    def __init__(self, eos, table=None, max_events=32, max_particles=0, hbm_fraction=0.0, pinned_bytes=0,
                 polish=False, max_inflight=2, stream=None, newton_tol=0.0, groups=0):
        ed, self._keep_eos = eos_desc(eos, table)
        self.eos = sph_set_eos_table(ed)
        d = ServerDesc()
        d.max_events, d.max_inflight, d.max_particles = int(max_events), int(max_inflight), int(max_particles)
        d.hbm_fraction, d.pinned_bytes, d.stream, d.polish = float(hbm_fraction), int(pinned_bytes), stream, int(polish)
        d.newton_tol = float(newton_tol)
        d.groups = int(groups)
        self.h = sph_server_create(d, self.eos)
        self.n_of = {}

    def submit(self, ev, nsteps: int) -> int:
        d, keep = event_desc(ev)
        t = sph_submit(self.h, d, nsteps)
        self.n_of[t] = ev.n
        return t

    def pump(self, max_steps: int = 1) -> int:
        return sph_server_pump(self.h, max_steps)

    def poll(self, ticket: int):
        return sph_poll(self.h, ticket)

    def collect(self, ticket: int, names=("X", "U", "S", "NQ", "BV", "PV", "T", "MU", "S_DENS", "N_DENS", "NNB")):
        n = self.n_of.pop(ticket)
        b = FieldBufs()
        out, mask = {}, 0
        for nm in names:
            rows, attr = _FIELD_SHAPES[nm]
            dt = np.uint32 if nm == "STATUS" else (np.int32 if nm == "NNB" else np.float64)
            arr = np.zeros((rows, n) if rows > 1 else n, dtype=dt)
            out[nm] = arr
            setattr(b, attr, arr.ctypes.data)
            mask |= F[nm]
        t = Totals()
        sph_collect(self.h, ticket, mask, b, t)
        out["totals"] = {"tau": t.tau, "E": t.E, "S": t.S, "N": np.array(t.N[:]), "work": t.work,
                         "status_or": t.status_or, "steps": t.steps, "pairs": t.pairs,
                         "eos_work": tuple(t.eos_work[:]), "shell_tests": t.shell_tests, "pair_overflows": t.pair_overflows}
        return out

    def stats(self) -> dict:
        return sph_server_stats_get(self.h)

    def autotune(self, trials: int = 3, lanes: bool = False):
        """Tunes the tiled passes' shape; returns the threads per block (and the lane-split warps
        with lanes=True)."""
        c, lw = C.c_int32(0), C.c_int32(0)
        _check(lib().sph_server_autotune(self.h, int(trials), C.byref(c), C.byref(lw)))
        return (c.value, lw.value) if lanes else c.value

    def set_shape(self, threads: int, lane_warps: int):
        """Fixes the tiled passes' shape (threads per block, lane-split warps)."""
        _check(lib().sph_server_set_shape(self.h, int(threads), int(lane_warps)))

    def drain(self, timeout_s: float = 0.0):
        sph_server_drain(self.h, timeout_s)

    def profile(self, every: int):
        """Sampled per-kernel-group timing of every every-th batch step (0: off)."""
        _check(lib().sph_server_profile(self.h, int(every)))

    def kernel_times(self):
        return sph_server_kernel_times(self.h)

    def free(self):
        if self.h is not None:
            sph_server_free(self.h)
            self.h = None
        if self.eos is not None:
            sph_free_eos(self.eos)
            self.eos = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class GpuEvent:
    """One event on the GPU, built from an ``inputs.Event``."""

    def __init__(self, ev, use_graph=True, fatal_mask=0, eos_handle=None, stream=None, profile=False,
                 precision=SPH_FP64):
        self.ev = ev
        self.dim, self.n = ev.dim, ev.n
        self.npi = 3 if ev.dim == 2 else 5
        self.nv = 2 * ev.dim + 2 + self.npi
        self._own_eos = eos_handle is None
        if eos_handle is None:
            ed, keep = eos_desc(ev.eos, ev.table)
            eos_handle = sph_set_eos_table(ed)
        self.eos = eos_handle
        d, self._keep = event_desc(ev)
        d.fatal_mask, d.use_graph = fatal_mask, int(use_graph)
        d.stream = stream
        d.profile = int(profile)
        d.precision = int(precision)
        self.h = sph_init_event(d, self.eos)
        inv = getattr(ev, "inverse", None)
        if inv is not None:
            sph_eos_build_inverse(self.eos, inv)
            sph_set_eos_mode(self.h, SPH_EOS_OFFLINE)
        jets = getattr(ev, "jets", None)
        if jets is not None and len(jets.tracks):
            sph_set_jets(self.h, jets.tracks, jets.sigma)
        dnmr = getattr(ev.transport, "dnmr", None)
        if dnmr is not None:
            sph_set_viscous_eom(self.h, SPH_EOM_DNMR, dnmr)
        src = getattr(ev, "partons", None)
        if src is not None and len(src.partons):
            sph_set_partons(self.h, src.partons, src.norm, src.h, getattr(src, "charges", None))
        bk = getattr(ev, "eos_backup", None)
        if bk is not None:
            sph_set_eos_backup(self.h, True, bk[0], bk[1])

    def step(self, nsteps: int, sync: bool = False):
        sph_step(self.h, nsteps, SPH_SYNC if sync else 0)

    def read(self, names=("X", "U", "S", "NQ", "BV", "PV")):
        """Fields in original particle order, as numpy arrays."""
        shapes = {"X": (self.dim, "x"), "U": (self.dim, "u"), "S": (1, "S"), "NQ": (3, "Nq"), "BV": (1, "Bv"),
                  "PV": (self.npi, "Pv"), "SIGMA_STAR": (1, "sigstar"), "S_DENS": (1, "s"), "N_DENS": (3, "nq"),
                  "T": (1, "T"), "MU": (3, "mu"), "P": (1, "p"), "E": (1, "e"), "PI_BULK": (1, "Pi"),
                  "STATUS": (1, "status"), "NNB": (1, "nnb"), "CELL": (self.dim, "cell"), "GUESS": (4, "guess"),
                  "JV": (6, "Jv")}
        b = FieldBufs()
        out, mask = {}, 0
        for nm in names:
            rows, attr = shapes[nm]
            dt = np.uint32 if nm == "STATUS" else (np.int32 if nm in ("NNB", "CELL") else np.float64)
            arr = np.zeros((rows, self.n), dtype=dt)
            out[nm] = arr if rows > 1 else arr[0]
            setattr(b, attr, arr.ctypes.data)
            mask |= F[nm]
        sph_read_fields(self.h, mask, b, None)
        return out

    def totals(self):
        t = Totals()
        sph_read_fields(self.h, 0, None, t)
        return {"tau": t.tau, "E": t.E, "S": t.S, "N": np.array(t.N[:]), "work": t.work,
                "status_or": t.status_or, "steps": t.steps, "pairs": t.pairs, "kernel_launches": t.kernel_launches,
                "eos_work": tuple(t.eos_work[:]), "shell_tests": t.shell_tests, "pair_overflows": t.pair_overflows}

    def kernel_times(self):
        return sph_kernel_times(self.h)

    def neighbors(self):
        cnt = sph_debug_neighbors(self.h, 0, None, None)
        pa = np.zeros(max(cnt, 1), dtype=np.int32)
        pb = np.zeros(max(cnt, 1), dtype=np.int32)
        sph_debug_neighbors(self.h, cnt, pa, pb)
        return pa[:cnt], pb[:cnt]

    def rates(self):
        r = np.zeros((self.nv, self.n))
        g = np.zeros((self.dim * self.dim + self.dim, self.n))
        sph_debug_rates(self.h, r, g)
        return r, g

    def write_state(self, x=None, u=None, S=None, Bv=None, Pv=None, guess=None):
        b = FieldBufs()
        keep, mask = [], 0
        for nm, arr, attr in [("X", x, "x"), ("U", u, "u"), ("S", S, "S"), ("BV", Bv, "Bv"), ("PV", Pv, "Pv"),
                              ("GUESS", guess, "guess")]:
            if arr is not None:
                a = _f64(arr)
                keep.append(a)
                setattr(b, attr, a.ctypes.data)
                mask |= F[nm]
        sph_write_state(self.h, mask, b)

    def freezeout_setup(self, e_fo: float, capacity: int):
        sph_freezeout_setup(self.h, e_fo, capacity)
        self._fo_cap = int(capacity)

    def read_freezeout(self):
        """(records [count][SPH_FO_NREC], original particle ids [count]) sorted by (tau, id)."""
        cap = self._fo_cap
        rec = np.zeros((cap, SPH_FO_NREC))
        ids = np.zeros(cap, dtype=np.int64)
        cnt = sph_read_freezeout(self.h, cap, rec, ids)
        return rec[:cnt].copy(), ids[:cnt].copy()

    def free(self):
        if self.h is not None:
            sph_free_event(self.h)
            self.h = None
        if self._own_eos and self.eos is not None:
            sph_free_eos(self.eos)
            self.eos = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
