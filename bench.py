"""Benchmark: SPH particle-steps/s, events/hr and p50/p99 event latency of the serving form
against the plain FP64 form, on the serving stream.

Workload: 512 viscous 2+1D BSQ events (Milne, boost invariant, minimal Israel-Stewart shear +
bulk with eta/s = 0.08 and a Gaussian zeta/s, synthetic 64 x 32^3 FP64 EoS table), particle
counts log-uniform in 5k-200k at the single event's resolution (spacing 0.062 fm, h = 0.3 fm,
200 seeded Gaussian hotspots), each evolved tau 0.6 -> 8 fm/c (1480 Heun steps of 0.005 fm),
arriving as a Poisson stream at a mean 20 events/s.  Events are submitted at their arrival
times through the C ABI with host arrays; the server batches all resident events into one
CUDA-graph batch step per Heun step (mixed precision: FP32 compensated neighbour sums, FP64
EoS inversion, equations of motion and totals).  particle-steps/s = the stream's particles x
steps / the summed device time of its batch steps; events/hr and the latency percentiles are
wall-clock figures of the whole stream.  The plain FP64 form, one event at a time, is timed on
a sample of whole events and extrapolated to the stream.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
    python bench.py --profile-case serving|fp64|mixed|diffusion [--events E] [--profile-steps K]
        (a short fixed run of the timed kernels for profiler captures; measures nothing)

N > 1 runs under torchrun, one independent stream per rank (replicas, weak scaling, no
collective on the data path); rank 0 prints one JSON line.  --impl reference times the CPU
oracle (FP64 C, all host cores) on a sample of the same stream.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SPH particle-steps/s"
UNIT = "particle-steps/s"

# algorithmic FP64 flops per accepted ordered neighbour pair (fused multiply-add = 2), with the
# kernel of each unordered pair evaluated once (its two ordered pairs share it):
#   density : [distance 5, sqrt 1, q 1, kernel and kernel-derivative polynomials with 1/r 12,
#             dW vector 2] / 2 shared, five accumulations 10                                = 20.5
#   gradient: sum of dW 2, stress divergence 8, velocity gradient 8                        = 18
FLOPS_PER_PAIR = {"density": 20.5, "gradient": 18.0}
# EoS inversion, per unit of work actually done (counted on the device):
#   table residual + Jacobian evaluation (the quadrilinear interpolant reduced axis by axis with
#   its four derivatives: 16 corner patches x 12, 8 x 9, 4 x 12; location 12; residual and
#   scaling 28) 352; 4x4 Gaussian elimination with pivoting 64; closed-form g(T), g'(T) 26
FLOPS_EOS = (352.0, 64.0, 26.0)
# nominal FP64 vector rate of GB300 (1.25 TFLOP/s at the 2070 MHz maximum SM clock), context only:
# the rooflines divide by the rates measured on the device (sph_measure_fma_peak)
FP64_PEAK_GFLOPS = 1250.0


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9 and parts[1].replace(".", "").isdigit():
                    rows.append(parts)
        except OSError:
            pass
        finally:
            try:
                os.unlink(self.path)
            except OSError:
                pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": float(rows[0][2]), "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None}


def combine_ranks(dev_ms: float, units: float, device=None):
    """(max over ranks of the timed device milliseconds, sum over ranks of the particle-steps).

    Replicas: every rank advances its own event, so the job's work is the sum and its time the
    slowest rank's.  Without an initialised process group this is the identity."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(dev_ms), float(units)
    t = torch.tensor([float(dev_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def cpu_baseline(ev, served, nsteps):
    """The CPU oracle, as it stands, on a bounded sample of the stream: one whole event (the
    stream's smallest) for all its Heun steps, on the host's cores.  The same run states the
    serving form's error against the oracle on that event: T, mu, s and n_q normwise (max |d| /
    max |ref|) and T per particle (max relative), and the neighbour counts' agreement."""
    import numpy as np
    from oracle import oracle as O
    run = O.OracleRun.start(ev)
    t = time.perf_counter()
    run.step(nsteps)
    dt = time.perf_counter() - t
    aux, _ = run.observe()
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    err = None
    if served is not None:
        nrm = lambda a, b: float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))
        T_ref = aux[O.AUX["T"]]
        err = {"T": nrm(served["T"], T_ref),
               "T_max_rel_per_particle": float(np.max(np.abs(served["T"] / T_ref - 1.0))),
               "mu": nrm(served["MU"], np.stack([aux[O.AUX[k]] for k in ("muB", "muS", "muQ")])),
               "s": nrm(served["S_DENS"], aux[O.AUX["s"]]),
               "n_q": nrm(served["N_DENS"], np.stack([aux[O.AUX[k]] for k in ("nB", "nS", "nQ")])),
               "parity_tolerance_300_steps": 1e-5,
               "note": "whole evolution (1480 steps): the served form's error against the oracle grows with "
                       "the evolution; the parity tests hold 1e-5 over 300 steps, and the FP64 form stays "
                       "within 1e-13 of the oracle over the whole evolution"}
    return {"value": ev.n * nsteps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one whole event of the stream (its smallest, {ev.n} particles): all {nsteps} Heun steps, "
                      f"tau 0.6 -> 8 fm/c ({dt:.1f} s, FP64 C oracle, OpenMP over particles)"}, err


# ---------------------------------------------------------------------------
# the serving workload: a Poisson stream of viscous 2+1D BSQ events
# ---------------------------------------------------------------------------
C4_EVENTS = 512
C4_RATE = 20.0     # mean arrivals per second
C4_STEPS = 1480    # Heun steps of dtau = 0.005 fm: tau 0.6 -> 8 fm/c
C4_ARENA = 1 << 20  # resident particles (the batch step saturates the GPU from about 0.5 M)
C4_WORKLOAD = (f"serving stream: {C4_EVENTS} viscous 2+1D BSQ events (eta/s 0.08, Gaussian zeta/s, 64x32^3 EoS table), "
               f"particle counts log-uniform in 5k-200k, each tau 0.6 -> 8 fm/c ({C4_STEPS} Heun steps, dtau 0.005 fm, "
               f"h 0.3 fm, spacing 0.062 fm), Poisson arrivals at {C4_RATE:g} events/s; batched mixed precision "
               f"(FP32 compensated neighbour sums, FP64 EoS/EoM/totals)")


def c4_sizes(nevents: int = C4_EVENTS, seed_sizes: int = 4):
    """Particle counts of the stream: floor(exp(U(ln 5e3, ln 2e5))) from the sizes seed."""
    import math
    import numpy as np
    from paper_2511_22852_gb300 import inputs as I
    u = I.uniform01(seed_sizes, nevents)
    return np.floor(np.exp(math.log(5e3) + u * (math.log(2e5) - math.log(5e3)))).astype(int)


# matter colder than 0.10 GeV (below the 0.15 GeV freeze-out surface, above the EoS table's
# 0.05 GeV lower edge) streams freely: it has left the fluid
C4_T_STOP_GEV = 0.10


def c4_event(e: int, n: int):
    """Event e of the stream: the single-event workload's spacing (0.062 fm), hotspot width
    (0.4 fm) and hotspot density (200 per 154 fm^2) on a disc of radius 7 fm sqrt(n / 40000),
    so round(200 n / 40000) hotspots; hotspot seed 1000 + e, charge seed 500000 + e.  Particles
    colder than 0.10 GeV stream freely (below the freeze-out surface)."""
    import math
    from paper_2511_22852_gb300 import inputs as I
    ev = I.viscous_bsq_2p1(n_target=int(n), R=7.0 * math.sqrt(n / 40000.0), n_hot=max(1, round(200 * n / 40000)),
                           seed_hot=1000 + e, seed_charge=500000 + e, with_table=False)
    ev.transport.T_stop_GeV = C4_T_STOP_GEV
    return ev


def _c4_event_job(arg):
    return c4_event(*arg)


def c4_events(sizes, workers: int = 8, offset: int = 0):
    """All events of the stream (event e with seeds of event e + offset), generated in a spawned
    process pool before the timed region."""
    import multiprocessing as mp
    jobs = [(e + offset, int(n)) for e, n in enumerate(sizes)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(max(1, min(workers, os.cpu_count() or 1))) as pool:
        return pool.map(_c4_event_job, jobs, chunksize=8)


def c4_arrivals(nevents: int = C4_EVENTS, rate: float = C4_RATE, seed: int = 3):
    """Poisson arrival times (s): exponential gaps from the arrivals seed, the first at 0."""
    import numpy as np
    from paper_2511_22852_gb300 import inputs as I
    u = I.uniform01(seed, nevents)
    gaps = -np.log1p(-u) / rate
    return np.cumsum(gaps) - gaps[0]


def replica_stream(rank: int, nevents: int = C4_EVENTS):
    """The stream of one rank (replicas): sizes and arrival times from rank-shifted seeds; its
    events use the event seeds shifted by 100000 rank."""
    return c4_sizes(nevents, seed_sizes=4 + 1000 * rank), c4_arrivals(nevents, seed=3 + 1000 * rank), 100000 * rank


def serve_stream(Bd, srv, evs, arrivals, nsteps, names=("T", "MU", "S_DENS", "N_DENS", "STATUS"), keep=()):
    """Runs the stream through the server: each event submitted (host arrays, the public API) at
    its arrival time, batch steps pumped in between, each finished event's fields collected to
    host memory.  Returns per-event latency (scheduled arrival to results readable in host
    memory), the wall time from the first arrival to the last collection, bytes copied in and
    out, the EoS work and pairs summed over the events, and the collected fields of `keep`."""
    import numpy as np
    ne = len(evs)
    lat = np.zeros(ne)
    ticket_ev = {}
    submit_off = np.zeros(ne)
    h2d = d2h = 0
    eos_work = np.zeros(3)
    pairs = 0
    kept = {}
    status_counts = {"FALLBACK": 0, "OUT_OF_TABLE": 0, "NOCONV": 0, "CS2_CAPPED": 0}
    i = 0
    done = 0
    t0 = time.perf_counter()
    while done < ne:
        now = time.perf_counter() - t0
        while i < ne and arrivals[i] <= now:
            tk = srv.submit(evs[i], nsteps)
            submit_off[i] = time.perf_counter() - t0 - arrivals[i]
            ticket_ev[tk] = i
            h2d += 12 * 8 * evs[i].n
            i += 1
        running = srv.pump(1)
        if srv.stats()["done"] > 0:
            for tk in [t for t in ticket_ev if srv.poll(t)[0] == Bd.SPH_TICKET_DONE]:
                e = ticket_ev.pop(tk)
                lat[e] = srv.poll(tk)[1] + submit_off[e]
                out = srv.collect(tk, names=names)
                d2h += sum(v.nbytes for k, v in out.items() if k != "totals")
                eos_work += np.array(out["totals"]["eos_work"], dtype=float)
                pairs += out["totals"]["pairs"]
                st = out["STATUS"] if "STATUS" in out else None
                if st is not None:
                    for nm, bit in (("FALLBACK", 1), ("OUT_OF_TABLE", 2), ("NOCONV", 4), ("CS2_CAPPED", 16)):
                        status_counts[nm] += int(np.count_nonzero(st & bit))
                if e in keep:
                    kept[e] = out
                done += 1
        if running == 0 and i < ne and not ticket_ev:
            time.sleep(max(0.0, min(0.002, arrivals[i] - (time.perf_counter() - t0))))
        if time.perf_counter() - t0 > 3000:
            raise RuntimeError("serving stream did not finish within 3000 s")
    wall = time.perf_counter() - t0
    return {"latency": lat, "wall": wall, "h2d": h2d, "d2h": d2h, "eos_work": eos_work, "pairs": pairs,
            "kept": kept, "status_counts": status_counts}


def fp64_one_at_a_time(Bd, I, evs, sizes, nsteps):
    """The plain FP64 form, one event at a time, end to end (upload, nsteps steps, read T), on a
    sample of whole events of the stream -- its smallest, the size quartiles and its largest --
    and the time of the whole stream extrapolated by a least-squares fit t(N) = a + b N."""
    import numpy as np
    order = np.argsort(sizes)
    pick = sorted({int(order[0]), int(order[len(order) // 4]), int(order[len(order) // 2]),
                   int(order[3 * len(order) // 4]), int(order[-1])})
    table = I.synthetic_eos_table(I.BJ_EOS)
    ed, keep = Bd.eos_desc(I.BJ_EOS, table)
    eh = Bd.sph_set_eos_table(ed)
    warm = Bd.GpuEvent(evs[pick[0]], use_graph=True, eos_handle=eh)
    warm.step(4, sync=True)
    warm.free()
    samples = []
    for e in pick:
        t = time.perf_counter()
        g = Bd.GpuEvent(evs[e], use_graph=True, eos_handle=eh)
        g.step(nsteps, sync=True)
        g.read(("T",))
        g.free()
        samples.append((int(sizes[e]), time.perf_counter() - t))
    Bd.sph_free_eos(eh)
    n_s = np.array([s[0] for s in samples], dtype=float)
    t_s = np.array([s[1] for s in samples])
    b, a = np.polyfit(n_s, t_s, 1)
    total = float(np.sum(a + b * sizes.astype(float)))
    return {"sample_events": [{"event": e, "particles": n, "seconds": t} for e, (n, t) in zip(pick, samples)],
            "fit_seconds": {"a": float(a), "b_per_particle": float(b)},
            "stream_seconds_extrapolated": total,
            "events_per_hr": 3600.0 * len(sizes) / total,
            "particle_steps_per_s": float(np.sum(sizes)) * nsteps / total,
            "how": f"{len(pick)} whole events ({nsteps} steps each; the smallest, the size quartiles, the largest) "
                   f"timed end to end (upload, steps, read of T), one at a time; the stream's time is the sum over "
                   f"its {len(sizes)} events of the least-squares line through them"}


def mixed_vs_fp64(fm, f64):
    """Normwise error (max |d| / max |ref|) of the mixed form's fields against the FP64 form's
    after the same steps (the FP64 form follows the oracle to 1e-11 per step, tests/)."""
    import numpy as np
    out = {}
    for k in ("T", "MU", "S_DENS", "N_DENS"):
        a, b = np.asarray(fm[k], dtype=np.float64), np.asarray(f64[k], dtype=np.float64)
        den = float(np.max(np.abs(b)))
        if den > 0:
            out[k] = float(np.max(np.abs(a - b)) / den)
    return out


def bench_mixed_single(Bd, I, steps: int = 50):
    """The 40k-particle event in the mixed-precision forms: the per-event SPH_MIXED path (cell-tiled
    passes over the 2h-cells, one CUDA graph per step) and the serving form holding this one
    event (cell-tiled passes over h-cells, one CUDA graph per batch step); device or wall ms per
    step after warm-up, and the per-event form's error against the FP64 form after the same
    steps."""
    import torch
    ev = I.viscous_bsq_2p1()
    st = torch.cuda.Stream()
    g = Bd.GpuEvent(ev, use_graph=True, stream=st.cuda_stream, precision=Bd.SPH_MIXED)
    g.step(3, sync=True)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(st):
        a.record(st)
        g.step(steps)
        b.record(st)
    torch.cuda.synchronize()
    per_event = a.elapsed_time(b) / steps
    names = ("T", "MU", "S_DENS", "N_DENS")
    fm = g.read(names)
    g.free()
    g64 = Bd.GpuEvent(ev, use_graph=True, precision=Bd.SPH_FP64)
    g64.step(3 + steps, sync=True)
    err = mixed_vs_fp64(fm, g64.read(names))
    g64.free()
    srv = Bd.GpuServer(ev.eos, ev.table, max_events=2, max_particles=1 << 17)
    t = srv.submit(ev, steps + 8)
    srv.pump(4)
    srv.autotune(2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    srv.pump(steps)
    torch.cuda.synchronize()
    served = 1e3 * (time.perf_counter() - t0) / steps
    srv.drain(60.0)
    srv.collect(t, names=("T",))
    srv.free()
    return {"workload": "40k-particle viscous BSQ event, mixed precision", "per_event_ms_per_step": per_event,
            "per_event_particle_steps_per_s": ev.n / (per_event / 1e3),
            "serving_one_event_ms_per_step": served,
            "serving_one_event_particle_steps_per_s": ev.n / (served / 1e3),
            "per_event_vs_fp64": {**err, "steps": 3 + steps},
            "note": "per-event: CUDA events; serving: wall clock over pumped batch steps (host pacing included)"}


def bench_freezeout(Bd, I, steps: int = 40):
    """Cost of recording the freeze-out surface on the 40k-particle event: device ms per step
    with and without recording (CUDA graphs, CUDA events), and the elements recorded, for a
    surface at the 20 % quantile of the initial energy density (it sweeps through the cooling
    edge during the window)."""
    import numpy as np
    import torch
    ev = I.viscous_bsq_2p1()
    g0 = Bd.GpuEvent(ev)
    e0 = g0.read(("E",))["E"]
    g0.free()
    se = np.sort(e0)
    k = int(0.2 * len(se))
    while se[k + 1] - se[k] < 1e-6 * se[k]:
        k += 1
    e_fo = 0.5 * float(se[k] + se[k + 1])
    out = {"workload": f"40k-particle viscous BSQ event, e_fo = {e_fo:.4g} fm^-4 (20 % quantile of the initial e), "
                       f"{steps} steps", "e_fo": e_fo}
    for name, on in (("without", False), ("with", True)):
        st = torch.cuda.Stream()
        g = Bd.GpuEvent(ev, use_graph=True, stream=st.cuda_stream)
        if on:
            g.freezeout_setup(e_fo, 100000)
        g.step(2, sync=True)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):
            a.record(st)
            g.step(steps)
            b.record(st)
        torch.cuda.synchronize()
        out[name + "_ms_per_step"] = a.elapsed_time(b) / steps
        if on:
            rec, ids = g.read_freezeout()
            out["elements"] = int(len(ids))
        g.free()
    out["overhead"] = out["with_ms_per_step"] / out["without_ms_per_step"] - 1.0
    return out


def bench_dnmr(Bd, I, steps: int = 40):
    """The DNMR equations of motion (14-moment coefficients) against minimal Israel-Stewart on
    the 40k-particle event: device ms per step (CUDA graphs, CUDA events) and the EoM pass."""
    import torch
    out = {"workload": f"40k-particle viscous BSQ event, {steps} steps, DNMR (14-moment coefficients) vs minimal IS"}
    for name, dn in (("min_is", None), ("dnmr", I.DNMR_14_MOMENT)):
        ev = I.viscous_bsq_2p1()
        ev.transport.dnmr = dn
        st = torch.cuda.Stream()
        g = Bd.GpuEvent(ev, use_graph=True, stream=st.cuda_stream)
        g.step(2, sync=True)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):
            a.record(st)
            g.step(steps)
            b.record(st)
        torch.cuda.synchronize()
        out[name + "_ms_per_step"] = a.elapsed_time(b) / steps
        g.free()
        gp = Bd.GpuEvent(ev, use_graph=False, stream=st.cuda_stream, profile=True)
        gp.step(4)
        torch.cuda.synchronize()
        kt = gp.kernel_times()
        out[name + "_eom_ms_per_pass"] = kt["eom"][0] / max(1, kt["eom"][1])
        gp.free()
    out["overhead"] = out["dnmr_ms_per_step"] / out["min_is_ms_per_step"] - 1.0
    return out


def bench_partons(Bd, I, steps: int = 40, per_step: int = 100):
    """Cost of dynamical-initialisation sources on the 40k-particle event: partons forming at
    per_step per step over the window (h_src = 1.4 fm, the paper's smearing width), device ms
    per step with and without them (CUDA graphs, CUDA events)."""
    import torch
    ev = I.viscous_bsq_2p1()
    npart = per_step * steps
    src = I.parton_sources(npart, (ev.tau0, ev.tau0 + steps * ev.dtau), 4.0, 2, E_GeV=(0.1, 0.3), norm=0.42, h=1.4)
    out = {"workload": f"40k-particle viscous BSQ event, {npart} partons forming over {steps} steps "
                       f"({per_step} per step, h_src = 1.4 fm, |x|, |y| <= 4 fm)"}
    for name, on in (("without", False), ("with", True)):
        ev.partons = src if on else None
        st = torch.cuda.Stream()
        g = Bd.GpuEvent(ev, use_graph=True, stream=st.cuda_stream)
        g.step(1, sync=True)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):
            a.record(st)
            g.step(steps)
            b.record(st)
        torch.cuda.synchronize()
        out[name + "_ms_per_step"] = a.elapsed_time(b) / steps
        g.free()
    out["overhead"] = out["with_ms_per_step"] / out["without_ms_per_step"] - 1.0
    return out


def bench_offline_eos(Bd, I, steps: int = 20):
    """The offline EoS inverter (interpolation in an inverted (s, n/s) table) against the online
    Newton inversion on the 40k-particle event: device ms per step and per EoS pass (profile
    mode), table build time, and the accuracy of T and mu_B against the online inversion."""
    import numpy as np
    import torch
    out = {}
    grid = I.InverseGrid(per_decade=90, decade_lo=-3, decades=6, nx=17, xmax=0.04)
    res = {}
    for name in ("online", "offline"):
        ev = I.viscous_bsq_2p1()
        if name == "offline":
            ev.inverse = grid
        t0 = time.perf_counter()
        g = Bd.GpuEvent(ev, use_graph=False, profile=True)
        build_s = time.perf_counter() - t0
        f = g.read(("T", "MU"))
        g.step(2)
        k0 = g.kernel_times()
        g.step(steps)
        k1 = g.kernel_times()
        torch.cuda.synchronize()
        eos_ms = (k1["eos"][0] - k0["eos"][0]) / (2 * steps)
        tot_ms = sum(k1[k][0] - k0[k][0] for k in k1) / steps
        res[name] = (f, eos_ms, tot_ms, build_s)
        g.free()
    fo, fn = res["offline"][0], res["online"][0]
    out = {"workload": "40k-particle viscous BSQ event; inverted table: s on 10^-3..10^3 with 90 nodes per decade, "
                       "n_q/s on 17 nodes in +-0.04 (2.66M nodes, 85 MB)",
           "online_eos_ms_per_pass": res["online"][1], "offline_eos_ms_per_pass": res["offline"][1],
           "online_ms_per_step": res["online"][2], "offline_ms_per_step": res["offline"][2],
           "eos_speedup": res["online"][1] / res["offline"][1],
           "table_build_s": res["offline"][3] - res["online"][3],
           "T_max_rel_err": float(np.max(np.abs(fo["T"] / fn["T"] - 1))),
           "T_mean_rel_err": float(np.mean(np.abs(fo["T"] / fn["T"] - 1))),
           "muB_err_normwise": float(np.max(np.abs(fo["MU"][0] - fn["MU"][0])) / np.max(np.abs(fn["MU"][0])))}
    return out


def bench_3p1d(Bd, I, steps: int = 3):
    """The 3+1D hyperbolic viscous BSQ event (about 10^6 particles): device ms per Heun step of
    the plain FP64 form next to the mixed form (FP32 neighbour sums, FP64 EoS and equations of
    motion), CUDA events on the event's stream after one untimed step."""
    import torch
    import numpy as np
    ev = I.viscous_bsq_3p1()
    out = {"workload": f"3+1D Milne viscous BSQ event, {ev.n} particles, dx = dy = 0.124 fm, d_eta = 0.1, "
                       f"h = 0.3 fm, dtau = 0.005 fm, 64x32^3 EoS table", "steps": steps}
    e_fo = None
    fields = {}
    for name, prec in (("fp64", Bd.SPH_FP64), ("mixed", Bd.SPH_MIXED), ("fp64_freezeout", Bd.SPH_FP64)):
        st = torch.cuda.Stream()
        g = Bd.GpuEvent(ev, use_graph=True, stream=st.cuda_stream, precision=prec)
        if name == "fp64":  # a freeze-out surface at the 20 % quantile of the initial e (cooling edge)
            se = np.sort(g.read(("E",))["E"])
            k = int(0.2 * len(se))
            while se[k + 1] - se[k] < 1e-6 * se[k]:
                k += 1
            e_fo = 0.5 * float(se[k] + se[k + 1])
        if name == "fp64_freezeout":
            g.freezeout_setup(e_fo, 400000)
        g.step(1, sync=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):
            e0.record(st)
            g.step(steps)
            e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[name] = {"ms_per_step": ms, "particle_steps_per_s": ev.n / (ms / 1e3)}
        if prec == Bd.SPH_MIXED:
            out[name]["shell_tests"] = g.totals()["shell_tests"]
        if name in ("fp64", "mixed"):
            fields[name] = g.read(("T", "MU", "S_DENS", "N_DENS"))
        if name == "fp64_freezeout":
            out[name]["e_fo"] = e_fo
            out[name]["elements"] = int(len(g.read_freezeout()[1]))
        g.free()
    out["mixed_speedup"] = out["fp64"]["ms_per_step"] / out["mixed"]["ms_per_step"]
    out["mixed_vs_fp64"] = {**mixed_vs_fp64(fields["mixed"], fields["fp64"]), "steps": 1 + steps}
    out["freezeout_overhead"] = out["fp64_freezeout"]["ms_per_step"] / out["fp64"]["ms_per_step"] - 1.0
    return out


def bench_stress(Bd, I, steps: int = 3):
    """The stress configuration: 3+1D Cartesian viscous BSQ event with 10 jet tracks, about
    8 10^6 particles, 128 x 64^3 EoS table; device ms per Heun step of the FP64 form next to the
    mixed form (CUDA events on the event's stream after one untimed step)."""
    import torch
    ev = I.stress_cartesian_3d()
    out = {"workload": f"3+1D Cartesian viscous BSQ event with 10 jet tracks (5 GeV/fm, sigma 0.3 fm), "
                       f"{ev.n} particles, spacing {ev.meta['dx']:.4f} fm, h = 0.15 fm, dt = 0.005 fm, "
                       f"128x64^3 EoS table", "steps": steps}
    fields = {}
    for name, prec in (("fp64", Bd.SPH_FP64), ("mixed", Bd.SPH_MIXED)):
        st = torch.cuda.Stream()
        g = Bd.GpuEvent(ev, use_graph=True, stream=st.cuda_stream, precision=prec)
        g.step(1, sync=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):
            e0.record(st)
            g.step(steps)
            e1.record(st)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        out[name] = {"ms_per_step": ms, "particle_steps_per_s": ev.n / (ms / 1e3),
                     "status_or": g.totals()["status_or"]}
        fields[name] = g.read(("T", "MU", "S_DENS", "N_DENS"))
        g.free()
    out["mixed_speedup"] = out["fp64"]["ms_per_step"] / out["mixed"]["ms_per_step"]
    out["mixed_vs_fp64"] = {**mixed_vs_fp64(fields["mixed"], fields["fp64"]), "steps": 1 + steps}
    return out


def run_reference(args):
    """The oracle (FP64 C, all host cores) on a bounded sample of the serving stream: W untimed and
    K timed Heun steps of the stream's median-size event."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    from oracle import oracle as O
    sizes = c4_sizes()
    e = int(np.argsort(sizes)[len(sizes) // 2])
    ev = c4_event(e, int(sizes[e]))
    ev.table = None
    run = O.OracleRun.start(_with_table(ev))
    for _ in range(args.warmup):
        run.step(1)
    t = time.perf_counter()
    run.step(args.steps)
    dt = time.perf_counter() - t
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    val = ev.n * args.steps / dt
    line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": C4_WORKLOAD, "events": C4_EVENTS, "l2": "host run (no GPU)"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} Heun steps (after {args.warmup} untimed) of event {e} of the "
                                       f"stream, its median size ({ev.n} particles), plain FP64"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


_TABLE = {}


def _with_table(ev):
    """The event with the shared 64 x 32^3 EoS table attached (built once)."""
    from paper_2511_22852_gb300 import inputs as I
    if "t" not in _TABLE:
        _TABLE["t"] = I.synthetic_eos_table(I.BJ_EOS)
    ev.table = _TABLE["t"]
    return ev


def traffic_of(kernel: str, particles_per_launch: float | None = None):
    """DRAM bytes (read + write) per launch of a kernel from the committed ncu summary
    (profiles/traffic.json: bytes per particle of one captured launch), scaled to the launch's
    particle count when it differs from the capture's; None when a source file of the kernel
    changed since the capture (the counters then no longer describe it)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))[kernel]
        h = hashlib.sha256()
        for f in rec["sources"]:
            h.update(open(os.path.join(ROOT, "paper_2511_22852_gb300", "csrc", f), "rb").read())
    except (OSError, KeyError, ValueError):
        return None
    if h.hexdigest()[:16] != rec["source_sha16"]:
        return None
    n = float(particles_per_launch) if particles_per_launch else float(rec["particles"])
    out = {"bytes_per_launch": rec["bytes_per_particle"] * n, "bytes_per_particle": rec["bytes_per_particle"],
           "capture": rec["capture"], "captured_particles": rec["particles"]}
    if "counters" in rec:  # pipe and issue activity of the captured launch (ncu)
        out["counters"] = rec["counters"]
    if "note" in rec:
        out["note"] = rec["note"]
    if abs(n - rec["particles"]) > 0.5:
        out["scaled"] = (f"captured on {rec['particles']} particles, scaled to {n:.0f} per launch "
                         "(DRAM bytes taken proportional to the particles processed)")
    return out


def bench_fp64_event(Bd, I, stream, flush, first_k: int):
    """The 40k-particle viscous BSQ event in the plain FP64 form over its whole evolution (tau 0.6
    -> 8 fm/c): every step timed with CUDA events on the event's stream after an L2 flush, and the
    kernel groups timed in profile mode over the same evolution (rooflines of the FP64 kernels)."""
    import numpy as np
    import torch
    ev = I.viscous_bsq_2p1()
    nsteps = ev.nsteps
    g = Bd.GpuEvent(ev, use_graph=True, stream=stream.cuda_stream)
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(nsteps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(nsteps)]
    t_before = g.totals()
    with torch.cuda.stream(stream):
        for k in range(nsteps):
            flush.fill_(float(k))
            e0[k].record(stream)
            g.step(1)
            e1[k].record(stream)
    torch.cuda.synchronize()
    ms = np.array([a.elapsed_time(b) for a, b in zip(e0, e1)])
    t_after = g.totals()
    st = g.read(("STATUS",))["STATUS"]
    g.free()
    # profile mode: CUDA events around each kernel group, same evolution
    gp = Bd.GpuEvent(ev, use_graph=False, stream=stream.cuda_stream, profile=True)
    tot0 = gp.totals()
    with torch.cuda.stream(stream):
        for k in range(nsteps):
            gp.step(1)
    torch.cuda.synchronize()
    tot1 = gp.totals()
    times = gp.kernel_times()
    gp.free()
    pairs = tot1["pairs"] - tot0["pairs"]
    ew = [b - a for a, b in zip(tot0["eos_work"], tot1["eos_work"])]
    flops = {"density": FLOPS_PER_PAIR["density"] * pairs,
             "gradient": FLOPS_PER_PAIR["gradient"] * (pairs - 2 * nsteps * ev.n),
             "eos": sum(f * w for f, w in zip(FLOPS_EOS, ew))}
    total_ms = sum(v[0] for v in times.values())
    return {"workload": "viscous 2+1D BSQ single event, plain FP64: 39,997 particles, 64x32^3 EoS table, h 0.3 fm, "
                        f"tau 0.6 -> 8 fm/c ({nsteps} Heun steps), CUDA graph, L2 flushed between timed steps",
            "ms_per_step": float(ms.mean()), "particle_steps_per_s": ev.n / (ms.mean() / 1e3),
            "ms_per_step_first_k": float(ms[:first_k].mean()), "first_k": first_k,
            "ms_per_step_by_tenth": [float(x.mean()) for x in np.array_split(ms, 10)],
            "status_counts_final": {nm: int(np.count_nonzero(st & bit)) for nm, bit in
                                    (("FALLBACK", 1), ("OUT_OF_TABLE", 2), ("NOCONV", 4), ("CS2_CAPPED", 16))},
            "status_or": int(t_after["status_or"]),
            "pair_list_overflow_stages": int(t_after["pair_overflows"] - t_before["pair_overflows"]),
            "kernel_share": {k: round(v[0] / total_ms, 4) for k, v in times.items()},
            "_times": times, "_flops": flops, "_launches": int(t_after["kernel_launches"] - t_before["kernel_launches"])}


def alu_roof(name, flops, ms, launches, peak, peak_name, kernel, traffic=None):
    achieved = flops / (ms / 1e3) / 1e9
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "GFLOP/s", "frac": achieved / peak,
            "traffic": traffic["bytes_per_launch"] if traffic else None, "traffic_source": traffic,
            "kernel": kernel, "group": name, "peak_source": peak_name,
            "avg_launch_ms": ms / max(1, launches), "flops_per_launch": flops / max(1, launches)}


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2511_22852_gb300 import binding as Bd
    from paper_2511_22852_gb300 import build_lib
    from paper_2511_22852_gb300 import inputs as I

    if rank == 0 or not os.path.exists(build_lib.LIB):
        build_lib.build()
    if ws > 1:
        dist.barrier()
    # the stream of this rank (replicas: rank r shifts the event and arrival seeds)
    sizes, arrivals, offset = replica_stream(rank, args.events)
    evs = c4_events(sizes, offset=offset)
    table = I.synthetic_eos_table(I.BJ_EOS)
    # measured arithmetic peaks (the rooflines' denominators)
    fp64_gflops, fp64_ms = Bd.sph_measure_fma_peak(True, 5)
    fp32_gflops, fp32_ms = Bd.sph_measure_fma_peak(False, 5)
    pin = int(sum(200 * n + 4096 for n in sizes)) + (256 << 20)
    srv = Bd.GpuServer(I.BJ_EOS, table, max_events=256, max_particles=C4_ARENA, pinned_bytes=pin)
    # warm-up: W batch steps of the stream's first four events (untimed), the autotuner's choice
    tw = [srv.submit(evs[k], args.warmup + 2) for k in range(4)]
    srv.pump(args.warmup)
    tuned = srv.autotune(3, lanes=True)
    srv.drain(600.0)
    for t in tw:
        srv.collect(t, names=("T",))
    srv.profile(25)
    st0 = srv.stats()
    kt0 = srv.kernel_times()
    smallest = int(np.argmin(sizes))
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        res = serve_stream(Bd, srv, evs, arrivals, C4_STEPS, keep=(smallest,))
    torch.cuda.synchronize()
    st1 = srv.stats()
    kt1 = srv.kernel_times()
    clocks = clk.summary()
    srv.free()
    batch_steps = st1["batch_steps"] - st0["batch_steps"]
    dev_ms = st1["device_ms"] - st0["device_ms"]
    psteps = float(st1["particle_steps"] - st0["particle_steps"])
    dev_ms_max, units = combine_ranks(dev_ms, psteps, device="cuda")
    wall_max, _ = combine_ranks(1e3 * res["wall"], 0.0, device="cuda")
    value = units / (dev_ms_max / 1e3)
    e2e_value = units / (wall_max / 1e3)

    out = None
    if rank == 0:
        lat = res["latency"]
        kt = {k: (v[0] - kt0[k][0], v[1] - kt0[k][1]) for k, v in kt1.items()}
        ktot = sum(v[0] for v in kt.values())
        share = {k: round(v[0] / ktot, 4) for k, v in kt.items()}
        # group times over the whole stream: the sampled shares applied to the device time of all
        # batch steps; launches: two stages per batch step
        g_ms = {k: share[k] * dev_ms for k in kt}
        launches_g = 2 * batch_steps
        ew = res["eos_work"]
        flops = {"eos": float(sum(f * w for f, w in zip(FLOPS_EOS, ew))),
                 "density": FLOPS_PER_PAIR["density"] * res["pairs"],
                 "gradient": FLOPS_PER_PAIR["gradient"] * res["pairs"]}
        peak64 = f"measured FP64 FMA rate of this GPU ({fp64_gflops:.0f} GFLOP/s, sph_measure_fma_peak)"
        peak32 = f"measured FP32 FMA rate of this GPU ({fp32_gflops:.0f} GFLOP/s, sph_measure_fma_peak)"
        ppl = psteps / max(1, batch_steps)  # mean particles per launch (resident per batch step)
        rooflines = {
            "eos": alu_roof("eos", flops["eos"], g_ms["eos"], launches_g, fp64_gflops, peak64, "k_eos2_seg",
                            traffic_of("k_eos2_seg", ppl)),
            "density": alu_roof("density", flops["density"], g_ms["density"], launches_g, fp32_gflops, peak32,
                                "k_seg_density", traffic_of("k_seg_density", ppl)),
            "gradient": alu_roof("gradient", flops["gradient"], g_ms["gradient"], launches_g, fp32_gflops, peak32,
                                 "k_seg_gradient", traffic_of("k_seg_gradient", ppl)),
        }
        rooflines["eos"]["work_per_particle_stage"] = {
            "table_evals": float(ew[0] / (2.0 * psteps)), "solves": float(ew[1] / (2.0 * psteps)),
            "closed_form_evals": float(ew[2] / (2.0 * psteps))}
        for k in ("density", "gradient"):
            rooflines[k]["note"] = ("FP32 neighbour pass: algorithmic FP64-equivalent flops of the accepted pairs "
                                    "against the FP32 FMA rate; the pass is issue-bound (compensated sums, the "
                                    "exact FP64 shell test, cell staging)")
        roof = rooflines[max(("eos", "density", "gradient"), key=lambda k: g_ms[k])]
        fp64_arm = fp64_one_at_a_time(Bd, I, evs, sizes, C4_STEPS)
        stream = torch.cuda.Stream()
        flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
        fp64ev = bench_fp64_event(Bd, I, stream, flush, max(1, args.steps))
        t64, f64 = fp64ev.pop("_times"), fp64ev.pop("_flops")
        fp64ev.pop("_launches")
        fp64ev["kernel_rooflines"] = {
            k: alu_roof(k, f64[k], t64[k][0], t64[k][1], fp64_gflops, peak64,
                        {"density": "k_pairs_density_fwd+bwd", "gradient": "k_pairs_gradient", "eos": "k_eos2"}[k],
                        traffic_of({"density": "k_pairs_density", "gradient": "k_pairs_gradient", "eos": "k_eos2"}[k]))
            for k in f64}
        events_hr = 3600.0 * args.events / res["wall"]
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": dev_ms_max / max(1, batch_steps), "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64 (mixed)", "data": "synthetic",
               "config": {"workload": C4_WORKLOAD, "events": args.events, "particles_total": int(np.sum(sizes)),
                          "heun_steps_per_event": C4_STEPS, "batch_steps": int(batch_steps),
                          "arena_particles": C4_ARENA, "parallelism": f"replicas x{ws}", "cuda_graph": True,
                          "l2": "inputs larger than L2 (resident state of about 1 M particles, ~0.7 GB, and the "
                                "101 MB EoS table)",
                          "value_is": "particle-steps of the whole stream / summed device time of its batch steps "
                                      "(CUDA events around each step)",
                          "ms_per_step_is": "mean device time of one batch step (every resident event advanced "
                                            "one Heun step, both stages); the stream runs to completion, so --steps "
                                            "does not bound it: it sets the first-steps window of the FP64 "
                                            "single-event sub-entry",
                          "autotuned_shape": {"block_threads": tuned[0], "lane_split_warps": tuned[1]}},
               "events_per_hr": events_hr,
               "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                             "mean": float(lat.mean()), "max": float(lat.max()),
                             "from": "scheduled Poisson arrival to the event's results readable in host memory"},
               "fp64_one_at_a_time": fp64_arm,
               "events_per_hr_vs_fp64": events_hr / fp64_arm["events_per_hr"],
               "roofline": roof, "kernel_rooflines": rooflines, "kernel_share": share,
               "peaks_measured": {"fp64_gflops": fp64_gflops, "fp32_gflops": fp32_gflops,
                                  "fp64_launch_ms": fp64_ms, "fp32_launch_ms": fp32_ms,
                                  "nominal_fp64_gflops": FP64_PEAK_GFLOPS},
               "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": res["h2d"] / max(1, batch_steps),
                       "d2h_bytes_per_step": res["d2h"] / max(1, batch_steps), "wall_s": res["wall"],
                       "how": "wall clock from the first scheduled arrival to the last event's results in host "
                              "memory, through sph_submit / sph_server_pump / sph_collect with host arrays"},
               "gpu_launches": int(st1["kernel_launches"] - st0["kernel_launches"]), "clocks": clocks,
               "status_counts_final": res["status_counts"],
               "failed_events": int(st1["failed"] - st0["failed"]),
               "fp64_single_event": fp64ev}
        if not args.no_extras:
            out["mixed_single_event"] = bench_mixed_single(Bd, I)
            out["freezeout"] = bench_freezeout(Bd, I)
            out["dnmr"] = bench_dnmr(Bd, I)
            out["partons"] = bench_partons(Bd, I)
            out["offline_eos"] = bench_offline_eos(Bd, I)
        if not args.no_3d:
            out["config_3p1d"] = bench_3p1d(Bd, I)
            out["config_stress"] = bench_stress(Bd, I)
        if not args.no_cpu_baseline and ws == 1:
            cb, err = cpu_baseline(_with_table(evs[smallest]), res["kept"].get(smallest), C4_STEPS)
            out["cpu_baseline"] = cb
            out["mixed_vs_oracle"] = dict(err or {}, event=smallest, particles=int(sizes[smallest]),
                                          how="the stream's smallest event as served (batched, mixed precision) "
                                              "against the FP64 oracle after its whole evolution")
        print(json.dumps(out), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_profile_case(args):
    """A short, fixed run of the timed kernels for profiler captures (no timing, no reference
    legs): 'serving' -- the stream's first --events events resident at once in the serving
    arena (one event group), --profile-steps batch steps in the tiled-pass shape --profile-shape; 'fp64' -- the
    40k-particle viscous BSQ event in the plain FP64 form, --profile-steps Heun steps (kernels
    launched one by one); 'mixed' -- the same event in the per-event mixed form; 'diffusion' --
    the same event with BSQ diffusion (FP64).  Prints one JSON
    line describing what ran."""
    import numpy as np
    import torch
    from paper_2511_22852_gb300 import binding as Bd
    from paper_2511_22852_gb300 import build_lib
    from paper_2511_22852_gb300 import inputs as I

    build_lib.build()
    k = args.profile_steps
    if args.profile_case == "serving":
        sizes = c4_sizes(C4_EVENTS)[:args.events]
        evs = c4_events(sizes)
        tt, lw = (int(v) for v in args.profile_shape.split(","))
        # one event group: every launch covers every event (the stream's two-group schedule runs
        # the same kernels over about half the events each)
        srv = Bd.GpuServer(I.BJ_EOS, I.synthetic_eos_table(I.BJ_EOS), max_events=max(4, len(evs)),
                           max_particles=C4_ARENA, groups=1)
        srv.set_shape(tt, lw)
        for ev in evs:
            srv.submit(ev, C4_STEPS)
        srv.pump(k)
        st = srv.stats()
        srv.free()
        desc = {"events": len(evs), "particles": int(np.sum(sizes)), "batch_steps": int(st["batch_steps"]),
                "shape": [tt, lw], "kernel_launches": int(st["kernel_launches"])}
    else:
        ev = I.viscous_bsq_2p1()
        if args.profile_case == "diffusion":
            ev.diffusion = I.Diffusion(kappaT2=I.KAPPA_BSQ)
        prec = Bd.SPH_MIXED if args.profile_case == "mixed" else Bd.SPH_FP64
        g = Bd.GpuEvent(ev, use_graph=False, precision=prec)
        g.step(k, sync=True)
        g.free()
        desc = {"particles": ev.n, "steps": k}
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": args.profile_case, **desc}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the freeze-out, DNMR, parton, offline-EoS "
                                                               "and single-event mixed sub-entries")
    ap.add_argument("--no-3d", action="store_true")
    ap.add_argument("--events", type=int, default=C4_EVENTS,
                    help="events of the stream (the configuration has 512; fewer only for quick checks)")
    ap.add_argument("--profile-case", choices=["serving", "fp64", "mixed", "diffusion"], default=None,
                    help="a short fixed run of the timed kernels for profiler captures (no measurement)")
    ap.add_argument("--profile-steps", type=int, default=40)
    ap.add_argument("--profile-shape", default="64,2", help="threads,lane-split warps of the tiled passes")
    args = ap.parse_args()
    if args.profile_case:
        return run_profile_case(args)
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    return run_reference(args) if args.impl == "reference" else run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
