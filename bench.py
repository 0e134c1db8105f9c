"""Benchmark: SPH particle-steps/s of the viscous 2+1D BSQ single event (FP64).

Workload: 40k particles in a 7 fm disc (200 seeded Gaussian hotspots, sigma
0.4 fm), Milne 2+1D boost invariant, minimal Israel-Stewart shear + bulk
(eta/s = 0.08, Gaussian zeta/s), synthetic 64 x 32^3 FP64 EoS table, h = 0.3 fm,
dtau = 0.005 fm.  One step = one full Heun (RK2) step of the event: both stages,
each with cell list, kernel sums, EoS inversion, gradients, equations of motion
and update.  particle-steps/s = particles x steps / time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun, one independent event per rank (replicas, weak
scaling, no collective on the data path); rank 0 prints one JSON line.
--impl reference times the CPU oracle (FP64 C, all host cores) on the same event.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SPH particle-steps/s"
UNIT = "particle-steps/s"
WORKLOAD = "viscous 2+1D BSQ single event, FP64: 40k particles, 64x32^3 EoS table, h=0.3 fm, dtau=0.005 fm"

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
# FP64 vector peak of GB300 (nominal 1.25 TFLOP/s at the 2070 MHz maximum SM clock)
FP64_PEAK_GFLOPS = 1250.0
# DRAM bytes (read + write) per launch of the FP64 40k-event kernels, from one ncu capture of
# the current kernels (profiles/ncu_fp64_kernels_viscous_bsq_40k.md; "density" is the forward
# plus the backward pair pass: 6.85 + 130.68 + 104.67 + 15.14 MB); None once a kernel changes
DRAM_BYTES_PER_LAUNCH = {"gradient": 180.3e6, "density": 257.3e6, "eos": 7.33e6, "eom": None}


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


def replica_event(rank: int):
    """The event of one rank: the 40k-particle viscous BSQ workload with rank-shifted seeds."""
    from paper_2511_22852_gb300 import inputs as I
    return I.viscous_bsq_2p1(seed_hot=1 + 1000 * rank, seed_charge=2 + 1000 * rank)


def fp64_dgemm_rate(n: int = 8192, reps: int = 5):
    """Context for the FP64 roofline: cuBLAS DGEMM (torch.matmul in float64, 2 n^3 flops) timed
    with CUDA events, best of reps -- the FP64 rate a library reaches on this GPU, next to the
    nominal vector rate the roofline uses."""
    import torch
    a = torch.rand(n, n, dtype=torch.float64, device="cuda")
    b = torch.rand(n, n, dtype=torch.float64, device="cuda")
    torch.matmul(a, b)
    torch.cuda.synchronize()
    best = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    del a, b
    return {"gflops": 2.0 * n ** 3 / (best / 1e3) / 1e9, "n": n, "best_ms": best,
            "how": "torch.matmul float64 (cuBLAS DGEMM), best of %d, CUDA events" % reps}


def cpu_baseline(ev, target_s=15.0):
    """The CPU oracle, as it stands, on a bounded sample: whole Heun steps of the same event."""
    from oracle import oracle as O
    run = O.OracleRun.start(ev)
    t = time.perf_counter()
    run.step(1)
    t1 = time.perf_counter() - t
    nsteps = max(1, min(60, int(target_s / max(t1, 1e-3))))
    t = time.perf_counter()
    run.step(nsteps)
    dt = time.perf_counter() - t
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": ev.n * nsteps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{nsteps} Heun steps of the full {ev.n}-particle event after 1 untimed step "
                      f"({dt:.1f} s, FP64 C oracle, OpenMP over particles)"}


def serving_events(nevents: int, seed_sizes: int = 4):
    """Serving workload: viscous 2+1D BSQ events with particle counts log-uniform in 5k-200k.

    Every event has the single-event workload's particle spacing (0.062 fm) and hotspot shape,
    on a disc of radius 7 fm sqrt(N / 40000) (the same resolution for systems of different
    size), 200 seeded hotspots, charges within +-1% of s; event e uses seeds 1000 + e."""
    import math
    import numpy as np
    from paper_2511_22852_gb300 import inputs as I
    u = I.uniform01(seed_sizes, nevents)
    sizes = np.floor(np.exp(math.log(5e3) + u * (math.log(2e5) - math.log(5e3)))).astype(int)
    evs = [I.viscous_bsq_2p1(n_target=int(n), R=7.0 * math.sqrt(n / 40000.0), seed_hot=1000 + e,
                             seed_charge=500000 + e, with_table=False) for e, n in enumerate(sizes)]
    return evs


def serving_bench(Bd, I, nevents: int, ksteps: int, load: float = 0.7, max_events: int = 32):
    """events/hr and p50/p99 latency of the serving form against the plain FP64 form run one
    event at a time, on the same events (each advanced ksteps Heun steps from tau0)."""
    import numpy as np
    import torch
    evs = serving_events(nevents)
    ntot = int(sum(e.n for e in evs))
    table = I.synthetic_eos_table(I.BJ_EOS)
    # plain FP64, one event at a time, end to end: upload, ksteps steps, read back T
    ed, keep = Bd.eos_desc(I.BJ_EOS, table)
    eh = Bd.sph_set_eos_table(ed)
    warm = Bd.GpuEvent(evs[0], use_graph=True, eos_handle=eh)
    warm.step(2, sync=True)
    warm.free()
    torch.cuda.synchronize()
    t_fp64 = []
    for e in evs:
        t = time.perf_counter()
        g = Bd.GpuEvent(e, use_graph=True, eos_handle=eh)
        g.step(ksteps, sync=True)
        g.read(("T",))
        g.free()
        t_fp64.append(time.perf_counter() - t)
    Bd.sph_free_eos(eh)
    T64 = sum(t_fp64)
    # serving form, closed loop (every event submitted at once): capacity
    srv = Bd.GpuServer(I.BJ_EOS, table, max_events=max_events, max_particles=int(1.25 * ntot) + 65536,
                       pinned_bytes=int(400 * ntot) + (64 << 20))
    # warm-up batch (8 events), on which the autotuner picks the tiled passes' launch shape
    tw = [srv.submit(e, 4) for e in evs[:8]]
    srv.pump(2)
    tuned = srv.autotune(3)
    srv.drain(120.0)
    for t in tw:
        srv.collect(t, names=("T",))
    st0 = srv.stats()
    t0 = time.perf_counter()
    tk = [srv.submit(e, ksteps) for e in evs]
    srv.drain(600.0)
    lat_closed = [srv.poll(t)[1] for t in tk]
    makespan = max(lat_closed)  # every event submitted at t0
    wall_closed = time.perf_counter() - t0
    torch.cuda.synchronize()
    st1 = srv.stats()
    ew = np.zeros(3)
    for t in tk:
        ew += np.array(srv.collect(t, names=("T",))["totals"]["eos_work"], dtype=float)
    # EoS work per particle and stage (the observe pass of each event counted as one stage)
    eos_per_pstage = (ew / (ntot * (2 * ksteps + 1))).tolist()
    cap_eps = nevents / makespan
    # open loop: Poisson arrivals at `load` x the measured capacity (exponential gaps, seed 3)
    u = I.uniform01(3, nevents)
    gaps = -np.log1p(-u) / (load * cap_eps)
    arrivals = np.cumsum(gaps) - gaps[0]
    tk2 = []
    t0 = time.perf_counter()
    i = 0
    while i < nevents or any(srv.poll(t)[0] != Bd.SPH_TICKET_DONE for t in tk2):
        now = time.perf_counter() - t0
        while i < nevents and arrivals[i] <= now:
            tk2.append(srv.submit(evs[i], ksteps))
            i += 1
        running = srv.pump(1)
        if running == 0 and i < nevents:
            time.sleep(max(0.0, min(0.002, arrivals[i] - (time.perf_counter() - t0))))
        if time.perf_counter() - t0 > 900:
            raise RuntimeError("serving benchmark did not finish")
    lat_open = np.array([srv.poll(t)[1] for t in tk2])
    wall_open = time.perf_counter() - t0
    for t in tk2:
        srv.collect(t, names=("T",))
    st2 = srv.stats()
    srv.free()
    ps = float(ntot * ksteps)
    return {
        "workload": f"{nevents} viscous 2+1D BSQ events, particle counts log-uniform in 5k-200k "
                    f"(total {ntot}), {ksteps} Heun steps each from tau0 = 0.6 fm, dtau = 0.005 fm, "
                    f"spacing 0.062 fm, h = 0.3 fm, shared 64x32^3 EoS table",
        "events_per_hr": 3600.0 * cap_eps,
        "particle_steps_per_s": ps / makespan,
        "fp64_one_at_a_time": {"events_per_hr": 3600.0 * nevents / T64, "particle_steps_per_s": ps / T64,
                               "seconds": T64, "per_event_e2e": "init (upload) + steps + read of T"},
        "events_per_hr_vs_fp64": T64 / makespan,
        "closed_loop": {"makespan_s": makespan, "wall_s": wall_closed, "p50_s": float(np.median(lat_closed)),
                        "p99_s": float(np.percentile(lat_closed, 99)),
                        "batch_steps": st1["batch_steps"] - st0["batch_steps"],
                        "device_s_of_batch_steps": 1e-3 * (st1["device_ms"] - st0["device_ms"]),
                        "device_particle_steps_per_s": ps / max(1e-9, 1e-3 * (st1["device_ms"] - st0["device_ms"])),
                        "kernel_launches": st1["kernel_launches"] - st0["kernel_launches"]},
        "open_loop": {"arrivals": f"Poisson, rate {load:.2f} x closed-loop capacity = {load * cap_eps:.2f} events/s",
                      "p50_s": float(np.median(lat_open)), "p99_s": float(np.percentile(lat_open, 99)),
                      "mean_s": float(lat_open.mean()), "wall_s": wall_open,
                      "batch_steps": st2["batch_steps"] - st1["batch_steps"]},
        "eos_work_per_particle_stage": {"table_evals": eos_per_pstage[0], "solves": eos_per_pstage[1],
                                        "closed_form_evals": eos_per_pstage[2]},
        "max_events": max_events, "tiled_block_threads": tuned,
        "latency": "submit (host arrays) to results readable in host memory",
        "precision": "mixed: FP32 neighbour sums (compensated), FP64 EoS/EoM/totals; no Newton polish",
    }


def bench_mixed_single(Bd, I, steps: int = 50):
    """The 40k-particle event in the mixed-precision forms: the per-event SPH_MIXED path (warp
    per particle neighbour passes) and the serving form holding this one event (cell-tiled
    passes, one CUDA graph per batch step); device or wall ms per step after warm-up."""
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
    g.free()
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
        if name == "fp64_freezeout":
            out[name]["e_fo"] = e_fo
            out[name]["elements"] = int(len(g.read_freezeout()[1]))
        g.free()
    out["mixed_speedup"] = out["fp64"]["ms_per_step"] / out["mixed"]["ms_per_step"]
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
        g.free()
    out["mixed_speedup"] = out["fp64"]["ms_per_step"] / out["mixed"]["ms_per_step"]
    return out


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle as O
    from paper_2511_22852_gb300 import inputs as I
    ev = I.viscous_bsq_2p1()
    run = O.OracleRun.start(ev)
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
            "config": {"workload": WORKLOAD, "particles": ev.n, "l2": "host run (no GPU)"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} Heun steps of the full {ev.n}-particle event"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


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
    # one independent event per rank (replicas): rank r uses hotspot/charge seeds shifted by r
    ev = replica_event(rank)
    stream = torch.cuda.Stream()
    g = Bd.GpuEvent(ev, use_graph=True, stream=stream.cuda_stream)
    for _ in range(args.warmup):
        g.step(1)
    torch.cuda.synchronize()
    # L2 (129 MB) flush between timed steps: a 256 MiB write, outside the timed events
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    t_before = g.totals()
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t_wall = time.perf_counter()
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                flush.fill_(float(k))
                e0[k].record(stream)
                g.step(1)
                e1[k].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    dev_ms = sum(a.elapsed_time(b) for a, b in zip(e0, e1))
    t_after = g.totals()
    # diagnostic only (not the reported value): the same steps without the L2 flush in between
    with torch.cuda.stream(stream):
        for k in range(min(args.steps, 50)):
            e0[k].record(stream)
            g.step(1)
            e1[k].record(stream)
    torch.cuda.synchronize()
    noflush_ms = sum(a.elapsed_time(b) for a, b in zip(e0[:min(args.steps, 50)], e1[:min(args.steps, 50)]))
    noflush_ms /= min(args.steps, 50)
    launches = t_after["kernel_launches"] - t_before["kernel_launches"]
    status_or = t_after["status_or"]
    clocks = clk.summary()

    dev_ms_max, units = combine_ranks(dev_ms, float(ev.n * args.steps), device="cuda")
    value = units / (dev_ms_max / 1e3)

    out = None
    if rank == 0:
        # --- per-kernel device times (profile mode: CUDA events around each kernel group,
        #     on the event's stream), same workload, for the roofline of the dominant kernel
        gp = Bd.GpuEvent(ev, use_graph=False, stream=stream.cuda_stream, profile=True)
        gp.step(2)
        gp_times0 = gp.kernel_times()
        tot0 = gp.totals()
        p0 = tot0["pairs"]
        kp = max(4, min(args.steps, 40))
        with torch.cuda.stream(stream):
            for k in range(kp):
                flush.fill_(float(k))
                gp.step(1)
        torch.cuda.synchronize()
        tot1 = gp.totals()
        p1 = tot1["pairs"]
        times = {k: (v[0] - gp_times0[k][0], v[1] - gp_times0[k][1]) for k, v in gp.kernel_times().items()}
        gp.free()
        pairs_incl_self = (p1 - p0)  # summed over both stages of kp steps
        dom = max(times, key=lambda k: times[k][0])
        ew = [b - a for a, b in zip(tot0["eos_work"], tot1["eos_work"])]
        flops = {"density": FLOPS_PER_PAIR["density"] * pairs_incl_self,
                 "gradient": FLOPS_PER_PAIR["gradient"] * (pairs_incl_self - 2 * kp * ev.n),
                 "eos": sum(f * w for f, w in zip(FLOPS_EOS, ew))}
        rooflines = {}
        for k in flops:
            ms = times[k][0]
            achieved = flops[k] / (ms / 1e3) / 1e9
            rooflines[k] = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                            "frac": achieved / FP64_PEAK_GFLOPS, "traffic": DRAM_BYTES_PER_LAUNCH.get(k),
                            "kernel": k,
                            "peak_source": "nominal FP64 vector rate of GB300 (1.25 TFLOP/s at 2070 MHz)",
                            "avg_launch_ms": ms / times[k][1], "flops_per_launch": flops[k] / times[k][1]}
        rooflines["eos"]["work_per_launch"] = {"table_evals": ew[0] / times["eos"][1], "solves": ew[1] / times["eos"][1],
                                               "closed_form_evals": ew[2] / times["eos"][1]}
        dgemm = fp64_dgemm_rate()
        for r in rooflines.values():
            r["frac_of_measured_dgemm"] = r["achieved"] / dgemm["gflops"]
        roof = rooflines.get(dom)
        total_ms = sum(v[0] for v in times.values())
        kernel_share = {k: round(v[0] / total_ms, 4) for k, v in times.items()}

        # --- end to end through the C ABI with host buffers: each step copies the state in
        #     from pinned host memory, steps, and reads the state back
        ge = Bd.GpuEvent(ev, use_graph=True, stream=stream.cuda_stream)
        st = ge.read(("X", "U", "S", "BV", "PV"))
        pinned = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory().numpy() for k, v in st.items()}
        ge.step(1)
        torch.cuda.synchronize()
        ke = max(3, min(args.steps, 30))
        bytes_state = sum(v.nbytes for v in pinned.values())
        t = time.perf_counter()
        for _ in range(ke):
            ge.write_state(x=pinned["X"], u=pinned["U"], S=pinned["S"], Bv=pinned["BV"], Pv=pinned["PV"])
            ge.step(1)
            o = ge.read(("X", "U", "S", "BV", "PV"))
        torch.cuda.synchronize()
        te = time.perf_counter() - t
        ge.free()
        e2e = {"value": ev.n * ke / te, "unit": UNIT, "h2d_bytes_per_step": bytes_state,
               "d2h_bytes_per_step": sum(v.nbytes for v in o.values()), "steps": ke}

        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": dev_ms_max / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
               "config": {"workload": WORKLOAD, "particles": ev.n, "l2": "flushed (256 MiB write) between timed steps",
                          "parallelism": f"replicas x{ws}", "cuda_graph": True},
               "roofline": roof, "kernel_share": kernel_share, "kernel_rooflines": rooflines,
               "fp64_dgemm_measured": dgemm,
               "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks,
               "wall_s_timed": t_wall, "status_or": int(status_or),
               "diagnostics": {"ms_per_step_without_l2_flush": noflush_ms,
                               "pair_list_overflow_stages_timed": int(t_after["pair_overflows"] - t_before["pair_overflows"]),
                               "profile_mode_group_ms_per_step": total_ms / kp}}
        if not args.no_serving:
            out["serving"] = serving_bench(Bd, I, args.serving_events, args.serving_steps)
        out["mixed_single_event"] = bench_mixed_single(Bd, I)
        out["freezeout"] = bench_freezeout(Bd, I)
        out["dnmr"] = bench_dnmr(Bd, I)
        out["partons"] = bench_partons(Bd, I)
        out["offline_eos"] = bench_offline_eos(Bd, I)
        if not args.no_3d:
            out["config_3p1d"] = bench_3p1d(Bd, I)
            out["config_stress"] = bench_stress(Bd, I)
        if not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(ev)
        print(json.dumps(out), flush=True)
    g.free()
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-3d", action="store_true")
    ap.add_argument("--serving-events", type=int, default=32)
    ap.add_argument("--serving-steps", type=int, default=60)
    ap.add_argument("--serving-only", action="store_true",
                    help="run only the serving comparison (profiling helper; prints its own JSON line)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.serving_only:
        from paper_2511_22852_gb300 import binding as Bd
        from paper_2511_22852_gb300 import build_lib
        from paper_2511_22852_gb300 import inputs as I
        build_lib.build()
        print(json.dumps({"serving": serving_bench(Bd, I, args.serving_events, args.serving_steps)}), flush=True)
        return 0
    return run_reference(args) if args.impl == "reference" else run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
