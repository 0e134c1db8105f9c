"""Host logic of the benchmark (CPU): the serving stream's recipe (event sizes and Poisson
arrivals), the rank-shifted replica streams, the DRAM-traffic record (scaling per particle,
staleness by source hash) and the mixed-vs-FP64 error measure."""
import hashlib
import json
import math

import numpy as np

import bench


def test_stream_sizes_are_log_uniform_in_range():
    sizes = bench.c4_sizes(512)
    assert len(sizes) == 512 and sizes.dtype.kind == "i"
    assert sizes.min() >= 5000 and sizes.max() < 200000
    # floor(exp(U(ln 5e3, ln 2e5))): log-sizes uniform, mean at the midpoint, spread (b - a)/sqrt(12)
    ls = np.log(sizes + 0.5)
    a, b = math.log(5e3), math.log(2e5)
    assert abs(ls.mean() - 0.5 * (a + b)) < 3.0 * (b - a) / math.sqrt(12.0 * 512)
    assert np.array_equal(sizes, bench.c4_sizes(512))  # seeded


def test_arrivals_are_poisson_at_the_stated_rate():
    t = bench.c4_arrivals(512)
    assert t[0] == 0.0 and np.all(np.diff(t) > 0.0)
    gaps = np.diff(t)
    # exponential gaps with mean 1/20 s: the sample mean within 4 standard errors, and the
    # coefficient of variation near 1 (an exponential's)
    assert abs(gaps.mean() - 1.0 / bench.C4_RATE) < 4.0 * (1.0 / bench.C4_RATE) / math.sqrt(len(gaps))
    assert 0.8 < gaps.std() / gaps.mean() < 1.2


def test_replica_streams_differ_by_rank():
    s0, a0, o0 = bench.replica_stream(0, 64)
    s1, a1, o1 = bench.replica_stream(1, 64)
    assert o0 == 0 and o1 == 100000
    assert not np.array_equal(s0, s1) and not np.array_equal(a0, a1)
    assert np.array_equal(s0, bench.c4_sizes(64))


def test_traffic_record_scales_per_particle_and_goes_stale(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2511_22852_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    src = b"__global__ void k(){}\n"
    (csrc / "k.cu").write_bytes(src)
    rec = {"k_x": {"sources": ["k.cu"], "source_sha16": hashlib.sha256(src).hexdigest()[:16], "particles": 1000,
                   "bytes_per_launch": 64000, "bytes_per_particle": 64.0, "capture": "profiles/x.md",
                   "counters": {"fp64_pipe_active_pct": 87.0}}}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    t = bench.traffic_of("k_x")
    assert t["bytes_per_launch"] == 64000.0 and "scaled" not in t
    assert t["counters"]["fp64_pipe_active_pct"] == 87.0
    t2 = bench.traffic_of("k_x", 2500.0)
    assert t2["bytes_per_launch"] == 160000.0 and "scaled" in t2
    assert bench.traffic_of("k_missing") is None
    (csrc / "k.cu").write_bytes(src + b"// changed\n")  # the kernel changed since the capture
    assert bench.traffic_of("k_x") is None


def test_mixed_vs_fp64_is_normwise():
    ref = {"T": np.array([1.0, 2.0, 4.0]), "MU": np.zeros((3, 3)), "S_DENS": np.array([10.0, 20.0, 40.0]),
           "N_DENS": np.array([[1.0, -2.0, 0.5]] * 3)}
    mixed = {k: v.copy() for k, v in ref.items()}
    mixed["T"][0] += 4e-7  # 1e-7 of max |T|
    mixed["S_DENS"][2] -= 8e-6  # 2e-7 of max |s|
    e = bench.mixed_vs_fp64(mixed, ref)
    assert abs(e["T"] - 1e-7) < 1e-12 and abs(e["S_DENS"] - 2e-7) < 1e-12 and e["N_DENS"] == 0.0
    assert "MU" not in e  # an all-zero reference has no norm
