#!/usr/bin/env python
"""KPM throughput benchmark on GB300: Chebyshev nnz*R*moments/s and % HBM roofline.

Workload (the 3D cubic configuration): L=64 periodic cubic lattice
(N = 262,144), complex hoppings t_ij = cos(th_i/2)cos(th_j/2) +
sin(th_i/2)sin(th_j/2)exp(-i(ph_i - ph_j)) from seeded random unit spins,
no on-site term, M = 1024 moments, R = 64 random-phase vectors, Jackson DOS
on K = 1024 Chebyshev nodes.  One step = one full solve through the C ABI:
random block, M/2 fused Chebyshev steps, moment reduction/doubling, Jackson
damping and DCT.  The headline is the FP32-vector / FP64-moment path; the
FP64 path on the same input is reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank solves its own realisation (independent random
blocks, no data-path collective: weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "Chebyshev nnz*R*moments/s"
UNIT = "nnz*R*moments/s"
WORKLOAD = dict(name="cubic_spin_L64", L=(64, 64, 64), R=64, M=1024, K=1024, seed=2,
                lanczos_steps=30, pad_eps=0.01)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


STEP_SOURCES = ["paper_1105_5481_gb300/csrc/kpm_step.cuh",
                "paper_1105_5481_gb300/csrc/kpm_step_dispatch.cuh",
                "paper_1105_5481_gb300/csrc/kpm_step_f32.cu",
                "paper_1105_5481_gb300/csrc/kpm_args.h"]
BATCH_SOURCES = STEP_SOURCES + ["paper_1105_5481_gb300/csrc/kpm_batch.cuh",
                                "paper_1105_5481_gb300/csrc/kpm_batch_res.cuh",
                                "paper_1105_5481_gb300/csrc/kpm_chunk16.cuh",
                                "paper_1105_5481_gb300/csrc/kpm_batch_dispatch.cuh",
                                "paper_1105_5481_gb300/csrc/kpm_batch_f32.cu"]
# DRAM bytes (read + write) per launch of the dominant kernel from one ncu capture,
# keyed by workload (and launch configuration), with the hash of the kernel sources
# it was taken on (profiles/cheb_step_fp32_cubic_spin_L64.md and
# profiles/cheb_step_fp32_csr_spin_dilute_L160.md: steady state of consecutive steps,
# caches not flushed between launches; profiles/batch_kernel_fp32_batch_2d_256.md);
# reported only while the hash matches.
MEASURED_TRAFFIC = {"cubic_spin_L64": (347.67e6, "step", "3b00c719cc0d365a"),
                    "csr_spin_dilute_L160": (3438.84e6, "step", "3b00c719cc0d365a"),
                    "batch_2d_256/C4/chunk4/clusters74/rt1/top0": (68.05e9, "batch", "721b534bb2268f1c"),
                    "batch_2d_256/C4/chunk2/clusters74/rt2/top8": (59.14e9, "batch", "721b534bb2268f1c")}


def accuracy_vs_fp64(K, mu32, mu64, a, b, n_nodes):
    """Error of an FP32-vector result against the FP64 path on the same inputs and random
    vectors (the FP64 path is parity-tested against the FP64 oracle): the largest moment
    difference and the L1 distance of the Jackson DOS, integral of |rho32 - rho64| dE by
    the Gauss-Chebyshev rule on the DOS nodes."""
    mu32, mu64 = np.asarray(mu32, dtype=np.float64), np.asarray(mu64, dtype=np.float64)
    _, r32 = K.kpm_dos(mu32, a, b, n_nodes)
    _, r64 = K.kpm_dos(mu64, a, b, n_nodes)
    x = np.cos(np.pi * (np.arange(n_nodes) + 0.5) / n_nodes)
    wq = np.pi / n_nodes * np.sqrt(1 - x * x)
    return {"max_abs_dmu": float(np.abs(mu32 - mu64).max()),
            "dos_l1": float(np.sum(np.abs(r32 - r64) * wq * a))}


def per_matvec(value):
    """The same throughput counted per matrix-vector product (two moments per
    product in the doubling form): nnz*R*(M/2)/t."""
    return {"value": value / 2, "unit": "nnz*R*matvecs/s"}


def step_source_hash(kind="step"):
    import hashlib

    h = hashlib.sha256()
    for f in (STEP_SOURCES if kind == "step" else BATCH_SOURCES):
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(key):
    t = MEASURED_TRAFFIC.get(key)
    return t[0] if t and t[2] == step_source_hash(t[1]) else None


# FP64 FMA issue rate of GB300: 152 SMs x 2 FP64 FMA per SM per clock x 2 flop at the
# sustained clock.  A dependent-chain probe measured 1.20 TFLOP/s (1.97 GHz).
FP64_PEAK_TFLOPS = 1.20


def algorithmic(nnz, N, R, M, fp32, dims=3):
    """Bytes and flops of one solve's fused steps (M/2 products).

    bytes/step = 3 N R s_v (read v_n, read v_{n-1}, write v_{n+1}) + N d s_hop
    flops/site/vector/step (complex) = 8 nnz/N + 4 + 8 (dots)."""
    s_v = 8 if fp32 else 16
    s_hop = s_v  # one complex hopping per forward bond, same precision as the vectors
    bytes_step = 3 * N * R * s_v + N * dims * s_hop
    flops_step = N * R * (8 * nnz / N + 4 + 8)
    return bytes_step, flops_step


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.proc = None
        self.dev = device_index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for k, n in enumerate(names):
                if f[4 + k].lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample(hop, L, R_s, M_s, seed):
    """The FP64 oracle as it stands on a bounded sample: R_s of the R vectors, M_s moments."""
    import oracle as O
    from paper_1105_5481_gb300 import inputs as I

    H = O.lattice_hamiltonian(L, hop=hop)
    N = H.n
    v0 = I.phase_block(seed, N, R_s)
    gmin, gmax = O.gershgorin(H)
    a, b = O.rescale(gmin, gmax, 0.01)
    t0 = time.perf_counter()
    mu, _ = O.moments_doubling(H, a, b, v0, M_s)
    O.dos(mu, a, b, 64)
    dt = time.perf_counter() - t0
    return H.nnz * R_s * M_s / dt, dt, H.nnz


def oracle_c_sample(hop, L, seed):
    """The oracle's doubling form restated in C (OpenMP over rows), on bounded samples
    of the same workload: all host threads with R=64, M=64, and one thread with R=8,
    M=32.  Returns (all-thread value, threads, one-thread value, seconds)."""
    import oracle as O
    from oracle import kpm_cpu as OC
    from paper_1105_5481_gb300 import inputs as I

    H = O.lattice_hamiltonian(L, hop=hop)
    a, b = O.rescale(*O.gershgorin(H), 0.01)
    nthreads = OC.max_threads()
    v0 = I.phase_block(seed, H.n, 64)
    OC.moments_doubling(H, a, b, v0[:, :8], 4, threads=nthreads)  # warm-up
    t0 = time.perf_counter()
    OC.moments_doubling(H, a, b, v0, 64, threads=nthreads)
    dt_all = time.perf_counter() - t0
    t0 = time.perf_counter()
    OC.moments_doubling(H, a, b, v0[:, :8], 32, threads=1)
    dt_one = time.perf_counter() - t0
    return (H.nnz * 64 * 64 / dt_all, nthreads, H.nnz * 8 * 32 / dt_one, dt_all + dt_one)


def reference_arm(args):
    """The oracle on the machine's host cores (its C restatement, OpenMP over all host
    threads), each step a bounded sample of the same workload: all 64 vectors,
    M=16 moments of the doubling form, plus the DOS on 64 nodes."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle as O
    from oracle import kpm_cpu as OC
    from paper_1105_5481_gb300 import inputs as I

    w = I.workload("cubic_spin_L64")
    R_s, M_s = 64, 16
    H = O.lattice_hamiltonian(w["L"], hop=w["hop"])
    a, b = O.rescale(*O.gershgorin(H), 0.01)
    v0 = I.phase_block(WORKLOAD["seed"], H.n, R_s)
    nthreads = OC.max_threads()

    def sample():
        t0 = time.perf_counter()
        mu, _ = OC.moments_doubling(H, a, b, v0, M_s, threads=nthreads)
        O.dos(mu, a, b, 64)
        return time.perf_counter() - t0

    for _ in range(args.warmup):
        sample()
    times = [sample() for _ in range(args.steps)]
    dt = float(np.median(times))
    value = H.nnz * R_s * M_s / dt
    desc = (f"3D L=64 spin lattice (N=262144, nnz={H.nnz}), all {R_s} random-phase vectors, "
            f"M={M_s} moments (the oracle's doubling form in C, FP64, OpenMP on {nthreads} host "
            f"threads) + DOS on 64 nodes, per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD["name"], "lattice": "3D cubic L=64 periodic, spin hoppings",
                   "R": 64, "M": 1024, "sample": "bounded oracle sample"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads,
                         "kind": "oracle (C, OpenMP)", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def csr_handle(K, w):
    rp, col, val = K.kpm_stencil_to_csr(3, w["L"], hop=w["hop"], bond_mask=w["mask"], complex_=True)
    return K.kpm_create_csr(rp.size - 1, rp, col, val, complex_=True)


def profile_run(prec, workload, batch_chunk=2, batch_cluster=4, batch_chunk_bytes=32,
                batch_rtiles=1, batch_top=0):
    """Two solves of the workload with Gershgorin bounds (no Lanczos products, so
    the only fused-step launches are those of the two solves); prec "bounds":
    three spectral-bound estimates of the headline lattice (Gershgorin and the
    30-step FP64 Lanczos), for captures of the bound kernels."""
    import torch

    from paper_1105_5481_gb300 import build as B
    from paper_1105_5481_gb300 import inputs as I
    from paper_1105_5481_gb300 import kpm as K

    B.build()
    if prec == "bounds":
        w = I.workload("cubic_spin_L64")
        h = K.kpm_create_stencil(3, w["L"], hop=w["hop"], complex_=True)
        t = []
        for _ in range(3):
            t0 = time.perf_counter()
            r = K.kpm_bounds(h, WORKLOAD["lanczos_steps"], WORKLOAD["pad_eps"], seed=6)
            t.append(1e3 * (time.perf_counter() - t0))
        h.close()
        print(json.dumps({"profile": "bounds", "ms_per_call": t, "emin": r[0], "emax": r[1]}))
        return 0
    if workload == "batch_2d_256":
        insts = I.batch_workload(3, 256)
        hs = [K.kpm_create_stencil(2, x["L"], onsite=x["onsite"]) for x in insts]
        ab = [K.kpm_bounds(h, 0, WORKLOAD["pad_eps"])[2:] for h in hs]
        with K.kpm_batch_create(hs, [x["M"] for x in insts], 16, [p[0] for p in ab],
                                [p[1] for p in ab], [x["seed"] for x in insts], prec) as bt:
            K.kpm_batch_set_chunk_bytes(bt, batch_chunk_bytes)
            K.kpm_batch_set_config(bt, batch_cluster, batch_chunk, 100)
            K.kpm_batch_set_rtiles(bt, batch_rtiles, batch_top)
            for _ in range(2):
                mu = K.kpm_batch_run(bt)
        print(json.dumps({"profile": prec, "workload": workload, "mu0": float(mu[0])}))
        return 0
    w = I.workload(workload)
    if workload == "csr_spin_dilute_L160":
        h = csr_handle(K, w)
        M, R = 64, w["R"]   # a short solve: the fused steps are identical at any M
    else:
        h = K.kpm_create_stencil(3, w["L"], hop=w["hop"], complex_=True)
        M, R = WORKLOAD["M"], WORKLOAD["R"]
    with h:
        _, _, a, b = K.kpm_bounds(h, 0, WORKLOAD["pad_eps"])
        for i in range(2):
            mu = K.kpm_moments(h, M, R, a, b, seed=1000 + i, precision=prec)
        torch.cuda.synchronize()
    print(json.dumps({"profile": prec, "workload": workload, "mu0": float(mu[0]), "mu2": float(mu[2])}))
    return 0


def square_leg(args):
    """The small FP64 configuration (2D L=32, R=8, M=256, Jackson DOS on 1024 nodes):
    latency-bound, reported as microseconds per solve with its L2-resident rate."""
    import torch

    from paper_1105_5481_gb300 import build as B
    from paper_1105_5481_gb300 import inputs as I
    from paper_1105_5481_gb300 import kpm as K

    B.build()
    w = I.workload("square_L32_fp64")
    N, R, M, Kn = int(np.prod(w["L"])), w["R"], w["M"], w["K"]
    h = K.kpm_create_stencil(2, w["L"], onsite=w["onsite"])
    nnz = K.kpm_info(h)["nnz"]
    emin, emax, a, b = K.kpm_bounds(h, WORKLOAD["lanczos_steps"], WORKLOAD["pad_eps"], seed=6)
    stream = torch.cuda.Stream()
    mu_d = torch.empty(M, dtype=torch.float64, device="cuda")
    E_d = torch.empty(Kn, dtype=torch.float64, device="cuda")
    rho_d = torch.empty(Kn, dtype=torch.float64, device="cuda")
    warm = max(args.warmup, 3)
    for i in range(warm):
        K.kpm_moments(h, M, R, a, b, seed=10 + i, precision="fp64", out=mu_d, stream=stream)
    stream.synchronize()
    steps = max(args.steps, 1) * 20  # 20 solves per step: one solve is well under a millisecond
    l0 = K.kpm_kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with Clocks(0) as clk:
        e0.record(stream)
        for i in range(steps):
            K.kpm_moments(h, M, R, a, b, seed=100 + i, precision="fp64", out=mu_d, stream=stream)
            K.kpm_dos(mu_d, a, b, Kn, "jackson", E=E_d, rho=rho_d, stream=stream)
        e1.record(stream)
        stream.synchronize()
    ms = e0.elapsed_time(e1) / steps
    launches = K.kpm_kernel_launches() - l0
    chain_ms, nsteps = K.kpm_step_timing(h)
    # the same solve as a batch of one: one persistent cluster launch, vectors in
    # global memory or resident in the cluster's shared memory
    batch_of_one = {}
    with K.kpm_batch_create([h], [M], R, [a], [b], [100], "fp64") as b1:
        for resident in (False, True):
            K.kpm_batch_set_resident(b1, resident)
            for C in (8, 16):
                K.kpm_batch_set_config(b1, C, 1, 100)
                for _ in range(3):
                    K.kpm_batch_run(b1, out=mu_d, stream=stream)
                e0.record(stream)
                for _ in range(steps):
                    K.kpm_batch_run(b1, out=mu_d, stream=stream)
                e1.record(stream)
                stream.synchronize()
                batch_of_one["%s_C%d_us" % ("resident" if resident else "global", C)] = (
                    e0.elapsed_time(e1) / steps * 1e3)
    bytes_step = 3 * N * R * 8 + N * 8  # vectors + on-site energies (uniform hopping)
    hbm, peak_kind = peaks()
    rate = bytes_step / (chain_ms / nsteps / 1e3) / 1e9
    value = nnz * R * M / (ms / 1e3)
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "per_matvec": per_matvec(value),
        "steps": steps, "warmup": warm, "ms_per_step": ms, "us_per_solve": ms * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "square_L32_fp64",
                   "lattice": "2D square L=32 periodic, t=1, on-site U[-0.5,0.5]",
                   "N": N, "nnz": nnz, "R": R, "M": M, "K": Kn, "step": "one solve + Jackson DOS",
                   "bounds": {"emin": emin, "emax": emax, "a": a, "b": b},
                   "l2": "working set (vectors 128 KB) L1/L2-resident"},
        "roofline": {"bound": "latency", "achieved": rate, "peak": hbm, "unit": "GB/s",
                     "frac": rate / hbm, "traffic": None, "bytes_per_launch": bytes_step,
                     "launch_ms": chain_ms / nsteps, "peak_kind": peak_kind,
                     "note": "127 dependent steps on 128 KB of vectors: each step is one "
                             "launch's latency; achieved = the L2-resident rate"},
        "batch_of_one_moments": batch_of_one,
        "gpu_launches": launches, "clocks": clk.summary()}))
    h.close()
    return 0


def csr_leg(args):
    """The large diluted CSR lattice: one solve per step (a JSON line of its own)."""
    import torch

    from paper_1105_5481_gb300 import build as B
    from paper_1105_5481_gb300 import inputs as I
    from paper_1105_5481_gb300 import kpm as K

    B.build()
    w = I.workload("csr_spin_dilute_L160")
    N, R, M = int(np.prod(w["L"])), w["R"], w["M"]
    h = csr_handle(K, w)
    nnz = K.kpm_info(h)["nnz"]
    emin, emax, a, b = K.kpm_bounds(h, WORKLOAD["lanczos_steps"], WORKLOAD["pad_eps"], seed=6)
    stream = torch.cuda.Stream()
    mu_d = torch.empty(M, dtype=torch.float64, device="cuda")
    E_d = torch.empty(w["K"], dtype=torch.float64, device="cuda")
    rho_d = torch.empty(w["K"], dtype=torch.float64, device="cuda")
    mu_chk = K.kpm_moments(h, M, R, a, b, seed=1, precision="fp32", stream=stream)
    assert abs(mu_chk[0] - 1.0) < 1e-5 and np.all(np.abs(mu_chk) <= 1 + 1e-5)
    steps = min(args.steps, 3)
    for i in range(min(args.warmup, 3)):
        K.kpm_moments(h, M, R, a, b, seed=10 + i, precision="fp32", out=mu_d, stream=stream)
    stream.synchronize()
    l0 = K.kpm_kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with Clocks(0) as clk:
        e0.record(stream)
        for i in range(steps):
            K.kpm_moments(h, M, R, a, b, seed=100 + i, precision="fp32", out=mu_d, stream=stream)
            K.kpm_dos(mu_d, a, b, w["K"], "jackson", E=E_d, rho=rho_d, stream=stream)
        e1.record(stream)
        stream.synchronize()
    ms = e0.elapsed_time(e1) / steps
    launches = K.kpm_kernel_launches() - l0
    chain_ms, nsteps = K.kpm_step_timing(h)
    # accuracy against the FP64 path on the first 512 moments (a prefix of the same
    # recursion: an FP64 solve of all 4096 would take ~12 s)
    m_pref = 512
    mu64 = K.kpm_moments(h, m_pref, R, a, b, seed=1, precision="fp64", stream=stream)
    accuracy = accuracy_vs_fp64(K, mu_chk[:m_pref], mu64, a, b, w["K"])
    accuracy["moments_compared"] = m_pref
    bytes_step = 3 * N * R * 8 + nnz * (8 + 4) + 8 * (N + 1)
    hbm, peak_kind = peaks()
    ach = bytes_step / (chain_ms / nsteps / 1e3) / 1e9
    print(json.dumps({
        "metric": METRIC, "value": nnz * R * M / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
        "per_matvec": per_matvec(nnz * R * M / (ms / 1e3)),
        "steps": steps, "warmup": min(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 vectors, f64 moments",
        "data": "synthetic",
        "config": {"workload": "csr_spin_dilute_L160",
                   "lattice": "3D cubic L=160 periodic, spin hoppings, 10% bond dilution, CSR",
                   "N": N, "nnz": nnz, "R": R, "M": M, "K": w["K"],
                   "bounds": {"emin": emin, "emax": emax, "a": a, "b": b},
                   "l2": "inputs larger than L2"},
        "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                     "traffic": measured_traffic("csr_spin_dilute_L160"), "bytes_per_launch": bytes_step,
                     "launch_ms": chain_ms / nsteps, "peak_kind": peak_kind},
        "accuracy_vs_fp64": accuracy,
        "gpu_launches": launches, "clocks": clk.summary()}))
    h.close()
    return 0


def dense_leg(args):
    """The paper's dense formulation at its largest matrix (Sec. IV-C: H_SIZE =
    4096, N = 128 moments, R x S = 1792 vectors), FP64 as in the paper: a real
    Wigner matrix, all 1792 vectors in one block, one solve per step."""
    import torch

    from paper_1105_5481_gb300 import build as B
    from paper_1105_5481_gb300 import inputs as I
    from paper_1105_5481_gb300 import kpm as K

    B.build()
    w = I.workload(args.workload)
    A, D, R, M, Kn = w["H"], w["D"], w["R"], w["M"], w["K"]
    h = K.kpm_create_dense(A)
    nnz = K.kpm_info(h)["nnz"]
    emin, emax, a, b = K.kpm_bounds(h, WORKLOAD["lanczos_steps"], WORKLOAD["pad_eps"], seed=6)
    stream = torch.cuda.Stream()
    mu_d = torch.empty(M, dtype=torch.float64, device="cuda")
    E_d = torch.empty(Kn, dtype=torch.float64, device="cuda")
    rho_d = torch.empty(Kn, dtype=torch.float64, device="cuda")
    mu_chk = K.kpm_moments(h, M, R, a, b, seed=1, stream=stream)
    assert abs(mu_chk[0] - 1.0) < 1e-12 and np.all(np.abs(mu_chk) <= 1 + 1e-9)
    steps = max(1, min(args.steps, 3))
    warm = 3
    for i in range(warm):
        K.kpm_moments(h, M, R, a, b, seed=10 + i, out=mu_d, stream=stream)
    stream.synchronize()
    l0 = K.kpm_kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with Clocks(0) as clk:
        e0.record(stream)
        for i in range(steps):
            K.kpm_moments(h, M, R, a, b, seed=100 + i, out=mu_d, stream=stream)
            K.kpm_dos(mu_d, a, b, Kn, "jackson", E=E_d, rho=rho_d, stream=stream)
        e1.record(stream)
        stream.synchronize()
    ms = e0.elapsed_time(e1) / steps
    launches = K.kpm_kernel_launches() - l0
    chain_ms, nsteps = K.kpm_step_timing(h)
    h.close()
    # the contraction dominates: 2 D^2 FP64 FMA-flops per vector and product
    flops_step = 2.0 * D * D * R
    ach = flops_step / (chain_ms / nsteps / 1e3) / 1e12
    value = nnz * R * M / (ms / 1e3)

    # end to end through the public API: pinned host matrix -> handle -> bounds ->
    # moments -> DOS -> host results
    A_pin = torch.from_numpy(A).pin_memory().numpy()

    def e2e_once(i):
        with K.kpm_create_dense(A_pin) as he:
            _, _, ae, be = K.kpm_bounds(he, WORKLOAD["lanczos_steps"], WORKLOAD["pad_eps"], seed=6)
            mu = K.kpm_moments(he, M, R, ae, be, seed=200 + i, stream=stream)
            K.kpm_dos(mu, ae, be, Kn, stream=stream)

    e2e_once(0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(2):
        e2e_once(i + 1)
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / 2

    cpu = None
    if not args.no_cpu_baseline:
        import oracle as O
        from oracle import kpm_cpu as OC

        H = O.from_dense(A)
        R_s, M_s = 448, 64
        v0 = I.rademacher_block(1, D, R_s)
        nthreads = OC.max_threads()
        t0 = time.perf_counter()
        OC.moments_doubling(H, a, b, v0, M_s, threads=nthreads)
        dt = time.perf_counter() - t0
        cpu = {"value": nnz * R_s * M_s / dt, "unit": UNIT, "cores": nthreads,
               "kind": "oracle (C, OpenMP)",
               "sample": f"the oracle's doubling form in C over all {D * D} stored elements, "
                         f"{R_s} of the {R} vectors, M={M_s} ({dt:.1f} s)"}
    print(json.dumps({
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "per_matvec": per_matvec(value),
        "steps": steps, "warmup": warm, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload,
                   "matrix": f"dense real Wigner matrix D={D} (entries U[-1,1)/sqrt(D)), every "
                             "element stored and used (the paper's formulation)",
                   "N": D, "nnz": nnz, "R": R, "M": M, "K": Kn,
                   "bounds": {"emin": emin, "emax": emax, "a": a, "b": b},
                   "step": "random block + M/2 dense products + moment reduction + Jackson DOS",
                   "l2": "matrix (134 MB) larger than L2"},
        "roofline": {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": ach / FP64_PEAK_TFLOPS, "traffic": None,
                     "kernel": "dense_step_kernel<real, STEP, 64-row tiles>",
                     "flops_per_launch": flops_step, "launch_ms": chain_ms / nsteps,
                     "peak_kind": "FP64 pipe, 2 FMA per SM and clock at 1.97 GHz (measured)"},
        "cpu_baseline": cpu,
        "e2e": {"value": nnz * R * M / (e2e_ms / 1e3), "unit": UNIT, "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": int(A.nbytes), "d2h_bytes_per_step": int(8 * (M + 2 * Kn)),
                "includes": "create from a pinned host matrix, bounds, moments, DOS, destroy"},
        "gpu_launches": launches, "clocks": clk.summary()}))
    return 0


def batch_leg(args):
    """256 independent 2D disorder realisations of uneven size, R=16 FP32 real
    vectors, one persistent cluster launch per batch (graph replay, autotuned),
    against the same solves issued as plain per-instance kpm_moments calls."""
    import torch

    from paper_1105_5481_gb300 import build as B
    from paper_1105_5481_gb300 import inputs as I
    from paper_1105_5481_gb300 import kpm as K

    B.build()
    insts = I.batch_workload(3, 256)
    R = 16
    hs = [K.kpm_create_stencil(2, x["L"], onsite=x["onsite"]) for x in insts]
    ab = [K.kpm_bounds(h, 0, WORKLOAD["pad_eps"])[2:] for h in hs]
    Ms = [x["M"] for x in insts]
    seeds = [x["seed"] for x in insts]
    bt = K.kpm_batch_create(hs, Ms, R, [p[0] for p in ab], [p[1] for p in ab], seeds, "fp32")
    t0 = time.perf_counter()
    info = K.kpm_batch_tune(bt, reps=1)
    info["rtiles"], info["tiled_instances"], _ = K.kpm_batch_get_rtiles(bt)
    info["resident"] = K.kpm_batch_get_resident(bt)[0]
    info["chunk_bytes"], info["threads_per_row"] = K.kpm_batch_get_chunk_bytes(bt)
    tune_s = time.perf_counter() - t0
    mu_host = K.kpm_batch_run(bt)  # host output: divergence check
    assert np.all(np.abs(mu_host) <= 1 + 1e-5)
    stream = torch.cuda.Stream()
    out = torch.empty(int(sum(Ms)), dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        K.kpm_batch_run(bt, out=out, stream=stream)
    stream.synchronize()
    l0 = K.kpm_kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with Clocks(0) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            K.kpm_batch_run(bt, out=out, stream=stream)
        e1.record(stream)
        stream.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    launches = K.kpm_kernel_launches() - l0
    Ns = [x["L"][0] * x["L"][1] for x in insts]
    nnz = [5 * n for n in Ns]                 # 4 bonds + on-site per row
    units = sum(z * R * m for z, m in zip(nnz, Ms))
    byts = sum((m // 2) * (3 * n * R * 4 + n * 4) for n, m in zip(Ns, Ms))
    # the same solves as plain per-instance calls (one graph per instance, sequential)
    mu1 = torch.empty(max(Ms), dtype=torch.float64, device="cuda")
    for h, m, p, sd in zip(hs[:4], Ms, ab, seeds):
        K.kpm_moments(h, m, R, p[0], p[1], seed=sd, precision="fp32", out=mu1[:m], stream=stream)
    stream.synchronize()
    e0.record(stream)
    for h, m, p, sd in zip(hs, Ms, ab, seeds):
        K.kpm_moments(h, m, R, p[0], p[1], seed=sd, precision="fp32", out=mu1[:m], stream=stream)
    e1.record(stream)
    stream.synchronize()
    ms_single = e0.elapsed_time(e1)
    # accuracy: every 32nd instance against its FP64 solve on the same random vectors
    acc_b = []
    for k, (mu_i, h_i, m_i, p_i, sd) in enumerate(zip(bt.split(mu_host), hs, Ms, ab, seeds)):
        if k % 32 == 0:
            mu64 = K.kpm_moments(h_i, m_i, R, p_i[0], p_i[1], seed=sd, precision="fp64")
            acc_b.append(accuracy_vs_fp64(K, mu_i, mu64, p_i[0], p_i[1], 1024))
    accuracy = {"max_abs_dmu": max(x["max_abs_dmu"] for x in acc_b),
                "dos_l1": max(x["dos_l1"] for x in acc_b), "instances_compared": len(acc_b)}
    # the resident form (each instance's vectors in its cluster's shared memory)
    # at the smallest cluster size where the largest instance fits
    resident = None
    K.kpm_batch_set_resident(bt, True)
    cmin = K.kpm_batch_get_resident(bt)[1]
    if cmin:
        K.kpm_batch_set_config(bt, cmin, info["chunk"], 100)
        K.kpm_batch_run(bt, out=out, stream=stream)
        stream.synchronize()
        e0.record(stream)
        for _ in range(2):
            K.kpm_batch_run(bt, out=out, stream=stream)
        e1.record(stream)
        stream.synchronize()
        resident = {"cluster": cmin, "clusters": K.kpm_batch_info(bt)["clusters"],
                    "ms": e0.elapsed_time(e1) / 2}
    hbm, peak_kind = peaks()
    ach = byts / (ms / 1e3) / 1e9
    print(json.dumps({
        "metric": METRIC, "value": units / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 vectors, f64 moments",
        "data": "synthetic",
        "config": {"workload": "batch_2d_256",
                   "instances": "256 x 2D periodic L~U{16..128}, W~U[0,4), M even ~U{128..2048}, R=16",
                   "sites_total": sum(Ns), "moments_total": sum(Ms),
                   "bounds": "Gershgorin per instance, pad 0.01",
                   "launch": "one persistent cluster kernel per batch, CUDA graph replay",
                   "autotuned": info, "tune_s": tune_s, "l2": "instances' vectors mostly L2-resident"},
        "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
                     "traffic": measured_traffic("batch_2d_256/C%d/chunk%d/clusters%d/rt%d/top%d%s" % (
                         info["cluster"], info["chunk"], info["clusters"], info["rtiles"],
                         info["tiled_instances"], ("/resident" if info["resident"] else "") +
                         ("/chunk16B" if info["chunk_bytes"] == 16 else ""))),
                     "bytes_per_launch": byts, "peak_kind": peak_kind,
                     "note": "algorithmic bytes of all instances per batch launch; the working "
                             "set of the active instances is L2-resident, so frac can exceed 1"},
        "per_instance_calls": {"ms": ms_single, "speedup_of_batch": ms_single / ms},
        "resident_form": resident,
        "accuracy_vs_fp64": accuracy,
        "solves_per_s": 256 / (ms / 1e3),
        "per_matvec": per_matvec(units / (ms / 1e3)),
        "gpu_launches": launches, "clocks": clk.summary()}))
    bt.close()
    for h in hs:
        h.close()
    return 0


def serve_leg(args, count=48, rate_hz=40.0, K_nodes=1024):
    """Poisson stream of DOS requests (2D/3D, N log-uniform in [1e3, 4e6], M in
    256..8192, R in {8,16,32,64}, real or complex spin hoppings) through the
    serving loop with FP32 vectors, against the same arrivals served as plain
    per-request FP64 calls (first come first served), with each served result's
    error against its FP64 counterpart."""
    import threading

    from paper_1105_5481_gb300 import build as B
    from paper_1105_5481_gb300 import inputs as I
    from paper_1105_5481_gb300 import kpm as K

    B.build()
    reqs = I.serving_stream(5, count, rate_hz)
    hs, ab = [], []
    for r in reqs:
        N = int(np.prod(r["L"]))
        th, ph = I.spins(r["spin_seed"], N)
        if not r["complex"]:
            ph = np.zeros(N)
        hop = I.spin_hoppings(r["L"], th, ph)
        h = K.kpm_create_stencil(r["dims"], r["L"], hop=hop if r["complex"] else hop.real,
                                 complex_=r["complex"])
        hs.append(h)
        ab.append(K.kpm_bounds(h, 0, WORKLOAD["pad_eps"])[2:])

    def run_served(prec):
        srv = K.kpm_server_create(48 << 30, steps_per_tick=32, cluster=4)
        ids = [None] * len(reqs)
        t0 = time.perf_counter()

        def feed():
            for k, r in enumerate(reqs):
                dt = t0 + r["t"] - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                ids[k] = K.kpm_server_submit(srv, hs[k], r["M"], r["R"], ab[k][0], ab[k][1],
                                             seed=r["seed"], precision=prec, K=K_nodes)

        th = threading.Thread(target=feed)
        th.start()
        th.join()
        res = []
        for rid in ids:
            K.kpm_server_wait(srv, rid, 600.0)
            res.append(K.kpm_server_poll(srv, rid))
        wall = time.perf_counter() - t0
        st = K.kpm_server_stats(srv)
        srv.close()
        return res, st, wall

    l0 = K.kpm_kernel_launches()
    with Clocks(0) as clk:
        served, st, wall = run_served("fp32")
    launches = K.kpm_kernel_launches() - l0
    # plain per-request FP64 calls, first come first served, on arrival
    t0 = time.perf_counter()
    lat64, res64 = [], []
    for k, r in enumerate(reqs):
        dt = t0 + r["t"] - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        mu = K.kpm_moments(hs[k], r["M"], r["R"], ab[k][0], ab[k][1], seed=r["seed"], precision="fp64")
        E, rho = K.kpm_dos(mu, ab[k][0], ab[k][1], K_nodes)
        res64.append((mu, rho))
        lat64.append(time.perf_counter() - (t0 + r["t"]))
    wall64 = time.perf_counter() - t0
    err_mu = max(float(np.abs(a_[0] - b_[0]).max()) for a_, b_ in zip(served, res64))
    x = np.cos(np.pi * (np.arange(K_nodes) + 0.5) / K_nodes)
    w = np.pi / K_nodes * np.sqrt(1 - x * x)
    err_dos = max(float(np.sum(np.abs(a_[2] - b_[1]) * w * ab[k][0]))
                  for k, (a_, b_) in enumerate(zip(served, res64)))
    units = sum(int(np.prod(r["L"])) * (2 * r["dims"]) * r["R"] * r["M"] for r in reqs)
    print(json.dumps({
        "metric": "served DOS solves/s, p50/p99", "value": st["completed"] / wall, "unit": "solves/s",
        "n_gpus": 1, "steps": count, "warmup": 0, "ms_per_step": 1e3 * wall / count,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 vectors, f64 moments", "data": "synthetic",
        "config": {"workload": "serve_poisson", "requests": count, "arrival_rate_hz": rate_hz,
                   "mix": "2D/3D cubic, N log-uniform [1e3, 4e6], M even log-uniform [256, 8192], "
                          "R in {8,16,32,64}, real or complex spin hoppings, K=1024 Jackson DOS",
                   "server": "48 GiB arena, 32 products per tick, clusters of 4, large requests "
                             "(>= 8 MB per product) as full-GPU steps on 4 streams",
                   "bounds": "Gershgorin per request, pad 0.01"},
        "latency_s": {"p50": st["p50_s"], "p99": st["p99_s"], "mean": st["mean_s"], "max": st["max_s"]},
        "throughput": {"solves_per_s": st["completed"] / wall, "nnz_R_moments_per_s": units / wall,
                       "nnz_R_matvecs_per_s": units / wall / 2},
        "server": {k: st[k] for k in ("completed", "failed", "ticks", "peak_resident", "peak_bytes")},
        "per_request_fp64": {"solves_per_s": count / wall64, "p50_s": float(np.percentile(lat64, 50)),
                             "p99_s": float(np.percentile(lat64, 99)), "wall_s": wall64},
        "accuracy_vs_fp64": {"max_abs_dmu": err_mu, "max_dos_l1": err_dos},
        "gpu_launches": launches, "clocks": clk.summary()}))
    for h in hs:
        h.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-chunk", type=int, default=2,
                    help="--profile with the batch workload: passes per chunk")
    ap.add_argument("--batch-cluster", type=int, default=4,
                    help="--profile with the batch workload: CTAs per cluster")
    ap.add_argument("--batch-chunk-bytes", type=int, default=32, choices=[16, 32],
                    help="--profile with the batch workload: bytes of a row per thread")
    ap.add_argument("--batch-rtiles", type=int, default=1,
                    help="--profile with the batch workload: column tiles of the largest instances")
    ap.add_argument("--batch-top", type=int, default=0,
                    help="--profile with the batch workload: instances tiled (0: all)")
    ap.add_argument("--workload", default="cubic_spin_L64",
                    choices=["cubic_spin_L64", "csr_spin_dilute_L160", "batch_2d_256",
                             "serve_poisson", "square_L32_fp64", "dense_wigner_D4096"],
                    help="cubic_spin_L64 (default, the headline) or the large diluted CSR "
                         "lattice (L=160, N=4.1M, R=32, M=4096, FP32 vectors)")
    ap.add_argument("--profile", default=None, choices=["fp32", "fp64", "bounds"],
                    help="run two solves of the workload at the given precision and exit "
                         "(a short command for ncu captures of the fused step)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    if args.profile:
        return profile_run(args.profile, args.workload, args.batch_chunk, args.batch_cluster,
                           args.batch_chunk_bytes, args.batch_rtiles, args.batch_top)
    if args.workload == "square_L32_fp64":
        return square_leg(args)
    if args.workload == "csr_spin_dilute_L160":
        return csr_leg(args)
    if args.workload == "batch_2d_256":
        return batch_leg(args)
    if args.workload.startswith("dense_wigner_D"):
        return dense_leg(args)
    if args.workload == "serve_poisson":
        return serve_leg(args)

    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    from paper_1105_5481_gb300 import build as B
    from paper_1105_5481_gb300 import inputs as I
    from paper_1105_5481_gb300 import kpm as K

    B.build()
    w = I.workload("cubic_spin_L64")
    L, R, M, Kn = w["L"], WORKLOAD["R"], WORKLOAD["M"], WORKLOAD["K"]
    N = int(np.prod(L))
    hop = np.ascontiguousarray(w["hop"])
    h = K.kpm_create_stencil(3, L, hop=hop, complex_=True)
    info = K.kpm_info(h)
    nnz = info["nnz"]
    emin, emax, a, b = K.kpm_bounds(h, WORKLOAD["lanczos_steps"], WORKLOAD["pad_eps"], seed=6)
    stream = torch.cuda.Stream()
    mu_d = torch.empty(M, dtype=torch.float64, device="cuda")
    E_d = torch.empty(Kn, dtype=torch.float64, device="cuda")
    rho_d = torch.empty(Kn, dtype=torch.float64, device="cuda")
    seed0 = 1000 + 7919 * rank

    def solve(i, prec):
        K.kpm_moments(h, M, R, a, b, seed=seed0 + i, precision=prec, out=mu_d, stream=stream)
        K.kpm_dos(mu_d, a, b, Kn, "jackson", E=E_d, rho=rho_d, stream=stream)

    # sanity: a host-output solve must not diverge and must keep mu_0 = 1
    mu_chk = K.kpm_moments(h, M, R, a, b, seed=seed0, precision="fp32", stream=stream)
    assert abs(mu_chk[0] - 1.0) < 1e-5 and np.all(np.abs(mu_chk) <= 1 + 1e-5)

    def timed(prec, steps, warmup):
        for i in range(warmup):
            solve(i, prec)
        stream.synchronize()
        barrier()
        torch.cuda.synchronize()
        l0 = K.kpm_kernel_launches()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        with Clocks(local) as clk:
            e0.record(stream)
            for i in range(steps):
                solve(warmup + i, prec)
            e1.record(stream)
            stream.synchronize()
        torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1) / steps
        launches = K.kpm_kernel_launches() - l0
        chain_ms, nsteps = K.kpm_step_timing(h)
        if dist is not None:
            t = torch.tensor([ms], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms, launches, chain_ms / nsteps, clk.summary()

    ms32, launches32, step_ms32, clk32 = timed("fp32", args.steps, args.warmup)
    ms64, launches64, step_ms64, clk64 = timed("fp64", args.fp64_steps, min(args.warmup, 3))
    # the FP32-vector result against the FP64 path on the same random vectors
    mu64_chk = K.kpm_moments(h, M, R, a, b, seed=seed0, precision="fp64", stream=stream)
    accuracy = accuracy_vs_fp64(K, mu_chk, mu64_chk, a, b, Kn)

    combined = None
    if dist is not None:
        # replicas ran disjoint random vectors (seed per rank): the job's moments
        # are the vector-weighted mean over ranks (one all-reduce of M+1 doubles)
        from paper_1105_5481_gb300.replicas import combine_moments

        mu_last = K.kpm_moments(h, M, R, a, b, seed=seed0, precision="fp32", stream=stream)
        combined = combine_moments(mu_last, R)
    units = nnz * R * M  # per solve
    value = world * units / (ms32 / 1e3)
    bytes32, flops = algorithmic(nnz, N, R, M, True)
    bytes64, _ = algorithmic(nnz, N, R, M, False)
    hbm, peak_kind = peaks()
    ach32 = bytes32 / (step_ms32 / 1e3) / 1e9
    ach64_tf = flops / (step_ms64 / 1e3) / 1e12

    # end to end through the public API: host inputs (pinned) -> handle -> bounds ->
    # moments -> DOS -> host results, every step
    hop_pin = torch.from_numpy(hop.view(np.float64)).pin_memory().numpy()
    e2e_steps = max(2, min(args.steps, 5))

    def e2e_once(i):
        with K.kpm_create_stencil(3, L, hop=hop_pin.view(np.complex128), complex_=True) as he:
            _, _, ae, be = K.kpm_bounds(he, WORKLOAD["lanczos_steps"], WORKLOAD["pad_eps"], seed=6)
            mu = K.kpm_moments(he, M, R, ae, be, seed=seed0 + i, precision="fp32", stream=stream)
            E, rho = K.kpm_dos(mu, ae, be, Kn, stream=stream)
        return mu, E, rho

    e2e_once(0)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        e2e_once(i + 1)
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps
    if dist is not None:
        t = torch.tensor([e2e_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())

    cpu = cpu_c = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, dt, _ = oracle_sample(w["hop"], L, 8, 32, WORKLOAD["seed"])
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"FP64 NumPy oracle, same lattice, 8 of the 64 vectors, M=32 moments "
                         f"+ DOS ({dt:.1f} s)"}
        v_all, nthr, v_one, dtc = oracle_c_sample(w["hop"], L, WORKLOAD["seed"])
        cpu_c = {"value": v_all, "unit": UNIT, "cores": nthr, "kind": "oracle (C, OpenMP)",
                 "sample": f"the oracle's doubling form in C, FP64 CSR, same lattice: all "
                           f"{nthr} host threads with R=64, M=64; one thread with R=8, M=32 "
                           f"({dtc:.1f} s)",
                 "one_core": {"value": v_one, "cores": 1}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms32, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 vectors, f64 moments", "data": "synthetic",
            "config": {"workload": WORKLOAD["name"],
                       "lattice": "3D cubic L=64 periodic (N=262144), spin-derived complex hoppings",
                       "N": N, "nnz": nnz, "R": R, "M": M, "K": Kn, "S_per_rank": 1,
                       "bounds": {"emin": emin, "emax": emax, "a": a, "b": b,
                                  "method": "Gershgorin + 30-step Lanczos, pad 0.01"},
                       "step": "random block + M/2 fused steps + moment reduction + Jackson DOS",
                       "l2": "inputs larger than L2 (two 134 MB vector blocks)",
                       "parallelism": f"replicas x{world}",
                       "replicas_combined": combined is not None},
            "roofline": {"bound": "hbm", "achieved": ach32, "peak": hbm, "unit": "GB/s",
                         "frac": ach32 / hbm, "traffic": measured_traffic(WORKLOAD["name"]),
                         "kernel": "cheb_step_kernel<float, complex, STEP, StencilOp<3,hop>>",
                         "bytes_per_launch": bytes32, "launch_ms": step_ms32,
                         "peak_kind": f"{peak_kind} (copy bandwidth)"},
            "per_matvec": per_matvec(value),
            "accuracy_vs_fp64": accuracy,
            "fp64_path": {"value": world * units / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64,
                          "per_matvec": per_matvec(world * units / (ms64 / 1e3)),
                          "steps": args.fp64_steps, "dtype": "f64",
                          "roofline": {"bound": "alu", "achieved": ach64_tf, "peak": FP64_PEAK_TFLOPS,
                                       "unit": "TFLOP/s", "frac": ach64_tf / FP64_PEAK_TFLOPS,
                                       "hbm_frac": bytes64 / (step_ms64 / 1e3) / 1e9 / hbm,
                                       "launch_ms": step_ms64},
                          "clocks": clk64, "gpu_launches": launches64},
            "cpu_baseline": cpu,
            "cpu_baseline_c": cpu_c,
            "e2e": {"value": world * units / (e2e_ms / 1e3), "unit": UNIT, "ms_per_step": e2e_ms,
                    "h2d_bytes_per_step": int(hop.nbytes),
                    "d2h_bytes_per_step": int(8 * (M + 2 * Kn)),
                    "includes": "create from pinned host arrays, bounds, moments, DOS, destroy"},
            "gpu_launches": launches32,
            "clocks": clk32,
        }
        print(json.dumps(line))
    h.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
