#!/usr/bin/env python
"""KPM throughput benchmark on GB300: Chebyshev nnz*R*moments/s, % HBM roofline,
and served DOS solves/s with p50/p99 latency.

Headline workload (the largest single-GPU configuration): a 3D cubic lattice
L = 160 (N = 4,096,000), periodic, complex hoppings t_ij = cos(th_i/2)cos(th_j/2)
+ sin(th_i/2)sin(th_j/2)exp(-i(ph_i - ph_j)) from seeded random unit spins, 10 %
seeded bond dilution, handed to the library as CSR (nnz = 22,117,096), M = 4096
moments, R = 32 random-phase vectors stored in FP32 with FP64 moment sums,
Jackson DOS on K = 4096 nodes.  One step = one full solve through the C ABI:
random block, M/2 fused Chebyshev steps, moment reduction and doubling, Jackson
damping and DCT, with all inputs resident in device memory.

The same JSON line carries the other configurations as extra keys (measured in
the same run, after the headline's timed region): the 3D L = 64 spin lattice
in both precisions, the small 2D L = 32 FP64 solve, the batch of 256 uneven 2D
instances in one persistent launch, and the Poisson serving stream swept over
arrival rates, against plain per-request FP64 calls.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--no-extras] [--no-cpu-baseline]

With --gpus N > 1 (outside torchrun) the script relaunches itself under
torch.distributed.run with N processes.  Every rank then solves its own
realisation of the headline's random vectors (kpm_params.s0 = rank, no
data-path collective: weak scaling), the moments are combined by one
all-reduce of M + 1 doubles, and rank 0 prints one JSON line.
--workload runs a single configuration and prints its own line.
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
HEADLINE = "csr_spin_dilute_L160"
LANCZOS_STEPS, PAD_EPS = 30, 0.01


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
TMA_SOURCES = STEP_SOURCES + ["paper_1105_5481_gb300/csrc/kpm_step_tma.cu"]
BATCH_SOURCES = STEP_SOURCES + ["paper_1105_5481_gb300/csrc/kpm_batch.cuh",
                                "paper_1105_5481_gb300/csrc/kpm_batch_res.cuh",
                                "paper_1105_5481_gb300/csrc/kpm_chunk16.cuh",
                                "paper_1105_5481_gb300/csrc/kpm_batch_dispatch.cuh",
                                "paper_1105_5481_gb300/csrc/kpm_batch_f32.cu",
                                "paper_1105_5481_gb300/csrc/kpm_batch_stg.cuh",
                                "paper_1105_5481_gb300/csrc/kpm_batch_stg_f32.cu",
                                "paper_1105_5481_gb300/csrc/kpm_mbar.cuh",
                                "paper_1105_5481_gb300/csrc/kpm_fastdiv.cuh"]
# DRAM bytes (read + write) per launch of the dominant kernel from one ncu
# capture (steady state of consecutive launches, caches not flushed between
# them), keyed by workload and launch configuration, with the hash of the
# kernel sources it was taken on; reported only while the hash matches.
MEASURED_TRAFFIC = {"cubic_spin_L64": (347.93e6, "step", "9d89b353287cea2a"),
                    "csr_spin_dilute_L160": (3394.59e6, "tma", "2ff2a33ede954230"),
                    "batch_2d_256/C4/chunk2/clusters74/rt1/top0": (69.20e9, "batch", "f1a1fabd8beeef38"),
                    "batch_2d_256/C4/chunk4/clusters74/rt1/top0": (68.25e9, "batch", "f1a1fabd8beeef38"),
                    "batch_2d_256/C4/chunk2/clusters74/rt2/top8": (61.17e9, "batch", "f1a1fabd8beeef38"),
                    "batch_2d_256/C4/chunk4/clusters74/rt1/top0/staged": (71.20e9, "batch", "f1a1fabd8beeef38")}

# FP64 FMA issue rate of GB300: 152 SMs x 2 FP64 FMA per SM per clock x 2 flop at the
# sustained clock.  A dependent-chain probe measured 1.20 TFLOP/s (1.97 GHz).
FP64_PEAK_TFLOPS = 1.20


def step_source_hash(kind="step"):
    """Hash of the kernel sources with comments and blank space taken out, so
    that a change of wording leaves the recorded traffic valid."""
    import hashlib
    import re

    h = hashlib.sha256()
    for f in {"step": STEP_SOURCES, "tma": TMA_SOURCES, "batch": BATCH_SOURCES}[kind]:
        with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
            code = re.sub(r"/\*.*?\*/", " ", fh.read(), flags=re.S)
        code = re.sub(r"//[^\n]*", " ", code)
        h.update(" ".join(code.split()).encode())
    return h.hexdigest()[:16]


def measured_traffic(key):
    t = MEASURED_TRAFFIC.get(key)
    return t[0] if t and t[2] == step_source_hash(t[1]) else None


def gc_weights(K):
    """Chebyshev nodes x_k = cos(pi (k + 1/2) / K) and the Gauss-Chebyshev weights of
    int g(x) dx = sum_k g(x_k) pi sqrt(1 - x_k^2) / K."""
    x = np.cos(np.pi * (np.arange(K) + 0.5) / K)
    return x, np.pi / K * np.sqrt(1 - x * x)


def dos_l1(rho1, rho2, a, K):
    """int |rho1 - rho2| dE on the DOS nodes (dE = a dx)."""
    _, w = gc_weights(K)
    return float(np.sum(np.abs(np.asarray(rho1) - np.asarray(rho2)) * w * a))


def accuracy_vs_fp64(K, mu32, mu64, a, b, n_nodes):
    """Error of an FP32-vector result against the FP64 path on the same inputs and random
    vectors: the largest moment difference and the L1 distance of the Jackson DOS."""
    mu32, mu64 = np.asarray(mu32, dtype=np.float64), np.asarray(mu64, dtype=np.float64)
    _, r32 = K.kpm_dos(mu32, a, b, n_nodes)
    _, r64 = K.kpm_dos(mu64, a, b, n_nodes)
    return {"max_abs_dmu": float(np.abs(mu32 - mu64).max()), "dos_l1": dos_l1(r32, r64, a, n_nodes)}


def accuracy_vs_oracle(K, mu_gpu, mu_oracle, a, b, n_nodes):
    """Error of a GPU result against the FP64 oracle on the same inputs and random
    vectors: largest moment difference and L1 distance of the Jackson DOS (the GPU
    DOS from the library, the oracle DOS from the oracle)."""
    import oracle as O

    mu_gpu, mu_oracle = np.asarray(mu_gpu, dtype=np.float64), np.asarray(mu_oracle, dtype=np.float64)
    _, r_gpu = K.kpm_dos(mu_gpu, a, b, n_nodes)
    _, r_or = O.dos(mu_oracle, a, b, n_nodes)
    return {"max_abs_dmu": float(np.abs(mu_gpu - mu_oracle).max()),
            "dos_l1": dos_l1(r_gpu, r_or, a, n_nodes)}


def per_matvec(value):
    """The same throughput counted per matrix-vector product (two moments per
    product in the doubling form): nnz*R*(M/2)/t."""
    return {"value": value / 2, "unit": "nnz*R*matvecs/s"}


def stencil_algorithmic(nnz, N, R, M, fp32, dims=3):
    """Bytes and flops of one fused step of a complex stencil solve.

    bytes/step = 3 N R s_v (read v_n, read v_{n-1}, write v_{n+1}) + N d s_hop
    flops/site/vector/step (complex) = 8 nnz/N + 4 + 8 (dots)."""
    s_v = 8 if fp32 else 16
    bytes_step = 3 * N * R * s_v + N * dims * s_v
    flops_step = N * R * (8 * nnz / N + 4 + 8)
    return bytes_step, flops_step


def csr_bytes_per_step(N, nnz, R, s_v=8):
    """Algorithmic bytes of one fused CSR step: 3 N R s_v for the vectors plus
    nnz (s_val + 4) + 8 (N + 1) for the matrix (FP32 complex: s_val = 8)."""
    return 3 * N * R * s_v + nnz * (s_v + 4) + 8 * (N + 1)


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


def lib():
    from paper_1105_5481_gb300 import build as B
    from paper_1105_5481_gb300 import kpm as K

    B.build()
    K.lib()
    return K


def csr_inputs(K, w):
    """CSR arrays of a lattice workload from the library's host-side builder."""
    rp, col, val = K.kpm_stencil_to_csr(w["dims"], w["L"], hop=w["hop"], onsite=w["onsite"],
                                        bond_mask=w["mask"], complex_=w["complex"])
    return rp, col, val


def timed_solves(K, stream, solve, steps, warmup, device=0, barrier=None):
    """Runs warmup + steps solves on `stream`, the timed ones bracketed by CUDA events
    (and a barrier / device synchronisation on both sides); returns (ms per solve,
    library kernels launched, clock summary)."""
    import torch

    for i in range(warmup):
        solve(i)
    stream.synchronize()
    if barrier:
        barrier()
    torch.cuda.synchronize()
    l0 = K.kpm_kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with Clocks(device) as clk:
        e0.record(stream)
        for i in range(steps):
            solve(warmup + i)
        e1.record(stream)
        stream.synchronize()
    torch.cuda.synchronize()
    if barrier:
        barrier()
    return e0.elapsed_time(e1) / steps, K.kpm_kernel_launches() - l0, clk.summary()


# ================================================================ reference arm
def reference_arm(args):
    """The oracle on the machine's host cores (its C restatement, OpenMP over all host
    threads), each step a bounded sample of the headline workload: all 32 vectors,
    M = 16 moments of the doubling form, plus the DOS on 64 nodes."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle as O
    from oracle import kpm_cpu as OC
    from paper_1105_5481_gb300 import inputs as I

    w = I.workload(HEADLINE)
    R_s, M_s = w["R"], 16
    H = O.lattice_hamiltonian(w["L"], hop=w["hop"], mask=w["mask"])
    a, b = O.rescale(*O.gershgorin(H), PAD_EPS)
    v0 = I.phase_block(w["seed"], H.n, R_s)
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
    desc = (f"3D L=160 diluted spin lattice as CSR (N={H.n}, nnz={H.nnz}), all {R_s} random-phase "
            f"vectors, M={M_s} moments (the oracle's doubling form in C, FP64, OpenMP on {nthreads} "
            f"host threads) + DOS on 64 nodes, per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": HEADLINE,
                   "lattice": "3D cubic L=160 periodic, spin hoppings, 10% bond dilution, CSR",
                   "N": int(H.n), "nnz": int(H.nnz), "R": R_s, "M": M_s, "M_workload": w["M"],
                   "sample": f"bounded oracle sample: M={M_s} of the workload's {w['M']} moments"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads,
                         "kind": "oracle (C, OpenMP)", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ================================================================ ncu helper
def profile_run(prec, workload, batch_chunk=2, batch_cluster=4, batch_chunk_bytes=32,
                batch_rtiles=1, batch_top=0, batch_staged=False):
    """Two solves of the workload with Gershgorin bounds (no Lanczos products, so
    the only fused-step launches are those of the two solves); prec "bounds":
    three spectral-bound estimates of the 3D L=64 lattice (Gershgorin and the
    30-step FP64 Lanczos), for captures of the bound kernels."""
    import torch

    from paper_1105_5481_gb300 import inputs as I

    K = lib()
    if prec == "bounds":
        w = I.workload("cubic_spin_L64")
        h = K.kpm_create_stencil(3, w["L"], hop=w["hop"], complex_=True)
        t = []
        for _ in range(3):
            t0 = time.perf_counter()
            r = K.kpm_bounds(h, LANCZOS_STEPS, PAD_EPS, seed=6)
            t.append(1e3 * (time.perf_counter() - t0))
        h.close()
        print(json.dumps({"profile": "bounds", "ms_per_call": t, "emin": r[0], "emax": r[1]}))
        return 0
    if workload == "batch_2d_256":
        insts = I.batch_workload(3, 256)
        hs = [K.kpm_create_stencil(2, x["L"], onsite=x["onsite"]) for x in insts]
        ab = [K.kpm_bounds(h, 0, PAD_EPS)[2:] for h in hs]
        with K.kpm_batch_create(hs, [x["M"] for x in insts], 16, [p[0] for p in ab],
                                [p[1] for p in ab], [x["seed"] for x in insts], prec) as bt:
            K.kpm_batch_set_chunk_bytes(bt, batch_chunk_bytes)
            K.kpm_batch_set_config(bt, batch_cluster, batch_chunk, 100)
            K.kpm_batch_set_rtiles(bt, batch_rtiles, batch_top)
            if batch_staged:
                K.kpm_batch_set_staged(bt, True)
            for _ in range(2):
                mu = K.kpm_batch_run(bt)
        print(json.dumps({"profile": prec, "workload": workload, "mu0": float(mu[0])}))
        return 0
    if workload == "square_L32_fp64_csr":
        # the small configuration as a CSR matrix (padded ELL of width 6)
        w = I.workload("square_L32_fp64")
        rp, col, val = K.kpm_stencil_to_csr(2, w["L"], onsite=w["onsite"])
        with K.kpm_create_csr(rp.size - 1, rp, col, val) as h:
            _, _, a, b = K.kpm_bounds(h, 0, PAD_EPS)
            for i in range(2):
                mu = K.kpm_moments(h, w["M"], w["R"], a, b, seed=1000 + i, precision=prec)
            torch.cuda.synchronize()
        print(json.dumps({"profile": prec, "workload": workload, "mu0": float(mu[0]),
                          "mu2": float(mu[2])}))
        return 0
    w = I.workload(workload)
    if workload.startswith("csr_spin_dilute_L"):
        rp, col, val = csr_inputs(K, w)
        h = K.kpm_create_csr(rp.size - 1, rp, col, val, complex_=True)
        M, R = 64, w["R"]   # a short solve: the fused steps are identical at any M
    elif workload == "square_L32_fp64":
        h = K.kpm_create_stencil(2, w["L"], onsite=w["onsite"])
        M, R = w["M"], w["R"]
    else:
        h = K.kpm_create_stencil(3, w["L"], hop=w["hop"], complex_=True)
        M, R = w["M"], w["R"]
    with h:
        _, _, a, b = K.kpm_bounds(h, 0, PAD_EPS)
        for i in range(2):
            mu = K.kpm_moments(h, M, R, a, b, seed=1000 + i, precision=prec)
        torch.cuda.synchronize()
    print(json.dumps({"profile": prec, "workload": workload, "mu0": float(mu[0]), "mu2": float(mu[2])}))
    return 0


# ================================================================ headline: large diluted CSR
def headline_leg(args):
    """The largest single-GPU configuration: 3D L=160 diluted spin lattice as CSR,
    R=32, M=4096, FP32 vectors with FP64 moments, one full solve per step.  Under
    torchrun every rank runs its own realisation (s0 = rank) and rank 0 prints."""
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

    def max_over_ranks(x):
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    from paper_1105_5481_gb300 import inputs as I

    K = lib()
    t_setup = time.perf_counter()
    w = I.workload(HEADLINE)
    L, R, M, Kn, seed = w["L"], w["R"], w["M"], w["K"], w["seed"]
    N = int(np.prod(L))
    rp, col, val = csr_inputs(K, w)
    h = K.kpm_create_csr(N, rp, col, val, complex_=True)
    nnz = K.kpm_info(h)["nnz"]
    emin, emax, a, b = K.kpm_bounds(h, LANCZOS_STEPS, PAD_EPS, seed=6)
    setup_s = time.perf_counter() - t_setup
    stream = torch.cuda.Stream()
    mu_d = torch.empty(M, dtype=torch.float64, device="cuda")
    E_d = torch.empty(Kn, dtype=torch.float64, device="cuda")
    rho_d = torch.empty(Kn, dtype=torch.float64, device="cuda")

    # a host-output solve with the per-vector moments: divergence check, and the
    # GPU side of the oracle comparison below
    mu_chk, pv_chk = K.kpm_moments(h, M, R, a, b, seed=seed, s0=rank, precision="fp32", per_vec=True,
                                   stream=stream)
    assert abs(mu_chk[0] - 1.0) < 1e-5 and np.all(np.abs(mu_chk) <= 1 + 1e-5)

    def solve(i):
        K.kpm_moments(h, M, R, a, b, seed=seed + 1 + i, s0=rank, precision="fp32", out=mu_d,
                      stream=stream)
        K.kpm_dos(mu_d, a, b, Kn, "jackson", E=E_d, rho=rho_d, stream=stream)

    ms, launches, clk = timed_solves(K, stream, solve, args.steps, args.warmup, local, barrier)
    ms = max_over_ranks(ms)
    chain_ms, nsteps = K.kpm_step_timing(h)
    step_ms = max_over_ranks(chain_ms / nsteps)
    combined = None
    if dist is not None:
        # the ranks ran realisations s0 = 0 .. world-1 of one seed: the job's
        # moments are their vector-weighted mean (one all-reduce of M + 1 doubles)
        from paper_1105_5481_gb300.replicas import combine_moments

        comb = combine_moments(mu_chk, R)
        combined = {"realisations": world, "mu0": float(comb[0]),
                    "max_abs_mu": float(np.abs(comb).max())}

    units = nnz * R * M  # per solve
    value = world * units / (ms / 1e3)
    bytes_step = csr_bytes_per_step(N, nnz, R)
    hbm, peak_kind = peaks()
    ach = bytes_step / (step_ms / 1e3) / 1e9

    # end to end through the public API: pinned host CSR arrays -> handle ->
    # bounds -> moments -> DOS -> host results, every step
    rp_pin = torch.from_numpy(rp).pin_memory().numpy()
    col_pin = torch.from_numpy(col).pin_memory().numpy()
    val_pin = torch.from_numpy(val.view(np.float64)).pin_memory().numpy().view(np.complex128)
    e2e_steps = 2

    def e2e_once(i):
        with K.kpm_create_csr(N, rp_pin, col_pin, val_pin, complex_=True) as he:
            _, _, ae, be = K.kpm_bounds(he, LANCZOS_STEPS, PAD_EPS, seed=6, stream=stream)
            mu = K.kpm_moments(he, M, R, ae, be, seed=seed + 100 + i, s0=rank, precision="fp32",
                               stream=stream)
            E, rho = K.kpm_dos(mu, ae, be, Kn, stream=stream)
        return mu

    e2e_once(0)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(e2e_steps):
        e2e_once(i + 1)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / e2e_steps)
    h.close()
    del rp_pin, col_pin, val_pin

    accuracy = cpu = cpu_c = None
    extras = {}
    if rank == 0 and world == 1:
        import oracle as O
        from oracle import kpm_cpu as OC

        H = O.lattice_hamiltonian(L, hop=w["hop"], mask=w["mask"])
        assert H.nnz == nnz
        nthreads = OC.max_threads()
        # accuracy: the first random vector's moments, all M of them, against the
        # FP64 oracle (its C form) on the same vector
        t0 = time.perf_counter()
        v0c = I.random_columns(seed, N, R, [0], True)
        _, per_o = OC.moments_doubling(H, a, b, v0c, M, threads=nthreads)
        accuracy = accuracy_vs_oracle(K, pv_chk[0], per_o[0], a, b, Kn)
        accuracy.update({"vectors_compared": 1, "moments_compared": M,
                         "oracle": f"C form of the FP64 oracle, {nthreads} threads "
                                   f"({time.perf_counter() - t0:.1f} s)"})
        if not args.no_cpu_baseline:
            v0 = I.phase_block(seed, N, 2)
            t0 = time.perf_counter()
            mu_o, _ = O.moments_doubling(H, a, b, v0, 8)
            O.dos(mu_o, a, b, 64)
            dt = time.perf_counter() - t0
            cpu = {"value": H.nnz * 2 * 8 / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"FP64 NumPy oracle, same lattice, 2 of the {R} vectors, M=8 moments "
                             f"+ DOS ({dt:.1f} s)"}
            v32 = I.phase_block(seed, N, R)
            OC.moments_doubling(H, a, b, v32[:, :2], 4, threads=nthreads)  # warm-up
            t0 = time.perf_counter()
            OC.moments_doubling(H, a, b, v32, 16, threads=nthreads)
            dt_all = time.perf_counter() - t0
            t0 = time.perf_counter()
            OC.moments_doubling(H, a, b, v32[:, :2], 8, threads=1)
            dt_one = time.perf_counter() - t0
            cpu_c = {"value": H.nnz * R * 16 / dt_all, "unit": UNIT, "cores": nthreads,
                     "kind": "oracle (C, OpenMP)",
                     "sample": f"the oracle's doubling form in C, FP64 CSR, same lattice: all "
                               f"{nthreads} host threads with R={R}, M=16; one thread with R=2, M=8 "
                               f"({dt_all + dt_one:.1f} s)",
                     "one_core": {"value": H.nnz * 2 * 8 / dt_one, "cores": 1}}
        del H
        if not args.no_extras:
            extras = run_extras(args, K)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 vectors, f64 moments", "data": "synthetic",
            "config": {"workload": HEADLINE,
                       "lattice": "3D cubic L=160 periodic (N=4,096,000), spin-derived complex "
                                  "hoppings, 10% bond dilution, CSR (padded ELL in the library)",
                       "N": N, "nnz": nnz, "R": R, "M": M, "K": Kn, "S_per_rank": 1,
                       "bounds": {"emin": emin, "emax": emax, "a": a, "b": b,
                                  "method": "Gershgorin + 30-step Lanczos, pad 0.01"},
                       "step": "random block + M/2 fused steps + moment reduction + Jackson DOS",
                       "l2": "inputs larger than L2 (two 1.05 GB vector blocks)",
                       "parallelism": f"replicas x{world}", "setup_s": setup_s},
            "roofline": {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                         "frac": ach / hbm, "traffic": measured_traffic(HEADLINE),
                         "kernel": "ell_tma_step_kernel<float, complex, W=6> (TMA-fed, "
                                   "2 stages x 64 rows, 2 CTAs/SM)",
                         "bytes_per_launch": bytes_step, "launch_ms": step_ms,
                         "peak_kind": f"{peak_kind} (copy bandwidth)"},
            "per_matvec": per_matvec(value),
            "accuracy_vs_oracle": accuracy,
            "cpu_baseline": cpu,
            "cpu_baseline_c": cpu_c,
            "e2e": {"value": world * units / (e2e_ms / 1e3), "unit": UNIT, "ms_per_step": e2e_ms,
                    "h2d_bytes_per_step": int(rp.nbytes + col.nbytes + val.nbytes),
                    "d2h_bytes_per_step": int(8 * (M + 2 * Kn)),
                    "includes": "create from pinned host CSR arrays (padded-ELL copy built on the "
                                "device), bounds, moments, DOS, destroy"},
            "replicas_combined": combined,
            "gpu_launches": launches,
            "clocks": clk,
        }
        line.update(extras)
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_extras(args, K):
    """The other configurations of the metric, each measured after the headline
    and reported under its own key; a failure is reported, not hidden."""
    out = {}
    for key, fn in (("cubic_spin_L64", cubic_result), ("square_L32_fp64", square_result),
                    ("batch_2d_256", batch_result), ("serve_poisson", serve_result)):
        t0 = time.perf_counter()
        try:
            r = fn(args, K)
            for k in ("metric", "n_gpus", "higher_is_better", "scaling", "vs_baseline", "data"):
                r.pop(k, None)
        except Exception as e:  # noqa: BLE001
            r = {"error": f"{type(e).__name__}: {e}"}
        r["leg_s"] = time.perf_counter() - t0
        out[key] = r
    return out


# ================================================================ other configurations
def cubic_result(args, K):
    """3D L=64 spin lattice (N=262144), R=64, M=1024: FP32-vector path (HBM-bound)
    and FP64 path (FP64-ALU-bound) on the same input, the FP32 result against the
    FP64 oracle on one full vector."""
    import torch

    import oracle as O
    from oracle import kpm_cpu as OC
    from paper_1105_5481_gb300 import inputs as I

    w = I.workload("cubic_spin_L64")
    L, R, M, Kn, seed = w["L"], w["R"], w["M"], w["K"], w["seed"]
    N = int(np.prod(L))
    h = K.kpm_create_stencil(3, L, hop=w["hop"], complex_=True)
    nnz = K.kpm_info(h)["nnz"]
    emin, emax, a, b = K.kpm_bounds(h, LANCZOS_STEPS, PAD_EPS, seed=6)
    stream = torch.cuda.Stream()
    mu_d = torch.empty(M, dtype=torch.float64, device="cuda")
    E_d = torch.empty(Kn, dtype=torch.float64, device="cuda")
    rho_d = torch.empty(Kn, dtype=torch.float64, device="cuda")

    def solver(prec):
        def solve(i):
            K.kpm_moments(h, M, R, a, b, seed=1000 + i, precision=prec, out=mu_d, stream=stream)
            K.kpm_dos(mu_d, a, b, Kn, "jackson", E=E_d, rho=rho_d, stream=stream)
        return solve

    steps32 = min(max(args.steps, 1), 10)
    ms32, l32, clk32 = timed_solves(K, stream, solver("fp32"), steps32, 3)
    step32 = K.kpm_step_timing(h)
    ms64, l64, clk64 = timed_solves(K, stream, solver("fp64"), 2, 1)
    step64 = K.kpm_step_timing(h)
    _, pv32 = K.kpm_moments(h, M, R, a, b, seed=seed, precision="fp32", per_vec=True, stream=stream)
    _, pv64 = K.kpm_moments(h, M, R, a, b, seed=seed, precision="fp64", per_vec=True, stream=stream)
    h.close()
    H = O.lattice_hamiltonian(L, hop=w["hop"])
    _, per_o = OC.moments_doubling(H, a, b, I.random_columns(seed, N, R, [0], True), M,
                                   threads=OC.max_threads())
    units = nnz * R * M
    bytes32, flops = stencil_algorithmic(nnz, N, R, M, True)
    bytes64, _ = stencil_algorithmic(nnz, N, R, M, False)
    hbm, peak_kind = peaks()
    ach32 = bytes32 / (step32[0] / step32[1] / 1e3) / 1e9
    ach64 = flops / (step64[0] / step64[1] / 1e3) / 1e12
    return {
        "value": units / (ms32 / 1e3), "unit": UNIT, "ms_per_step": ms32, "steps": steps32,
        "dtype": "f32 vectors, f64 moments",
        "config": {"workload": "cubic_spin_L64", "N": N, "nnz": nnz, "R": R, "M": M, "K": Kn,
                   "bounds": {"a": a, "b": b}, "l2": "inputs larger than L2 (two 134 MB blocks)"},
        "roofline": {"bound": "hbm", "achieved": ach32, "peak": hbm, "unit": "GB/s",
                     "frac": ach32 / hbm, "traffic": measured_traffic("cubic_spin_L64"),
                     "kernel": "cheb_step_kernel<float, complex, STEP, StencilOp<3,hop>>",
                     "bytes_per_launch": bytes32, "launch_ms": step32[0] / step32[1],
                     "peak_kind": f"{peak_kind} (copy bandwidth)"},
        "accuracy_vs_oracle": dict(accuracy_vs_oracle(K, pv32[0], per_o[0], a, b, Kn),
                                   vectors_compared=1, moments_compared=M, path="fp32"),
        "accuracy_fp64_vs_oracle": dict(accuracy_vs_oracle(K, pv64[0], per_o[0], a, b, Kn),
                                        vectors_compared=1, moments_compared=M, path="fp64"),
        "fp64_path": {"value": units / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64, "steps": 2,
                      "dtype": "f64",
                      "roofline": {"bound": "alu", "achieved": ach64, "peak": FP64_PEAK_TFLOPS,
                                   "unit": "TFLOP/s", "frac": ach64 / FP64_PEAK_TFLOPS,
                                   "hbm_frac": bytes64 / (step64[0] / step64[1] / 1e3) / 1e9 / hbm,
                                   "launch_ms": step64[0] / step64[1]},
                      "gpu_launches": l64, "clocks": clk64},
        "gpu_launches": l32, "clocks": clk32}


def square_result(args, K):
    """The small FP64 configuration (2D L=32, R=8, M=256, Jackson DOS on 1024 nodes):
    latency-bound, reported as microseconds per solve with its L2-resident rate,
    beside the same solve as a batch of one."""
    import torch

    from paper_1105_5481_gb300 import inputs as I

    w = I.workload("square_L32_fp64")
    N, R, M, Kn = int(np.prod(w["L"])), w["R"], w["M"], w["K"]
    h = K.kpm_create_stencil(2, w["L"], onsite=w["onsite"])
    nnz = K.kpm_info(h)["nnz"]
    emin, emax, a, b = K.kpm_bounds(h, LANCZOS_STEPS, PAD_EPS, seed=6)
    stream = torch.cuda.Stream()
    mu_d = torch.empty(M, dtype=torch.float64, device="cuda")
    E_d = torch.empty(Kn, dtype=torch.float64, device="cuda")
    rho_d = torch.empty(Kn, dtype=torch.float64, device="cuda")

    def solve(i):
        K.kpm_moments(h, M, R, a, b, seed=100 + i, precision="fp64", out=mu_d, stream=stream)
        K.kpm_dos(mu_d, a, b, Kn, "jackson", E=E_d, rho=rho_d, stream=stream)

    steps = max(args.steps, 1) * 20  # one solve is well under a millisecond
    ms, launches, clk = timed_solves(K, stream, solve, steps, max(args.warmup, 3))
    chain_ms, nsteps = K.kpm_step_timing(h)
    form = K.kpm_testing_last_step_form(h)
    # the same solve as a chain of dependent step launches (the form the
    # column-resident solve replaces), on a handle planned with it turned off
    old = os.environ.get("KPM_COLRES")
    os.environ["KPM_COLRES"] = "0"
    try:
        hc = K.kpm_create_stencil(2, w["L"], onsite=w["onsite"])

        def solve_chain(i):
            K.kpm_moments(hc, M, R, a, b, seed=100 + i, precision="fp64", out=mu_d, stream=stream)
            K.kpm_dos(mu_d, a, b, Kn, "jackson", E=E_d, rho=rho_d, stream=stream)

        chain_solve_ms, _, _ = timed_solves(K, stream, solve_chain, steps, max(args.warmup, 3))
        chain_steps_ms, _ = K.kpm_step_timing(hc)
        hc.close()
    finally:
        if old is None:
            os.environ.pop("KPM_COLRES", None)
        else:
            os.environ["KPM_COLRES"] = old
    batch_of_one = {}
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
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
    h.close()
    bytes_step = 3 * N * R * 8 + N * 8  # vectors + on-site energies (uniform hopping)
    hbm, peak_kind = peaks()
    rate = bytes_step / (chain_ms / nsteps / 1e3) / 1e9
    value = nnz * R * M / (ms / 1e3)
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "per_matvec": per_matvec(value),
        "steps": steps, "warmup": max(args.warmup, 3), "ms_per_step": ms, "us_per_solve": ms * 1e3,
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
                     "note": ("128 dependent products on 128 KB of vectors, all in one launch "
                              "of 8 independent clusters (one per vector column, both vector "
                              "blocks in shared memory): launch_ms is the average product "
                              "inside it; achieved = the vector bytes of a product over that time"
                              if form == "column-resident solve" else
                              "127 dependent steps on 128 KB of vectors: each step is one "
                              "launch's latency; achieved = the L2-resident rate")},
        "form": form,
        "step_chain": {"us_per_solve": chain_solve_ms * 1e3,
                       "us_per_step": chain_steps_ms / nsteps * 1e3,
                       "note": "the same solves as a chain of dependent fused-step launches "
                               "(KPM_COLRES=0)"},
        "batch_of_one_moments": batch_of_one,
        "gpu_launches": launches, "clocks": clk}


def batch_result(args, K):
    """256 independent 2D disorder realisations of uneven size, R=16 FP32 real
    vectors, one persistent cluster launch per batch (graph replay, autotuned),
    against the same solves issued as plain per-instance kpm_moments calls in FP32
    and in FP64."""
    import torch

    from paper_1105_5481_gb300 import inputs as I

    insts = I.batch_workload(3, 256)
    R = 16
    hs = [K.kpm_create_stencil(2, x["L"], onsite=x["onsite"]) for x in insts]
    ab = [K.kpm_bounds(h, 0, PAD_EPS)[2:] for h in hs]
    Ms = [x["M"] for x in insts]
    seeds = [x["seed"] for x in insts]
    bt = K.kpm_batch_create(hs, Ms, R, [p[0] for p in ab], [p[1] for p in ab], seeds, "fp32")
    t0 = time.perf_counter()
    info = K.kpm_batch_tune(bt, reps=1)
    info["rtiles"], info["tiled_instances"], _ = K.kpm_batch_get_rtiles(bt)
    info["resident"] = K.kpm_batch_get_resident(bt)[0]
    info["staged"] = K.kpm_batch_get_staged(bt)[0]
    info["chunk_bytes"], info["threads_per_row"] = K.kpm_batch_get_chunk_bytes(bt)
    tune_s = time.perf_counter() - t0
    mu_host = K.kpm_batch_run(bt)  # host output: divergence check
    assert np.all(np.abs(mu_host) <= 1 + 1e-5)
    stream = torch.cuda.Stream()
    out = torch.empty(int(sum(Ms)), dtype=torch.float64, device="cuda")
    steps = max(args.steps, 1)

    def run(i):
        K.kpm_batch_run(bt, out=out, stream=stream)

    ms, launches, clk = timed_solves(K, stream, run, steps, max(args.warmup, 3))
    Ns = [x["L"][0] * x["L"][1] for x in insts]
    nnz = [5 * n for n in Ns]                 # 4 bonds + on-site per row
    units = sum(z * R * m for z, m in zip(nnz, Ms))
    byts = sum((m // 2) * (3 * n * R * 4 + n * 4) for n, m in zip(Ns, Ms))
    # the same solves as plain per-instance calls (one graph per instance, sequential)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    mu1 = torch.empty(max(Ms), dtype=torch.float64, device="cuda")
    per_instance = {}
    for prec in ("fp32", "fp64"):
        for h, m, p, sd in zip(hs, Ms, ab, seeds):  # first call of a shape, then the captured form
            K.kpm_moments(h, m, R, p[0], p[1], seed=sd, precision=prec, out=mu1[:m], stream=stream)
            K.kpm_moments(h, m, R, p[0], p[1], seed=sd, precision=prec, out=mu1[:m], stream=stream)
        stream.synchronize()
        e0.record(stream)
        for h, m, p, sd in zip(hs, Ms, ab, seeds):
            K.kpm_moments(h, m, R, p[0], p[1], seed=sd, precision=prec, out=mu1[:m], stream=stream)
        e1.record(stream)
        stream.synchronize()
        per_instance[prec] = {"ms": e0.elapsed_time(e1), "speedup_of_batch": e0.elapsed_time(e1) / ms}
    # accuracy: every 32nd instance against its FP64 solve on the same random vectors
    acc_b = []
    for k, (mu_i, h_i, m_i, p_i, sd) in enumerate(zip(bt.split(mu_host), hs, Ms, ab, seeds)):
        if k % 32 == 0:
            mu64 = K.kpm_moments(h_i, m_i, R, p_i[0], p_i[1], seed=sd, precision="fp64")
            acc_b.append(accuracy_vs_fp64(K, mu_i, mu64, p_i[0], p_i[1], 1024))
    accuracy = {"max_abs_dmu": max(x["max_abs_dmu"] for x in acc_b),
                "dos_l1": max(x["dos_l1"] for x in acc_b), "instances_compared": len(acc_b)}
    bt.close()
    for h in hs:
        h.close()
    hbm, peak_kind = peaks()
    ach = byts / (ms / 1e3) / 1e9
    traffic = measured_traffic("batch_2d_256/C%d/chunk%d/clusters%d/rt%d/top%d%s" % (
        info["cluster"], info["chunk"], info["clusters"], info["rtiles"],
        info["tiled_instances"], ("/resident" if info["resident"] else "") +
        ("/staged" if info["staged"] else "") +
        ("/chunk16B" if info["chunk_bytes"] == 16 else "")))
    return {
        "metric": METRIC, "value": units / (ms / 1e3), "unit": UNIT, "n_gpus": 1,
        "steps": steps, "warmup": max(args.warmup, 3), "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 vectors, f64 moments",
        "data": "synthetic",
        "config": {"workload": "batch_2d_256",
                   "instances": "256 x 2D periodic L~U{16..128}, W~U[0,4), M even ~U{128..2048}, R=16",
                   "sites_total": sum(Ns), "moments_total": sum(Ms),
                   "bounds": "Gershgorin per instance, pad 0.01",
                   "launch": "one persistent cluster kernel per batch, CUDA graph replay",
                   "autotuned": info, "tune_s": tune_s, "l2": "instances' vectors mostly L2-resident"},
        "roofline": {"bound": "latency", "achieved": ach, "peak": hbm, "unit": "GB/s",
                     "frac": ach / hbm, "traffic": traffic, "bytes_per_launch": byts,
                     "peak_kind": peak_kind,
                     "dram_frac": (traffic / (ms / 1e3) / 1e9 / hbm) if traffic else None,
                     "note": "achieved = algorithmic bytes of all instances per batch launch over "
                             "its duration; the active instances' vectors mostly stay in L2, so "
                             "this is not a DRAM rate: dram_frac = the measured DRAM traffic "
                             "over the duration, against the copy bandwidth.  The kernel is "
                             "latency-bound (chains of dependent products per cluster)"},
        "per_instance_calls": per_instance,
        "accuracy_vs_fp64": accuracy,
        "solves_per_s": 256 / (ms / 1e3),
        "per_matvec": per_matvec(units / (ms / 1e3)),
        "gpu_launches": launches, "clocks": clk}


def serve_result(args, K, rates=(10.0, 20.0, 40.0, 80.0, 160.0), count=128, count64=48,
                 rate64=40.0, K_nodes=1024):
    """Poisson streams of DOS requests (2D/3D, N log-uniform in [1e3, 4e6], M in
    256..8192, R in {8,16,32,64}, real or complex spin hoppings) through the serving
    loop with FP32 vectors, the arrival rate swept to saturation (the same requests
    at every rate, arrival times scaled); beside it, the first `count64` requests at
    `rate64` served as plain per-request FP64 calls (first come first served), and
    each served result's error against its FP64 counterpart."""
    import threading

    from paper_1105_5481_gb300 import inputs as I

    reqs = I.serving_stream(5, count, 1.0)   # arrival times at 1 Hz, scaled per rate
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
        ab.append(K.kpm_bounds(h, 0, PAD_EPS)[2:])

    def run_served(rate, n):
        srv = K.kpm_server_create(48 << 30, steps_per_tick=32, cluster=4)
        ids = [None] * n
        t0 = time.perf_counter()

        def feed():
            for k in range(n):
                r = reqs[k]
                dt = t0 + r["t"] / rate - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                ids[k] = K.kpm_server_submit(srv, hs[k], r["M"], r["R"], ab[k][0], ab[k][1],
                                             seed=r["seed"], precision="fp32", K=K_nodes)

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

    units = [int(np.prod(r["L"])) * (2 * r["dims"]) * r["R"] * r["M"] for r in reqs]
    sweep = []
    l0 = K.kpm_kernel_launches()
    first = None
    with Clocks(0) as clk:
        for rate in rates:
            res, st, wall = run_served(rate, count)
            if first is None:
                first = res
            sweep.append({"rate_hz": rate, "offered_solves_per_s": count / (reqs[-1]["t"] / rate),
                          "solves_per_s": st["completed"] / wall,
                          "nnz_R_moments_per_s": sum(units) / wall,
                          "p50_s": st["p50_s"], "p99_s": st["p99_s"], "mean_s": st["mean_s"],
                          "max_s": st["max_s"], "completed": st["completed"], "failed": st["failed"],
                          "ticks": st["ticks"], "peak_resident": st["peak_resident"],
                          "wall_s": wall})
    launches = K.kpm_kernel_launches() - l0
    # plain per-request FP64 calls, first come first served, on arrival
    t0 = time.perf_counter()
    lat64, res64 = [], []
    for k in range(count64):
        r = reqs[k]
        dt = t0 + r["t"] / rate64 - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        mu = K.kpm_moments(hs[k], r["M"], r["R"], ab[k][0], ab[k][1], seed=r["seed"], precision="fp64")
        E, rho = K.kpm_dos(mu, ab[k][0], ab[k][1], K_nodes)
        res64.append((mu, rho))
        lat64.append(time.perf_counter() - (t0 + r["t"] / rate64))
    wall64 = time.perf_counter() - t0
    served40 = next((s for s in sweep if s["rate_hz"] == rate64), None)
    err_mu = max(float(np.abs(first[k][0] - res64[k][0]).max()) for k in range(count64))
    err_dos = max(dos_l1(first[k][2], res64[k][1], ab[k][0], K_nodes) for k in range(count64))
    for h in hs:
        h.close()
    best = max(sweep, key=lambda s: s["solves_per_s"])
    return {
        "metric": "served DOS solves/s, p50/p99", "value": best["solves_per_s"], "unit": "solves/s",
        "n_gpus": 1, "steps": count * len(rates), "warmup": 0,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 vectors, f64 moments", "data": "synthetic",
        "config": {"workload": "serve_poisson", "requests_per_rate": count, "rates_hz": list(rates),
                   "mix": "2D/3D cubic, N log-uniform [1e3, 4e6], M even log-uniform [256, 8192], "
                          "R in {8,16,32,64}, real or complex spin hoppings, K=1024 Jackson DOS",
                   "server": "48 GiB arena, 32 products per tick, clusters of 4, large requests "
                             "(>= 8 MB per product) as full-GPU steps on 4 streams",
                   "bounds": "Gershgorin per request, pad 0.01"},
        "sweep": sweep,
        "served_at_fp64_rate": served40,
        "per_request_fp64": {"rate_hz": rate64, "requests": count64,
                             "solves_per_s": count64 / wall64,
                             "p50_s": float(np.percentile(lat64, 50)),
                             "p99_s": float(np.percentile(lat64, 99)), "wall_s": wall64},
        "accuracy_vs_fp64": {"max_abs_dmu": err_mu, "max_dos_l1": err_dos, "requests": count64},
        "gpu_launches": launches, "clocks": clk.summary()}


def dense_result(args, K):
    """The paper's dense formulation at its largest matrix (Sec. IV-C: H_SIZE =
    4096, N = 128 moments, R x S = 1792 vectors), FP64 as in the paper: a real
    Wigner matrix, all 1792 vectors in one block, one solve per step."""
    import torch

    from paper_1105_5481_gb300 import inputs as I

    w = I.workload(args.workload)
    A, D, R, M, Kn = w["H"], w["D"], w["R"], w["M"], w["K"]
    h = K.kpm_create_dense(A)
    nnz = K.kpm_info(h)["nnz"]
    emin, emax, a, b = K.kpm_bounds(h, LANCZOS_STEPS, PAD_EPS, seed=6)
    stream = torch.cuda.Stream()
    mu_d = torch.empty(M, dtype=torch.float64, device="cuda")
    E_d = torch.empty(Kn, dtype=torch.float64, device="cuda")
    rho_d = torch.empty(Kn, dtype=torch.float64, device="cuda")
    mu_chk = K.kpm_moments(h, M, R, a, b, seed=1, stream=stream)
    assert abs(mu_chk[0] - 1.0) < 1e-12 and np.all(np.abs(mu_chk) <= 1 + 1e-9)

    def solve(i):
        K.kpm_moments(h, M, R, a, b, seed=100 + i, out=mu_d, stream=stream)
        K.kpm_dos(mu_d, a, b, Kn, "jackson", E=E_d, rho=rho_d, stream=stream)

    steps = max(1, min(args.steps, 3))
    ms, launches, clk = timed_solves(K, stream, solve, steps, 3)
    chain_ms, nsteps = K.kpm_step_timing(h)
    h.close()
    flops_step = 2.0 * D * D * R
    step_s = chain_ms / nsteps / 1e3
    value = nnz * R * M / (ms / 1e3)
    tensor = os.environ.get("KPM_DENSE_TENSOR", "") != "0" and D >= 512
    # the same solve on the FP64 pipe, for comparison
    os.environ["KPM_DENSE_TENSOR"] = "0"
    try:
        with K.kpm_create_dense(A) as h64:
            fp64_ms, _, _ = timed_solves(K, stream, lambda i: K.kpm_moments(
                h64, M, R, a, b, seed=300 + i, out=mu_d, stream=stream), 1, 1)
            c64, n64 = K.kpm_step_timing(h64)
            mu64 = K.kpm_moments(h64, M, R, a, b, seed=1, stream=stream)
    finally:
        del os.environ["KPM_DENSE_TENSOR"]
    fp64_form = {"ms_per_solve": fp64_ms, "step_ms": c64 / n64,
                 "fp64_tflops": flops_step / (c64 / n64 / 1e3) / 1e12,
                 "max_abs_dmu_vs_tensor_form": float(np.abs(mu64 - mu_chk).max())}
    A_pin = torch.from_numpy(A).pin_memory().numpy()

    def e2e_once(i):
        with K.kpm_create_dense(A_pin) as he:
            _, _, ae, be = K.kpm_bounds(he, LANCZOS_STEPS, PAD_EPS, seed=6)
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
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "per_matvec": per_matvec(value),
        "steps": steps, "warmup": 3, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload,
                   "matrix": f"dense real Wigner matrix D={D} (entries U[-1,1)/sqrt(D)), every "
                             "element stored and used (the paper's formulation)",
                   "N": D, "nnz": nnz, "R": R, "M": M, "K": Kn,
                   "bounds": {"emin": emin, "emax": emax, "a": a, "b": b},
                   "step": "random block + M/2 dense products + moment reduction + Jackson DOS",
                   "l2": "matrix (134 MB) larger than L2"},
        "roofline": dense_roofline(tensor, D, R, flops_step, step_s),
        "fp64_equivalent_tflops": flops_step / step_s / 1e12,
        "fp64_pipe_form": fp64_form,
        "cpu_baseline": cpu,
        "e2e": {"value": nnz * R * M / (e2e_ms / 1e3), "unit": UNIT, "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": int(A.nbytes), "d2h_bytes_per_step": int(8 * (M + 2 * Kn)),
                "includes": "create from a pinned host matrix, bounds, moments, DOS, destroy"},
        "gpu_launches": launches, "clocks": clk}


def dense_roofline(tensor, D, R, flops_step, step_s):
    """Roofline of the dense step.  Tensor-core form: the bf16 slice products
    (k(k+1)/2 products of 2 D^2 Rp flops, beta and k as the library chooses
    them) per step duration, against the measured sustained bf16 GEMM rate;
    FP64-pipe form: 2 D^2 R FP64 flops against the FP64 FMA rate."""
    if not tensor:
        ach = flops_step / step_s / 1e12
        return {"bound": "alu", "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP64_PEAK_TFLOPS, "traffic": None,
                "kernel": "dense_step_kernel<real, STEP, 64-row tiles>", "flops_per_launch": flops_step,
                "launch_ms": step_s * 1e3,
                "peak_kind": "FP64 pipe, 2 FMA per SM and clock at 1.97 GHz (measured)"}
    lg = max(0, (D - 1).bit_length())
    beta = max(1, min(7, (24 - lg) // 2))
    k = (54 + beta - 1) // beta
    Rp = R + (R % 2)
    tc_flops = k * (k + 1) // 2 * 2.0 * D * D * Rp
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak, kind = float(json.load(f)["bf16_tflops_sustained"]), "measured (sustained cuBLAS bf16)"
    except Exception:
        peak, kind = 1700.0, "fallback"
    ach = tc_flops / step_s / 1e12
    return {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "traffic": None, "kernel": f"Ozaki split: {k * (k + 1) // 2} bf16 slice products "
                                      f"(beta={beta}, k={k}) + slicing and FP64 epilogue",
            "flops_per_launch": tc_flops, "launch_ms": step_s * 1e3, "peak_kind": kind}


def single_leg(args):
    """--workload NAME (other than the headline): one configuration, its own line."""
    K = lib()
    fn = {"cubic_spin_L64": cubic_result, "square_L32_fp64": square_result,
          "batch_2d_256": batch_result, "serve_poisson": serve_result}.get(args.workload)
    if fn is None and args.workload.startswith("dense_wigner_D"):
        fn = dense_result
    if fn is None:
        raise SystemExit(f"--workload {args.workload} runs only with --profile")
    r = fn(args, K)
    base = {"metric": METRIC, "n_gpus": 1, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "data": "synthetic", "steps": args.steps, "warmup": args.warmup}
    base.update(r)
    print(json.dumps(base))
    return 0


def relaunch_distributed(args):
    """--gpus N > 1 outside torchrun: run this script as N processes, one per GPU."""
    import socket

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
           f"--nproc-per-node={args.gpus}", "--master-addr", "127.0.0.1",
           "--master-port", str(port), os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline only: skip the other configurations' keys")
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
    ap.add_argument("--batch-staged", action="store_true",
                    help="--profile with the batch workload: the staged form (tiles copied "
                         "into shared-memory rings; --batch-chunk sets the tile size)")
    ap.add_argument("--workload", default=HEADLINE,
                    choices=[HEADLINE, "cubic_spin_L64", "batch_2d_256", "serve_poisson",
                             "square_L32_fp64", "dense_wigner_D4096", "csr_spin_dilute_L100",
                             "square_L32_fp64_csr"],
                    help="csr_spin_dilute_L160 (default: the headline line with the other "
                         "configurations as extra keys) or one configuration alone")
    ap.add_argument("--profile", default=None, choices=["fp32", "fp64", "bounds"],
                    help="run two solves of the workload at the given precision and exit "
                         "(a short command for ncu captures of the fused step)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)
    if args.profile:
        return profile_run(args.profile, args.workload, args.batch_chunk, args.batch_cluster,
                           args.batch_chunk_bytes, args.batch_rtiles, args.batch_top,
                           args.batch_staged)
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        return relaunch_distributed(args)
    if args.workload == "csr_spin_dilute_L100":
        ap.error("csr_spin_dilute_L100 (a smaller lattice for profiler captures) is for --profile only")
    if args.workload != HEADLINE:
        return single_leg(args)
    return headline_leg(args)


if __name__ == "__main__":
    sys.exit(main())
