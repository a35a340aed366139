#!/usr/bin/env python
"""Benchmark of the CDFCI column update on GB300: H elements/s into the hash table of b.

Workload (one GPU): synthetic ab initio Hamiltonian, N = 24 spatial orbitals,
6 alpha + 6 beta electrons, seed 2, 48 Cholesky vectors, aufbau start,
compression tau = 1e-5, one coordinate per iteration (CDFCI, Algorithm 1),
a 2^27-slot (4 GiB) device hash table.  Column length 16,471.

A step is `iters_per_step` iterations of the whole hot path (choice, step size,
column enumeration, Slater-Condon elements, compression, hash scatter,
recalculation of b_i), i.e. one cdfci_step call.  The table (4 GiB) is larger
than L2, so no flush is needed between steps.

Extra keys: roofline of the fused column kernel, the CPU oracle as the
baseline, end-to-end throughput through the C-ABI from host buffers, time to
reach a stored exact energy within 1e-6 Ha on the 8-site chain, SM clocks
sampled during the timed region, and the batched paths: mCDFCI (m = 128) on
the same workload, the 4x4 Hubbard lattice with m = 256, 96 uneven problems
stepped in one launch, and the RDM/derivative pass on the N = 16 workload.

Multi-GPU (torchrun): every rank runs an independent replica of the same solve
(one CDFCI trajectory does not shard without an exchange step); value = all
ranks' elements / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

ALGO_BYTES_PER_ELEMENT = 40      # 16 B key compare + 8 B c read + 8 B b read + 8 B b write
WORKLOAD = dict(name="abinitio_N24_6a6b_seed2", N=24, n_alpha=6, n_beta=6, seed=2, tau=1e-5, log2_capacity=27, m=1)
KERNEL_SOURCES = ["paper_2605_04483_gb300/csrc/cdfci_kernels.cu", "paper_2605_04483_gb300/csrc/cdfci_internal.cuh"]
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "k_cd_loop_grid_abinitio_N24.txt")
SCATTER_SOURCES = ["paper_2605_04483_gb300/csrc/cdfci_block.cu", "paper_2605_04483_gb300/csrc/cdfci_internal.cuh"]
SCATTER_PROFILE = os.path.join(ROOT, "profiles", "k_mc_scatter_abinitio_N24_m128.txt")


def kernel_hash(sources) -> str:
    """Hash of the kernel sources' code: comments, trailing blanks and blank lines removed, so that a
    comment edit keeps a profile summary valid while any code change invalidates it."""
    import re
    h = hashlib.sha256()
    for f in sources:
        with open(os.path.join(ROOT, f)) as fh:
            text = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        for line in text.splitlines():
            line = re.sub(r"//.*", "", line).rstrip()
            if line:
                h.update(line.encode() + b"\n")
    return h.hexdigest()[:16]


def profiled_traffic(path, sources, key):
    """A DRAM figure from a committed ncu summary, if it was taken on the current kernel sources."""
    try:
        vals = {}
        for line in open(path):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
        if vals.get("kernel_source_hash") != kernel_hash(sources):
            return None
        return float(vals[key])
    except (OSError, KeyError, ValueError):
        return None


def slot_probe(torch, api, log2_slots: int = 27, n_ops: int = 1 << 26, reps: int = 5) -> dict:
    """The hash scatter's access pattern at its ceiling (cdfci_probe_slots, a hand-written kernel of the
    library): independent random 32-byte slots of a 2^27-slot (4 GiB > L2) table, each a 16-byte key load,
    a 16-byte {c, b} load and an FP64 add to b, several in flight per lane.  Reported per operation as the
    scatter's 40 algorithmic bytes and as the 64 bytes of DRAM sectors it moves (read + write-back)."""
    table = torch.zeros((1 << log2_slots) * 4, dtype=torch.float64, device="cuda")
    st = torch.cuda.Stream()
    for r in range(2):
        api.cdfci_probe_slots(table, log2_slots, n_ops, seed=r + 1, stream=st.cuda_stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for r in range(reps):
        api.cdfci_probe_slots(table, log2_slots, n_ops, seed=100 + r, stream=st.cuda_stream)
    e1.record(st)
    e1.synchronize()
    dt = e0.elapsed_time(e1) * 1e-3 / reps
    del table
    torch.cuda.empty_cache()
    ops = n_ops / dt
    peak, _ = measured_peaks()
    return {"ops_per_s": ops, "gbs_40B": ops * ALGO_BYTES_PER_ELEMENT / 1e9,
            "frac_40B": ops * ALGO_BYTES_PER_ELEMENT / 1e9 / peak, "sector_gbs_64B": ops * 64 / 1e9,
            "frac_64B": ops * 64 / 1e9 / peak, "ops": n_ops, "table_gib": (1 << log2_slots) * 32 / 2 ** 30}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.idx = gpu_index
        self.proc = None

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def load_reference_energy(name: str) -> float:
    for line in open(os.path.join(ROOT, "tests", "golden", "reference_energies.txt")):
        if line.startswith(name + " "):
            return float(line.split()[-1])
    raise KeyError(name)


def paper_hubbard_ed(na: int, nb: int, U: float) -> float:
    """Exact energy of the 4x4 periodic lattice that the paper prints (tests/golden/paper_hubbard_ed.txt)."""
    for line in open(os.path.join(ROOT, "tests", "golden", "paper_hubbard_ed.txt")):
        f = line.split()
        if f and not line.startswith("#") and (int(f[0]), int(f[1]), float(f[2])) == (na, nb, U):
            return float(f[3])
    raise KeyError((na, nb, U))


def hubbard_k_leg(api, inputs) -> dict:
    """The paper's own lattice setting: the 4x4 periodic Hubbard model in momentum space built by the library
    (cdfci_create_hubbard_k: momentum-conserving enumeration), half filling, from the degenerate-subspace
    start, m = 128: seconds until the running energy is within 1e-5 Ha of the paper's exact value, at
    U/t = 0.5 (2^24 slots with z_threshold_search; the paper's CDFCI run took 13 s) and at U/t = 4 (2^26
    slots, tau = 0; the paper's run took 9 minutes), and the exact Rayleigh quotient reached."""
    out = {}
    for U, budget, kw in ((0.5, 30.0, dict(log2_capacity=24, z_threshold_search=1)),
                          (4.0, 60.0, dict(log2_capacity=26))):
        ref = paper_hubbard_ed(8, 8, U)
        s = api.Solver.hubbard_k((4, 4), 8, 8, t=1.0, U=U, num_coordinates=128, **kw)
        try:
            t0 = time.perf_counter()
            n_det, E_start = s.set_initial_degenerate()
            t_start = time.perf_counter() - t0
            reached = None
            while time.perf_counter() - t0 < budget:
                st = s.step(200)
                if abs(st["energy"] - ref) < 1e-5:
                    reached = time.perf_counter() - t0
                    break
            st = s.stats()
            out[f"U{U:g}"] = {"E_paper_ed": ref, "seconds_to_1e-5": reached, "energy": st["energy"],
                              "exact_rq": s.energy(1), "gap_ha": st["energy"] - ref,
                              "seconds": time.perf_counter() - t0,
                              "iterations": st["iterations"], "determinants": st["n_slots"],
                              "degenerate_start": {"determinants": n_det, "E": E_start, "seconds": t_start}}
        finally:
            s.close()
    return out


def host_info() -> dict:
    """The host the CPU numbers were taken on: online cores and CPU model."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model, "machine": os.uname().machine}


def cpu_baseline(seconds: float) -> dict:
    """The CPU oracle's serial CDFCI on the same workload, one host core, bounded sample."""
    import oracle
    from paper_2605_04483_gb300 import inputs
    w = inputs.config2()
    o = oracle.CDFCI(w.N, w.n_alpha, w.n_beta, w.h, w.g, (0, 0), WORKLOAD["tau"], 1)
    o.step(20)
    e0 = o.info()["elements"]
    it = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        o.step(20)
        it += 20
    dt = time.perf_counter() - t0
    el = o.info()["elements"] - e0
    o.close()
    return {"value": el / dt, "unit": "elements/s", "cores": 1, "kind": "oracle", "host": host_info(),
            "sample": f"{it} CDFCI iterations of the same workload after 20 warm-up iterations "
                      f"({dt:.1f} s, serial C oracle, 1 thread)"}


def workload_name(log2_capacity: int) -> str:
    return WORKLOAD["name"] + f", tau={WORKLOAD['tau']}, m=1, 2^{log2_capacity}-slot table"


def run_reference_arm(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_2605_04483_gb300 import inputs
    w = inputs.config2()
    iters = args.ref_iters_per_step
    o = oracle.CDFCI(w.N, w.n_alpha, w.n_beta, w.h, w.g, (0, 0), WORKLOAD["tau"], 1)
    for _ in range(args.warmup):
        o.step(iters)
    e0 = o.info()["elements"]
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.step(iters)
    dt = time.perf_counter() - t0
    el = o.info()["elements"] - e0
    value = el / dt
    line = {"impl": "reference", "metric": "H elements/s into hash b (CDFCI, Algorithm 1)", "value": value,
            "unit": "elements/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.log2_capacity),
                       "iters_per_step": iters, "note": "CPU oracle (serial C, its own hash map), bounded sample per step"},
            "cpu_baseline": {"value": value, "unit": "elements/s", "cores": 1, "kind": "oracle", "host": host_info(),
                             "sample": f"{args.steps} steps x {iters} iterations after {args.warmup} warm-up steps"},
            "e2e": {"value": value, "unit": "elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def timed_block_run(api, w, m, tau, log2_capacity, warm_iters, iters, kernel_iters=0, **kw) -> dict:
    """mCDFCI (Algorithm 2) throughput: elements/s over `iters` block iterations after `warm_iters`.
    With kernel_iters > 0, then that many more iterations launch by launch with CUDA events around each
    kernel (cdfci_time_kernels): the per-kernel split and the scatter's achieved bandwidth."""
    s = api.Solver(w.h, w.g, w.N, w.n_alpha, w.n_beta, num_coordinates=m, z_threshold=tau,
                   log2_capacity=log2_capacity, ref_alpha=int(w.ref[0]), ref_beta=int(w.ref[1]), **kw)
    kt = None
    try:
        s.step(warm_iters)
        st0 = s.stats()
        t0 = time.perf_counter()
        st = s.step(iters)
        dt = time.perf_counter() - t0
        if kernel_iters > 0:
            k0 = s.stats()
            t = s.time_kernels(kernel_iters)
            k1 = s.stats()
            kt = (t, (k1["elements"] - k0["elements"]) / kernel_iters, (k1["applied"] - k0["applied"]) / kernel_iters)
    finally:
        s.close()
    el = st["elements"] - st0["elements"]
    out = {"value": el / dt, "unit": "elements/s", "us_per_iteration": dt / iters * 1e6,
           "elements_per_iteration": el / iters, "iterations": iters, "after_warmup_iterations": warm_iters,
           "reduced_eig_iterations_per_iteration": (st["reduced_iterations"] - st0["reduced_iterations"]) / iters,
           "energy": st["energy"], "load": st["load"]}
    if kt is not None:
        t, el_k, app_k = kt
        us = {k: v * 1e3 / kernel_iters for k, v in t.items()}
        peak, kind = measured_peaks()
        achieved = el_k * ALGO_BYTES_PER_ELEMENT / (us["scatter"] * 1e-6) / 1e9
        out["us_per_kernel"] = {k: round(v, 2) for k, v in us.items()}
        out["scatter_roofline"] = {"bound": "hbm", "achieved": achieved, "peak": peak, "peak_kind": kind,
                                   "unit": "GB/s", "frac": achieved / peak,
                                   "algorithmic_bytes_per_element": ALGO_BYTES_PER_ELEMENT,
                                   "elements_per_iteration": el_k, "iterations_timed": kernel_iters,
                                   "applied_per_iteration": app_k,
                                   "applied_per_s": app_k / (us["scatter"] * 1e-6)}
    return out


def timed_xcd_run(api, w, k1, tau, log2_capacity, warm_iters, iters) -> dict:
    """xCDFCI (Algorithm 3, K + 1 = k1 states) throughput: elements/s (one column of k1-wide
    updates per iteration) over `iters` iterations after `warm_iters`, and the energies."""
    s = api.Solver(w.h, w.g, w.N, w.n_alpha, w.n_beta, num_states=k1, z_threshold=tau,
                   log2_capacity=log2_capacity, ref_alpha=int(w.ref[0]), ref_beta=int(w.ref[1]))
    try:
        s.step(warm_iters)
        st0 = s.stats()
        t0 = time.perf_counter()
        st = s.step(iters)
        dt = time.perf_counter() - t0
        E = [float(x) for x in s.energies()]
    finally:
        s.close()
    el = st["elements"] - st0["elements"]
    return {"value": el / dt, "unit": "elements/s", "us_per_iteration": dt / iters * 1e6,
            "elements_per_iteration": el / iters, "iterations": iters, "after_warmup_iterations": warm_iters,
            "energies": E, "load": st["load"]}


def fci_dim(N: int, na: int, nb: int) -> int:
    import math
    return math.comb(N, na) * math.comb(N, nb)


def loop_kernel_name(st: dict, ips: int) -> str:
    """The m = 1 loop kernel the library launched, with its shape."""
    if st.get("grid_wide"):
        return f"k_cd_loop_grid (persistent cooperative grid of {st['grid_blocks']} CTAs, {ips} iterations per launch)"
    return f"k_cd_loop (persistent {st['grid_blocks']}-CTA cluster, {ips} iterations per launch)"


def c4_tables(w):
    """Table size and tau of a config-4 instance: the next power of two >= dim / 0.6, capped at 2^24;
    tau = 0 where the FCI space fits, else 1e-5."""
    import math
    dim = fci_dim(w.N, w.n_alpha, w.n_beta)
    need = dim / 0.6
    lc = max(10, min(24, math.ceil(math.log2(need))))
    return lc, (0.0 if need <= 2 ** 24 else 1e-5)


def column_length(w) -> int:
    import math
    va, vb = w.N - w.n_alpha, w.N - w.n_beta
    return (1 + w.n_alpha * va + w.n_beta * vb + math.comb(w.n_alpha, 2) * math.comb(va, 2) +
            math.comb(w.n_beta, 2) * math.comb(vb, 2) + w.n_alpha * va * w.n_beta * vb)


def c4_block_sizes(api, ws, seconds: float = 0.6) -> tuple:
    """m for every config-4 instance from cdfci_autotune: the tuner runs on the instances with the
    shortest, the median and the longest column, and every instance takes the choice of the nearest
    of them in column length, capped by its table (below)."""
    import math
    order = sorted(range(len(ws)), key=lambda i: column_length(ws[i]))
    reps = sorted({order[0], order[len(order) // 2], order[-1]})
    chosen = {}
    for i in reps:
        w = ws[i]
        lc, tau = c4_tables(w)
        p, _ = api.cdfci_autotune(w.h, w.g, w.N, w.n_alpha, w.n_beta, seconds=seconds, log2_capacity=lc,
                                  z_threshold=tau, ref_alpha=int(w.ref[0]), ref_beta=int(w.ref[1]))
        chosen[i] = max(p["num_coordinates"], 4)           # the batch's m > 1 path
    ms = []
    for w in ws:
        L = column_length(w)
        near = min(reps, key=lambda i: abs(column_length(ws[i]) - L))
        # a space larger than its capped table (tau > 0): early iterations insert nearly every element
        # (eta is large), so one iteration of m columns may fill at most 1/16 of the table:
        # m <= 0.79 capacity / (16 L), a power of two, at least 4 (a table that holds the whole space
        # cannot fill)
        lc, tau = c4_tables(w)
        cap_m = max(4, 1 << max(0, int(math.floor(math.log2(max(1.0, 0.79 * (1 << lc) / (16 * L)))))))
        ms.append(min(chosen[near], cap_m) if tau > 0 else chosen[near])
    return ms, {column_length(ws[i]): chosen[i] for i in reps}


def batch_c4(api, inputs, iters: int, grid_blocks: int = 1, ms=None) -> dict:
    """The uneven batch (64 ab initio + 32 Hubbard problems) stepped together: with ms = None every
    problem runs Algorithm 1 (one thread-block cluster of grid_blocks CTAs per problem, one persistent
    launch); otherwise problem k runs Algorithm 2 with m = ms[k], all problems as branches of one
    captured graph."""
    ws = inputs.config4_instances()
    solvers = []
    total_bytes = 0
    try:
        for k, w in enumerate(ws):
            lc, tau = c4_tables(w)
            total_bytes += (1 << lc) * 32
            # Algorithm 2 on a space larger than its capped table: the compression threshold search
            # keeps the table from filling (tau raised tenfold as the load passes 50 %, 75 %, ...)
            kw = dict(grid_blocks=grid_blocks) if ms is None else dict(num_coordinates=ms[k],
                                                                       z_threshold_search=1 if tau > 0 else 0)
            solvers.append(api.Solver(w.h, w.g, w.N, w.n_alpha, w.n_beta, log2_capacity=lc, z_threshold=tau,
                                      ref_alpha=int(w.ref[0]), ref_beta=int(w.ref[1]), **kw))
        b = api.Batch(solvers)
        try:
            b.step(20 if ms is None else 16)
            st0 = [s.stats() for s in solvers]
            t0 = time.perf_counter()
            st = b.step(iters)
            dt = time.perf_counter() - t0
        finally:
            b.close()
        el = sum(x["elements"] - y["elements"] for x, y in zip(st, st0))
        peak, _ = measured_peaks()
        out = {"value": el / dt, "unit": "elements/s", "problems": len(ws), "iterations_each": iters,
               "ms_per_batch_step": dt * 1e3, "tables_gib": total_bytes / 2 ** 30,
               "algorithmic_frac": el * ALGO_BYTES_PER_ELEMENT / dt / 1e9 / peak,
               "column_lengths": [min(x["last_column"] for x in st), max(x["last_column"] for x in st)],
               "energies": [round(x["energy"], 10) for x in st]}
        if ms is None:
            out.update(cluster_ctas_per_problem=grid_blocks, m=1, gpu_launches_timed=2)
        else:
            out.update(m=sorted(set(ms)), m_counts={m: ms.count(m) for m in sorted(set(ms))},
                       graph_launches_timed=iters // 8)
        return out
    finally:
        for s in solvers:
            s.close()


def adjoint_c5(api, inputs, m: int, iters: int) -> dict:
    """RDMs and dE/dh, dE/dg, dE/dkappa of a config-5 mCDFCI vector after `iters` iterations, and the
    largest relative difference from central differences (step 1e-5) of the vector's exact Rayleigh
    quotient under perturbed integrals (cdfci_energy_with), one random direction each for h, g, kappa."""
    import numpy as np
    import scipy.linalg
    w = inputs.config5()
    s = api.Solver(w.h, w.g, w.N, w.n_alpha, w.n_beta, num_coordinates=m, log2_capacity=25,
                   ref_alpha=int(w.ref[0]), ref_beta=int(w.ref[1]))

    def sym8(G):
        return (G + G.transpose(1, 0, 2, 3) + G.transpose(0, 1, 3, 2) + G.transpose(1, 0, 3, 2) +
                G.transpose(2, 3, 0, 1) + G.transpose(3, 2, 0, 1) + G.transpose(2, 3, 1, 0) +
                G.transpose(3, 2, 1, 0)) / 8

    def rotated(K):
        U = scipy.linalg.expm(K)
        h2 = U.T @ w.h @ U
        return 0.5 * (h2 + h2.T), sym8(np.einsum("ap,bq,cr,ds,abcd->pqrs", U, U, U, U, w.g, optimize=True))

    try:
        t0 = time.perf_counter()
        st = s.step(iters)
        t_solve = time.perf_counter() - t0
        t0 = time.perf_counter()
        dh, dg, dk = s.gradient()
        t_grad = time.perf_counter() - t0
        nnz = st["nnz_c"]
        rng = np.random.default_rng(7)
        eps = 1e-5
        D = rng.normal(size=(16, 16)); D = D + D.T
        G = sym8(rng.normal(size=(16, 16, 16, 16)))
        K = rng.normal(size=(16, 16)); K = K - K.T
        t0 = time.perf_counter()
        fd = {"h": (s.energy_with(w.h + eps * D, w.g) - s.energy_with(w.h - eps * D, w.g)) / (2 * eps),
              "g": (s.energy_with(w.h, w.g + eps * G) - s.energy_with(w.h, w.g - eps * G)) / (2 * eps),
              "kappa": (s.energy_with(*rotated(eps * K)) - s.energy_with(*rotated(-eps * K))) / (2 * eps)}
        t_fd = time.perf_counter() - t0
        an = {"h": float(np.sum(D * dh)), "g": float(np.sum(G * dg)), "kappa": 0.5 * float(np.sum(dk * K))}
        err = {k: abs(fd[k] - an[k]) / max(1.0, abs(fd[k])) for k in fd}
    finally:
        s.close()
    return {"workload": "abinitio_N16_5a5b_seed5 (FCI dim 19,079,424, column 4,236), m=%d" % m,
            "solve_iterations": iters, "solve_seconds": t_solve, "energy": st["energy"],
            "nonzeros_c": nnz, "gradient_seconds": t_grad,
            "rdm_lookups_per_s": nnz * 4236 / t_grad, "dE_dkappa_norm": float((dk ** 2).sum() ** 0.5),
            "trace_dE_dh": float(dh.trace()), "central_difference_rel_err": err,
            "central_difference_seconds": t_fd}


def time_to_energy(api, w, E_ref: float, m: int, check_every: int, log2_capacity: int, cap_s: float = 30.0):
    """Seconds from cdfci_create's return to the first check with |E - E_ref| <= 1e-6 Ha."""
    s = api.Solver(w.h, w.g, w.N, w.n_alpha, w.n_beta, num_coordinates=m, log2_capacity=log2_capacity,
                   ref_alpha=int(w.ref[0]), ref_beta=int(w.ref[1]))
    try:
        t0 = time.perf_counter()
        it = 0
        while time.perf_counter() - t0 < cap_s:
            st = s.step(check_every)
            it += check_every
            if abs(st["energy"] - E_ref) <= 1e-6:
                return {"seconds": time.perf_counter() - t0, "iterations": it, "check_every": check_every,
                        "elements": st["elements"]}
        return {"seconds": None, "iterations": it, "check_every": check_every, "note": f"not reached in {cap_s} s"}
    finally:
        s.close()


def time_to_e_batched_vs_plain(api, inputs) -> list:
    import math
    out = []
    cases = [("config1_hubbard_chain8_obc_U4", inputs.config1()),
             ("abinitio_N12_3a3b_seed2", inputs.ab_initio(12, 3, 3, seed=2)),
             ("abinitio_N10_4a4b_seed7", inputs.ab_initio(10, 4, 4, seed=7)),
             ("hubbard_chain10_obc_U4_5a5b", inputs.hubbard((10,), 5, 5, U=4.0, periodic=False))]
    for name, w in cases:
        E_ref = load_reference_energy(name)
        lc = max(12, math.ceil(math.log2(w.fci_dim / 0.6)))
        ref = dict(ref_alpha=int(w.ref[0]), ref_beta=int(w.ref[1]), log2_capacity=lc)
        t0 = time.perf_counter()
        tuned, rep = api.cdfci_autotune(w.h, w.g, w.N, w.n_alpha, w.n_beta, seconds=1.0, **ref)
        t_tune = time.perf_counter() - t0
        m = tuned["num_coordinates"]
        plain = time_to_energy(api, w, E_ref, 1, 2000, lc)
        batched = time_to_energy(api, w, E_ref, m, 16 if m > 1 else 2000, lc)
        out.append({"workload": f"{name} (FCI dim {w.fci_dim:,})", "E_ref": E_ref, "threshold_ha": 1e-6,
                    "plain_m1": plain, "batched": dict(batched, m=m, autotune_seconds=t_tune,
                                                       autotune_seconds_to_target=dict(zip(rep["m"], rep["score"])))})
    return out


def batched_summary(line: dict, probe: dict) -> dict:
    """The m = 128 scatter's roofline and the batched-vs-plain figures in a few scalars."""
    out = {}
    mc = line.get("mcdfci", {})
    sr = mc.get("scatter_roofline")
    if sr:
        out["mcdfci_scatter"] = {
            "workload": f"config 2 (N=24, 6+6, tau=1e-5), m=128, iterations {mc['after_warmup_iterations'] + mc['iterations']}.."
                        f"{mc['after_warmup_iterations'] + mc['iterations'] + sr['iterations_timed']}",
            "elements_per_iteration": round(sr["elements_per_iteration"]),
            "scatter_us": mc["us_per_kernel"]["scatter"], "iteration_us": round(mc["us_per_iteration"], 2),
            "achieved": round(sr["achieved"], 1), "frac": round(sr["frac"], 4),
            "applied_per_iteration": round(sr["applied_per_iteration"]),
            # elements that reach the table (applied: a slot read and an add each) per second of the
            # scatter, against the probe's independent random slots per second
            "applied_frac_of_slot_probe": round(sr["applied_per_s"] / probe["ops_per_s"], 4),
            "dram_bytes_per_element": profiled_traffic(SCATTER_PROFILE, SCATTER_SOURCES, "dram_bytes_per_element"),
            "kernel_source_hash": kernel_hash(SCATTER_SOURCES)}
    b = line.get("batch_96")
    if b:
        out["batch_96"] = {k: b.get(k) for k in ("value", "m_counts", "problems", "ms_per_batch_step",
                                                 "algorithmic_frac") if b.get(k) is not None}
        b1 = line.get("batch_96_m1")
        if b1:
            out["batch_96"]["m1_value"] = b1.get("value")
    ad = line.get("adjoint")
    if ad and "central_difference_rel_err" in ad:
        out["adjoint_c5_max_rel_err_vs_central_difference"] = max(ad["central_difference_rel_err"].values())
    hk = line.get("hubbard_k_4x4")
    if hk and "U4" in hk:
        out["hubbard_4x4_U4_seconds_to_paper_ed"] = hk["U4"].get("seconds_to_1e-5")
    tt = line.get("time_to_E_batched_vs_plain")
    if tt:
        out["time_to_E_s"] = [[x["workload"].split(" ")[0], x["plain_m1"].get("seconds"),
                               x["batched"].get("seconds"), x["batched"].get("m")] for x in tt]
    return out


def aggregate_ranks(ms: float, elements: float, dist=None, device: str = "cpu"):
    """Replicas: the slowest rank's time and all ranks' elements (weak scaling,
    no data-path collective; this reduction only reports)."""
    if dist is None:
        return ms, elements
    import torch
    t = torch.tensor([ms, elements], dtype=torch.float64, device=device)
    tmax, tsum = t.clone(), t.clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(tsum, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(tsum[1])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--iters-per-step", type=int, default=4000)
    ap.add_argument("--ref-iters-per-step", type=int, default=200)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-extras", action="store_true", help="only the device-timed value (for profiling)")
    ap.add_argument("--log2-capacity", type=int, default=WORKLOAD["log2_capacity"],
                    help="hash table size (smaller only for profiling captures)")
    ap.add_argument("--only", choices=["mcdfci", "xcdfci"], default=None,
                    help="run only the m = 128 block leg or the K + 1 = 4 xCDFCI leg on the same workload "
                         "(for profiling captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    if args.impl == "reference":
        run_reference_arm(args)
        return
    if args.only == "mcdfci":
        import __graft_entry__
        __graft_entry__.build()
        from paper_2605_04483_gb300 import api, inputs
        r = timed_block_run(api, inputs.config2(), 128, WORKLOAD["tau"], args.log2_capacity, args.warmup * 10,
                            args.iters_per_step, kernel_iters=min(200, args.iters_per_step))
        print(json.dumps({"mcdfci_m128": r}))
        return
    if args.only == "xcdfci":
        import __graft_entry__
        __graft_entry__.build()
        from paper_2605_04483_gb300 import api, inputs
        r = timed_xcd_run(api, inputs.config2(), 4, WORKLOAD["tau"], args.log2_capacity, args.warmup * 10,
                          args.iters_per_step)
        print(json.dumps({"xcdfci_k4": r}))
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        dist.barrier()
    from paper_2605_04483_gb300 import api, inputs

    w = inputs.config2()
    h_host = torch.tensor(w.h).pin_memory()
    g_host = torch.tensor(w.g).pin_memory()
    h_dev = h_host.cuda()
    g_dev = g_host.cuda()
    stream = torch.cuda.Stream()
    params = dict(log2_capacity=args.log2_capacity, z_threshold=WORKLOAD["tau"],
                  cuda_stream=stream.cuda_stream)
    ips = args.iters_per_step

    # ---- device-resident throughput -------------------------------------------------
    s = api.Solver(h_dev, g_dev, w.N, w.n_alpha, w.n_beta, **params)
    for _ in range(args.warmup):
        s.step(ips)
    st0 = s.stats()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        ev0.record(stream)
    for _ in range(args.steps):
        st = s.step(ips)
    with torch.cuda.stream(stream):
        ev1.record(stream)
    ev1.synchronize()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    elements = st["elements"] - st0["elements"]
    launches = st["iterations"] - st0["iterations"]
    ms_max, total_el = aggregate_ranks(ms, float(elements), dist if world > 1 else None, "cuda")
    value = total_el / (ms_max * 1e-3)
    final_energy = st["energy"]
    s.close()

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    peak, peak_kind = measured_peaks()
    # one k_cd_loop launch per step runs all its iterations (plus one small finalisation launch)
    loop_launches = args.steps
    avg_launch_s = ms * 1e-3 / loop_launches
    el_per_launch = elements / loop_launches
    achieved = el_per_launch * ALGO_BYTES_PER_ELEMENT / avg_launch_s / 1e9
    # DRAM bytes per iteration from the committed small-case capture (same column length per
    # iteration, so a launch's traffic grows in proportion to its iterations), times this launch's
    per_it = profiled_traffic(PROFILE_SUMMARY, KERNEL_SOURCES, "dram_bytes_per_iteration")
    traffic = None if per_it is None else per_it * ips
    probe = slot_probe(torch, api)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "slot_probe": {k: probe[k] for k in ("gbs_40B", "frac_40B", "sector_gbs_64B")},
                "traffic": traffic, "kernel": loop_kernel_name(st, ips),
                "algorithmic_bytes_per_launch": el_per_launch * ALGO_BYTES_PER_ELEMENT,
                "peak_kind": f"{peak_kind} HBM copy bandwidth (burst)"}

    line = {"metric": "H elements/s into hash b (CDFCI, Algorithm 1)", "value": value, "unit": "elements/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.log2_capacity),
                       "iters_per_step": ips, "column_length": 16471,
                       "l2": "inputs larger than L2 (4 GiB hash table), no flush",
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": roofline, "gpu_launches": int(2 * args.steps), "clocks": clk,
            "energy_after_timed_steps": final_energy,
            "us_per_iteration": ms / max(launches, 1) * 1e3, "iterations_timed": int(launches)}

    if not args.no_extras:
        # ---- end to end through the C-ABI from pinned host buffers ----------------------
        # the job as a user runs it: create from host h, g (H2D copy, table set-up, initial column),
        # then the same W + K steps of ips iterations as the device-timed run, the stats (energy) read
        # back to the host after every step; it covers iterations 0 .. (W + K) ips, the device-timed
        # window and the W warm-up steps before it
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s2 = api.Solver(h_host, g_host, w.N, w.n_alpha, w.n_beta, **params)
        for _ in range(args.warmup + args.steps):
            st2 = s2.step(ips)
        e_dt = time.perf_counter() - t0
        e_el = st2["elements"]
        s2.close()
        nst = args.warmup + args.steps
        line["e2e"] = {"value": e_el / e_dt, "unit": "elements/s",
                       "h2d_bytes_per_step": int((h_host.numel() * 8 + g_host.numel() * 8) / nst),
                       "d2h_bytes_per_step": int(__import__("ctypes").sizeof(api.cdfci_stats)),
                       "iterations": [0, nst * ips],
                       "note": f"create(host h, g) once ({int(h_host.numel() * 8 + g_host.numel() * 8)} B H2D) "
                               f"+ {nst} steps of {ips} iterations with a stats read each; wall clock"}
        # ---- time to E within 1e-6 Ha on the 8-site chain (stored exact energy) ------------
        wc = inputs.config1()
        E_ref = load_reference_energy("config1_hubbard_chain8_obc_U4")
        s3 = api.Solver(wc.h, wc.g, wc.N, wc.n_alpha, wc.n_beta, log2_capacity=16,
                        ref_alpha=int(wc.ref[0]), ref_beta=int(wc.ref[1]))
        t0 = time.perf_counter()
        it = 0
        reached = None
        while it < 400000:
            st3 = s3.step(1000)
            it += 1000
            if abs(st3["energy"] - E_ref) <= 1e-6:
                reached = time.perf_counter() - t0
                break
        s3.close()
        line["time_to_E"] = {"workload": "hubbard_chain8_obc_U4 (FCI dim 4,900), m=1", "threshold_ha": 1e-6,
                             "seconds": reached, "iterations": it, "check_every": 1000, "E_ref": E_ref}
        # ---- time to E within 1e-6 Ha: batched (autotuned m) vs plain (m = 1) -------------------
        line["time_to_E_batched_vs_plain"] = time_to_e_batched_vs_plain(api, inputs)
        # ---- batched coordinate updates (mCDFCI, Algorithm 2) on the same workload ------------
        line["mcdfci"] = dict(workload=WORKLOAD["name"] + f", tau={WORKLOAD['tau']}, m=128, 2^27-slot table",
                              **timed_block_run(api, w, 128, WORKLOAD["tau"], 27, 1000, 500, kernel_iters=200))
        # ---- excited states (xCDFCI, Algorithm 3), K + 1 = 4, same workload -------------------
        line["xcdfci"] = dict(workload=WORKLOAD["name"] + f", tau={WORKLOAD['tau']}, K+1=4 states, 2^26-slot table",
                              **timed_xcd_run(api, w, 4, WORKLOAD["tau"], 26, 500, 2000))
        # ---- 2D Hubbard 4x4 periodic, U=8, 8+8 (FCI dim 165,636,900), m=256, 2^28 slots ------------
        line["hubbard_4x4"] = dict(workload="hubbard_4x4_pbc_U8 (dim 1.66e8, column <= 65), m=256, 2^28-slot table",
                                   **timed_block_run(api, inputs.config3(8.0), 256, 0.0, 28, 100, 200, kernel_iters=50))
        # ---- the paper's k-space 4x4 lattice, half filling, degenerate start ------------------------
        try:
            kleg = hubbard_k_leg(api, inputs)
        except Exception as e:                       # an informational leg: report, keep the line
            kleg = {"error": f"{type(e).__name__}: {e}"}
        line["hubbard_k_4x4"] = dict(workload="hubbardk_4x4_pbc_8a8b (momentum basis, dim 1.66e8), m=128", **kleg)
        # ---- uneven batch of 96 problems: Algorithm 2 with autotuned m, one graph; and at m = 1 ----
        ws4 = inputs.config4_instances()
        try:                                           # informational legs: report, keep the line
            ms, tuned = c4_block_sizes(api, ws4)
            line["batch_96"] = dict(workload="64 ab initio (N 12..32, 3..8 electrons per spin) + 32 Hubbard "
                                             "problems, Algorithm 2 per problem (m autotuned), one graph per 8 "
                                             "iterations", **batch_c4(api, inputs, 200, ms=ms),
                                    autotuned_m_by_column_length=tuned)
        except Exception as e:
            line["batch_96"] = {"error": f"{type(e).__name__}: {e}"}
        try:
            line["batch_96_m1"] = dict(workload="the same 96 problems, m=1, one persistent launch (8-CTA cluster "
                                                "each)", **batch_c4(api, inputs, 200, 8))
        except Exception as e:
            line["batch_96_m1"] = {"error": f"{type(e).__name__}: {e}"}
        # ---- adjoint: RDMs and energy derivatives ----------------------------------------------
        line["adjoint"] = adjoint_c5(api, inputs, 512, 8000)
        # ---- compact copies of the batched paths' figures inside the roofline object ------------
        roofline.update(batched_summary(line, probe))
        if world == 1:
            line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
