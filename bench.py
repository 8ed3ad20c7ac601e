#!/usr/bin/env python3
"""Benchmark: one GKBA second-Born Heun step at N = 96 with a 2000-point history.

A step is one pass of the whole hot path through the C ABI (gkba_step): the
mean field, two collision integrals (history of n+1 and n+2 points: GKBA
reconstruction, the four-stage split-TF32 tensor-core contraction of
Eq. (2bse), the FP64 weighted history sum), the propagator exp(-i dt h), the
T(t,t_k) recursion and the Heun update.  Inputs are seeded and synthetic
(random Hermitian rho_k with eigenvalues in [0,1], T(t,t_k) products of
exp(-i H_j dt) with random Hermitian H_j, v from 64 Gaussian factors).

Printed JSON line (rank 0):
  value        algorithmic contraction TFLOP/s over the step (24 N^5 real flops
               per (t_k, component) unit; 2 (2n+3) units per step)
  e2e          the same metric for gkba_collision called with pinned host
               buffers (history copied host->device inside the timed region)
  roofline     the dominant stage kernel: its algorithmic flops per launch over
               its CUDA-event launch time, against the TF32 tensor peak
               (measured bf16 sustained peak x 1.1/2.25)
  cpu_baseline the CPU oracle on one (t_k, component) unit of the same workload
  fp64_path    the FP64 CUDA path timed on a 3-point history and extrapolated
               (cost is linear in the number of units), with the split-TF32
               error against it
  time_linear  the same Heun step with the time-linear history (FP64, the
               history sum kept as one N^4 accumulator; cost independent of L)

--impl reference times the CPU oracle (the reference arm) on a
bounded sample per step: one (t_k, component) unit at N = 96.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

TF32_OVER_BF16 = 1.1 / 2.25  # nominal dense TF32 / BF16 tensor rates (GB300)
METRIC = "GKBA-2B step time & contraction TFLOP/s (% peak), TC vs FP64 path at stated err"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--N", type=int, default=96)
    ap.add_argument("--L", type=int, default=2000)
    ap.add_argument("--nP", type=int, default=64)
    ap.add_argument("--dt", type=float, default=0.02)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-time-linear", action="store_true")
    ap.add_argument("--no-rho-check", action="store_true",
                    help="skip the stated-error leg (1000 config-1 steps against the FP64 path)")
    ap.add_argument("--precision", default="tf32", choices=["tf32", "tf32acc"],
                    help="split-TF32 mode of the timed step")
    ap.add_argument("--adjoint", action="store_true",
                    help="gradients of the final dipole at N=32, 800 steps (adjoint run)")
    ap.add_argument("--fd-samples", type=int, default=6,
                    help="field samples checked by finite differences (--adjoint)")
    ap.add_argument("--fd-dirs", type=int, default=32,
                    help="Coulomb-factor directions checked by finite differences (--adjoint)")
    ap.add_argument("--batch", action="store_true",
                    help="time 32 systems of uneven N and L stacked in one batch vs one by one")
    ap.add_argument("--chains", action="store_true",
                    help="time the Sec. IV propagations at N_b = 10 (Table I context)")
    ap.add_argument("--time-linear", action="store_true",
                    help="time gkba_step with the time-linear history (FP64) at N and exit")
    ap.add_argument("--profile-case", action="store_true",
                    help="run one split-TF32 collision over one history point at N "
                         "with a two-unit workspace (the small case for ncu captures) and exit")
    return ap.parse_args()


def unit_flops(N):
    return 24.0 * float(N) ** 5


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return dict(bf16_burst=d["bf16_tflops"], bf16_sustained=d["bf16_tflops_sustained"],
                    hbm=d["hbm_gbs"], src="measured")
    return dict(bf16_burst=1900.0, bf16_sustained=1700.0, hbm=6800.0, src="fallback")


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = max(mx, float(f[1]))
            except ValueError:
                continue
            for nm, val in zip(names, f[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_unit_sample(N, nP, seed=0):
    """Time the CPU oracle on one (t_k, component) unit of the workload: Eq.
    (2bse) through the paper's N^5 route, Eq. (2b-opt)."""
    import gkba_inputs as gi
    import oracle as O
    s = gi.system(N, nP, seed=seed)
    rho, T = gi.history(N, 2, 0.02, seed=seed)
    P = T[0] @ rho[0]
    Q = T[0] - P
    t0 = time.perf_counter()
    O.sigma_paper(s["v"], P, Q.conj().T)
    dt = time.perf_counter() - t0
    return dt


_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS",
                "BLIS_NUM_THREADS", "VECLIB_MAXIMUM_THREADS", "NUMEXPR_NUM_THREADS")


def oracle_unit_timed(N, nP, threads, seed=0):
    """oracle_unit_sample in a fresh interpreter whose BLAS and OpenMP thread
    pools are pinned to `threads` (set before numpy loads), so the core count
    of the CPU baseline is the one the oracle actually ran with."""
    env = dict(os.environ)
    for k in _THREAD_VARS:
        env[k] = str(threads)
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_unit_sample(%d, %d, %d)))" % (ROOT, N, nP, seed))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=900)
    if r.returncode != 0:
        raise RuntimeError("oracle timing failed: " + r.stderr[-500:])
    return float(r.stdout.strip().splitlines()[-1])


def rho_gate(P, precision, stream, n=1000):
    """The stated error of the timed mode on rho(t): the N = 24 model (32
    factors, seed 0, dt = 0.02, the pulse on [0, 10]) propagated n Heun steps
    in `precision` and on the FP64 path (its time-linear history, equal to the
    history sum up to rounding), max over steps of ||rho - rho_64|| / ||rho_64||."""
    import gkba_inputs as gi
    s = gi.system(24, 32, seed=0)
    dt = 0.02
    E = gi.field(dt * np.arange(n + 1))
    ref = P.Context(s["h"], s["v"], s["d"], s["rho0"], dt, max_steps=n, history="time_linear",
                    stream=stream.cuda_stream)
    tc = P.Context(s["h"], s["v"], s["d"], s["rho0"], dt, max_steps=n, precision=precision,
                   stream=stream.cuda_stream)
    worst, t0 = 0.0, time.perf_counter()
    for k in range(n):
        r64, _, _ = ref.step(E[k], E[k + 1])
        rtc, _, _ = tc.step(E[k], E[k + 1])
        worst = max(worst, float(np.linalg.norm(rtc - r64) / np.linalg.norm(r64)))
    wall = time.perf_counter() - t0
    ref.close()
    tc.close()
    return {"rho_rel_err_max_config1_1000_steps": worst, "rho_gate": 1e-5,
            "rho_check": f"N=24, 32 factors, dt=0.02, {n} Heun steps with the pulse, "
                         f"max over steps vs the FP64 GPU path ({wall:.1f} s)"}


def profile_case(a):
    """One split-TF32 collision over one history point (two units) at N: each
    stage kernel launches once on a batch of two units."""
    import gkba_inputs as gi
    from paper_1905_01180_gb300 import build as b
    b.build()
    import paper_1905_01180_gb300 as P
    N = a.N
    s = gi.system(N, a.nP, seed=0)
    rho, T = gi.history(N, 2, a.dt, seed=0)
    per_unit = 2 * 2 * (((N + 15) // 16) * 16) ** 4 * 4
    ctx = P.Context(s["h"], s["v"], s["d"], s["rho0"], a.dt, precision="tf32",
                    workspace_bytes=int(2.4 * per_unit) + (64 << 20))
    I = ctx.collision(rho[:1], T[:1], np.array([a.dt]))
    ctx.close()
    print(json.dumps({"profile_case": f"N={N}, 2 units", "max_abs_I": float(np.abs(I).max())}))


def captured_traffic(kernel, units_per_launch):
    """DRAM bytes per launch of the kernel class `kernel`, scaled by units from
    a committed ncu summary line 'dram_bytes_per_unit[<class>]: <bytes>' under
    profiles/ (kernels whose traffic is proportional to the units), or None."""
    import glob
    import re
    pat = re.compile(r"dram_bytes_per_unit\[" + re.escape(kernel) + r"\]:\s*([0-9.eE+]+)")
    for f in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        m = pat.search(open(f).read())
        if m:
            return float(m.group(1)) * units_per_launch, os.path.basename(f)
    return None, None


def job_timing(ms_local, units_local, dist=None):
    """Whole-job timing over replicas: the slowest rank's time and the units
    all ranks processed (each rank runs its own history, weak scaling)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms_local, units_local
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms_local], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([units_local], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def run_reference(a, rank, world):
    if rank != 0:
        return
    N = a.N
    import gkba_inputs  # noqa: F401  (warm imports outside the timed region)
    times = []
    cores = os.cpu_count() or 1
    for i in range(a.warmup + a.steps):
        t = oracle_unit_timed(N, a.nP, cores, seed=i)
        if i >= a.warmup:
            times.append(t)
    ms = 1e3 * float(np.mean(times))
    val = unit_flops(N) / (ms * 1e-3) / 1e12
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s",
        "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"gkba2b_heun_step_N{N}_L{a.L}", "N": N, "n_P": a.nP, "L": a.L,
                   "dt": a.dt, "parallelism": "replicas"},
        "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                         "threads": f"BLAS/OpenMP pools pinned to {cores} threads",
                         "sample": f"one (t_k, component) unit of Eq. (2bse) at N={N} per step "
                                   "through the paper's N^5 route, Eq. (2b-opt)"},
        "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_chains(a):
    """The paper's Sec. IV propagations at N_b = 10, each a whole GKBA run of
    N_t Heun steps through gkba_step (field-free, from the initial state):
    (1) Hubbard chain, diagonal basis, 5000 x 0.01; (2) Ohno chain, symmetric
    basis, 2000 x 0.025; (3) general basis (the seeded stand-in for the CH4
    integrals, 2 occupied orbitals), 1000 x 0.05, also with the time-linear
    history (FP64 and split-TF32).  One JSON line per run; the paper's single-core CPU times
    (Table I, tensor-contraction column) are context, not a target."""
    import torch
    import gkba_inputs as gi
    from paper_1905_01180_gb300 import build as b
    b.build()
    import paper_1905_01180_gb300 as P
    cases = [("hubbard_chain_N10", "diagonal", 0.01, 5000, "fp64", "sum", 164.0),
             ("ohno_chain_N10", "symmetric", 0.025, 2000, "fp64", "sum", 731.0),
             ("general_basis_N10", "general", 0.05, 1000, "fp64", "sum", 1333.0),
             ("general_basis_N10", "general", 0.05, 1000, "tf32acc", "sum", 1333.0),
             ("general_basis_N10", "general", 0.05, 1000, "fp64", "time_linear", 1333.0),
             ("general_basis_N10", "general", 0.05, 1000, "tf32", "time_linear", 1333.0)]
    for name, kind, dt, n, prec, history, paper in cases:
        s = gi.system(10, 8, seed=0) if kind == "general" else gi.chain(10, kind)
        ctx = P.Context(s["h"], s["v"], s["d"], s["rho0"], dt, max_steps=n, precision=prec,
                        interaction=kind, history=history)
        tr0 = float(np.trace(s["rho0"]).real)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tr, en = [], []
        for _ in range(n):
            _, _, diag = ctx.step(0.0, 0.0)
            tr.append(diag[0])
            en.append(diag[1])
        wall = time.perf_counter() - t0
        _, launches = ctx.stats(reset=True)
        ctx.close()
        print(json.dumps({"workload": name, "metric": "GKBA propagation wall time (N_t steps)",
                          "value": wall, "unit": "s", "higher_is_better": False,
                          "interaction": kind, "precision": prec, "history": history,
                          "N": 10, "steps": n, "dt": dt,
                          "ms_per_step": 1e3 * wall / n, "gpu_launches": launches,
                          "trace_drift": float(np.abs(np.array(tr) - tr0).max()),
                          "energy_drift": float(np.abs(np.array(en) - en[0]).max()),
                          "paper_table1_s": paper,
                          "paper_hardware": "Intel i5-4460, 1 core, NumPy/Armadillo (context)"}),
              flush=True)


def time_linear_sample(P, s, N, dt, stream, warmup, steps, precision="fp64"):
    """gkba_step with cfg.history = GKBA_HISTORY_TIME_LINEAR at N: the history
    sum kept as one N^4 accumulator (FP64), so a step's cost does not depend on
    the history length; its contractions in FP64 or on the tensor cores
    (split-TF32).  `warmup` steps from the initial state, then `steps` timed
    steps (CUDA events on the context's stream); the per-step work is the same
    at any step index."""
    import torch
    ctx = P.Context(s["h"], s["v"], s["d"], s["rho0"], dt, max_steps=warmup + steps + 1,
                    precision=precision, stream=stream.cuda_stream, timing=True,
                    history="time_linear")
    for _ in range(warmup):
        ctx.step(0.0, 0.0)
    ctx.stats(reset=True)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(steps):
        _, _, diag = ctx.step(0.0, 0.0)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    stats, launches = ctx.stats(reset=True)
    ctx.close()
    flops = sum(v["flops"] for v in stats.values()) / steps
    return {"ms_per_step": ms, "flops_per_step": flops,
            "tflops": flops / (ms * 1e-3) / 1e12, "gpu_launches": launches,
            "classes": {k: {"ms": v["ms"] / steps, "launches": v["launches"] // steps}
                        for k, v in stats.items() if v["launches"]},
            "trace": float(diag[0])}


def run_time_linear(a):
    """The time-linear step alone at N (see time_linear_sample), FP64 and split-TF32."""
    import torch
    import gkba_inputs as gi
    from paper_1905_01180_gb300 import build as b
    b.build()
    import paper_1905_01180_gb300 as P
    N, dt = a.N, a.dt
    s = gi.system(N, a.nP, seed=0)
    for prec in ("fp64", "tf32"):
        r = time_linear_sample(P, s, N, dt, torch.cuda.current_stream(), a.warmup, a.steps, prec)
        print(json.dumps({"workload": f"gkba_time_linear_step_N{N}", "metric": "GKBA Heun step time",
                          "value": r["ms_per_step"] / 1e3, "unit": "s", "higher_is_better": False,
                          "precision": prec, "history": "time_linear", "N": N, "n_P": a.nP,
                          "steps": a.steps, "warmup": a.warmup, **r}), flush=True)


def run_batch(a):
    """Many systems of uneven size and history length: 32 seeded systems with
    N in {8, 12, 16, 24, 32, 48} and L in U[500, 3000] (then U[20, 200]), one Heun step each
    (after one warm-up step), split-TF32.  The stacked batch (gkba_batch_step)
    against the same systems stepped one after another (each alone on the GPU
    with the default workspace).  Histories: the last L points of one seeded
    history per N (a valid history of L points)."""
    from paper_1905_01180_gb300 import build as b
    b.build()
    for lo, hi in ((500, 3000), (20, 200)):
        run_batch_case(a, lo, hi)


def run_batch_case(a, lo, hi):
    import torch
    import gkba_inputs as gi
    import paper_1905_01180_gb300 as P
    rng = np.random.default_rng(7)
    Ns = rng.choice([8, 12, 16, 24, 32, 48], size=32)
    Ls = rng.integers(lo, hi + 1, size=32)
    dt = 0.02
    hist = {int(N): gi.history(int(N), int(Ls[Ns == N].max()) + 2, dt, seed=100 + int(N))
            for N in sorted(set(Ns.tolist()))}

    def make(i):
        N, L = int(Ns[i]), int(Ls[i])
        s = gi.system(N, 8, seed=i)
        rho, T = hist[N]
        ctx = P.Context(s["h"], s["v"], s["d"], s["rho0"], dt, max_steps=L + 2, precision="tf32")
        ctx.set_history(L - 1, rho[-L:], T[-L:])
        return ctx

    # units of the timed step: history of n + 1 = L + 1 and n + 2 points (after the warm-up)
    flops = float(sum(2 * (2 * (int(L) + 1) + 1) * 24.0 * int(N) ** 5 for N, L in zip(Ns, Ls)))

    def batched(use_graph, tune):
        ctxs = [make(i) for i in range(32)]
        with P.Batch(ctxs) as bt:
            bt.set_options(use_graph=use_graph)
            tuned = bt.autotune() if tune else None
            bt.step(0.0, 0.0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            bt.step(0.0, 0.0)
            t = time.perf_counter() - t0
        for c in ctxs:
            c.close()
        return t, tuned

    t_batch, _ = batched(False, False)
    t_graph, _ = batched(True, False)
    t_tuned, tuned = batched(True, True)
    t_seq = 0.0
    for i in range(32):
        c = make(i)
        c.step(0.0, 0.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c.step(0.0, 0.0)
        t_seq += time.perf_counter() - t0
        c.close()
    best = min(t_batch, t_graph, t_tuned)
    print(json.dumps({"workload": f"32_systems_N8-48_L{lo}-{hi}_one_step",
                      "metric": "contraction TFLOP/s over one Heun step of all systems",
                      "value": flops / t_tuned / 1e12, "unit": "TFLOP/s", "higher_is_better": True,
                      "batched_autotuned_graph_s": t_tuned, "batched_graph_s": t_graph,
                      "batched_eager_s": t_batch, "one_by_one_s": t_seq,
                      "speedup": t_seq / t_tuned, "speedup_best": t_seq / best,
                      "one_by_one_tflops": flops / t_seq / 1e12, "precision": "split_tf32",
                      "autotuned": tuned,
                      "N": sorted(Ns.tolist()), "L_range": [int(Ls.min()), int(Ls.max())],
                      "algorithmic_flops": flops}), flush=True)


def dipole_fd_forward(P, s, dt, E, B=None):
    """Final dipole Re Tr[d rho(t_n)] of an FP64 propagation with the history
    sum kept as one N^4 accumulator (the same discrete trajectory as the
    history-sum stepper up to rounding), for central finite differences."""
    v = s["v"] if B is None else np.ascontiguousarray(np.einsum("pil,pjk->ijkl", B, B))
    n = len(E) - 1
    ctx = P.Context(s["h"], v, s["d"], s["rho0"], dt, max_steps=n, precision="fp64",
                    history="time_linear")
    for k in range(n):
        rho, _, _ = ctx.step(E[k], E[k + 1])
    ctx.close()
    return float(np.real(np.trace(s["d"] @ rho)))


def run_adjoint(a):
    """Gradients of the final dipole L = Re Tr[d rho(T)] at N = 32 with 32
    Coulomb factors, 800 Heun steps of dt = 0.025 under the pulse E(t) of the
    seeded generator: dL/dE(t_k) for all 801 samples and dL/dB^P for the 32
    factors, from the split-TF32 forward (history sum) and gkba_adjoint over
    the recorded trajectory.  Checked by central finite differences (h = 1e-6)
    of FP64 propagations (time-linear history) on a subset of the samples and
    on one symmetric direction per factor."""
    import torch
    import gkba_inputs as gi
    from paper_1905_01180_gb300 import build as b
    b.build()
    import paper_1905_01180_gb300 as P
    from paper_1905_01180_gb300 import gkba
    N, nP, n, dt = 32, 32, 800, 0.025
    s = gi.system(N, nP, seed=0)
    E = gi.field(np.arange(n + 1) * dt)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx = P.Context(s["h"], s["v"], s["d"], s["rho0"], dt, max_steps=n, precision=a.precision)
    for k in range(n):
        rho, _, _ = ctx.step(E[k], E[k + 1])
    t1 = time.perf_counter()
    E_bar, rho0_bar, vb = ctx.adjoint(s["d"], want_v=True)
    t2 = time.perf_counter()
    ctx.close()
    L = float(np.real(np.trace(s["d"] @ rho)))
    B_bar = gkba.coulomb_factor_grad(s["B"], vb)
    h = 1e-6
    t3 = time.perf_counter()
    L64 = dipole_fd_forward(P, s, dt, E)
    fdE = {}
    for k in [int(x) for x in np.linspace(0, 400, a.fd_samples)]:
        Ep, Em = E.copy(), E.copy()
        Ep[k] += h
        Em[k] -= h
        fdE[k] = (dipole_fd_forward(P, s, dt, Ep) - dipole_fd_forward(P, s, dt, Em)) / (2 * h)
    rng = np.random.default_rng(3)
    fdB = []
    for Pf in range(min(nP, a.fd_dirs)):
        X = rng.normal(size=(N, N))
        D = np.zeros_like(s["B"])
        D[Pf] = 0.5 * (X + X.T)
        fd = (dipole_fd_forward(P, s, dt, E, s["B"] + h * D)
              - dipole_fd_forward(P, s, dt, E, s["B"] - h * D)) / (2 * h)
        fdB.append((Pf, float(np.sum(B_bar * D)), fd))
    t4 = time.perf_counter()
    errE = max(abs(E_bar[k] - f) for k, f in fdE.items()) / max(abs(f) for f in fdE.values())
    errB = max(abs(ad - fd) for _, ad, fd in fdB) / max(abs(fd) for _, _, fd in fdB)
    print(json.dumps({
        "workload": f"gkba_adjoint_N{N}_nP{nP}_{n}_steps_dt{dt}",
        "metric": "gradient of the final dipole w.r.t. all field samples and Coulomb factors",
        "value": t2 - t0, "unit": "s", "higher_is_better": False,
        "forward_s": t1 - t0, "adjoint_s": t2 - t1, "precision": a.precision,
        "L_split_tf32": L, "L_fp64": L64, "L_rel_diff": abs(L - L64) / abs(L64),
        "fd": {"h": h, "forward": "fp64, time-linear history", "seconds": t4 - t3,
               "E_samples": {str(k): [float(E_bar[k]), f] for k, f in fdE.items()},
               "E_max_rel_err": errE,
               "B_directions": [[p_, ad, fd] for p_, ad, fd in fdB],
               "B_max_rel_err": errB},
        "E_bar_norm": float(np.linalg.norm(E_bar)), "B_bar_norm": float(np.linalg.norm(B_bar)),
        "data": "synthetic (seeded generator, seed 0)"}), flush=True)


def main():
    a = parse()
    if a.adjoint:
        run_adjoint(a)
        return
    if a.batch:
        run_batch(a)
        return
    if a.chains:
        run_chains(a)
        return
    if a.time_linear:
        run_time_linear(a)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        run_reference(a, rank, world)
        return
    if a.profile_case:
        profile_case(a)
        return

    import torch
    import gkba_inputs as gi
    from paper_1905_01180_gb300 import build as b
    b.build()
    import paper_1905_01180_gb300 as P

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    N, L, dt = a.N, a.L, a.dt
    s = gi.system(N, a.nP, seed=0)
    rho_h, T_h = gi.history(N, L, dt, seed=1 + rank)
    stream = torch.cuda.current_stream()
    steps_total = a.warmup + a.steps
    ctx = P.Context(s["h"], s["v"], s["d"], s["rho0"], dt, max_steps=L - 1 + steps_total + 1,
                    precision=a.precision, stream=stream.cuda_stream, timing=True)
    ctx.set_history(L - 1, rho_h, T_h)

    for _ in range(a.warmup):
        ctx.step(0.0, 0.0)
    ctx.stats(reset=True)

    clocks = Clocks(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n0 = L - 1 + a.warmup
    ev0.record(stream)
    for _ in range(a.steps):
        ctx.step(0.0, 0.0)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    ms_local = ev0.elapsed_time(ev1)
    stats, launches = ctx.stats(reset=True)
    units = sum(2 * (2 * (n0 + k) + 3) for k in range(a.steps))
    ms_total, units_job = job_timing(ms_local, units, dist)
    value = units_job * unit_flops(N) / (ms_total * 1e-3) / 1e12
    ms_step = ms_total / a.steps

    # roofline: dominant stage kernel over the timed region.  Peak: the larger of
    # the TF32 rate derived from the measured bf16 peak and the tcgen05 kind::tf32
    # MMA rate measured now on this GPU (gkba_measure_tf32_mma, the stage
    # kernels' MMA shape with nothing else running).
    pk = peaks()
    tf32_derived = pk["bf16_sustained"] * TF32_OVER_BF16
    tf32_mma = ctx.measure_tf32_mma(100000)
    tf32_peak = max(tf32_derived, tf32_mma)
    stage = {k: v for k, v in stats.items() if k.startswith("S") and v["launches"] > 0}
    dom = max(stage, key=lambda k: stage[k]["ms"])
    d = stage[dom]
    achieved = d["flops"] / (d["ms"] * 1e-3) / 1e12
    units_per_launch = units / d["launches"]  # (t_k, component) units per launch of dom
    traffic, traffic_src = captured_traffic(dom, units_per_launch)
    # Compulsory bytes (what the problem itself must move): per collision the v
    # and w tensors (16 N^4 B), the rho / T history (2 x 16 N^2 B per point) and
    # I; per step two collisions.  Materialised bytes: what the kernels stream by
    # design (the N^4 intermediates of every unit), from the library's counters.
    L_avg = n0 + 1.5 + (a.steps - 1) / 2.0
    compulsory_step = 2.0 * (16.0 * N ** 4 + 2 * L_avg * 16.0 * N ** 2 + 16.0 * N ** 2)
    materialised_step = sum(v["bytes"] for v in stage.values()) / a.steps
    roof = {"bound": "tensor", "kernel": dom, "achieved": achieved, "peak": tf32_peak,
            "unit": "TFLOP/s", "frac": achieved / tf32_peak,
            "executed_frac": 3.0 * achieved / tf32_peak,
            "peak_source": ("tcgen05 kind::tf32 MMA rate measured in this run"
                            if tf32_mma >= tf32_derived else
                            f"bf16 sustained ({pk['src']}) x 1.1/2.25"),
            "peak_candidates": {"tf32_mma_measured": tf32_mma, "tf32_from_bf16": tf32_derived},
            "peak_note": "executed_frac counts the 3 TF32 products per algorithmic product",
            "traffic": traffic, "traffic_unit": "bytes per launch",
            "traffic_source": traffic_src,
            "algorithmic_bytes_per_launch": compulsory_step * units_per_launch / (units / a.steps),
            "algorithmic_bytes_note": "the step's compulsory bytes apportioned by units",
            "bytes_per_step": {"compulsory": compulsory_step, "materialised": materialised_step,
                               "materialised_over_compulsory": materialised_step / compulsory_step},
            "ms_per_launch": d["ms"] / d["launches"], "launches": d["launches"],
            "share": d["ms"] / sum(v["ms"] for v in stage.values()),
            "stages": {k: {"ms": v["ms"], "tflops": v["flops"] / max(v["ms"], 1e-9) / 1e9,
                           "launches": v["launches"]} for k, v in stage.items()}}

    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "tf32x3+f64", "data": "synthetic",
        "config": {"workload": f"gkba2b_heun_step_N{N}_L{L}", "N": N, "n_P": a.nP, "L": L,
                   "dt": dt, "precision": {"tf32": "split_tf32", "tf32acc": "split_tf32_acc"}[a.precision],
                   "acc_window": 32, "stated_err": {},
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "inputs larger than L2 (per-unit intermediates 680 MB each)",
                   "units_per_step": units / a.steps},
        "gpu_launches": launches,
        "roofline": roof,
        "clocks": clk,
    }

    if rank == 0 and not a.no_e2e:
        # e2e: gkba_collision with pinned host buffers, copies inside the timed region
        Lh = L
        rh = torch.from_numpy(rho_h).pin_memory()
        th = torch.from_numpy(T_h).pin_memory()
        Iout = torch.empty((N, N), dtype=torch.complex128).pin_memory()
        e0 = time.perf_counter()
        ctx.collision(rh.numpy(), th.numpy())
        e_s = time.perf_counter() - e0
        line["e2e"] = {"value": 2 * Lh * unit_flops(N) / e_s / 1e12, "unit": "TFLOP/s",
                       "h2d_bytes_per_step": int(rh.numel() * 16 + th.numel() * 16),
                       "d2h_bytes_per_step": int(Iout.numel() * 16),
                       "call": f"gkba_collision(L={Lh}) host buffers"}
    ctx.close()

    if rank == 0 and not a.no_fp64:
        Ls = 3
        c64 = P.Context(s["h"], s["v"], s["d"], s["rho0"], dt, precision="fp64",
                        stream=stream.cuda_stream)
        ctc = P.Context(s["h"], s["v"], s["d"], s["rho0"], dt, precision=a.precision,
                        stream=stream.cuda_stream)
        r3, t3 = rho_h[:Ls].copy(), T_h[:Ls].copy()
        I64 = c64.collision(r3, t3)  # warm
        torch.cuda.synchronize()
        e0 = time.perf_counter()
        I64 = c64.collision(r3, t3)
        t64 = time.perf_counter() - e0
        Itc = ctc.collision(r3, t3)
        err = float(np.linalg.norm(Itc - I64) / np.linalg.norm(I64))
        per_unit = t64 / (2 * Ls)
        ms64 = 1e3 * per_unit * units / a.steps
        fp = {"sample": f"collision over {Ls} history points ({2 * Ls} units) at N={N}",
              "extrapolated_from_units": 2 * Ls,
              "ms_per_step_extrapolated": ms64,
              "tflops": unit_flops(N) / per_unit / 1e12,
              "speedup_split_tf32": ms64 / ms_step,
              "speedup_note": "FP64 path time per unit x units per step (cost is linear in the "
                              "units), over the measured split-TF32 step",
              "split_tf32_rel_err_I": err}
        # kept inside recorded objects: the metric is quoted at a stated error
        line["roofline"]["fp64_path"] = fp
        line["config"]["stated_err"]["I_rel_err_vs_fp64_path"] = err
        c64.close()
        ctc.close()

    if rank == 0 and not a.no_rho_check:
        line["config"]["stated_err"].update(rho_gate(P, a.precision, stream))

    if rank == 0 and not a.no_time_linear:
        # the same Heun step with the history sum kept as one N^4 accumulator
        # (FP64; its cost does not depend on L)
        r = time_linear_sample(P, s, N, dt, stream, 1, 2)
        r32 = time_linear_sample(P, s, N, dt, stream, 1, 3, a.precision)
        line["time_linear"] = {"fp64": {"ms_per_step": r["ms_per_step"], "tflops": r["tflops"],
                                        "speedup_vs_history_sum_step": ms_step / r["ms_per_step"]},
                               "split_tf32": {"ms_per_step": r32["ms_per_step"], "tflops": r32["tflops"],
                                              "precision": a.precision,
                                              "speedup_vs_history_sum_step": ms_step / r32["ms_per_step"]},
                               "sample": f"2-3 steps after 1 warm-up from rho0 at N={N} "
                                         "(per-step work independent of the history length)"}

    if rank == 0 and not a.no_cpu:
        ncpu = os.cpu_count() or 1
        t_all = oracle_unit_timed(N, a.nP, ncpu)
        t_one = oracle_unit_timed(N, a.nP, 1)
        line["cpu_baseline"] = {"value": unit_flops(N) / t_all / 1e12, "unit": "TFLOP/s",
                                "cores": ncpu, "kind": "oracle",
                                "threads": f"BLAS/OpenMP pools pinned to {ncpu} threads",
                                "one_core": {"value": unit_flops(N) / t_one / 1e12, "cores": 1,
                                             "s": t_one},
                                "sample": f"one (t_k, component) unit of Eq. (2bse) at N={N} "
                                          f"through the paper's N^5 route, Eq. (2b-opt) "
                                          f"({t_all:.1f} s on {ncpu} threads, {t_one:.1f} s on 1)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
