#!/usr/bin/env python
"""Throughput of the multi-product imaginary-time step on GB300.

One step = itp_propagate (order-2k multi-product propagator on all states,
Eq. 3) + itp_orthonormalize (Eq. 4) + itp_energies with the Ritz values of
the subspace (the rotation onto Ritz vectors does not change the span, so it
is left to the read-out).
The metric is state-steps per second: (n + guard states) x steps / time.

Default workload: the C60-like Gaussian well on a 128^3 grid (box 32 bohr),
n = 120 wanted + 8 guard states, order 12, tau = 0.25, in the mixed form
(FP32 FFT passes; FP64 combination, Cholesky and energies).  The FP64 form
of the same workload is measured beside it.  Inputs are seeded and
synthetic (itp_workloads).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload (the reference arm; there is no other implementation to run).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

if "--impl" in sys.argv and "reference" in sys.argv or "--cpu-sample" in sys.argv:
    # the oracle leg runs single-threaded (numpy FFT is; pin BLAS too)
    for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[_v] = "1"

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "c60_128": dict(n=128, box=32.0, potential="c60", n_states=120, n_guard=8, order=12,
                    tau=0.25, seed=1234,
                    desc="C60-like Gaussian well (60 wells, depth 2.0 Ha, sigma 0.8 bohr, "
                         "radius 6.7 bohr), 128^3 grid, box 32 bohr, n=120 + 8 guard states, "
                         "order 12 (k_i = 1..6), tau = 0.25"),
    # the same grid and potential with 16 states: a case small enough for
    # full ncu captures (the half spectrum, 136 MB, still exceeds L2)
    "c60_128_m16": dict(n=128, box=32.0, potential="c60", n_states=16, n_guard=0, order=12,
                        tau=0.25, seed=1234,
                        desc="C60-like Gaussian well, 128^3 grid, box 32 bohr, 16 states, "
                             "order 12, tau = 0.25 (profiling case)"),
    # 128 states on a 64^3 grid: the tensor-core kernels' full tile height with
    # a state block (134 MB FP32) just above L2, small enough for full ncu captures
    "c60_64_m128": dict(n=64, box=32.0, potential="c60", n_states=120, n_guard=8, order=12,
                        tau=0.25, seed=1234,
                        desc="C60-like Gaussian well, 64^3 grid, box 32 bohr, 120 + 8 states, "
                             "order 12, tau = 0.25 (profiling case of the tensor-core kernels)"),
    "ho_32": dict(n=32, box=16.0, potential="ho", n_states=10, n_guard=2, order=4, tau=0.1,
                  seed=1234, desc="3D harmonic oscillator, 32^3 grid, box [-8,8)^3, n=10 + 2 "
                                  "guard, order 4, tau = 0.1"),
}


def make_inputs(w, rank=0):
    from itp_workloads import build_native, c60_like_potential, cubic, harmonic_potential, \
        normal_states
    try:
        build_native()
    except Exception:
        pass
    g = cubic(w["n"], w["box"])
    V = c60_like_potential(g) if w["potential"] == "c60" else harmonic_potential(g)
    m = w["n_states"] + w["n_guard"]
    psi = normal_states(m, g.n_points, seed=w["seed"], problem=rank)
    return g, V, psi


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum)
# from ncu captures summarised in profiles/, scaled to the full launch by the
# number of states, with the SHA-1 of the kernel source the counters were
# taken on: a kernel changed since then reports no traffic.
NCU_TRAFFIC = {
    # DRAM bytes (read + write) per full launch from one ncu capture of the
    # 16-state case, scaled by the number of states; valid only while the
    # kernel's source file is the one that was profiled
    ("c60_128", "plane_merged"): {"bytes": 1.784e9,
                                  "source": "paper_0809_3739_gb300/csrc/fft_passes.cuh",
                                  "sha1": "6982298585d4fd2f311b2719a76cc47cd560377c",
                                  "profile": "profiles/plane_merged_c60_128.md"},
    ("c60_128", "pencil"): {"bytes": 1.697e9,
                            "source": "paper_0809_3739_gb300/csrc/fft_tmem.cuh",
                            "sha1": "5657d3abdd160f6831798c09342aa04ad0083a70",
                            "profile": "profiles/pencil_tmem_c60_128.md"},
}


def max_over_ranks(x, device="cuda"):
    """The largest value of x over all ranks (x itself without a process
    group): every replica's time is taken as the slowest rank's."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replicas_value(units_per_rank, seconds, world):
    """Whole-job throughput of `world` independent replicas that each
    processed units_per_rank units, over the slowest rank's seconds."""
    return world * units_per_rank / seconds


def ncu_traffic(workload, kind):
    import hashlib
    rec = NCU_TRAFFIC.get((workload, kind))
    if rec is None:
        return None
    try:
        with open(os.path.join(ROOT, rec["source"]), "rb") as f:
            if hashlib.sha1(f.read()).hexdigest() != rec["sha1"]:
                return None
    except OSError:
        return None
    return rec["bytes"]


def measure_peaks(P):
    """The GPU's measured arithmetic rates (itp_peak_probe: FP32 FMA, packed
    FP32 FMA, FP64 FMA, tcgen05 TF32 MMA), with the SM clocks sampled while
    the probes run."""
    clocks = ClockSampler()
    clocks.begin()
    out = {}
    for kind in ("ffma", "ffma2", "dfma", "tf32_mma"):
        try:
            t, ms = P.itp_peak_probe(kind)
            out[f"{kind}_tflops"] = round(t, 2)
            out[f"{kind}_ms"] = round(ms, 2)
        except Exception as ex:   # an auxiliary figure never takes the bench line down
            out[f"{kind}_error"] = f"{type(ex).__name__}: {ex}"
    out["clocks"] = clocks.stop()
    out["how"] = ("itp_peak_probe: long chains of independent operations on every SM, best of "
                  "3 launches (CUDA events); an FMA counts 2 flops, an MxNxK MMA 2MNK")
    return out


def fft_pass_flops(kind, g, m):
    """Algorithmic flops of one FFT pass over m states: a complete complex
    FFT of length L counts 5 L log2 L, a real one half that; the plane pass
    does the 2D real transform(s) of its plane (two for the merged pass),
    the pencil pass a forward and an inverse complex transform along z of
    each of the nx/2+1 columns, plus one multiply per point for the factors."""
    import math
    P2 = g.nx * g.ny
    Nh = g.nz * g.ny * (g.nx // 2 + 1)
    real2d = 2.5 * P2 * math.log2(P2) if P2 > 1 else 0.0
    zfft = 5.0 * g.nz * math.log2(g.nz) if g.nz > 1 else 0.0
    per = {"plane_merged": 2 * real2d + P2, "plane_fwd": real2d + P2,
           "plane_combine": real2d + 3 * P2, "plane_hpsi": real2d + 2 * P2}
    if kind in per:
        return m * g.nz * per[kind]
    if kind in ("pencil", "pencil_kinetic"):
        return m * (Nh // g.nz) * (2 * zfft + 2 * g.nz)
    return None


def _hbm_peak():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    except Exception:
        return 6800.0


def algorithmic_bytes(kind, g, m, s, mixed=False):
    """Bytes a launch of `kind` must move over m states (s = bytes per real):
    every pass reads and writes the half spectrum once; the potential factor
    is read once per launch.  mixed: the FP32 path's forms of the last pass
    of a term (the term's contribution c_i f u_i written over its own plane)
    and of H psi (FP32 output, FP32 potential)."""
    N = g.n_points
    Nh = g.nz * g.ny * (g.nx // 2 + 1)
    spec = m * Nh * 2 * s
    return {
        "pencil": 2 * spec,
        "plane_merged": 2 * spec + N * s,
        "plane_fwd": m * N * s + N * s + spec,
        "plane_combine": (spec + N * s + m * N * s) if mixed else (spec + N * s + 2 * m * N * 8),
        "pencil_kinetic": 2 * spec,
        "plane_hpsi": (spec + 2 * m * N * s + N * s) if mixed
                      else (spec + m * N * s + N * 8 + m * N * 8),
    }.get(kind)


def step_bytes(g, m, k, s=4):
    """Algorithmic bytes of one whole mixed-path step (order 2k, Ritz values)
    over m states on grid g with whole-plane passes: per term i a forward
    plane pass, i pencils, i - 1 merged plane passes and the term pass; the
    exact sum of the k FP32 term contributions into phi (k reads, one write);
    the overlap Gram (phi once) and the update psi = L^-1 phi (read phi,
    write psi); the energies (forward pass, kinetic pencil, H psi pass, the
    subspace Gram reading psi and H psi).  The n x n work moves no
    appreciable bytes."""
    N = g.n_points
    b = 0
    for i in range(1, k + 1):
        b += algorithmic_bytes("plane_fwd", g, m, s, mixed=True)
        b += i * algorithmic_bytes("pencil", g, m, s, mixed=True)
        b += (i - 1) * algorithmic_bytes("plane_merged", g, m, s, mixed=True)
        b += algorithmic_bytes("plane_combine", g, m, s, mixed=True)
    b += (k + 1) * m * N * 4                    # term sum
    b += m * N * 4 + 2 * m * N * 4              # overlap Gram, update
    b += (m * N * s + m * g.nz * g.ny * (g.nx // 2 + 1) * 2 * s   # forward (no factor)
          + algorithmic_bytes("pencil_kinetic", g, m, s, mixed=True)
          + algorithmic_bytes("plane_hpsi", g, m, s, mixed=True)
          + 2 * m * N * 4)                      # subspace Gram
    return b


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id=None):
        self.f = tempfile.NamedTemporaryFile("w", suffix=".csv", delete=False)
        self.path = self.f.name
        self.proc = None
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        if gpu_id:
            cmd.insert(1, f"--id={gpu_id}")
        try:
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:   # no nvidia-smi: no clock record
            self.f.close()
            os.unlink(self.path)
        self.offset = 0

    def begin(self):
        """Wait (at most 5 s) until the sampler has written its first line,
        then mark the start of the timed window: stop() reads only the
        samples written after this call."""
        if self.proc is None:
            return
        t0 = time.perf_counter()
        while (os.path.getsize(self.path) == 0 and self.proc.poll() is None
               and time.perf_counter() - t0 < 5.0):
            time.sleep(0.02)
        self.offset = os.path.getsize(self.path)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            f.seek(self.offset)
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# the bounded CPU-oracle sample of the workload (about 10 s of one core)
CPU_SAMPLE_STATES, CPU_SAMPLE_STEPS = 4, 3


def cpu_sample(w, n_sample, steps):
    """Time the FP64 oracle on n_sample states of the workload (one oracle
    step per timed step).  Returns state-steps per second."""
    from oracle import itp_oracle as O
    from itp_workloads import c60_like_potential, cubic, harmonic_potential, normal_states
    g = cubic(w["n"], w["box"])
    V = c60_like_potential(g) if w["potential"] == "c60" else harmonic_potential(g)
    psi = normal_states(n_sample, g.n_points, seed=w["seed"])
    times = []
    for _ in range(steps):
        t0 = time.perf_counter()
        psi, E = O.itp_step(psi, V, g, w["order"], w["tau"], ritz=True)
        times.append(time.perf_counter() - t0)
    return n_sample / (sum(times) / len(times)), sum(times)


def _cpu_worker(job):
    """One oracle process of the all-cores sample: set up, wait for the
    common start time, then time its steps on one state."""
    w, start_at, steps = job
    from oracle import itp_oracle as O
    from itp_workloads import c60_like_potential, cubic, harmonic_potential, normal_states
    g = cubic(w["n"], w["box"])
    V = c60_like_potential(g) if w["potential"] == "c60" else harmonic_potential(g)
    psi = normal_states(1, g.n_points, seed=w["seed"])
    while time.time() < start_at:
        time.sleep(0.01)
    started = time.time()
    t0 = time.perf_counter()
    for _ in range(steps):
        psi, _ = O.itp_step(psi, V, g, w["order"], w["tau"], ritz=True)
    return steps / (time.perf_counter() - t0), started


def cpu_sample_all_cores(w, steps=2, setup_s=15.0):
    """The oracle on every host core at once: one single-threaded process per
    core (spawned, no CUDA), each on one state, all starting together; the
    value is the sum of their state-step rates."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    workers = len(os.sched_getaffinity(0))
    start_at = time.time() + setup_s
    with ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        futs = [ex.submit(_cpu_worker, (w, start_at, steps)) for _ in range(workers)]
        res = [f.result(timeout=600) for f in futs]
    rates = [r[0] for r in res]
    starts = [r[1] for r in res]
    return {"value": float(sum(rates)), "unit": "state-steps/s", "cores": workers,
            "per_core_median": float(np.median(rates)),
            "start_skew_s": round(max(starts) - min(starts), 3),
            "sample": f"{workers} oracle processes, one state and {steps} steps each"}


def run_reference(args):
    w = WORKLOADS[args.workload]
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n_sample = 1
    from oracle import itp_oracle as O
    from itp_workloads import c60_like_potential, cubic, harmonic_potential, normal_states
    g = cubic(w["n"], w["box"])
    V = c60_like_potential(g) if w["potential"] == "c60" else harmonic_potential(g)
    psi = normal_states(n_sample, g.n_points, seed=w["seed"])
    for _ in range(args.warmup):
        psi, _ = O.itp_step(psi, V, g, w["order"], w["tau"], ritz=True)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        psi, _ = O.itp_step(psi, V, g, w["order"], w["tau"], ritz=True)
    dt = time.perf_counter() - t0
    value = n_sample * args.steps / dt
    sample = (f"{n_sample} state(s) of the workload per step: the oracle's propagation, "
              f"Cholesky and Ritz step on that block")
    line = {
        "impl": "reference", "metric": "state-steps/s", "value": value, "unit": "state-steps/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["desc"], "precision": "fp64 (CPU oracle)"},
        "cpu_baseline": {"value": value, "unit": "state-steps/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "state-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def ho_closed_shells(n):
    """E = n + 3/2 of the 3D oscillator, shell s with (s+1)(s+2)/2 states.
    On the 128^3 / [-8,8)^3 grid the grid spectrum equals these values to
    round-off for the first eight shells (120 states)."""
    E = []
    s = 0
    while len(E) < n:
        E += [s + 1.5] * ((s + 1) * (s + 2) // 2)
        s += 1
    return np.array(E[:n])


# Problems of the time-to-tolerance runs: grid edge, box, potential, the
# reference energies (exact closed shells for the oscillator; the oracle's
# certified eigenvalues of the grid Hamiltonian for the C60-like well, stored
# by tests/golden/make_c60_eref.py), seed of the random-normal start.
TTT_PROBLEMS = {
    "c60_128": {"desc": "C60-like Gaussian well (60 wells, depth 2.0 Ha, sigma 0.8 bohr, "
                        "radius 6.7 bohr), 128^3 grid, box 32 bohr",
                "n": 128, "box": 32.0, "potential": "c60",
                "eref": os.path.join("tests", "golden", "c60_128_eref.txt"), "seed": 4321},
    "osc_128": {"desc": "3D harmonic oscillator, 128^3 grid, box [-8,8)^3 (eight closed "
                        "shells, exact E = n + 3/2)",
                "n": 128, "box": 16.0, "potential": "ho", "eref": None, "seed": 4321},
}


# The C60-like time-to-tolerance run: n = 120 wanted states and 136 guard
# states (m = 256, two tensor-core tiles: the gap from state 120 to state 257
# sets the convergence rate; with 8 guard states it is ~0.008 Ha, with 136
# about ten times larger), order 12 at tau = 1.
C60_TTT = {"n": 120, "guard": 136, "order": 12, "tau": 1.0, "max_fp32": 400, "max_fp64": 300}


def fp64_step_extrapolation(P, mixed, n, guard, order, tau, **_):
    """The FP64 path's time to tolerance estimated (not measured) from its
    measured step time: the FP64 iteration is the same map as the FP32 one,
    so it needs about as many steps as the mixed path took in all."""
    from itp_workloads import c60_like_potential, cubic, normal_states
    pr = TTT_PROBLEMS["c60_128"]
    g = cubic(pr["n"], pr["box"])
    h = P.ItpGrid(g.nx, g.ny, g.nz, g.lx, g.ly, g.lz, n, guard, P.ITP_FP64)
    h.set_potential(c60_like_potential(g))
    h.set_states(normal_states(n + guard, g.n_points, seed=pr["seed"]))
    h.step_graph(order, tau)
    t0 = time.perf_counter()
    for _ in range(2):
        h.step_graph(order, tau)
    step_s = (time.perf_counter() - t0) / 2
    h.close()
    steps = mixed["fp32_steps"] + mixed["fp64_steps"]
    return {"seconds_estimated": step_s * steps, "step_seconds": step_s, "steps_assumed": steps,
            "how": "estimated, not measured: the measured FP64 step time x the mixed path's "
                   "total step count (run bench.py with --fp64-ttt to measure it)"}


def load_eref(path):
    """Reference eigenvalues from a stored table (column 2 of the data rows)."""
    vals = []
    with open(os.path.join(ROOT, path)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                vals.append(float(line.split()[1]))
    return np.array(vals)


def time_to_tol(P, precision, problem="c60_128", tol=1e-8, order=12, tau=0.5, n=120, guard=8,
                max_fp32=400, max_fp64=200, plateau_rel=1e-5, polish_order=None,
                per_state=False, fp64_eval=False, margin=1.0):
    """Wall time from itp_set_states of seeded random states until every one
    of the n lowest Ritz energies is within tol of its reference value.
    FP64: FP64 steps throughout.  Mixed: FP32 steps while the energies still
    change by more than plateau_rel * max|E| per step (the FP32-evaluated
    energies level off near 1e-5 relative while the FP32 states keep
    converging), then as many further FP32 steps as the observed convergence
    rate says the states need, then FP64 polish steps (itp_polish, one step
    per call) until within tol.  fp64_eval: before any polish step, the
    final energy evaluation in FP64 (ITP_EVAL_FP64), with ten more FP32 steps
    before each further one; margin: the FP32 phase aims its extra steps at
    tol / margin.  The reference is used only to stop the clock, never to
    steer the iteration.  per_state: also return every state's final error."""
    from itp_workloads import c60_like_potential, cubic, harmonic_potential, normal_states
    pr = TTT_PROBLEMS[problem]
    g = cubic(pr["n"], pr["box"])
    V = c60_like_potential(g) if pr["potential"] == "c60" else harmonic_potential(g)
    m = n + guard
    psi = normal_states(m, g.n_points, seed=pr["seed"])
    E_ref = load_eref(pr["eref"])[:n] if pr["eref"] else ho_closed_shells(n)
    h = P.ItpGrid(g.nx, g.ny, g.nz, g.lx, g.ly, g.lz, n, guard, precision)
    h.set_potential(V)
    h.set_states(psi)
    tuned, _ = h.autotune(order, tau)   # launch shapes for this state count (untimed)
    h.synchronize()
    t0 = time.perf_counter()
    h.set_states(psi)
    steps32 = steps64 = evals = 0
    err = float("inf")
    E_prev = None
    E = None
    if precision == P.ITP_MIXED:
        # FP32 steps until the FP32-evaluated energies stop moving; the
        # states keep converging below that floor at the rate the energy
        # changes showed before it, so a few more FP32 steps (as many as
        # that rate needs to bring an energy change of the last clean step
        # down to tol) precede the FP64 polish.
        dEs = []
        extra = None
        while steps32 < max_fp32:
            E = h.step_graph(order, tau)
            steps32 += 1
            err = float(np.max(np.abs(E[:n] - E_ref)))
            if err < tol:
                break
            if E_prev is not None:
                dE = float(np.max(np.abs(E[:n] - E_prev[:n])))
                if extra is not None:
                    extra -= 1
                    if extra <= 0:
                        break
                elif dE < plateau_rel * max(1.0, float(np.max(np.abs(E[:n])))):
                    clean = [d for d in dEs[-4:] if d > 0]
                    rates = [b / a for a, b in zip(clean, clean[1:]) if a > 0]
                    rho = min(0.9, max(0.05, float(np.median(rates)))) if rates else 0.5
                    goal = tol / margin
                    extra = int(np.ceil(np.log(max(dEs[-1], goal) / goal) / np.log(1.0 / rho)))
                    extra = min(extra, 60)
                    if extra <= 0:
                        break
                dEs.append(dE)
            E_prev = E
        if fp64_eval:
            # the final evaluation in FP64 (ITP_EVAL_FP64: no FP64
            # propagation); if the states were not yet converged, ten more
            # FP32 steps before each further evaluation
            while evals < 10:
                E = h.energies("values", fp64=True)
                evals += 1
                err = float(np.max(np.abs(E[:n] - E_ref)))
                if err < tol:
                    break
                for _ in range(10):
                    h.step_graph(order, tau)
                    steps32 += 1
        while err >= tol and steps64 < max_fp64:
            _, E = h.polish(polish_order or order, tau, 1e-300, 1)
            steps64 += 1
            err = float(np.max(np.abs(E[:n] - E_ref)))
    else:
        while err >= tol and steps64 < max_fp64:
            E = h.step_graph(order, tau)
            steps64 += 1
            err = float(np.max(np.abs(E[:n] - E_ref)))
    h.synchronize()
    dt = time.perf_counter() - t0
    h.close()
    out = {"seconds": dt, "fp32_steps": steps32, "fp64_steps": steps64,
           "max_abs_error_ha": err, "reached": err < tol, "launch_shapes": tuned}
    if fp64_eval:
        out["fp64_evaluations"] = evals
    if per_state and E is not None:
        out["errors_ha"] = [float(f"{x:.3e}") for x in (E[:n] - E_ref)]
    return out


# The 32^3 oscillator workload: box [-8,8)^3, V = r^2/2, n = 10 states (three
# closed shells, exact E = 1.5, 2.5 x 3, 3.5 x 6), order 4, tau = 0.1, FP64,
# seeded random-normal start (seed 1234), tolerance 1e-10 Ha.
OSC32 = {"n": 32, "box": 16.0, "n_states": 10, "order": 4, "tau": 0.1, "seed": 1234,
         "tol": 1e-10, "max_steps": 400}


def steps_to_tol(step, E_ref, tol, max_steps):
    """Call step() (returns the energies) until every energy is within tol
    of E_ref; returns (steps, max abs error)."""
    steps, err = 0, float("inf")
    while err >= tol and steps < max_steps:
        E = np.sort(np.asarray(step())[:len(E_ref)])
        steps += 1
        err = float(np.max(np.abs(E - E_ref)))
    return steps, err


def osc32_gpu(P):
    """Time to tolerance of the 32^3 oscillator on the GPU, FP64 graph steps
    (Ritz values each step), from itp_set_states to the last energy read."""
    from itp_workloads import cubic, harmonic_potential, normal_states
    c = OSC32
    g = cubic(c["n"], c["box"])
    psi = normal_states(c["n_states"], g.n_points, seed=c["seed"])
    E_ref = ho_closed_shells(c["n_states"])
    h = P.ItpGrid(g.nx, g.ny, g.nz, g.lx, g.ly, g.lz, c["n_states"], 0, P.ITP_FP64)
    try:
        h.set_potential(harmonic_potential(g))
        h.synchronize()
        t0 = time.perf_counter()
        h.set_states(psi)
        steps, err = steps_to_tol(lambda: h.step_graph(c["order"], c["tau"]), E_ref,
                                  c["tol"], c["max_steps"])
        h.synchronize()
        dt = time.perf_counter() - t0
    finally:
        h.close()
    return {"seconds": dt, "steps": steps, "max_abs_error_ha": err, "reached": err < c["tol"]}


def osc32_oracle():
    """The same with the FP64 CPU oracle (one core), in full."""
    from oracle import itp_oracle as O
    from itp_workloads import cubic, harmonic_potential, normal_states
    c = OSC32
    g = cubic(c["n"], c["box"])
    V = harmonic_potential(g)
    state = {"psi": normal_states(c["n_states"], g.n_points, seed=c["seed"])}

    def step():
        state["psi"], E = O.itp_step(state["psi"], V, g, c["order"], c["tau"], ritz=True)
        return E

    t0 = time.perf_counter()
    steps, err = steps_to_tol(step, ho_closed_shells(c["n_states"]), c["tol"], c["max_steps"])
    return {"seconds": time.perf_counter() - t0, "steps": steps, "max_abs_error_ha": err,
            "reached": err < c["tol"], "cores": 1}


def extrapolate_oracle(cpu, ttt, m):
    """The oracle's time to tolerance on the C60-like workload, extrapolated
    (not measured): m states x the FP64 path's step count there, divided by
    the oracle's measured state-steps per second on the same grid and order.
    None when either figure is missing."""
    if not cpu or not cpu.get("value") or not ttt or "fp64" not in ttt:
        return None
    steps = ttt["fp64"].get("fp64_steps") or ttt["fp64"].get("steps_assumed")
    if not steps:
        return None
    return {"value_s": round(m * steps / cpu["value"], 1),
            "how": f"extrapolated, not measured: {m} states x {steps} FP64 steps (the GPU "
                   "FP64 path's step count to the tolerance on the same workload, grid and "
                   "order as the oracle's sample) / the oracle's measured state-steps per "
                   "second"}


def adaptive_to_tol(P, precision, tol=1e-8, order=12, n=120, guard=8):
    """The adaptive iteration of Sec. III (itp_solve_adaptive: tau 0.5,
    halved between levels, converged leading states no longer propagated,
    stop on R^H) on the time-to-tolerance problem (3D oscillator, 128^3,
    box [-8,8)^3, n = 120 closed-shell states).  FP64: bound gamma = tol.
    Mixed: FP32 levels down to gamma = 1e-6 (on this grid, spacing 0.125
    bohr, the FP32 floor of R^H lies near 3e-7), then FP64 polish steps
    until the energies change by less than tol / 10.  Wall time from itp_set_states; the error against the
    exact n + 3/2 is measured after the clock stops."""
    from itp_workloads import cubic, harmonic_potential, normal_states
    g = cubic(128, 16.0)
    V = harmonic_potential(g)
    m = n + guard
    psi = normal_states(m, g.n_points, seed=4321)
    E_ref = ho_closed_shells(n)
    h = P.ItpGrid(g.nx, g.ny, g.nz, g.lx, g.ly, g.lz, n, guard, precision)
    h.set_potential(V)
    h.synchronize()
    t0 = time.perf_counter()
    h.set_states(psi)
    polish_steps = 0
    if precision == P.ITP_MIXED:
        r = h.solve_adaptive(order, 0.5, 0.5, 1e-6, max_steps=100, max_levels=2)
        polish_steps, E = h.polish(order, 0.5 * 0.5 ** (len(r["levels"]) - 1), tol / 10, 20)
    else:
        r = h.solve_adaptive(order, 0.5, 0.5, tol, max_steps=100, max_levels=4)
        E = r["E"]
    h.synchronize()
    dt = time.perf_counter() - t0
    h.close()
    err = float(np.max(np.abs(np.asarray(E)[:n] - E_ref)))
    return {"seconds": dt, "levels": r["levels"], "adaptive_converged": r["converged"],
            "max_RH": float(np.max(r["RH"][:n])), "fp64_polish_steps": polish_steps,
            "max_abs_error_ha": err, "reached": err < tol}


def precision_sweep(P, orders=(4, 8, 12), taus=(0.5, 0.25, 0.125, 0.05), n=20, guard=4):
    """Accuracy of the mixed form per order and time step: the 3D oscillator
    on a 64^3 grid in [-8,8)^3, n = 20 (closed shells) + 4 guard states.
    FP32 steps until the energies change by less than 1e-6 relative (at most
    400), then FP64 polish steps until they change by less than 1e-11 (at
    most 60).  Reports the largest |E - (n + 3/2)| over the 20 states after
    the FP32 phase and after the polish: the FP32 floor, and the time-step
    bias of the converged Rayleigh-Ritz values, which falls as tau^(4k)."""
    from itp_workloads import cubic, harmonic_potential, normal_states
    g = cubic(64, 16.0)
    V = harmonic_potential(g)
    E_ref = ho_closed_shells(n)
    psi = normal_states(n + guard, g.n_points, seed=2024)
    out = {}
    for order in orders:
        for tau in taus:
            h = P.ItpGrid(64, 64, 64, 16.0, 16.0, 16.0, n, guard, P.ITP_MIXED)
            h.set_potential(V)
            h.set_states(psi)
            E_prev, steps32 = None, 0
            for steps32 in range(1, 401):
                E = h.step_graph(order, tau)
                if E_prev is not None and np.max(np.abs(E[:n] - E_prev[:n])) < 1e-6 * np.max(
                        np.abs(E[:n])):
                    break
                E_prev = E
            err32 = float(np.max(np.abs(E[:n] - E_ref)))
            steps64, E = h.polish(order, tau, 1e-11, 60)
            h.close()
            out[f"order{order}_tau{tau}"] = {
                "fp32_steps": steps32, "fp64_steps": steps64,
                "max_abs_error_fp32_ha": err32,
                "max_abs_error_polished_ha": float(np.max(np.abs(E[:n] - E_ref)))}
    return out


def order_sweep_small(P, orders=(2, 4, 6, 8, 10, 12), gamma=1e-10):
    """Which order is fastest (the paper found 6 on one Itanium processor):
    the adaptive iteration (tau 0.5, halved between levels, stop on R^H <
    gamma) at each order on the 3D oscillator, 32^3 grid, box [-8,8)^3,
    n = 10 + 2 guard states, FP64; wall time, steps and the error of the 10
    energies against n + 3/2."""
    from itp_workloads import cubic, harmonic_potential, normal_states
    g = cubic(32, 16.0)
    V = harmonic_potential(g)
    psi = normal_states(12, g.n_points, seed=1234)
    E_ref = ho_closed_shells(10)
    out = {}
    for order in orders:
        h = P.ItpGrid(32, 32, 32, 16.0, 16.0, 16.0, 10, 2, P.ITP_FP64)
        h.set_potential(V)
        h.synchronize()
        t0 = time.perf_counter()
        h.set_states(psi)
        r = h.solve_adaptive(order, 0.5, 0.5, gamma, max_steps=300, max_levels=10)
        h.synchronize()
        dt = time.perf_counter() - t0
        h.close()
        out[str(order)] = {"seconds": round(dt, 4), "levels": len(r["levels"]),
                           "steps": sum(lv[1] for lv in r["levels"]),
                           "final_tau": r["levels"][-1][0] if r["levels"] else None,
                           "converged": r["converged"],
                           "max_abs_error_ha": float(np.max(np.abs(r["E"][:10] - E_ref)))}
    return out


def large_c60(P, torch, steps, warmup, n=120, guard=8, order=8, tau=0.25, seed=1234):
    """The large workload: C60-like well on a 256^3 grid (16.8 M points), box
    32 bohr, n = 120 + 8 guard states, order 8, mixed (planes too large for
    one CTA: row and column passes, or two-CTA clusters, as the autotuner
    picks).  Graph-replayed steps per second,
    the row/column passes' achieved GB/s, and the tensor-core Gram's TF32
    rate.  States from torch's seeded device generator (2.1 G values)."""
    from itp_workloads import c60_like_potential, cubic
    g = cubic(256, 32.0)
    V = c60_like_potential(g)
    m = n + guard
    stream = torch.cuda.Stream()
    h = P.ItpGrid(256, 256, 256, 32.0, 32.0, 32.0, n, guard, P.ITP_MIXED,
                  cuda_stream=stream.cuda_stream)
    h.set_potential(V)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    x = torch.randn((m, g.n_points), dtype=torch.float64, device="cuda", generator=gen)
    torch.cuda.synchronize()
    P.itp_set_states_device(h.h, x.data_ptr())
    h.synchronize()
    del x
    torch.cuda.empty_cache()
    tuned, report = h.autotune(order, tau)
    for _ in range(warmup):
        h.step_graph(order, tau)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        E = h.step_graph(order, tau)
    b.record(stream)
    b.synchronize()
    dt = a.elapsed_time(b) / 1e3
    h.profile(True)
    h.step(order, tau, ritz="values")
    prof = {k: v for k, v in h.profile_read().items() if v[0] > 0}
    h.profile(False)
    h.close()
    Nh = g.nz * g.ny * (g.nx // 2 + 1)
    spec = m * Nh * 8
    per = {k: {"launches": v[0], "avg_launch_ms": round(v[1] / v[0], 4)} for k, v in prof.items()}
    # a pencil pass moves the FP32 half spectrum in and out; the overlap
    # Gram reads the FP32 block and does 3 TF32 products per FP32 product
    if "pencil" in per:
        t = per["pencil"]["avg_launch_ms"] / 1e3
        per["pencil"]["achieved_gbs"] = round(2 * spec / t / 1e9, 1)
    if "gram" in per:
        t = per["gram"]["avg_launch_ms"] / 1e3
        per["gram"]["tf32_tflops"] = round(3 * 2 * 128 * 128 * g.n_points / t / 1e12, 1)
    return {"workload": f"C60-like well, 256^3 grid, box 32 bohr, n = {n} + {guard} guard, "
                        f"order {order}, tau = {tau}, mixed",
            "value": m * steps / dt, "unit": "state-steps/s", "ms_per_step": 1e3 * dt / steps,
            "steps": steps, "launch_shapes": tuned, "autotune": report, "per_kernel": per,
            "energies_head": [round(float(v), 8) for v in E[:3]]}


def planar_dots(P, torch, steps, warmup, order=12, tau=0.25):
    """The paper's planar case: a 9 x 9 array of quantum dots (sech wells,
    depth 2 Ha, width 0.6 bohr, spacing 3 bohr) on a 256 x 256 grid in a
    32 bohr box, n = 81 (one state per dot) + 8 guard states.  Mixed steps
    (graph replays) per second, and the FP64 adaptive iteration's wall time
    to R^H < 1e-10 for the 81 states."""
    from itp_workloads import normal_states, planar, quantum_dot_array
    g = planar(256, 256, 32.0, 32.0)
    V = quantum_dot_array(g)
    n, guard = 81, 8
    psi = normal_states(n + guard, g.n_points, seed=81)
    stream = torch.cuda.Stream()
    h = P.ItpGrid(256, 256, 1, 32.0, 32.0, 1.0, n, guard, P.ITP_MIXED,
                  cuda_stream=stream.cuda_stream)
    h.set_potential(V)
    h.set_states(psi)
    tuned, _ = h.autotune(order, tau)
    for _ in range(warmup):
        h.step_graph(order, tau)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        E = h.step_graph(order, tau)
    b.record(stream)
    b.synchronize()
    dt = a.elapsed_time(b) / 1e3
    h.close()
    h = P.ItpGrid(256, 256, 1, 32.0, 32.0, 1.0, n, guard, P.ITP_FP64)
    h.set_potential(V)
    h.synchronize()
    t0 = time.perf_counter()
    h.set_states(psi)
    r = h.solve_adaptive(order, 0.5, 0.5, 1e-10, max_steps=150, max_levels=3)
    h.synchronize()
    t_ad = time.perf_counter() - t0
    h.close()
    return {"workload": "9 x 9 quantum dots (sech wells, depth 2 Ha, width 0.6 bohr, "
                        "spacing 3 bohr), 256 x 256 grid, box 32 bohr, n = 81 + 8 guard, "
                        f"order {order}, tau = {tau}; no pencil pass (the kinetic factor "
                        "ends each forward plane pass)",
            "value": (n + guard) * steps / dt, "unit": "state-steps/s",
            "ms_per_step": 1e3 * dt / steps, "launch_shapes": tuned,
            "energies_head": [round(float(x), 8) for x in E[:3]],
            "fp64_adaptive": {"seconds": round(t_ad, 3), "levels": r["levels"],
                              "converged": r["converged"],
                              "max_RH": float(np.max(r["RH"][:n])),
                              "E_81": float(r["E"][n - 1])}}


def batch_throughput(P, torch, steps, warmup, count=64, order=8, tau=0.25, seed=1000):
    """The batched workload: `count` independent random-well problems (grid
    edges from {32, 48, 64, 96}, n ~ U{8..64} states, 4-60 Gaussian wells),
    order 8, mixed precision, every step of all problems one CUDA graph
    launch (itp_batch_step).  The same problems stepped one after another
    (each problem's own itp_step graph) are timed beside it.  Potentials come
    from the seeded Philox generator; the initial states (840 M values, too
    many to draw on the host in a bench) from torch's seeded device generator,
    which only throughput depends on."""
    from itp_workloads import random_wells_problem
    probs = [random_wells_problem(seed, p) for p in range(count)]
    stream = torch.cuda.Stream()
    dims = [(g.nx, g.ny, g.nz) for g, _, _ in probs]
    boxes = [(g.lx, g.ly, g.lz) for g, _, _ in probs]
    ns = [n for _, _, n in probs]
    b = P.ItpBatch(dims, boxes, ns, precision=P.ITP_MIXED, cuda_stream=stream.cuda_stream)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    for q, (g, V, n) in zip(b.problems, probs):
        q.set_potential(V)
        x = torch.randn((n, g.n_points), dtype=torch.float64, device="cuda", generator=gen)
        torch.cuda.synchronize()
        P.itp_set_states_device(q.h, x.data_ptr())
        q.synchronize()
        del x
    m_total = b.m_total
    # launch shapes (untimed): tuned on one problem per grid and shared by the
    # others of that grid, so that they form one group of grouped launches
    tuned_by_grid = {}
    for q, (g, _, _) in zip(b.problems, probs):
        key = (g.nx, g.ny, g.nz)
        if key not in tuned_by_grid:
            tuned_by_grid[key], _ = q.autotune(order, tau)
        else:
            t = tuned_by_grid[key]
            q.set_tuning(t["pencil_w"], t["split"], t["row_tb"], t["gram_ctas"])

    def timed(grouped):
        b.set_grouping(grouped)
        for _ in range(warmup):
            b.step(order, tau)
        n0 = b.kernel_launches
        torch.cuda.synchronize()
        start = torch.cuda.Event(enable_timing=True)
        end = torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for _ in range(steps):
            E = b.step(order, tau)
        end.record(stream)
        end.synchronize()
        return start.elapsed_time(end) / 1e3, (b.kernel_launches - n0) // steps, E

    # one graph branch of ~50 launches per problem, then grouped launches
    dt_br, per_step_br, _ = timed(False)
    dt, per_step, E = timed(True)
    n_groups = b.groups
    # the same problems one after another (each its own step graph)
    for q in b.problems:
        q.step_graph(order, tau)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        for q in b.problems:
            q.step_graph(order, tau)
    dt_serial = time.perf_counter() - t0
    b.close()
    sizes = {}
    for g, _, _ in probs:
        sizes[f"{g.nx}^3"] = sizes.get(f"{g.nx}^3", 0) + 1
    # whole-step roofline of the batch: every problem's algorithmic bytes
    # per step over the measured step time
    hbm_peak = _hbm_peak()
    step_b = sum(step_bytes(g, n, order // 2) for g, _, n in probs)
    return {"workload": f"{count} independent random-well problems (seed {seed}+p), grids "
                        f"{sizes}, n = 8..64 states each ({m_total} in all), order 8, "
                        f"tau = {tau}, mixed precision, grouped launches",
            "value": m_total * steps / dt, "unit": "state-steps/s",
            "ms_per_step": 1e3 * dt / steps, "steps": steps,
            "state_points": int(sum(n * g.n_points for g, _, n in probs)),
            "gpu_launches_per_step": per_step, "graph_launches_per_step": 1,
            "grouped": {"groups": n_groups,
                        "how": "each FFT pass of the problems that share a grid is one launch "
                               "over all their states (itp_batch_set_grouping); the n x n "
                               "kernels run as per-problem branches between those launches"},
            "branches": {"value": m_total * steps / dt_br, "ms_per_step": 1e3 * dt_br / steps,
                         "gpu_launches_per_step": per_step_br,
                         "how": "one graph branch per problem (itp_batch_set_grouping(b, 0))"},
            "roofline": {"bound": "hbm", "algorithmic_bytes_per_step": step_b,
                         "achieved": step_b / (dt / steps) / 1e9, "peak": hbm_peak,
                         "unit": "GB/s", "frac": step_b / (dt / steps) / 1e9 / hbm_peak,
                         "how": "sum over the problems of the whole step's algorithmic "
                                "bytes (FFT passes, term sum, overlap, update, energies) "
                                "over the measured time of one batch step"},
            "one_by_one": {"value": m_total * steps / dt_serial,
                           "ms_per_step": 1e3 * dt_serial / steps,
                           "how": "each problem's own itp_step graph, problems in turn "
                                  "(host wall clock)"},
            "energies_head_p0": [round(float(x), 8) for x in E[0][:3]]}


def time_steps(h, stream, order, tau, steps, torch):
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    E = None
    start.record(stream)
    for _ in range(steps):
        E = h.step(order, tau, ritz="values")
    end.record(stream)
    end.synchronize()
    return start.elapsed_time(end) / 1e3, E


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c60_128", choices=sorted(WORKLOADS))
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-path measurement")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-ttt", action="store_true", help="skip the time-to-tolerance runs")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched workload")
    ap.add_argument("--no-fp64-ttt", dest="fp64_ttt", action="store_false",
                    help="estimate the FP64 path's time to tolerance on the C60-like workload "
                         "from its step time instead of running it (about two minutes)")
    ap.add_argument("--ttt-orders", action="store_true",
                    help="also the C60-like time to tolerance (mixed, FP64 evaluation) at orders "
                         "4-12 and tau 0.5-1.5 (about seven minutes)")
    ap.add_argument("--adaptive-fp64", action="store_true",
                    help="also time the FP64 adaptive iteration (about two minutes)")
    ap.add_argument("--cpu-sample", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    w = WORKLOADS[args.workload]

    if args.cpu_sample:
        v, t = cpu_sample(w, CPU_SAMPLE_STATES, CPU_SAMPLE_STEPS)
        out = {"value": v, "seconds": t}
        for key, fn in (("osc32", osc32_oracle), ("all_cores", lambda: cpu_sample_all_cores(w))):
            try:   # the single-core figure above stands whatever these do
                out[key] = fn()
            except Exception as ex:
                out[key] = {"error": f"{type(ex).__name__}: {ex}"}
        print(json.dumps(out))
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.warmup < 3:
        raise SystemExit("timing rules: at least 3 warm-up steps")

    import torch
    import torch.distributed as dist
    import paper_0809_3739_gb300 as P

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.Stream()
    g, V, psi = make_inputs(w, rank)
    m = w["n_states"] + w["n_guard"]
    order, tau = w["order"], w["tau"]

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- end to end through the C ABI with host buffers (first, in a clean process) --
    e2e = None
    if not args.no_e2e:
        K = args.steps
        h = P.ItpGrid(g.nx, g.ny, g.nz, g.lx, g.ly, g.lz, w["n_states"], w["n_guard"],
                      P.ITP_MIXED)   # the library's own stream, as a host-side caller has
        h.set_potential(V)
        h.set_states(psi)
        h.autotune(order, tau)
        pin_in = torch.from_numpy(psi).pin_memory()
        pin_out = torch.empty_like(pin_in).pin_memory()
        E_host = np.empty(m)
        lib = P.load()
        ptr_in, ptr_out = pin_in.data_ptr(), pin_out.data_ptr()

        def host_step():   # host -> device [m][N] FP64, step, device -> host, energies
            P.itp_step_host(h.h, m, g.n_points, order, tau, ptr_in, ptr_out,
                            P.ITP_RITZ_VALUES, E_host)

        def sequential_calls():   # the same step as three calls, copies not overlapped
            lib.itp_set_states(h.h, ptr_in)
            P.itp_step(h.h, order, tau, P.ITP_RITZ_VALUES, E_host)
            lib.itp_get_states(h.h, ptr_out)

        for _ in range(3):   # warm-up of the whole end-to-end step, copies included
            host_step()
        barrier()
        per_step = []
        t0 = time.perf_counter()
        for _ in range(K):
            ta = time.perf_counter()
            host_step()
            per_step.append(time.perf_counter() - ta)
        barrier()
        t_e2e = max_over_ranks(time.perf_counter() - t0)
        # beside it, the unoverlapped sequence (not the value)
        for _ in range(3):
            sequential_calls()
        K2 = min(K, 10)
        seq = []
        for _ in range(K2):
            ta = time.perf_counter()
            sequential_calls()
            seq.append(time.perf_counter() - ta)
        e2e = {"value": replicas_value(m * K, t_e2e, world), "unit": "state-steps/s",
               "h2d_bytes_per_step": int(psi.nbytes),
               "d2h_bytes_per_step": int(psi.nbytes + E_host.nbytes), "steps": K,
               "calls": "itp_step_host (pinned host buffers in and out; the copies overlap "
                        "the device work in 4 state chunks)",
               "ms_per_step_each": [round(1e3 * t, 1) for t in per_step],
               "median_ms_per_step": round(1e3 * float(np.median(per_step)), 2),
               "sequential_calls": {
                   "calls": "itp_set_states + itp_step + itp_get_states (pinned host)",
                   "steps": K2, "ms_per_step_each": [round(1e3 * t, 1) for t in seq],
                   "median_ms_per_step": round(1e3 * float(np.median(seq)), 2)}}
        # the raw copy rate of the same pinned buffers, for comparison
        dev = torch.empty(pin_in.shape, dtype=pin_in.dtype, device="cuda")
        dev.copy_(pin_in, non_blocking=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dev.copy_(pin_in, non_blocking=True)
        pin_out.copy_(dev, non_blocking=True)
        torch.cuda.synchronize()
        e2e["raw_copy_gbs_h2d_plus_d2h"] = round(2 * psi.nbytes / (time.perf_counter() - t0) / 1e9, 1)
        del dev, pin_in, pin_out
        h.close()

    # ---- headline: mixed path, states resident in HBM --------------------------
    h = P.ItpGrid(g.nx, g.ny, g.nz, g.lx, g.ly, g.lz, w["n_states"], w["n_guard"],
                  P.ITP_MIXED, cuda_stream=stream.cuda_stream)
    h.set_potential(V)
    h.set_states(psi)
    # launch shapes picked by timing the candidates on this workload (untimed)
    tuned, tune_report = h.autotune(order, tau)
    for _ in range(args.warmup):
        h.step_graph(order, tau)   # the first call captures the step's graph
    gpu_id = None
    try:
        gpu_id = str(torch.cuda.get_device_properties(local).uuid)
        if not gpu_id.startswith("GPU-"):
            gpu_id = "GPU-" + gpu_id
    except Exception:
        gpu_id = None
    barrier()
    # timed: whole steps as CUDA-graph replays (itp_step), the library's step call
    clocks = ClockSampler(gpu_id)
    clocks.begin()
    n0 = h.kernel_launches
    torch.cuda.nvtx.range_push("itp_timed_steps")   # lets a profiler select the timed launches
    gstart = torch.cuda.Event(enable_timing=True)
    gend = torch.cuda.Event(enable_timing=True)
    gstart.record(stream)
    for _ in range(args.steps):
        E = h.step_graph(order, tau)
    gend.record(stream)
    gend.synchronize()
    torch.cuda.nvtx.range_pop()
    launches = h.kernel_launches - n0
    clk = clocks.stop()
    barrier()
    dt = max_over_ranks(gstart.elapsed_time(gend) / 1e3)
    value = replicas_value(m * args.steps, dt, world)
    # the same steps launched one kernel at a time with a CUDA-event pair around
    # each launch: the per-kernel times of the breakdown and the rooflines
    h.profile(True)
    dt_prof, _ = time_steps(h, stream, order, tau, args.steps, torch)
    prof = h.profile_read()
    h.profile(False)

    # dominant kernel of the step and its roofline
    kinds = {k: v for k, v in prof.items() if v[0] > 0}
    # dominant kernel among the FFT passes (the ones with a byte roofline)
    top = max((k for k in kinds if algorithmic_bytes(k, g, m, 4, mixed=True) is not None),
              key=lambda k: kinds[k][1])
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    # this GPU's own arithmetic rates (FP32, FP64, TF32 tensor), measured here
    probes = measure_peaks(P)
    roof = None
    ab = algorithmic_bytes(top, g, m, 4, mixed=True)
    if ab is not None:
        per_launch_s = kinds[top][1] / 1e3 / kinds[top][0]
        achieved = ab / per_launch_s / 1e9
        roof = {"kernel": top, "bound": "hbm", "achieved": achieved, "peak": hbm_peak,
                "peak_source": peak_src, "unit": "GB/s", "frac": achieved / hbm_peak,
                "traffic": ncu_traffic(args.workload, top), "algorithmic_bytes_per_launch": ab,
                "avg_launch_ms": per_launch_s * 1e3}
    # the same figure for every FFT pass (achieved GB/s of algorithmic bytes)
    roof_all = {}
    for k in kinds:
        b = algorithmic_bytes(k, g, m, 4, mixed=True)
        if b is not None:
            t = kinds[k][1] / 1e3 / kinds[k][0]
            roof_all[k] = {"avg_launch_ms": round(t * 1e3, 4),
                           "achieved_gbs": round(b / t / 1e9, 1),
                           "frac": round(b / t / 1e9 / hbm_peak, 4)}
    # the tensor-core Gram (overlap and subspace matrix, 128 x 128 blocks):
    # three TF32 products per FP32 product, against the measured TF32 MMA rate
    gram_tc = None
    if "gram" in kinds and probes.get("tf32_mma_tflops"):
        nb = (m + 127) // 128
        t = kinds["gram"][1] / 1e3 / kinds["gram"][0]
        # per launch on average: the overlap (nb(nb+1)/2 blocks) and the
        # subspace matrix (nb^2 blocks) alternate
        blocks = 0.5 * (nb * (nb + 1) / 2 + nb * nb)
        ach = 3 * 2 * 128 * 128 * blocks * g.n_points / t / 1e12
        gram_tc = {"bound": "tensor (TF32)", "achieved": ach, "peak": probes["tf32_mma_tflops"],
                   "unit": "TFLOP/s", "frac": ach / probes["tf32_mma_tflops"],
                   "avg_launch_ms": round(t * 1e3, 4),
                   "hbm_gbs": round(1.5 * m * g.n_points * 4 / t / 1e9, 1),
                   "how": "3 TF32 MMA products per FP32 product (hi*hi + hi*lo + lo*hi), "
                          "128 x 128 result blocks; hbm_gbs: the FP32 operands read (one "
                          "block for the overlap, two for the subspace matrix, averaged)"}
    # the whole timed step against the same roofline: its algorithmic bytes
    # (every pass, the term sum, overlap, update, energies) over the step time
    sb = step_bytes(g, m, order // 2)
    step_roof = {"bound": "hbm", "algorithmic_bytes_per_step": sb,
                 "achieved": sb / (dt / args.steps) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                 "frac": sb / (dt / args.steps) / 1e9 / hbm_peak}
    total_prof = sum(v[1] for v in kinds.values())
    dt_prof = max_over_ranks(dt_prof)
    eager = {"value": replicas_value(m * args.steps, dt_prof, world), "unit": "state-steps/s",
             "ms_per_step": 1e3 * dt_prof / args.steps, "steps": args.steps,
             "how": "itp_propagate + itp_orthonormalize + itp_energies, one kernel at a time, "
                    "an event pair around each launch, terms in turn"}
    breakdown = {k: {"launches": v[0], "ms": round(v[1], 3),
                     "share": round(v[1] / total_prof, 4)} for k, v in kinds.items()}
    # cost of one step at every order, and of the Romberg T_6 propagation
    # (Eq. sixp) against the multi-product T_6 (same workload, graph steps)
    order_cost = {}
    for o in (2, 4, 6, 8, 10, 12):
        for _ in range(2):
            h.step_graph(o, tau)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(3):
            h.step_graph(o, tau)
        b.record(stream)
        b.synchronize()
        order_cost[str(o)] = round(a.elapsed_time(b) / 3, 3)
    prop_ms = {}
    for name, fn in (("multi_product_t6", lambda: h.propagate(6, tau)),
                     ("romberg_t6", lambda: h.propagate_romberg6(tau))):
        fn()
        h.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(3):
            fn()
        b.record(stream)
        b.synchronize()
        prop_ms[name] = round(a.elapsed_time(b) / 3, 3)
    h.close()

    # ---- the FP64 form of the same workload -----------------------------------
    fp64 = None
    if not args.no_fp64:
        K = min(args.steps, 3)
        h = P.ItpGrid(g.nx, g.ny, g.nz, g.lx, g.ly, g.lz, w["n_states"], w["n_guard"],
                      P.ITP_FP64, cuda_stream=stream.cuda_stream)
        h.set_potential(V)
        h.set_states(psi)
        tuned64, _ = h.autotune(order, tau)
        for _ in range(3):
            h.step(order, tau, ritz="values")
        barrier()
        h.profile(True)
        dt64, _ = time_steps(h, stream, order, tau, K, torch)
        prof64 = {k: v for k, v in h.profile_read().items() if v[0] > 0}
        tot64 = sum(v[1] for v in prof64.values())
        dt64 = max_over_ranks(dt64)
        fp64 = {"value": replicas_value(m * K, dt64, world), "unit": "state-steps/s", "steps": K,
                "ms_per_step": 1e3 * dt64 / K, "launch_shapes": tuned64,
                "breakdown": {k: {"launches": v[0], "ms": round(v[1], 3),
                                  "share": round(v[1] / tot64, 4)} for k, v in prof64.items()}}
        # the FP64 path is bound by GB300's FP64 rate: its dominant FFT pass
        # against the measured DFMA rate
        top64 = max((k for k in prof64 if fft_pass_flops(k, g, m) is not None),
                    key=lambda k: prof64[k][1], default=None)
        if top64 is not None and probes.get("dfma_tflops"):
            t = prof64[top64][1] / 1e3 / prof64[top64][0]
            ach = fft_pass_flops(top64, g, m) / t / 1e12
            fp64["roofline"] = {"kernel": top64, "bound": "alu (FP64)", "achieved": ach,
                                "peak": probes["dfma_tflops"], "unit": "TFLOP/s",
                                "frac": ach / probes["dfma_tflops"],
                                "avg_launch_ms": round(t * 1e3, 3),
                                "peak_source": "measured (itp_peak_probe DFMA)"}
        h.close()

    # ---- time to n states at tol: mixed vs FP64 --------------------------------
    ttt = None
    ttt_osc = None
    if not args.no_ttt:
        barrier()
        # the metric's own workload: C60-like well, 128^3, n = 120, against
        # the oracle's certified eigenvalues of the grid Hamiltonian
        c60 = TTT_PROBLEMS["c60_128"]
        ttt = {"workload": f"{c60['desc']}, n = 120 + {C60_TTT['guard']} guard, order 12, "
                           f"tau = {C60_TTT['tau']}, seeded random-normal start",
               "reference": f"{c60['eref']} (the oracle's LOBPCG eigenvalues of the grid "
                            "Hamiltonian, certified by residual norms)",
               "tol_ha": 1e-8,
               "mixed": time_to_tol(P, P.ITP_MIXED, per_state=True, fp64_eval=True, margin=100.0,
                                    **C60_TTT),
               "mixed_fp64_polish_steps": time_to_tol(P, P.ITP_MIXED, **C60_TTT)}
        if args.fp64_ttt:
            ttt["fp64"] = time_to_tol(P, P.ITP_FP64, per_state=True, **C60_TTT)
            ttt["speedup_mixed_vs_fp64"] = ttt["fp64"]["seconds"] / ttt["mixed"]["seconds"]
        else:
            # one FP64 step measured; the FP64 path needs at least as many
            # steps as the mixed path took in all (same iteration, FP64 states)
            ttt["fp64"] = fp64_step_extrapolation(P, ttt["mixed"], **C60_TTT)
        if args.ttt_orders:
            # the fixed point of the iteration carries the propagator's time-step
            # error: which orders reach 1e-8 Ha at which tau, and how fast
            sweep_ttt = {}
            for o in (4, 6, 8, 12):
                for t in (0.5, 1.0, 1.5):
                    cfg = dict(C60_TTT, order=o, tau=t, max_fp64=0)
                    r = time_to_tol(P, P.ITP_MIXED, fp64_eval=True, margin=100.0, **cfg)
                    r.pop("launch_shapes", None)
                    sweep_ttt[f"order{o}_tau{t}"] = r
            ttt["by_order_and_tau"] = sweep_ttt
        # the 3D oscillator (exact closed-shell energies) with 8 guard states
        ttt_osc = {"workload": f"{TTT_PROBLEMS['osc_128']['desc']}, n = 120 + 8 guard, "
                               "order 12, tau = 0.5, seeded random-normal start",
                   "tol_ha": 1e-8,
                   "mixed": time_to_tol(P, P.ITP_MIXED, problem="osc_128"),
                   "fp64": time_to_tol(P, P.ITP_FP64, problem="osc_128")}
        ttt_osc["speedup_mixed_vs_fp64"] = (ttt_osc["fp64"]["seconds"]
                                            / ttt_osc["mixed"]["seconds"])
        # order 6 (the fastest order per converged state on one GB300, as the
        # paper found on one processor): FP32 steps at order 6, FP64 polish at
        # order 12; and the FP64 path at order 6
        ttt_osc["order6"] = {"mixed_fp32_order6_polish_order12":
                             time_to_tol(P, P.ITP_MIXED, problem="osc_128", order=6,
                                         polish_order=12),
                             "fp64_order6": time_to_tol(P, P.ITP_FP64, problem="osc_128",
                                                        order=6)}
        # the same problem with the adaptive iteration of Sec. III
        ttt_osc["adaptive"] = {"mixed": adaptive_to_tol(P, P.ITP_MIXED)}
        if args.adaptive_fp64:   # about two minutes on one GB300
            ttt_osc["adaptive"]["fp64"] = adaptive_to_tol(P, P.ITP_FP64)

    # ---- the 32^3 oscillator to 1e-10 Ha (GPU FP64; the oracle beside it) ----
    osc32 = None
    if not args.no_ttt:
        try:
            osc32 = {"workload": "3D harmonic oscillator, 32^3 grid, box [-8,8)^3, n = 10 "
                                 "(three closed shells), order 4, tau = 0.1, FP64, seeded "
                                 "random-normal start", "tol_ha": OSC32["tol"],
                     "gpu_fp64": osc32_gpu(P)}
        except Exception as ex:   # an auxiliary figure never takes the bench line down
            osc32 = {"error": f"{type(ex).__name__}: {ex}"}

    # ---- the batched workload: 64 independent problems, one graph per step ----
    batch = None
    if not args.no_batch:
        barrier()
        batch = batch_throughput(P, torch, args.steps, args.warmup)
        slow = max_over_ranks(batch["ms_per_step"])   # replicas: the slowest rank's time
        batch["value"] = replicas_value(batch["value"] * batch["ms_per_step"] / 1e3, slow / 1e3,
                                        world)
        batch["ms_per_step"] = slow

    sweep = None
    prec_sweep = None
    if not args.no_ttt:
        sweep = order_sweep_small(P)
        prec_sweep = precision_sweep(P)
    planar_case = None
    large = None
    if not args.no_batch:
        barrier()
        planar_case = planar_dots(P, torch, args.steps, args.warmup)
        barrier()
        large = large_c60(P, torch, min(args.steps, 5), args.warmup)

    # ---- CPU oracle on a bounded sample (rank 0, N = 1 only) -------------------
    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample",
                            "--workload", args.workload], capture_output=True, text=True,
                           timeout=900)
        try:
            res = json.loads(r.stdout.strip().splitlines()[-1])
            if osc32 is not None and "osc32" in res:
                osc32["cpu_oracle"] = res["osc32"]
            cpu = {"value": res["value"], "unit": "state-steps/s", "cores": 1, "kind": "oracle",
                   "sample": f"{CPU_SAMPLE_STATES} states of the workload, {CPU_SAMPLE_STEPS} "
                             "oracle steps (propagation, Cholesky, Ritz), "
                             f"{res['seconds']:.1f} s of CPU work",
                   "all_cores": res.get("all_cores")}
        except Exception:
            cpu = {"value": None, "unit": "state-steps/s", "cores": 1, "kind": "oracle",
                   "sample": "failed: " + (r.stderr.strip().splitlines() or ["?"])[-1]}

    if cpu is not None and ttt is not None:
        try:
            ttt["fp64_oracle_extrapolated"] = extrapolate_oracle(
                cpu, ttt, C60_TTT["n"] + C60_TTT["guard"])
        except Exception as ex:   # an auxiliary figure never takes the bench line down
            ttt["fp64_oracle_extrapolated"] = {"error": f"{type(ex).__name__}: {ex}"}

    if rank == 0:
        line = {
            "metric": "state-steps/s", "value": value, "unit": "state-steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "mixed: f32 FFT passes, f64 combination/Cholesky/energies",
            "data": "synthetic (seeded Philox4x32-10 states, C60-like potential)",
            "config": {"workload": w["desc"], "precision": "mixed", "grid": w["n"],
                       "box_bohr": w["box"], "n_states": w["n_states"],
                       "n_guard": w["n_guard"], "order": order, "tau": tau,
                       "l2": "inputs larger than L2 (FP32 state block "
                             f"{m * g.n_points * 4 / 1e9:.2f} GB, half spectrum "
                             f"{m * g.nz * g.ny * (g.nx // 2 + 1) * 8 / 1e9:.2f} GB)",
                       "parallelism": f"replicas x{world} (independent problems)",
                       "timed": "itp_step: each step one CUDA-graph launch of the whole "
                                "step's kernels in stream order (the expansion's terms one "
                                "after another, then the orthonormalisation and the Ritz "
                                "values)"},
            "gpu_launches": launches,
            "launch_shapes": {"chosen": tuned, "autotune": tune_report},
            "roofline": roof,
            "rooflines_fft_passes": roof_all,
            "step_roofline": step_roof,
            "measured_peaks": probes,
            "gram_tensor_roofline": gram_tc,
            "kernel_breakdown": breakdown,
            "eager_profiled": eager,
            "fp64_path": fp64,
            "time_to_tol": ttt,
            "time_to_tol_osc128": ttt_osc,
            "time_to_tol_osc32": osc32,
            "orders": {"ms_per_step_by_order": order_cost,
                       "propagation_ms": prop_ms,
                       "time_to_tol_by_order_ho32": sweep,
                       "mixed_accuracy_by_order_and_tau_ho64": prec_sweep},
            "batch": batch,
            "planar_quantum_dots": planar_case,
            "large_256": large,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "clocks": clk,
            "energies_head": [round(float(x), 8) for x in E[:4]],
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
