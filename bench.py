#!/usr/bin/env python
"""Benchmark: leaf-cell Strang updates per second on one GB300.

One "step" is one Strang step of the BZ reaction-diffusion system on the
adaptive multiresolution grid: grid adaptation, R_{dt/2} (Radau5 per leaf),
D_dt (ROCK4-type per species), R_{dt/2}.  One update is one leaf advanced
through a whole step; value = sum over steps of the leaves / device time.

Default workload (the one the metric is quoted on): 2D BZ, finest level
J = 10 (1024^2), eta = 1e-3, two crossing tanh fronts (w = 0.02) with smooth
seeded position noise, dt = 1e-3, rtol = atol = tol = 1e-6, FP64.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...    (the CPU oracle on the host cores)

Under torchrun (N > 1) every rank runs an independent replica of the
workload (the step does not shard); value = leaves of all ranks / the
slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1506_04651_gb300.inputs import CROSS_J10  # noqa: E402  (generator parameters only)

METRIC = "leaf-cell Strang updates/s on 1 GB300, mixed vs FP64 at rel-L1 ≤1e-5; % roofline"
UNIT = "leaf-updates/s"

WORKLOADS = {
    "bz2d_J10_eta1e-3": dict(d=2, J=10, eta=1e-3, dt=1e-3, gen="cross", seed=2, **CROSS_J10,
                             desc="2D BZ, J=10 (1024^2 finest), eta=1e-3, graded, two crossing "
                                  f"tanh fronts (w={CROSS_J10['w']}) with smooth seeded position noise (8 modes, "
                                  f"amplitude {CROSS_J10['amp']}): 12-17% of finest cells are leaves over steps "
                                  "5-25 (15% initially); dt=1e-3, FP64"),
    "bz2d_J10_cm": dict(d=2, J=10, eta=0.0, dt=1e-3, gen="cross", seed=2, **CROSS_J10, oracle_J=8,
                        desc="2D BZ on the uniform 1024^2 grid (Cartesian mesh: J=10, eta=0), the same crossing "
                             "fronts as the adaptive J=10 workload, dt=1e-3, FP64: the CM side of the paper's "
                             "MR-versus-CM comparison"),
    "bz2d_J7_uniform": dict(d=2, J=7, eta=0.0, dt=1e-3, gen="front", seed=1,
                            desc="2D BZ, uniform 128^2 (J=7, eta=0), tanh front + 1% seeded noise, "
                                 "dt=1e-3, FP64"),
    "bz3d_J7_eta1e-2": dict(d=3, J=7, eta=1e-2, dt=1e-3, gen="sphere", seed=3,
                            desc="3D BZ, J=7 (128^3 finest), eta=1e-2, spherical front r=0.3, "
                                 "w=0.02 + smooth seeded noise, dt=1e-3, FP64"),
    "bz3d_J9_eta1e-2": dict(d=3, J=9, eta=1e-2, dt=1e-3, gen="sphere", seed=3, oracle_J=6,
                            desc="3D BZ, J=9 (512^3 finest, 134M cells), eta=1e-2, spherical front r=0.3, "
                                 "w=0.02 + smooth seeded noise, dt=1e-3, FP64: the HBM-resident point of the "
                                 "3D BZ workload (leaf vectors larger than L2)"),
    "nagumo2d_J10_eta1e-4": dict(d=2, J=10, eta=1e-4, dt=1e-2, gen="nagumo", seed=0, model="nagumo",
                                 desc="2D NAGUMO (k=10, diffusion 0.1), J=10 (1024^2 finest), eta=1e-4, circular "
                                      "front of radius 0.3 with the travelling-front profile, dt=1e-2, FP64: "
                                      "a cheap, non-stiff reaction, so the adaptation's share of the step is "
                                      "large (the paper's Table 3 case)"),
    "nagumo3d_J8_eta1e-3": dict(d=3, J=8, eta=1e-3, dt=1e-2, gen="nagumo", seed=0, model="nagumo", oracle_J=6,
                                desc="3D NAGUMO (k=10, diffusion 0.1), J=8 (256^3 finest), eta=1e-3, spherical "
                                     "front of radius 0.3 with the travelling-front profile, dt=1e-2, FP64"),
    "net3d_J8_eta1e-3": dict(d=3, J=8, eta=1e-3, dt=1e-3, gen="network", seed=5, model="network",
                             oracle_J=4,
                             desc="3D stiff mass-action network, 16 species, 32 reversible reactions "
                                  "A+B<->C+D (seeded species, rates log-U[1e-2,1e6], D log-U[1e-4,1e-2]), "
                                  "J=8 (256^3 finest), eta=1e-3, Gaussian-bump initial state, dt=1e-3, "
                                  "Radau5 on 48x48 Newton systems, FP64"),
    "ionic2d_J9_eta1e-3": dict(d=2, J=9, eta=1e-3, dt=1e-3, gen="ionic", seed=7, model="ionic", oracle_J=6,
                               desc="2D synthetic 21-species membrane model (stand-in for the paper's STROKE "
                                    "case: steep sigmoid gates, log Nernst potentials, eigenvalues to -1e8, "
                                    "numerical Jacobian), J=9 (512^2 finest), eta=1e-3, depolarised ischaemic "
                                    "core r=0.2 (w=0.02, smooth seeded radius noise) in resting tissue, "
                                    "dt=1e-3, Radau5 on 63x63 Newton systems, FP64"),
}
BATCH = {"batch64_bz2d": dict(n=64, dt=1e-3,
                              desc="64 independent 2D BZ instances, seeded J ~ U{7..10}, f ~ U[0.9, 2.0], "
                                   "eta log-uniform in [1e-4, 1e-2], front position ~ U[0.2, 0.8] "
                                   "(master seed 2026); native batch: adaptation and diffusion of every "
                                   "instance on its own stream, reaction half steps as joint Radau5 launches "
                                   "over all instances' leaves; FP64")}
DEFAULT = "bz2d_J10_eta1e-3"
TOL = 1e-6


def initial_state(w, J=None):
    from paper_1506_04651_gb300 import inputs as I
    J = J or w["J"]
    if w["gen"] == "network":
        return I.network_bumps(w["d"], J, w["seed"])
    if w["gen"] == "nagumo":
        return I.nagumo_front(w["d"], J)
    if w["gen"] == "ionic":
        return I.ionic_core(w["d"], J, w["seed"])
    if w["gen"] == "cross":
        return I.bz_cross_2d(J, w["seed"], w=w.get("w", 0.02), amp=w.get("amp", 0.01))
    if w["gen"] == "front":
        return I.bz_front_2d(J, w["seed"])
    return I.bz_sphere_3d(J, w["seed"])


# Radau5 schedule of BZ and NAGUMO contexts (None: the library's default, one thread per cell)
RADAU_SCHEDULE = None


def make_context(mr, w, stream, precision=0):
    """A library context for workload w (BZ, or the network with its reactions set);
    w["max_leaves"], when set, caps the leaf capacity (profiling captures that
    must hold only a few GB on the device)."""
    from paper_1506_04651_gb300 import inputs as I
    cap = dict(precision=precision, max_leaves=w.get("max_leaves", 0))
    if w.get("model") == "network":
        sp, kf, kb, D = I.network_instance(w["seed"])
        c = mr.Context(mr.problem(w["d"], w["J"], model="network", D=D, **cap), stream=stream)
        c.set_network(sp, kf, kb)
        return c
    if w.get("model") == "ionic":
        return mr.Context(mr.problem(w["d"], w["J"], model="ionic", D=I.IONIC_D, **cap), stream=stream)
    if w.get("model") == "nagumo":
        c = mr.Context(mr.problem(w["d"], w["J"], model="nagumo", params=(I.NAGUMO_K,), D=(I.NAGUMO_D,), **cap),
                       stream=stream)
    else:
        c = mr.Context(mr.problem(w["d"], w["J"], **cap), stream=stream)
    if RADAU_SCHEDULE is not None:
        c.set_radau_schedule(RADAU_SCHEDULE)
    return c


def oracle_model(w):
    """(oracle model, diffusion coefficients, species) of workload w."""
    from oracle import oracle as O
    from paper_1506_04651_gb300 import inputs as I
    if w.get("model") == "network":
        sp, kf, kb, D = I.network_instance(w["seed"])
        return O.make_model("network", m=16, params=(sp, kf, kb)), D, 16
    if w.get("model") == "ionic":
        return O.make_model("ionic"), I.IONIC_D, I.IONIC_M
    if w.get("model") == "nagumo":
        return O.make_model("nagumo", params=(I.NAGUMO_K,)), (I.NAGUMO_D,), 1
    return O.make_model("bz"), I.BZ_D, 3


def moiety_basis(w):
    """Rows: a basis of the conserved moieties of the network (left null space
    of the stoichiometric matrix) and the total amount; for the membrane
    model its five linear invariants (ion totals c_k + e_k / beta, with the
    buffer for ion 3, and the charge Cm V - sum z_k c_k - 2 Bt B) followed by
    the sum of the ion totals; None for BZ."""
    from paper_1506_04651_gb300 import inputs as I
    if w.get("model") == "ionic":
        beta, cm, bt, z = 4.0, 3e-9, 0.05, (1.0, 1.0, -1.0, 2.0)
        W = np.zeros((6, 21))
        for k in range(4):
            W[k, 5 + k], W[k, k] = 1.0, 1.0 / beta
        W[3, 19] = bt
        W[4, 9], W[4, 5:9], W[4, 19] = cm, [-v for v in z], -2.0 * bt
        W[5] = W[0] + W[1] + W[2] + W[3]
        return W
    if w.get("model") != "network":
        return None
    sp = I.network_instance(w["seed"])[0]
    S = np.zeros((16, len(sp)))
    for r, (a, b, c, d) in enumerate(sp):
        S[a, r] -= 1
        S[b, r] -= 1
        S[c, r] += 1
        S[d, r] += 1
    _, sv, Vt = np.linalg.svd(S.T)
    return np.vstack([Vt[int((sv > 1e-10).sum()):], np.ones(16)])


def profiled_traffic(kernel_file, summary):
    """DRAM bytes per launch recorded in profiles/<summary> by an ncu capture,
    or None when the kernel's source has changed since that capture."""
    import hashlib
    import re
    try:
        text = open(os.path.join(ROOT, "profiles", summary)).read()
        src = open(os.path.join(ROOT, "paper_1506_04651_gb300", "csrc", kernel_file), "rb").read()
    except OSError:
        return None
    sha = re.search(r"source_sha256_16: ([0-9a-f]{16})", text)
    tb = re.search(r"traffic_bytes_per_launch: (\d+)", text)
    if not sha or not tb or hashlib.sha256(src).hexdigest()[:16] != sha.group(1):
        return None
    return int(tb.group(1))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in self.rows for q in range(4) if r[5 + q].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def aggregate_replicas(pg, ms, leaves, dev):
    """Replicas (one independent instance per rank): the job's time is the
    slowest rank's, its work the leaf updates of all ranks.  pg is
    torch.distributed (or None for one rank)."""
    if pg is None:
        return ms, leaves
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    n = torch.tensor([float(leaves)], dtype=torch.float64, device=dev)
    pg.all_reduce(n, op=pg.ReduceOp.SUM)
    return float(t.item()), float(n.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_oracle_rate(w, u0, budget_s=20.0, max_steps=100, threads=1, want_state=False):
    """The oracle as it stands (C, `threads` threads in its parallel-for),
    Strang steps on the same workload until the time budget is spent;
    returns (rate, steps, cores), plus its final leaves when want_state."""
    from oracle import oracle as O
    md, D, m = oracle_model(w)
    J = w.get("oracle_J", w["J"])
    T = O.Tree(w["d"], J, m, jmin=2)
    T.set_full(u0)
    assert T.adapt(w["eta"]) == 0
    O.set_threads(threads)
    leaves, t_tot, steps = 0, 0.0, 0
    try:
        while steps < max_steps and t_tot < budget_s:
            t0 = time.perf_counter()
            rc = T.strang(md, D, w["dt"], w["eta"], TOL, TOL, TOL)
            t_tot += time.perf_counter() - t0
            assert rc == 0, rc
            leaves += T.num_leaves()
            steps += 1
    finally:
        O.set_threads(1)
    if want_state:
        return leaves / t_tot, steps, threads, T.leaves()
    return leaves / t_tot, steps, threads


def radau_work(model, m):
    """FP64 operations per counted event of the one-thread-per-cell Radau5
    kernel, the closed forms in m counted from its source (include/mr.h,
    csrc/radau_common.cuh); None for the team-kernel models."""
    if model not in ("bz", "nagumo"):
        return None
    lu_real = m + m * (m - 1) / 2 + m * (m - 1) * (2 * m - 1) / 3
    lu_cplx = m * (m + 1) / 2 + 6 * m + 3 * m * (m - 1) + 4 * m * (m - 1) * (2 * m - 1) / 3
    sol_real = m + 2 * m * (m - 1)
    return {"rhs": 13 if model == "bz" else 4, "jac": 10 if model == "bz" else 5,
            "dec": 6 + 2 * m + lu_real + lu_cplx, "newton": 62 * m + 10 * m * (m - 1) + 3, "monitor": 6,
            "attempt": 19 + 18 * m, "extrap": 55 + 18 * m, "accept": (5 + 13 * m + sol_real) + 4 + (11 + m)}


def radau_flops(work, cnt):
    """Lower bound of a run's algorithmic FP64 operations from the Radau5
    counters (fev, jac, steps, accept, reject, newton, dec, cells)."""
    fev, jac, nstep, nacc, nrej, nnew, ndec, cells = cnt
    return (work["rhs"] * fev + work["jac"] * jac + work["dec"] * ndec + work["newton"] * nnew
            + work["monitor"] * max(0, nnew - nstep) + work["attempt"] * nstep
            + work["extrap"] * max(0, nstep - cells - nrej) + work["accept"] * nacc)


def run_reference(args, w):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    oj = w.get("oracle_J", w["J"])
    u0 = initial_state(w, oj)
    budget = min(240.0, 20.0 + 2.0 * args.steps)
    rate, steps, cores = cpu_oracle_rate(w, u0, budget_s=budget, max_steps=args.steps, threads=host_cores())
    form = (f"C oracle, parallel-for over leaves in the reaction and over rows in every diffusion sweep "
            f"on {cores} host threads, no algorithmic change")
    sample = (f"first {steps} Strang steps of the workload from its initial grid ({form})"
              if oj == w["J"] else
              f"first {steps} Strang steps of the same problem at finest level J={oj} instead of {w['J']} "
              f"({form}; the full size takes minutes per step)")
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": ws,
            "steps": steps, "warmup": 0, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "desc": w["desc"], "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(args, w):
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_1506_04651_gb300 import mr

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist
    stream = torch.cuda.current_stream()
    u0 = initial_state(w)
    ctx = make_context(mr, w, stream)
    ctx.build(torch.from_numpy(u0).to(dev), w["eta"])
    basis = moiety_basis(w)

    def step():
        ctx.strang(w["dt"], w["eta"], TOL, TOL, TOL)

    for _ in range(args.warmup):
        step()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    # the state at the start of the timed region, kept on the host: the
    # end-to-end measurement replays the same steps from it
    k_start, v_start = ctx.leaves()
    mass0 = ctx.mass()
    st0 = ctx.stats()
    clocks = ClockSampler(local)
    clocks.start()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    leaves, nmax = 0, len(k_start)
    phase_sum = {"adapt_and_tables": 0.0, "react_both_halves": 0.0, "diffuse": 0.0}
    nodes_sum = 0
    for k in range(args.steps):
        flush.zero_()
        ev0[k].record(stream)
        step()
        ev1[k].record(stream)
        sk = ctx.stats()
        nk = sk["leaves"]
        leaves += nk
        nmax = max(nmax, nk)
        phase_sum["adapt_and_tables"] += sk["ms_adapt"]
        phase_sum["react_both_halves"] += sk["ms_react"]
        phase_sum["diffuse"] += sk["ms_diffuse"]
        nodes_sum += sk["nodes"]
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    clk = clocks.stop()
    st1 = ctx.stats()
    mass1 = ctx.mass()
    ms = sum(a.elapsed_time(b) for a, b in zip(ev0, ev1))
    conservation = None
    if basis is not None:
        y0, y1 = basis @ mass0, basis @ mass1
        conservation = {"total_amount_rel_drift": float(abs(y1[-1] - y0[-1]) / abs(y0[-1])),
                        "moiety_max_drift_rel_to_total": float(np.max(np.abs(y1 - y0)) / abs(y0[-1])),
                        "moieties": int(len(basis)), "steps": args.steps}
    ms, total_leaves = aggregate_replicas(pg, ms, leaves, dev)
    value = total_leaves / (ms * 1e-3)

    # kernel-level roofline figures over the timed region
    rad_ms = st1["radau_kernel_ms"] - st0["radau_kernel_ms"]
    rad_n = st1["radau_kernel_launches"] - st0["radau_kernel_launches"]
    rad_fl = st1["radau_alg_flops"] - st0["radau_alg_flops"]
    rock_ms = st1["rock_kernel_ms"] - st0["rock_kernel_ms"]
    rock_n = st1["rock_kernel_launches"] - st0["rock_kernel_launches"]
    rock_b = st1["rock_alg_bytes"] - st0["rock_alg_bytes"]
    launches = st1["kernel_launches"] - st0["kernel_launches"]
    peaks = measured_peaks()
    fp64_tf, fp64_mhz = mr.fp64_fma_rate()
    hbm = peaks.get("hbm_gbs")
    if rad_ms >= rock_ms:
        ach = rad_fl / (rad_ms * 1e-3) / 1e12
        kname = ("k_radau_team (Radau5, one 16-lane team per cell, FP64)" if w.get("model") == "network"
                 else "k_radau_team (Radau5, one warp per cell, numerical Jacobian, FP64)"
                 if w.get("model") == "ionic" else "k_radau_pool (Radau5, phase-sorted cell pool, FP64)"
                 if RADAU_SCHEDULE == 1 else "k_radau (Radau5, one thread per cell, FP64)")
        roof = {"bound": "alu", "kernel": kname, "achieved": ach, "peak": fp64_tf,
                "unit": "TFLOP/s", "frac": ach / fp64_tf,
                "traffic": profiled_traffic("radau5.cu", "k_radau_pool_bz2d_J10.md" if RADAU_SCHEDULE == 1
                                            else "k_radau_bz2d_J10.md")
                if args.workload == DEFAULT else None,
                "peak_source": "measured FP64 FMA rate of this GPU (library probe, 2 flop/FMA)",
                "launches": rad_n, "ms_per_launch": rad_ms / max(rad_n, 1)}
    else:
        roof = rock_roofline(rock_b, st1["rock_alg_flops"] - st0["rock_alg_flops"], rock_ms, hbm, fp64_tf,
                             mixed_form=False)
        roof.update({"traffic": profiled_traffic("rock4.cu", "k_rock_persistent_bz2d_J10.md")
                     if args.workload == DEFAULT else None, "launches": rock_n,
                     "ms_per_launch": rock_ms / max(rock_n, 1)})
    # adaptation: algorithmic bytes per step = for the tree before and after
    # (about the same size), every node's m values (8 B each), code (4 B) and
    # level (1 B) read or written once, plus its tag byte
    m_sp = ctx.m
    adapt_ms = phase_sum["adapt_and_tables"] / args.steps
    adapt_b = 2.0 * (nodes_sum / args.steps) * (8.0 * m_sp + 4.0 + 1.0 + 1.0)
    adapt_ach = adapt_b / (adapt_ms * 1e-3) / 1e9 if adapt_ms else 0.0
    roof_adapt = {"bound": "hbm", "kernel": "adaptation and operator tables (the whole phase)",
                  "achieved": adapt_ach, "peak": hbm or 6800.0, "unit": "GB/s",
                  "frac": adapt_ach / (hbm or 6800.0),
                  "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if hbm else "fallback 6.8 TB/s",
                  "note": "algorithmic bytes (values, code, level and tag of every node of the old and new tree, "
                          "once) over the phase's event time per step; the phase is launch- and latency-bound "
                          "(tens of small kernels, a few host synchronisations to size the new tree)"}
    roof_rock = rock_roofline(rock_b, st1["rock_alg_flops"] - st0["rock_alg_flops"], rock_ms, hbm, fp64_tf,
                              mixed_form=False)
    rad_cnt = [b - a for a, b in zip(st0["radau_counters"], st1["radau_counters"])]
    work = radau_work(w.get("model", "bz"), ctx.m)
    kernels = {"radau": {"ms": rad_ms, "launches": rad_n, "tflops": rad_fl / max(rad_ms, 1e-9) / 1e9,
                         "counters": dict(zip(("fev", "jac", "steps", "accept", "reject", "newton", "dec", "cells"),
                                              rad_cnt)),
                         "work_per_event": work,
                         "alg_flops": rad_fl,
                         "alg_flops_from_counters": radau_flops(work, rad_cnt) if work else None,
                         "note": "achieved = alg_flops / ms; alg_flops = sum of counters x work_per_event "
                                 "(lower bound: extrapolated attempts >= steps - cells - reject, error "
                                 "estimates of accepted steps only)"},
               "rock": {"ms": rock_ms, "launches": rock_n,
                        "gbs": rock_b / max(rock_ms, 1e-9) / 1e6},
               "step_ms": ms / args.steps,
               # CUDA-event phases of every timed step, averaged; the rest of
               # the step is host time between the phases (synchronisations,
               # launches) and the call's entry and return
               "phase_ms_per_step": {k: v / args.steps for k, v in phase_sum.items()},
               "host_gap_ms_per_step": ms / args.steps - sum(phase_sum.values()) / args.steps}

    # end to end through the C-ABI with host buffers, replaying the timed
    # steps from the same starting state: every step the state goes in from
    # pinned host memory, the step runs, the state comes out
    m = ctx.m
    cap = nmax
    hk = torch.empty(cap, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
    hv = torch.empty(m * cap, dtype=torch.float64, pin_memory=True).numpy()
    hk2 = torch.empty(cap, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
    hv2 = torch.empty(m * cap, dtype=torch.float64, pin_memory=True).numpy()
    n0 = len(k_start)
    keys, vals = hk[:n0], hv[:m * n0].reshape(m, n0)
    keys[:] = k_start
    vals[:] = v_start
    del k_start, v_start
    n_e2e = args.steps
    h2d = d2h = 0
    e2e_leaves = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        ctx.set_leaves(keys, vals)
        h2d += keys.nbytes + vals.nbytes
        step()
        n = ctx.num_leaves()
        e2e_leaves += n
        keys, vals = ctx.leaves(hk2[:n], hv2[:m * n].reshape(m, n))
        d2h += keys.nbytes + vals.nbytes
        hk, hk2, hv, hv2 = hk2, hk, hv2, hv
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    e2e = {"value": e2e_leaves / t_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d // n_e2e,
           "d2h_bytes_per_step": d2h // n_e2e, "steps": n_e2e,
           "note": "the timed steps replayed from the same starting state: mr_set_leaves(host) + "
                   "strang_step + mr_get_leaves(host) per step, wall clock"}

    # mixed form (FP32 Newton factorisations in Radau5) on the same workload and
    # the same number of steps from the same initial grid; its final state is
    # compared with the FP64 path's after the same steps (relative L1 on the
    # finest grid)
    # the leaf operator in its compact form against the same operator as a
    # CSR matrix, on the tree the timed steps ended with (App. C, Table 5)
    forms = ctx.operator_forms(reps=50)
    forms["ratio_compact_over_csr"] = forms["ms_compact"] / forms["ms_csr"]
    mixed = None
    if not args.no_mixed:
        mixed = run_mixed(args, w, mr, torch, dev, stream, u0)
    hbm_point = None
    extras = None
    if args.workload == DEFAULT and not args.no_hbm_extra and not args.J:
        hbm_point = run_hbm_point(mr, torch, dev, stream, hbm, fp64_tf)
        extras = run_extras(args, mr, torch, dev, stream, fp64_tf, hbm)
    if pg:
        pg.barrier()
    if rank != 0:
        ctx.close()
        return
    cpu = None
    final = mixed.pop("_final") if mixed else None
    if ws == 1 and not args.no_cpu_baseline:
        oj = w.get("oracle_J", w["J"])
        where = ("the same workload" if oj == w["J"] else
                 f"the same problem at finest level J={oj} (the full size takes minutes per oracle step)")
        # at full size the oracle runs the same warm-up + timed steps as the
        # mixed comparison (within a bounded budget), and its final state is
        # the reference of the mixed and FP64 errors
        full = oj == w["J"] and final is not None
        nst = args.warmup + args.steps
        rate, steps, cores, ostate = cpu_oracle_rate(w, initial_state(w, oj), budget_s=45.0 if full else 12.0,
                                                     max_steps=nst if full else 50, threads=host_cores(),
                                                     want_state=True)
        if full and steps == nst:
            ko, vo = ostate
            mixed["rel_l1_vs_fp64_oracle"] = rel_l1_finest(*final["mixed"], ko, vo, w["d"], w["J"])
            mixed["fp64_path_rel_l1_vs_fp64_oracle"] = rel_l1_finest(*final["fp64"], ko, vo, w["d"], w["J"])
            mixed["fp64_path_grid_equals_oracle"] = bool(np.array_equal(final["fp64"][0], ko))
            mixed["f32_details"]["rel_l1_vs_fp64_oracle"] = rel_l1_finest(*final["f32_details"], ko, vo, w["d"],
                                                                          w["J"])
            mixed["oracle_steps"] = steps
        rate1, steps1, _ = cpu_oracle_rate(w, initial_state(w, oj), budget_s=12.0, max_steps=50, threads=1)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"first {steps} Strang steps of {where} from its initial grid (C oracle, "
                         f"parallel-for over leaves in the reaction and rows in every diffusion sweep, "
                         f"{cores} threads, no algorithmic change; ~12 s budget)",
               "single_thread": {"value": rate1, "cores": 1, "steps": steps1}}
    st = ctx.stats()
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "desc": w["desc"],
                       "l2": "flushed between timed steps (256 MB write)",
                       "leaves_last_step": st["leaves"], "compression_ratio": st["compression_ratio"],
                       "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                       "radau_schedule": "pool" if RADAU_SCHEDULE == 1 else "thread"},
            "roofline": roof, "roofline_rock4": roof_rock, "roofline_adapt": roof_adapt, "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clk, "mixed": mixed, "hbm_point": hbm_point, "extras": extras,
            "operator_forms": forms,
            "cm_over_mr_step_time": (extras["bz2d_J10_cm"]["ms_per_step"] / (ms / args.steps)) if extras else None,
            "fp64_probe": {"tflops": fp64_tf, "sm_mhz_attr": fp64_mhz}}
    if conservation:
        line["conservation"] = conservation
    print(json.dumps(line), flush=True)
    ctx.close()
    if pg:
        pg.destroy_process_group()


def finest_grid(keys, vals, d, J):
    """Leaf values injected piecewise-constant onto the level-J grid
    (lexicographic, x fastest)."""
    keys = np.asarray(keys, dtype=np.uint64)
    lev = (keys >> np.uint64(48)).astype(np.int64)
    code = (keys & np.uint64((1 << 48) - 1)).astype(np.int64)
    n = 1 << J
    out = np.zeros((vals.shape[0],) + (n,) * d)
    for j in np.unique(lev):
        sel = np.nonzero(lev == j)[0]
        k = np.zeros((d, len(sel)), dtype=np.int64)
        for b in range(j):
            for a in range(d):
                k[a] |= ((code[sel] >> (d * b + (d - 1 - a))) & 1) << b
        bsz = 1 << (J - j)
        offs = np.arange(bsz)
        idx = []
        for a in range(d):
            shape = [len(sel)] + [1] * d
            shape[1 + (d - 1 - a)] = bsz
            idx.append(((k[a] * bsz)[:, None] + offs[None, :]).reshape(shape))
        for i in range(vals.shape[0]):
            out[(i,) + tuple(idx[a] for a in reversed(range(d)))] = vals[i, sel].reshape([len(sel)] + [1] * d)
    return out.reshape(vals.shape[0], -1)


def rel_l1_finest(ka, va, kb, vb, d, J):
    """max over species of |a - b|_1 / |b|_1 over the finest grid (b the reference)."""
    A, B = finest_grid(ka, va, d, J), finest_grid(kb, vb, d, J)
    return max(float(np.sum(np.abs(A[i] - B[i])) / max(np.sum(np.abs(B[i])), 1e-300)) for i in range(len(B)))


def rock_roofline(nbytes, flops, ms, hbm, fp64_tf, mixed_form):
    """The ROCK4 sweeps against their binding limit: HBM bandwidth, or for
    the FP64 form the FP64 pipe at the sweeps' arithmetic intensity
    (flops per algorithmic byte), whichever is lower."""
    peak_hbm = hbm or 6800.0
    gbs = nbytes / (ms * 1e-3) / 1e9 if ms else 0.0
    fpb = flops / nbytes if nbytes else 0.0
    fp64_bound = fp64_tf * 1e3 / fpb if fpb and not mixed_form else None
    binding = min(peak_hbm, fp64_bound) if fp64_bound else peak_hbm
    return {"bound": "hbm" if binding == peak_hbm else "alu",
            "kernel": "k_rock_persistent (ROCK4 sweeps, whole diffusion sub-step)",
            "achieved": gbs, "peak": binding, "unit": "GB/s", "frac": gbs / binding,
            "hbm_peak": peak_hbm, "frac_of_hbm": gbs / peak_hbm,
            "peak_source": ("min(HBM, FP64 FMA rate x bytes per flop)" if not mixed_form else "HBM") +
                           (" -- HBM from MEASURED_PEAKS.json (of measured)" if hbm else " -- HBM fallback 6.8 TB/s"),
            "flops": flops, "flops_per_byte": fpb,
            "tflops": flops / (ms * 1e-3) / 1e12 if ms else 0.0,
            "frac_of_fp64_peak": (flops / (ms * 1e-3) / 1e12) / fp64_tf if ms and not mixed_form else None,
            "note": "algorithmic bytes of the sweeps (tables and merged rows once per sweep, vectors read and "
                    "written once) and their arithmetic, over the launch time"}


def run_hbm_point(mr, torch, dev, stream, hbm, fp64_tf, steps=3, warmup=2):
    """The HBM-resident point of the 3D BZ workload (J = 9, 512^3 finest,
    leaf vectors larger than L2) as a bounded extra of the default line: a
    few CUDA-event-timed steps with the L2 flushed before each, in the FP64
    and the mixed form, and the rooflines of its ROCK4 sweeps (against
    min(HBM, the FP64 pipe at their intensity) in FP64, against HBM in the
    mixed form), its Radau5 launches and its adaptation."""
    w = WORKLOADS["bz3d_J9_eta1e-2"]
    t0 = time.perf_counter()
    u0 = initial_state(w)
    peak = hbm or 6800.0
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    forms = {}
    out = {"workload": "bz3d_J9_eta1e-2", "desc": w["desc"], "steps": steps, "warmup": warmup, "unit": UNIT,
           "l2": "flushed before every timed step (256 MB write); state and work vectors exceed L2"}
    for prec, tag in ((mr.MR_FP64, "fp64"), (mr.MR_MIXED, "mixed")):
        ctx = make_context(mr, w, stream, precision=prec)
        ctx.build(torch.from_numpy(u0).to(dev), w["eta"])
        for _ in range(warmup):
            ctx.strang(w["dt"], w["eta"], TOL, TOL, TOL)
        st0 = ctx.stats()
        ms, leaves, nodes = 0.0, 0, 0
        ph = {"adapt_and_tables": 0.0, "react_both_halves": 0.0, "diffuse": 0.0}
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.strang(w["dt"], w["eta"], TOL, TOL, TOL)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            sk = ctx.stats()
            leaves += sk["leaves"]
            nodes += sk["nodes"]
            ph["adapt_and_tables"] += sk["ms_adapt"]
            ph["react_both_halves"] += sk["ms_react"]
            ph["diffuse"] += sk["ms_diffuse"]
        st1 = ctx.stats()
        if prec == mr.MR_FP64:
            forms = ctx.operator_forms(reps=20)
        ctx.close()
        rock_ms = st1["rock_kernel_ms"] - st0["rock_kernel_ms"]
        rock = rock_roofline(st1["rock_alg_bytes"] - st0["rock_alg_bytes"],
                             st1["rock_alg_flops"] - st0["rock_alg_flops"], rock_ms, hbm, fp64_tf,
                             mixed_form=prec != mr.MR_FP64)
        rock["ms_per_launch"] = rock_ms / max(1, st1["rock_kernel_launches"] - st0["rock_kernel_launches"])
        rad_ms = st1["radau_kernel_ms"] - st0["radau_kernel_ms"]
        rad_fl = st1["radau_alg_flops"] - st0["radau_alg_flops"]
        adapt_ms = ph["adapt_and_tables"] / steps
        adapt_b = 2.0 * (nodes / steps) * (8.0 * 3 + 6.0)
        rec = {"value": leaves / (ms * 1e-3), "ms_per_step": ms / steps, "leaves_last_step": st1["leaves"],
               "irregular_rows": st1["irregular_rows"], "irregular_nnz": st1["irregular_nnz"],
               "phase_ms_per_step": {k: v / steps for k, v in ph.items()}, "roofline_rock4": rock,
               "roofline_adapt": {"bound": "hbm", "achieved": adapt_b / (adapt_ms * 1e-3) / 1e9, "peak": peak,
                                  "unit": "GB/s", "frac": adapt_b / (adapt_ms * 1e-3) / 1e9 / peak}}
        if prec == mr.MR_FP64:
            rec["roofline_radau"] = {"bound": "alu", "achieved": rad_fl / (rad_ms * 1e-3) / 1e12, "peak": fp64_tf,
                                     "unit": "TFLOP/s", "frac": rad_fl / (rad_ms * 1e-3) / 1e12 / fp64_tf}
            out.update(rec)
        else:
            rec["speedup_vs_fp64"] = rec["value"] / out["value"]
            out["mixed"] = rec
    out["operator_forms"] = dict(forms, ratio_compact_over_csr=forms["ms_compact"] / forms["ms_csr"],
                                 paper_ratio_3d="0.67 (BZ 3D J=10, 40 Haswell threads, App. C Table 5)")
    out["wall_s"] = time.perf_counter() - t0
    return out


def run_extras(args, mr, torch, dev, stream, fp64_tf, hbm):
    """Bounded extras of the default line, so that one run of the default
    bench also measures the 3D J = 7 workload (cfg 3) and the 64-instance
    batch (cfg 4): a few CUDA-event-timed steps each, the L2 flushed before
    each 3D step, FP64 and the mixed form."""
    out = {}
    w = WORKLOADS["bz3d_J7_eta1e-2"]
    u0 = initial_state(w)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    res = {}
    for prec in (mr.MR_FP64, mr.MR_MIXED):
        c = make_context(mr, w, stream, precision=prec)
        c.build(torch.from_numpy(u0).to(dev), w["eta"])
        for _ in range(3):
            c.strang(w["dt"], w["eta"], TOL, TOL, TOL)
        st0 = c.stats()
        ms, leaves = 0.0, 0
        for _ in range(5):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            c.strang(w["dt"], w["eta"], TOL, TOL, TOL)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            leaves += c.stats()["leaves"]
        st1 = c.stats()
        res[prec] = (leaves / (ms * 1e-3), ms / 5, c.leaves(), st0, st1)
        c.close()
    v64, ms64, (kf, vf), st0, st1 = res[mr.MR_FP64]
    rad_ms = st1["radau_kernel_ms"] - st0["radau_kernel_ms"]
    rad_fl = st1["radau_alg_flops"] - st0["radau_alg_flops"]
    out["bz3d_J7_eta1e-2"] = {
        "desc": w["desc"], "steps": 5, "warmup": 3, "value": v64, "unit": UNIT, "ms_per_step": ms64,
        "leaves_last_step": st1["leaves"],
        "roofline_radau": {"bound": "alu", "achieved": rad_fl / (rad_ms * 1e-3) / 1e12, "peak": fp64_tf,
                           "unit": "TFLOP/s", "frac": rad_fl / (rad_ms * 1e-3) / 1e12 / fp64_tf},
        "roofline_rock4": rock_roofline(st1["rock_alg_bytes"] - st0["rock_alg_bytes"],
                                        st1["rock_alg_flops"] - st0["rock_alg_flops"],
                                        st1["rock_kernel_ms"] - st0["rock_kernel_ms"], hbm, fp64_tf, False),
        "mixed": {"value": res[mr.MR_MIXED][0], "speedup_vs_fp64": res[mr.MR_MIXED][0] / v64,
                  "rel_l1_vs_fp64_path": rel_l1_finest(*res[mr.MR_MIXED][2], kf, vf, w["d"], w["J"])},
        "l2": "flushed before every timed step"}
    # the uniform 1024^2 grid of the same fronts (Cartesian mesh, eta = 0):
    # the CM side of the paper's MR-versus-CM comparison (Tables 1-2)
    wc = WORKLOADS["bz2d_J10_cm"]
    c = make_context(mr, wc, stream)
    c.build(torch.from_numpy(initial_state(wc)).to(dev), wc["eta"])
    for _ in range(3):
        c.strang(wc["dt"], wc["eta"], TOL, TOL, TOL)
    ms = 0.0
    for _ in range(5):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c.strang(wc["dt"], wc["eta"], TOL, TOL, TOL)
        e1.record(stream)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
    cells = c.stats()["leaves"]
    c.close()
    out["bz2d_J10_cm"] = {"desc": wc["desc"], "steps": 5, "warmup": 3, "value": cells * 5 / (ms * 1e-3),
                          "unit": "cell-updates/s", "ms_per_step": ms / 5,
                          "note": "ms_per_step against the default line's adaptive step gives the CM/MR step-time "
                                  "ratio (the paper: 4.4 for BZ 2D J=10 on 40 Haswell threads, Table 1)"}
    del flush
    bargs = argparse.Namespace(**dict(vars(args), steps=3, warmup=4, no_mixed=False, threads=0, instances=0))
    line = run_batch(bargs, BATCH["batch64_bz2d"], print_line=False)
    out["batch64_bz2d"] = {k: line[k] for k in ("value", "unit", "ms_per_step", "steps", "warmup", "roofline",
                                                "mixed", "autotuner", "kernels", "e2e", "gpu_launches")}
    out["batch64_bz2d"]["desc"] = BATCH["batch64_bz2d"]["desc"]
    return out


def run_mixed(args, w, mr, torch, dev, stream, u0):
    nsteps = args.warmup + args.steps
    res = {}
    for prec in (mr.MR_FP64, mr.MR_MIXED, mr.MR_MIXED_F32_DETAILS):
        c = make_context(mr, w, stream, precision=prec)
        c.build(torch.from_numpy(u0).to(dev), w["eta"])
        for _ in range(args.warmup):
            c.strang(w["dt"], w["eta"], TOL, TOL, TOL)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ms, leaves = 0.0, 0
        for _ in range(args.steps):
            e0.record(stream)
            c.strang(w["dt"], w["eta"], TOL, TOL, TOL)
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
            leaves += c.stats()["leaves"]
        keys, vals = c.leaves()
        res[prec] = (leaves / (ms * 1e-3), ms / args.steps, keys, vals)
        c.close()
    kf, vf = res[mr.MR_FP64][2], res[mr.MR_FP64][3]
    km, vm = res[mr.MR_MIXED][2], res[mr.MR_MIXED][3]
    # on the finest grid, so that leaves one form refined and the other not
    # (a detail at the threshold rounded to the other side) still count
    err = rel_l1_finest(km, vm, kf, vf, w["d"], w["J"]) if w["d"] * w["J"] <= 24 else None
    # the same norm over the leaves both grids share: the arithmetic's part
    # of the difference, without the cells one form refined and the other not
    _, i_f, i_m = np.intersect1d(kf, km, assume_unique=True, return_indices=True)
    vol_c = np.ldexp(1.0, (w["d"] * (w["J"] - (kf[i_f] >> np.uint64(48)).astype(np.int64))).astype(np.int32))
    err_common = max(float(np.sum(vol_c * np.abs(vm[i][i_m] - vf[i][i_f])) / max(np.sum(vol_c * np.abs(vf[i][i_f])), 1e-300))
                     for i in range(len(vf)))
    # the option with FP32 details: the cells where its grid and the FP64
    # path's differ (leaves of one and not the other) are the grid flips
    kd, vd = res[mr.MR_MIXED_F32_DETAILS][2], res[mr.MR_MIXED_F32_DETAILS][3]
    f32d = {"value": res[mr.MR_MIXED_F32_DETAILS][0], "ms_per_step": res[mr.MR_MIXED_F32_DETAILS][1],
            "speedup_vs_fp64": res[mr.MR_MIXED_F32_DETAILS][0] / res[mr.MR_FP64][0],
            "rel_l1_vs_fp64_path": rel_l1_finest(kd, vd, kf, vf, w["d"], w["J"]) if w["d"] * w["J"] <= 24 else None,
            "grid_flips_vs_fp64_path": int(len(np.setxor1d(kd, kf, assume_unique=True))),
            "leaves": int(len(kd)),
            "form": "as the mixed form, and the MR details predicted and differenced in FP32 from the FP64 "
                    "node values (thresholds and normalisation in FP64)"}
    return {"value": res[mr.MR_MIXED][0], "ms_per_step": res[mr.MR_MIXED][1],
            "fp64_value_same_run": res[mr.MR_FP64][0], "speedup_vs_fp64": res[mr.MR_MIXED][0] / res[mr.MR_FP64][0],
            "rel_l1_vs_fp64_path": err, "steps": nsteps,
            "grids_equal": bool(np.array_equal(kf, km)), "leaves_fp64": int(len(kf)), "leaves_mixed": int(len(km)),
            "rel_l1_on_common_leaves": err_common,
            "form": "Radau5 Newton factorisations and solves, and the starting values and tolerance scales of each step attempt, in FP32; ROCK4 stage vectors in FP32; "
                    "Radau5 residuals, both error norms, step control, the state between sub-steps, "
                    "details and mass in FP64",
            "note": "no L2 flush between these steps; the FP64 path matches the oracle to 1e-9 per step",
            "f32_details": f32d,
            "_final": {"fp64": (kf, vf), "mixed": (km, vm), "f32_details": (kd, vd)}}


def run_batch(args, b, print_line=True):
    """Batched serving workload through the native batch (mr_batch_*): every
    instance adapts and diffuses on its own stream, the reaction half steps of
    all instances are joint Radau5 launches.  value = leaves of all instances
    and steps / the run's device time (CUDA events around mr_batch_run)."""
    import torch
    import __graft_entry__ as g
    g.build()
    from paper_1506_04651_gb300 import inputs as I
    from paper_1506_04651_gb300 import mr

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    insts = I.batch_instances(b["n"])
    eta = [inst["eta"] for inst in insts]
    u0s = [I.bz_front_smooth_2d(inst["J"], inst["seed"] & 0xFFFFFFFF, x0=inst["x0"], f=inst["f"]) for inst in insts]

    def make(prec):
        B = mr.Batch([mr.problem(2, inst["J"], params=(1e-2, 1e-5, inst["f"], 2e-3), precision=prec)
                      for inst in insts], threads=args.threads)
        for k, inst in enumerate(insts):
            B[k].build(torch.from_numpy(u0s[k]).to(dev), inst["eta"])
        return B

    B = make(mr.MR_FP64)
    # at least 4 warm-up steps: the autotuner's trials (4 Radau5 shapes and 2
    # ROCK4 shapes, each twice) are then over before the timed steps
    warm = max(args.warmup, 4)
    B.run(warm, b["dt"], eta, TOL, TOL, TOL)
    start = [B[k].leaves() for k in range(B.n)]  # the timed steps' starting state, for the e2e replay
    launches0 = sum(B[k].stats()["kernel_launches"] for k in range(B.n))
    clocks = ClockSampler(local)
    clocks.start()
    torch.cuda.synchronize()
    B.run(args.steps, b["dt"], eta, TOL, TOL, TOL)
    torch.cuda.synchronize()
    clk = clocks.stop()
    st = B.stats()
    tuning = B.tuning()  # the autotuner's trials (made during the warm-up steps) and its choice
    launches = sum(B[k].stats()["kernel_launches"] for k in range(B.n)) - launches0 + st["react_launches"]
    ms = st["ms_device"]
    value = st["leaf_updates"] / (ms * 1e-3)
    fp64_tf, _ = mr.fp64_fma_rate()
    ach = st["radau_alg_flops"] / (st["ms_react_kernel"] * 1e-3) / 1e12 if st["ms_react_kernel"] else 0.0
    chosen = [e for e in tuning if e["phase"] == "reaction" and e["chosen"]]
    kname = ("k_radau_pool" if not chosen or chosen[0]["schedule"] == "pool" else "k_radau")
    roof = {"bound": "alu", "kernel": kname + " (joint Radau5 launch over all instances, the autotuner's shape, FP64)",
            "achieved": ach,
            "peak": fp64_tf, "unit": "TFLOP/s", "frac": ach / fp64_tf, "traffic": None,
            "peak_source": "measured FP64 FMA rate of this GPU (library probe, 2 flop/FMA)",
            "launches": st["react_launches"], "ms_per_launch": st["ms_react_kernel"] / max(st["react_launches"], 1)}
    final64 = [B[k].leaves() for k in range(B.n)]

    # end to end: the timed steps replayed from the same starting state, every
    # step every instance's state in from pinned host memory and out again
    pinned = []
    for k, (keys, vals) in enumerate(start):
        cap = max(len(keys), max(len(f[0]) for f in [final64[k]])) * 2
        bufs = [torch.empty(cap, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64),
                torch.empty(3 * cap, dtype=torch.float64, pin_memory=True).numpy()]
        n0 = len(keys)
        bk, bv = bufs[0][:n0], bufs[1][:3 * n0].reshape(3, n0)
        bk[:] = keys
        bv[:] = vals
        pinned.append((bufs, bk, bv))
    n_e2e = min(args.steps, 5)
    h2d = d2h = 0
    e2e_leaves = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        for k in range(B.n):
            _, bk, bv = pinned[k]
            B[k].set_leaves(bk, bv)
            h2d += bk.nbytes + bv.nbytes
        B.run(1, b["dt"], eta, TOL, TOL, TOL)
        e2e_leaves += B.stats()["leaf_updates"]
        for k in range(B.n):
            bufs, _, _ = pinned[k]
            n = B[k].num_leaves()
            if 3 * n > len(bufs[1]):
                bufs[0] = torch.empty(2 * n, dtype=torch.int64, pin_memory=True).numpy().view(np.uint64)
                bufs[1] = torch.empty(6 * n, dtype=torch.float64, pin_memory=True).numpy()
            bk, bv = B[k].leaves(bufs[0][:n], bufs[1][:3 * n].reshape(3, n))
            d2h += bk.nbytes + bv.nbytes
            pinned[k] = (bufs, bk, bv)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    e2e = {"value": e2e_leaves / t_e2e, "unit": UNIT, "h2d_bytes_per_step": h2d // n_e2e,
           "d2h_bytes_per_step": d2h // n_e2e, "steps": n_e2e,
           "note": "the first timed steps replayed from the same starting state: every instance's "
                   "mr_set_leaves(host), mr_batch_run(1 step), every instance's mr_get_leaves(host); wall clock"}
    B.close()

    # mixed form: the same batch and steps with FP32 Newton factorisations and ROCK4 stages
    mixed = None
    if not args.no_mixed:
        Bm = make(mr.MR_MIXED)
        Bm.run(warm, b["dt"], eta, TOL, TOL, TOL)
        Bm.run(args.steps, b["dt"], eta, TOL, TOL, TOL)
        sm = Bm.stats()
        errs, errs_same, flipped = [], [], []
        for k in range(Bm.n):
            km, vm = Bm[k].leaves()
            kf, vf = final64[k]
            if np.array_equal(km, kf):
                vol = np.ldexp(1.0, (2 * (insts[k]["J"] - (kf >> np.uint64(48)).astype(np.int64))).astype(np.int32))
                errs.append(max(float(np.sum(vol * np.abs(vm[i] - vf[i])) / np.sum(vol * np.abs(vf[i])))
                                for i in range(3)))
                errs_same.append(errs[-1])
            else:
                # the two forms adapted differently (a detail at the threshold
                # rounded to the other side): compared on the finest grid
                f64 = finest_grid(kf, vf, 2, insts[k]["J"])
                mix = finest_grid(km, vm, 2, insts[k]["J"])
                errs.append(max(float(np.sum(np.abs(mix[i] - f64[i])) / np.sum(np.abs(f64[i]))) for i in range(3)))
                flipped.append({"instance": k, "J": insts[k]["J"], "eta": insts[k]["eta"],
                                "leaves_fp64": int(len(kf)), "leaves_mixed": int(len(km)), "rel_l1": errs[-1]})
        mvalue = sm["leaf_updates"] / (sm["ms_device"] * 1e-3)
        mixed = {"value": mvalue, "ms_per_step": sm["ms_device"] / args.steps, "speedup_vs_fp64": mvalue / value,
                 "rel_l1_vs_fp64_path_max_over_instances": max(errs),
                 "rel_l1_max_over_instances_with_equal_grids": max(errs_same) if errs_same else None,
                 "instances_with_different_grids": flipped,
                 "form": "Radau5 Newton factorisations and solves, and the starting values and tolerance scales of each step attempt, in FP32; ROCK4 stage vectors in FP32; "
                         "Radau5 residuals, both error norms, step control, the state between sub-steps, "
                         "details and mass in FP64"}
        Bm.close()

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": warm, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "desc": b["desc"], "instances": len(insts),
                       "J": [i["J"] for i in insts], "host_threads": st["threads"],
                       "leaves_total_last_step": sum(len(f[0]) for f in final64),
                       "l2": "inputs larger than L2 (all instances' state and work vectors)"},
            "roofline": roof, "e2e": e2e, "cpu_baseline": None, "gpu_launches": launches, "clocks": clk,
            "autotuner": {"trials": tuning,
                          "note": "launch shapes tried on the first launches (each twice), ranked by algorithmic "
                                  "work per ms; none changes a result"},
            "mixed": mixed, "kernels": {"joint_radau": {"ms": st["ms_react_kernel"], "launches": st["react_launches"],
                                                       "tflops": ach},
                                        "phases_ms_per_step": {"adapt_and_tables": st["ms_adapt_phase"] / args.steps,
                                                               "react_joint": st["ms_react_kernel"] / args.steps,
                                                               "diffuse": st["ms_diffuse_phase"] / args.steps}}}
    if rank == 0 and print_line:
        print(json.dumps(line), flush=True)
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS) + sorted(BATCH))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-hbm-extra", action="store_true",
                    help="skip the HBM-resident 3D J=9 extra of the default workload")
    ap.add_argument("--J", type=int, default=0,
                    help="run the workload at another finest level (profiling captures of a smaller case); "
                         "the line's config records it")
    ap.add_argument("--max-leaves", type=int, default=0,
                    help="leaf capacity of the context (0: the full finest grid); for profiling captures that "
                         "must hold only a few GB on the device")
    ap.add_argument("--threads", type=int, default=0,
                    help="batched workload: host threads driving the instances' adaptation (0: the library's "
                         "default, one per core up to 32)")
    ap.add_argument("--instances", type=int, default=0,
                    help="batched workload: the first N of its seeded instances (profiling captures of a "
                         "smaller case); the line's config records it")
    ap.add_argument("--radau-schedule", choices=("pool", "thread"), default=None,
                    help="Radau5 schedule of single-context BZ and NAGUMO workloads (default: the library's, "
                         "one thread per cell); both give bit-identical results")
    args = ap.parse_args()
    if args.radau_schedule is not None:
        global RADAU_SCHEDULE
        RADAU_SCHEDULE = 1 if args.radau_schedule == "pool" else 0
    if args.warmup < 3 and args.impl != "reference":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.workload in BATCH:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle arm covers the single-instance workloads"}))
            return
        b = BATCH[args.workload]
        if args.instances and args.instances != b["n"]:
            b = dict(b, n=max(1, min(args.instances, b["n"])),
                     desc=b["desc"] + f" -- run with the first {args.instances} instances")
        run_batch(args, b)
        return
    w = WORKLOADS[args.workload]
    if args.max_leaves:
        w = dict(w, max_leaves=args.max_leaves)
    if args.J and args.J != w["J"]:
        w = dict(w, J=args.J, oracle_J=min(w.get("oracle_J", args.J), args.J),
                 desc=w["desc"] + f" -- run at finest level J={args.J}")
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_gpu(args, w)


if __name__ == "__main__":
    main()
