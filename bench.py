"""Benchmark: Metropolis sampling of gauged Gaussian fermionic PEPS on GB300.

One step = one sweep of every chain (all 2V links proposed in order, ratio +
combine + decide + rank-r update per proposal, periodic refresh, per-sweep
observables).  Metric: effective samples per second, ESS = chains * sweeps /
(2 tau_int), tau_int the larger of the integrated autocorrelation times of
the plaquette and log N(G) series (Madras-Sokal window, c = 5), estimated
from all sweeps run after burn-in.

  python bench.py [--gpus N --steps K --warmup W] [--workload cfg3|cfg2]
                  [--impl ggf|reference] [--observables]

--impl reference times the FP64 CPU oracle (exact Metropolis, full Pfaffian
recompute per proposal) on the host cores on a bounded sample.
Multi-GPU: independent replicas (rank k runs the global chains k*chains .. ,
the Philox key of each chain is its global index), no data-path
collective; the timing is the max over ranks.
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

REFRESH_CFG3 = 2048   # accepts per chain between refreshes (about 4 sweeps at the workload's acceptance)
REFRESH_Z2 = 64       # Z2 cells of the uneven batch (as the 8x8 Z2 workload)

WORKLOADS = {
    # name: (L, group, n_v, K, chains, precision, refresh_every, delay, label)
    "cfg3": (16, 1, 2, 4, 256, 1, REFRESH_CFG3, 16,
             "16x16 periodic U(1), n_v=2 (M 4096x4096 complex), K=4, 256 chains, FP32 batched updates "
             "(16 links per batch, one rank-128 tensor-core flush per batch), FP64 refresh every "
             f"{REFRESH_CFG3} accepts per chain (site-by-site FP64 Pfaffian for the log-weights, one "
             "tensor-core Newton step for the inverses)"),
    "cfg3_fp64": (16, 1, 2, 4, 16, 0, REFRESH_CFG3, 16,
                  "16x16 periodic U(1), n_v=2, K=4 as cfg3 but the plain FP64 local sampler (FP64 inverses, "
                  "ratios and batched updates; FP64 SIMT flush), 16 chains (2 GiB of inverses each)"),
    "cfg2": (8, 0, 1, 1, 1024, 1, 64, 1,
             "8x8 periodic Z2, K=1 (M 512x512), 1024 chains, FP32 rank-r updates, FP64 refresh every 64 accepts"),
    "cfg2_fp64": (8, 0, 1, 1, 1024, 0, 1024, 1,
                  "8x8 periodic Z2, K=1 (M 512x512), 1024 chains, plain FP64 local updates"),
    "su2": (16, 2, 2, 2, 256, 1, REFRESH_CFG3, 16,
            "16x16 periodic SU(2), n_v=2 (one doublet per link end, M 4096x4096), K=2, 256 chains, FP32 "
            f"batched updates (16 links per batch), FP64 refresh every {REFRESH_CFG3} accepts"),
    "cfg4": (16, 1, 2, 4, 192, 1, REFRESH_CFG3, 32,
             "16x16 periodic U(1), n_v=2, K=4 with the learned 4x4-block proposal (BF16 conv net trained on "
             "plain-sampler configurations); step = 1 local sweep + 16 block moves; 192 resident chains; FP64 "
             f"refresh every {REFRESH_CFG3} accepts"),
}
# Bond covariances: B_n (n >= 2) is B_1 rotated by a link-local Gaussian
# unitary with generator entries of this standard deviation.
BOND_SCALE = 0.05
# dram__bytes_read.sum + dram__bytes_write.sum of one flush launch group per
# chain (ncu, 4 chains of the same workload; profiles/sweep_kernels_cfg3_4chains.md).
# Remove the entry when the split or flush kernels change.
FLUSH_TRAFFIC_PER_CHAIN = {
    "cfg3": {"bytes": 2.573e9, "source": "ncu capture of ps_split_kernel and flush_ps_kernel, 4 chains, scaled "
                                          "by the chains (profiles/sweep_kernels_cfg3_4chains.md)"},
}
BLOCK_MOVES_PER_STEP = 16

# Uneven batch: every (lattice, group, K) cell below is one problem; all cells
# sweep together, one parent CUDA graph launch per sweep.  Chains are spread
# so that every cell holds about the same inverse memory (at least one chain).
CFG5_CELLS = [(L, grp, K) for L in (8, 12, 16, 24) for grp in (0, 1) for K in (1, 2, 4, 8)]
CFG5_TUNE_MAX = 2 * 2**30      # cells whose chains hold more inverse memory run at delay 16 untuned
CFG5_CHAINS = 4096
CFG5_BUDGET = 120 * 2**30


def cfg5_cells():
    import ggf_inputs as gi
    cells = []
    for (L, grp, K) in CFG5_CELLS:
        nv = 1 if grp == 0 else 2
        p = gi.make_problem(L, grp, nv, K, seed=BASE_SEED + 31 * len(cells))
        mem = 4 * p.N * p.N * K * K                  # FP32 inverses of all K^2 pair entries
        cells.append([p, mem])
    inv = [1.0 / m for _, m in cells]
    scale = CFG5_CHAINS / sum(inv)
    out = []
    for (p, mem), w in zip(cells, inv):
        ch = max(1, int(round(w * scale)))
        ch = max(1, min(ch, int(CFG5_BUDGET / len(cells) // mem)))
        out.append((p, ch, mem))
    return out


def run_cfg5(args):
    """Uneven batch of problems in one graph launch per sweep."""
    import torch
    import ggf_inputs as gi
    from paper_2412_01737_gb300 import GGF
    from paper_2412_01737_gb300.ggf import sample_group
    from paper_2412_01737_gb300.tune import tune_delay
    cells = cfg5_cells()
    ctxs, tuned, t0 = [None] * len(cells), [None] * len(cells), time.time()
    # the largest cells are set up first, while the most memory is free
    order = sorted(range(len(cells)), key=lambda k: -cells[k][1] * cells[k][2])
    for k in order:
        p, ch, mem = cells[k]
        links = gi.cold_links(p, ch)
        t_cell = time.time()
        if mem <= CFG5_TUNE_MAX:
            d, tim = tune_delay(p, links, 1, candidates=(8, 16), use_cache=False, seed=BASE_SEED + k)
        else:
            d, tim = 16, {}       # the tuner would set these chains up once per candidate
        print(f"cfg5 cell {k}: L={p.L} group={p.group} K={p.K} chains={ch} delay={d} "
              f"tune {time.time() - t_cell:.1f}s {tim}", file=sys.stderr, flush=True)
        tuned[k] = {"L": p.L, "group": "Z2" if p.group == 0 else "U1", "K": p.K, "chains": ch, "delay": d,
                    "tuned": bool(tim), "ms_per_sweep": {str(a): round(b, 2) for a, b in tim.items()}}
        # Z2 flips are large moves: their FP32 tracked log-weight drifts ~1.5e-6
        # per accept, so Z2 cells refresh every REFRESH_Z2 accepts
        refresh = REFRESH_Z2 if p.group == gi.Z2 else REFRESH_CFG3
        tuned[k]["refresh_every_accepts"] = refresh
        t_init = time.time()
        c = GGF(0)
        c.init_problem(p)
        c.chains_init(links, precision=1, refresh_every=refresh, seed=BASE_SEED + k, delay=d, graph=1)
        tuned[k]["init_s"] = round(time.time() - t_init, 2)
        ctxs[k] = c
    t_setup = time.time() - t0
    obs = [[] for _ in ctxs]
    for o, s in zip(sample_group(ctxs, args.warmup), obs):
        s.append(o)
    torch.cuda.synchronize()
    clocks = Clocks()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    outs = sample_group(ctxs, args.steps)
    e1.record()
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    # the same sweeps cell by cell (one graph launch per cell and sweep, in
    # sequence): what the single grouped launch saves over separate launches
    torch.cuda.synchronize()
    t_sep = time.time()
    last = [c.sample(args.steps)[-1] for c in ctxs]
    torch.cuda.synchronize()
    t_sep = time.time() - t_sep
    # tracked log N at the last sweep against a fresh FP64 evaluation
    for k, (c, o) in enumerate(zip(ctxs, last)):
        fresh = c.logweight(np.ascontiguousarray(c.chains_links()))
        tuned[k]["dlogp_vs_fp64_recompute"] = float(np.nanmax(np.abs(fresh - o[:, 1])))
    ess, total_chains, launches = 0.0, 0, 0
    for k, (c, o) in enumerate(zip(ctxs, outs)):
        ser = np.concatenate([obs[k][0], o], axis=0).transpose(1, 0, 2)      # chains, sweeps, 3
        keep = ser[:, max(1, ser.shape[1] // 4):, :]
        tau, closed, _ = tau_report(keep)
        tuned[k]["tau_int"] = round(tau, 3)
        tuned[k]["tau_window_closed"] = closed
        ess += c.n_chains * args.steps / (2 * tau)
        total_chains += c.n_chains
        launches += c.chains_stats().launches
        c.close()
    line = {"metric": "effective samples/sec/GPU", "value": ess / (ms * 1e-3), "unit": "samples/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"uneven batch: {len(cells)} problems (L in 8,12,16,24; Z2 and U(1); K in 1,2,4,8), "
                                   f"{total_chains} chains, one parent CUDA graph launch per sweep, autotuned delay, "
                                   f"FP32 updates with the FP64 refresh every {REFRESH_CFG3} accepts (U(1) cells) or "
                                   f"{REFRESH_Z2} accepts (Z2 cells)",
                       "cells": tuned, "setup_s": t_setup,
                       "separate_launches_s": t_sep, "grouped_s": ms * 1e-3,
                       "separate_note": "the timed sweeps repeated cell by cell, one graph launch per cell"},
            "roofline": None, "roofline_note": "per-kernel timing is not collected inside grouped graph launches",
            "clocks": ck, "gpu_launches": int(launches)}
    print(json.dumps(line), flush=True)

BASE_SEED = 20241202


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self):
        self.rows, self.proc = [], None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", os.environ.get("LOCAL_RANK", "0"),
                                          f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if "Active" in r[3 + k]
                          and "Not" not in r[3 + k]})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def tau_int(series, c=5.0):
    """Integrated autocorrelation time of the (chains, sweeps) series with the
    Madras-Sokal window: the sum runs to the first lag t >= c tau.  Returns
    (tau, window, closed); closed is False when the series ended before the
    window condition was met (tau is then a truncated sum, a lower bound)."""
    x = np.asarray(series, dtype=np.float64)
    x = x - x.mean()
    T = x.shape[1]
    var = np.mean(x * x)
    if var == 0 or T < 2:
        return 0.5, 0, False
    tau = 0.5
    for t in range(1, T):
        tau += np.mean(x[:, :-t] * x[:, t:]) / var
        if t >= c * tau:
            return float(tau), t, True
    return float(tau), T - 1, False


def problem_for(name):
    import ggf_inputs as gi
    L, grp, nv, K, chains, prec, refresh, delay, label = WORKLOADS[name]
    p = gi.make_problem(L, grp, nv, K, seed=BASE_SEED, bond_scale=BOND_SCALE)
    label += f"; bond generators N(0, {BOND_SCALE}^2)"
    return p, chains, prec, refresh, delay, label


def unit_bytes(p, prec):
    """Algorithmic HBM bytes of one rank-r update of one chain: every pair's W
    read and written once (N^2 elements each)."""
    b = 8 if prec == 0 else 4
    return 2 * p.N * p.N * (p.K * b + p.K * (p.K - 1) // 2 * 2 * b)


def _oracle_pair_task(args):
    """One pair term log N_nm(G') of the oracle's exact Metropolis step at the
    workload's full size: the covariance route of oracle.weight (twist O(G'),
    O^T Gamma_A O + Gamma_X^{nm} on the full physical + virtual space, FP64
    Parlett-Reid Pfaffian).  G' is the cold start with one link proposed.
    Only the pair's own covariance is embedded (the oracle's table of all
    K^2 would not fit the workers' memory) and the constant log Pf(Gamma_A),
    which every ratio cancels, is left at 0.  Returns wall seconds."""
    name, k, link = args
    sys.path.insert(0, ROOT)
    import ggf_inputs as gi
    from oracle import weight
    p, *_ = problem_for(name)
    pairs = [(n, n) for n in range(p.K)] + [(n, m) for n in range(p.K) for m in range(n + 1, p.K)]
    n, m = pairs[k % len(pairs)]
    W = weight.Weights.__new__(weight.Weights)
    W.p = p
    W.GA = weight.gamma_A(p)
    W.bond = weight.BondData(p)
    W.log_pf_A = 0.0
    W.n_virt = 4 * p.n_v * p.V
    W.GX = {(n, m): W.bond.embedded(n, m)}
    links = gi.cold_links(p)[0].copy()
    if p.group == gi.Z2:
        links[link % p.n_links] *= -1
    else:
        links[link % p.n_links] += 0.25
    t0 = time.time()
    W.log_n_nm(links, n, m)
    return time.time() - t0


def start_cpu_baseline(name, workers):
    """Start the oracle's pair terms on `workers` spawned processes (one BLAS
    thread each); returns a handle for finish_cpu_baseline."""
    import multiprocessing as mp
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    ctx = mp.get_context("spawn")
    pool = ctx.Pool(workers)
    res = pool.map_async(_oracle_pair_task, [(name, w, 37 * w + 5) for w in range(workers)])
    return pool, res, workers, time.time()


def finish_cpu_baseline(name, handle, timeout=1800):
    """Collect the pair-term timings: proposals per second of the oracle's
    exact Metropolis on the host cores, and the sample description."""
    pool, res, workers, t0 = handle
    secs = res.get(timeout=timeout)
    pool.close()
    pool.join()
    p, *_ = problem_for(name)
    P = p.K * (p.K + 1) // 2
    t_pair = float(np.mean(secs))
    rate = workers / (P * t_pair)
    desc = (f"{workers} concurrent spawned workers, each the oracle's exact-Metropolis pair term log N_nm(G') "
            f"at the full {p.L}x{p.L} size (full-space {p.m_s * p.V}x{p.m_s * p.V} complex Pfaffian route), "
            f"mean {t_pair:.1f} s per term (wall {time.time() - t0:.0f} s); one proposal = the {P} pair terms, "
            f"so proposals/s = workers / ({P} x mean)")
    return rate, t_pair, workers, desc


def run_reference(args):
    """The oracle on the host cores (the reference arm): one round of full-size
    pair terms on every core; each core's chain would need P such terms per
    proposal and 2V proposals per sweep.  ESS uses tau_int = 1/2 (the bound
    that favours the oracle)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    p, chains, prec, refresh, delay, label = problem_for(args.workload)
    t0 = time.time()
    workers = os.cpu_count() or 1
    rate, t_pair, workers, desc = finish_cpu_baseline(args.workload, start_cpu_baseline(args.workload, workers))
    sweeps_per_s = rate / p.n_links
    value = sweeps_per_s / (2 * 0.5)      # tau_int >= 1/2: upper bound for the oracle
    line = {"metric": "effective samples/sec/GPU", "value": value, "unit": "samples/s", "impl": "reference",
            "n_gpus": args.gpus, "steps": 1, "warmup": 0,
            "ms_per_step": 1e3 / sweeps_per_s, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": label, "chains": workers,
                       "note": "one round of pair terms on every host core stands for the steps: a single "
                               "full-size pair term takes minutes, so --steps/--warmup sweeps cannot run"},
            "cpu_baseline": {"value": value, "unit": "samples/s", "cores": workers, "host_cores": os.cpu_count(),
                             "kind": "oracle", "sample": desc + "; ESS bound with tau_int = 1/2"},
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.time() - t0}
    print(json.dumps(line), flush=True)


def tau_report(series):
    """tau_int of the plaquette and log N(G) series (chains, sweeps) about each
    sweep's ensemble mean (removes a common drift of chains started together);
    the larger one is used.  Returns (tau, closed, details)."""
    out, taus = {}, []
    for k, name in ((0, "plaquette"), (1, "logN")):
        x = series[:, :, k] - series[:, :, k].mean(axis=0, keepdims=True)
        t, w, closed = tau_int(x)
        out[name] = {"tau": t, "window": w, "window_closed": closed}
        taus.append((t, closed))
    tau = max(max(t for t, _ in taus), 0.5)
    return tau, all(c for _, c in taus), out


def tau_calibration(args, p, prec, refresh, delay, local, keep=False):
    """tau_int of the same sampler from a longer run with fewer chains: the
    autocorrelation time is a property of the Markov chain (lattice, weights,
    proposal), not of how many independent chains run, and the benchmark's
    own series is too short for the Madras-Sokal window at this workload.
    Returns (tau, closed, details, sweeps, chains, seconds)."""
    import torch
    import ggf_inputs as gi
    from paper_2412_01737_gb300 import GGF
    t0 = time.time()
    n = args.tau_chains
    ctx = GGF(local)
    ctx.init_problem(p)
    ctx.chains_init(gi.cold_links(p, n), precision=prec, refresh_every=refresh, seed=BASE_SEED + 104729,
                    delay=delay)
    obs = torch.zeros((1, n, 3), dtype=torch.float64, device=f"cuda:{local}")
    for _ in range(args.tau_burn):
        ctx.sample(1, obs=obs)
    series = []
    for _ in range(args.tau_run):
        ctx.sample(1, obs=obs)
        series.append(obs[0].cpu().numpy().copy())
    ctx.close()
    ser = np.stack(series, axis=1)
    tau, closed, detail = tau_report(ser)
    if keep:
        return tau, closed, detail, args.tau_run, n, time.time() - t0, ser
    return tau, closed, detail, args.tau_run, n, time.time() - t0


def run_ggf(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    # the oracle's CPU baseline runs on the host cores while the GPU samples
    # (spawned before the first CUDA call; two cores stay with this process)
    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = start_cpu_baseline(args.workload, max(1, (os.cpu_count() or 1) - 2))
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    import ggf_inputs as gi
    from paper_2412_01737_gb300 import GGF
    from paper_2412_01737_gb300.ggf import KT_RATIO, KT_UPDATE, KT_REFRESH, KT_FLUSH, KT_GATHER, KT_APPLY

    p, chains, prec, refresh, delay, label = problem_for(args.workload)
    if args.chains:
        chains = args.chains
    if args.delay:
        delay = args.delay
    if args.refresh:
        refresh = args.refresh
    # replica r owns the chains r * chains .. (r + 1) * chains - 1 of one
    # global ensemble: Philox key (seed, global chain index)
    seed = BASE_SEED
    # ---- set-up through the public API from host buffers (part of the e2e time)
    torch.cuda.synchronize()
    t_setup0 = time.time()
    ctx = GGF(local)
    ctx.init_problem(p)
    start = gi.cold_links(p, chains)
    ctx.chains_init(start, precision=prec, refresh_every=refresh, seed=seed, delay=delay,
                    chain_offset=rank * chains)
    torch.cuda.synchronize()
    t_setup = time.time() - t_setup0
    dev_obs = torch.zeros((1, chains, 3), dtype=torch.float64, device=f"cuda:{local}")
    stream = torch.cuda.current_stream()
    net, train_info = None, None
    if args.workload == "cfg4":
        # training data from the plain local sampler, then MLE training of the proposal
        from paper_2412_01737_gb300 import Net
        t_tr = time.time()
        ctx.sample(args.burn_train)
        data = []
        for _ in range(args.train_sweeps):
            ctx.sample(1)
            data.append(ctx.chains_links())
        data = torch.from_numpy(np.concatenate(data)).cuda()
        t_gen = time.time() - t_tr
        net = Net(local, p.L, seed)
        t0n = time.time()
        losses = net.train(data, 128, args.train_steps, 2e-3)
        torch.cuda.synchronize()
        train_info = {"configs": int(data.shape[0]), "data_s": t_gen, "train_s": time.time() - t0n,
                      "train_steps": args.train_steps, "loss_first": float(losses[:10].mean()),
                      "loss_last": float(losses[-10:].mean())}
        blk_obs = torch.zeros((BLOCK_MOVES_PER_STEP, chains, 3), dtype=torch.float64, device=f"cuda:{local}")

    def one_step(obs):
        """One step; obs is a (1, chains, 3) device tensor or host array."""
        ctx.sample(1, obs=obs)
        if net is not None:
            ctx.sample_blocks(net, BLOCK_MOVES_PER_STEP, obs=blk_obs)
            if isinstance(obs, np.ndarray):
                obs[0] = blk_obs[-1].cpu().numpy()
            else:
                obs[0].copy_(blk_obs[-1])

    # ---- thermalisation from the cold start (discarded), then recorded
    # untimed sweeps for the autocorrelation estimate and the warm-up
    t_burn0 = time.time()
    for _ in range(args.burn):
        one_step(dev_obs)
    torch.cuda.synchronize()
    t_burn = time.time() - t_burn0
    series = []
    for _ in range(args.tau_sweeps + args.warmup):
        one_step(dev_obs)
        series.append(dev_obs[0].cpu().numpy().copy())
    st0 = ctx.chains_stats()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    # ---- timed region: the captured sweep graph replayed, observables read
    # back into host memory every step through the public API
    host_obs = np.zeros((args.steps, chains, 3))
    clocks = Clocks()
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.cudart().cudaProfilerStart()     # ncu --profile-from-start off sees the timed sweeps only
    t_wall0 = time.time()
    e0.record(stream)
    for k in range(args.steps):
        one_step(host_obs[k:k + 1])
    e1.record(stream)
    torch.cuda.synchronize()
    t_wall = time.time() - t_wall0
    torch.cuda.cudart().cudaProfilerStop()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    st1 = ctx.chains_stats()
    series.extend(list(host_obs))
    if dist:
        t = torch.tensor([ms, t_wall], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms, t_wall = float(t[0]), float(t[1])
    # ---- separate profiled pass (not timed): the same graph with timing-event
    # nodes around every launch group, for the kernel shares and the roofline
    ctx.profile(True)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sp0 = ctx.chains_stats()
    p0.record(stream)
    for _ in range(args.prof_sweeps):
        one_step(dev_obs)
    p1.record(stream)
    torch.cuda.synchronize()
    last_tracked = dev_obs[0, :, 1].cpu().numpy().copy()     # log N tracked at the last sweep run
    sp1 = ctx.chains_stats()
    prof_ms = p0.elapsed_time(p1)
    kt = {k: ctx.kernel_time(v) for k, v in (("ratio", KT_RATIO), ("update", KT_UPDATE),
                                             ("refresh", KT_REFRESH), ("flush", KT_FLUSH),
                                             ("gather", KT_GATHER), ("apply", KT_APPLY))}
    ctx.profile(False)
    obs_series = np.stack(series, axis=1)             # (chains, sweeps, 3) after thermalisation
    tau, closed, tau_detail = tau_report(obs_series)
    sweeps_timed = args.steps
    value = world * chains * sweeps_timed / (2 * tau) / (ms * 1e-3)
    accepts = sp1.accepts - sp0.accepts
    shares = {k: v[0] for k, v in kt.items()}
    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs", 6800.0)
    dom = max(shares, key=shares.get)
    wpairs = p.K + 4 * (p.K * (p.K - 1) // 2)             # real-MAC weight of all pairs
    if dom == "refresh":
        roof = {"kernel": "refresh (site-by-site FP64 Pfaffian + Newton step)", "bound": "alu",
                "achieved": None, "peak": None, "unit": None}
    elif dom == "flush":
        fl = accepts * 2.0 * p.N ** 2 * p.r * wpairs      # every accepted rank-r update folded once
        t_fl = kt["flush"][0] * 1e-3
        if prec == 1:
            # tensor-core flush: W read + written once per flush call and chain
            byts = kt["flush"][1] * chains * unit_bytes(p, prec)
            roof = {"kernel": "flush_tc_kernel (tcgen05 TF32x3, W -= U V)", "bound": "hbm",
                    "achieved": byts / t_fl / 1e9, "peak": hbm, "unit": "GB/s",
                    "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                    "algorithmic_bytes_per_launch_group": chains * unit_bytes(p, prec),
                    "avg_launch_group_ms": kt["flush"][0] / max(1, kt["flush"][1]),
                    "fp32_equivalent_tflops": fl / t_fl / 1e12}
            # the complex-pair tiles are tensor-bound (three TF32 products per
            # FP32 MAC): the same time against the tensor roofline, TF32 peak =
            # measured BF16 burst x the nominal TF32/BF16 ratio (1.1 / 2.25)
            tf32_peak = peaks.get("bf16_tflops", 1900.0) * 1.1 / 2.25
            roof["tensor"] = {"achieved": 3 * fl / t_fl / 1e12, "peak": tf32_peak, "unit": "TFLOP/s (TF32)",
                              "frac": 3 * fl / t_fl / 1e12 / tf32_peak,
                              "peak_source": "MEASURED_PEAKS.json bf16_tflops x 1.1/2.25 (nominal TF32/BF16 ratio)"}
        else:
            roof = {"kernel": "flush_kernel (FP64 SIMT, W -= U V)", "bound": "alu",
                    "achieved": fl / t_fl / 1e12, "peak": 1.25, "unit": "TFLOP/s",
                    "peak_source": "FP64 nominal 1.25 TFLOP/s (recipe)"}
    elif dom == "update" and delay <= 1:
        upd_bytes = accepts * unit_bytes(p, prec)
        roof = {"kernel": "update_kernel (rank-r SMW)", "bound": "hbm",
                "achieved": upd_bytes / (kt["update"][0] * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    elif dom == "update":
        # gather of the pending-panel path (block moves): per tentative update and pair,
        # panel rows U, V^T (2 N kr b) plus the rows of W at S and the new panel columns
        # (3 N r b), kr at its mean over a block.  Mostly L2-resident: no HBM peak applies.
        b = 8 if prec == 0 else 4
        kr_mean = 0.5 * 31 * p.r
        per = sum((2 if n == m else 4) * b * p.N * (kr_mean + 1.5 * p.r) for n in range(p.K) for m in range(n, p.K))
        n_upd = 32 * (sp1.block_proposals - sp0.block_proposals)
        roof = {"kernel": "gather_kernel (pending-panel rows/columns)", "bound": "l2",
                "achieved": n_upd * per / (kt["update"][0] * 1e-3) / 1e9, "peak": None, "unit": "GB/s",
                "peak_source": "no measured L2 peak; reported for the record"}
    elif dom == "ratio" and delay > 1:
        props = sp1.proposals - sp0.proposals
        roof = {"kernel": "batch_steps (link steps on W[T, T], FP64 ratios)", "bound": "latency",
                "achieved": props / (kt["ratio"][0] * 1e-3), "peak": None, "unit": "link proposals/s",
                "peak_source": "latency-bound (one CTA per chain, sequential links); no peak applies"}
    else:
        roof = {"kernel": "ratio_kernel", "bound": "alu", "achieved": None, "peak": None, "unit": None}
    roof["frac"] = (roof["achieved"] / roof["peak"]) if roof.get("achieved") and roof.get("peak") else None
    roof["traffic"] = None
    if dom == "flush" and prec == 1 and args.workload in FLUSH_TRAFFIC_PER_CHAIN:
        # DRAM bytes of one flush launch group (split passes + flushes, both
        # families), per chain from an ncu capture of these kernels, times the
        # chains: the traffic grows in proportion to them
        t = FLUSH_TRAFFIC_PER_CHAIN[args.workload]
        roof["traffic"] = t["bytes"] * chains / 1e9
        roof["traffic_unit"] = "GB per launch group"
        roof["traffic_source"] = t["source"]
        roof["traffic_over_algorithmic"] = t["bytes"] / unit_bytes(p, prec)
    roof["share"] = {k: round(v / max(prof_ms, 1e-9), 4) for k, v in shares.items()}
    # time between the graph's kernel groups (launch gaps, host work between
    # sweeps): what a single persistent kernel could at most remove
    roof["kernel_time_fraction"] = round(sum(shares.values()) / max(prof_ms, 1e-9), 4)
    roof["profiled_pass"] = {"sweeps": args.prof_sweeps, "ms": prof_ms,
                             "refreshes": int(sp1.refreshes - sp0.refreshes),
                             "note": "separate untimed pass of the same graph with timing-event nodes"}
    if kt["refresh"][1] > 0:
        roof["refresh_ms_per_chain"] = kt["refresh"][0] / max(1, sp1.refreshes - sp0.refreshes)
    if delay > 1 and kt["gather"][1] > 0:
        # batched mode: per batch and pair, the gather reads W[:, T] and W[T, :]
        # (2 N kr b) and writes the U and V^T panels (2 N kr b); the X product
        # reads and writes V^T (2 N kr b) and does N kr^2 MACs
        b = 8 if prec == 0 else 4
        kr = delay * p.r
        per_b = sum((1 if n == m else 2) * b * p.N * kr for n in range(p.K) for m in range(n, p.K))
        macs = sum((1 if n == m else 4) * p.N * kr * kr for n in range(p.K) for m in range(n, p.K))
        n_b = kt["gather"][1]
        roof["batch_kernels"] = {
            "batch_gather_gbs": n_b * chains * 4 * per_b / (kt["gather"][0] * 1e-3) / 1e9,
            "batch_apply_gbs": n_b * chains * 2 * per_b / (kt["apply"][0] * 1e-3) / 1e9,
            "batch_apply_fp32_tflops": n_b * chains * 2 * macs / (kt["apply"][0] * 1e-3) / 1e12,
            "note": "kr = delay r is the batch's rank; sizes per launch group over all chains"}
    # |Delta log N|: every chain's tracked log-weight at the end of the timed
    # region against a fresh FP64 factorisation of its configuration
    fin = ctx.chains_links()
    fresh = ctx.logweight(np.ascontiguousarray(fin))
    dlogp = float(np.nanmax(np.abs(fresh - last_tracked)))
    st2 = ctx.chains_stats()
    h2d = (p.gamma_site.nbytes + p.gamma_bond.nbytes + p.lam.nbytes + start.nbytes) / args.steps
    ess_timed = world * chains * sweeps_timed / (2 * tau)
    line = {"metric": "effective samples/sec/GPU", "value": value, "unit": "samples/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec == 1 else "f64", "data": "synthetic",
            "config": {"workload": label, "chains": chains, "delay": delay, "refresh_every_accepts": refresh,
                       "sweeps_timed": args.steps, "thermalisation_sweeps": args.burn,
                       "thermalisation_s": t_burn,
                       "thermalisation_note": "untimed, discarded; 200 sweeps of this workload would take about 25 min",
                       "tau_series_sweeps": obs_series.shape[1],
                       "tau_int": tau_detail, "tau_used": tau, "tau_window_closed": closed,
                       "ess_is_upper_bound": not closed,
                       "timed_path": "captured sweep graph replayed (graph mode), observables read back to host "
                                     "every step",
                       "parallelism": f"replicas x{world}", "l2": "inputs larger than L2 (W is "
                       f"{chains * unit_bytes(p, prec) / 2 / 2**30:.1f} GiB)",
                       "link_updates_per_s": world * chains * p.n_links * sweeps_timed / (ms * 1e-3),
                       "acceptance": (st1.accepts - st0.accepts) / max(1, st1.proposals - st0.proposals),
                       "refreshes_timed": int(st1.refreshes - st0.refreshes),
                       "refresh_max_resid": st2.max_resid, "refresh_dense_fallbacks": int(st2.dense_refreshes),
                       "refresh_newton_steps": int(st2.refine_steps),
                       "pfaffian_dense_fallbacks": int(st2.dense_pfaffians),
                       "flush_wave_chains": int(st2.flush_wave),
                       "init_s": t_setup},
            "dlogp_vs_fp64_recompute": dlogp, "max_drift_at_refresh": st2.max_drift,
            "roofline": roof, "clocks": ck,
            "gpu_launches": int(st1.launches - st0.launches),
            "e2e": {"value": ess_timed / (t_setup + t_wall), "unit": "samples/s",
                    "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(chains * 3 * 8),
                    "includes": "context creation, parameter and start-link upload (host buffers), FP64 chain "
                                "set-up, then the timed sweeps with every step's observables read back to host "
                                "memory (wall clock)"}}
    if train_info is not None:
        nb = st1.block_proposals - st0.block_proposals
        train_info["block_acceptance"] = (st1.block_accepts - st0.block_accepts) / max(1, nb)
        line["config"]["learned_proposal"] = train_info
        net.close()
    ctx.close()
    if args.tau_run > 0 and net is None:
        tau_c, closed_c, det_c, sw_c, ch_c, sec_c = tau_calibration(args, p, prec, refresh, delay, local)
        line["config"]["tau_calibration"] = {
            "chains": ch_c, "thermalisation_sweeps": args.tau_burn, "sweeps": sw_c, "tau_int": det_c,
            "tau": tau_c, "window_closed": closed_c, "seconds": sec_c,
            "note": "untimed run of the identical sampler (same problem, precision, batch size and refresh "
                    "cadence) with fewer chains and more sweeps; its tau is used for the ESS when its window "
                    "closed"}
        if closed_c:
            tau = tau_c
            line["config"]["tau_used"] = tau
            line["config"]["tau_window_closed"] = True
            line["config"]["ess_is_upper_bound"] = False
            ess_timed = world * chains * sweeps_timed / (2 * tau)
            line["value"] = ess_timed / (ms * 1e-3)
            line["e2e"]["value"] = ess_timed / (t_setup + t_wall)
    if cpu is not None:
        rate, t_pair, workers, desc = finish_cpu_baseline(args.workload, cpu)
        line["cpu_baseline"] = {"value": rate / p.n_links / (2 * tau), "unit": "samples/s",
                                "cores": workers, "host_cores": os.cpu_count(), "kind": "oracle",
                                "sample": desc + "; run concurrently with the GPU sweeps; same tau_int"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_compare(args):
    """Effective samples per second of three samplers of the same 16x16 U(1),
    K = 4 problem, i.e. the time each needs for a given error bar on the
    plaquette (error ~ sigma / sqrt(ESS)):
      * plain FP64 local updates (FP64 inverses, ratios and batched updates),
      * plain FP32 local updates with the FP64 refresh (the benchmark's sampler),
      * the learned block proposal on top of the FP32 sampler (one local sweep
        + 16 block moves per step, exact Metropolis-Hastings).
    tau_int of each sampler comes from its own recorded run (FP64 and FP32
    local updates are the same Markov chain, so they share the FP32 run's).
    ESS/s = chain-steps per second / (2 tau_int) at the chain count each
    sampler ran with (stated; the FP32 samplers gain a little per chain at
    the benchmark's 256).  Plaquette means are reported with their errors
    as a consistency check."""
    import torch
    import ggf_inputs as gi
    from paper_2412_01737_gb300 import GGF, Net
    p, chains, prec, refresh, delay, label = problem_for("cfg3")
    out = {"metric": "effective samples/sec/GPU (comparison)", "unit": "samples/s",
           "config": {"workload": label, "note": run_compare.__doc__.split("\n")[0]}}

    def mean_err(series, tau):
        x = series.reshape(-1)
        n_eff = series.size / (2 * tau)
        return float(x.mean()), float(x.std() / np.sqrt(max(n_eff, 1.0)))

    # plain FP32 local updates: tau from a long recorded run
    tau32, closed32, det32, sw32, ch32, sec32, ser32 = tau_calibration(args, p, 1, refresh, delay, 0, keep=True)
    pl32 = mean_err(ser32[:, :, 0], tau32)
    ctx = GGF(0)
    ctx.init_problem(p)
    n32 = args.tau_chains
    ctx.chains_init(gi.cold_links(p, n32), precision=1, refresh_every=refresh, seed=BASE_SEED + 7, delay=delay)
    ctx.sample(2)
    torch.cuda.synchronize()
    t0 = time.time()
    ctx.sample(3)
    torch.cuda.synchronize()
    s32 = (time.time() - t0) / (3 * n32)                 # seconds per chain-sweep
    ctx.close()
    # plain FP64 local updates
    n64 = 4
    ctx = GGF(0)
    ctx.init_problem(p)
    ctx.chains_init(gi.cold_links(p, n64), precision=0, refresh_every=refresh, seed=BASE_SEED + 11, delay=delay)
    ctx.sample(1)
    torch.cuda.synchronize()
    t0 = time.time()
    ctx.sample(2)
    torch.cuda.synchronize()
    s64 = (time.time() - t0) / (2 * n64)
    ctx.close()
    # learned block proposal on the FP32 sampler
    nl = args.learn_chains
    ctx = GGF(0)
    ctx.init_problem(p)
    ctx.chains_init(gi.cold_links(p, nl), precision=1, refresh_every=refresh, seed=BASE_SEED + 13, delay=32)
    obs = torch.zeros((1, nl, 3), dtype=torch.float64, device="cuda")
    for _ in range(args.tau_burn):
        ctx.sample(1, obs=obs)
    data = []
    for _ in range(args.train_sweeps):
        ctx.sample(1)
        data.append(ctx.chains_links())
    data = torch.from_numpy(np.concatenate(data)).cuda()
    net = Net(0, p.L, BASE_SEED)
    losses = net.train(data, 128, args.train_steps, 2e-3)
    blk = torch.zeros((BLOCK_MOVES_PER_STEP, nl, 3), dtype=torch.float64, device="cuda")
    series = []
    st0 = ctx.chains_stats()
    torch.cuda.synchronize()
    t0 = time.time()
    for _ in range(args.learn_steps):
        ctx.sample(1, obs=obs)
        ctx.sample_blocks(net, BLOCK_MOVES_PER_STEP, obs=blk)
        series.append(blk[-1].cpu().numpy().copy())
    torch.cuda.synchronize()
    sl = (time.time() - t0) / (args.learn_steps * nl)    # seconds per chain-step
    st1 = ctx.chains_stats()
    fin = ctx.chains_links()
    dlogp = float(np.nanmax(np.abs(ctx.logweight(np.ascontiguousarray(fin)) - blk[-1, :, 1].cpu().numpy())))
    ser = np.stack(series, axis=1)
    taul, closedl, detl = tau_report(ser)
    net.close()
    ctx.close()
    res = {}
    for name, sec, tau, closed, nch in (("fp64_local", s64, tau32, closed32, n64),
                                        ("fp32_local", s32, tau32, closed32, n32),
                                        ("fp32_learned", sl, taul, closedl, nl)):
        # chain-steps per second of the GPU at the measured chain count, over 2 tau
        res[name] = {"s_per_chain_step": sec, "tau_int": tau, "tau_window_closed": closed, "chains_measured": nch,
                     "ess_per_s": 1.0 / (sec * 2 * tau)}
    res["fp32_learned"].update({"tau_detail": detl, "block_acceptance":
                                (st1.block_accepts - st0.block_accepts) / max(1, st1.block_proposals - st0.block_proposals),
                                "plaquette_mean_err": mean_err(ser[:, :, 0], taul), "dlogp_vs_fp64_recompute": dlogp,
                                "train_configs": int(data.shape[0]), "train_steps": args.train_steps,
                                "train_loss_first_last": [float(losses[:10].mean()), float(losses[-10:].mean())],
                                "steps": args.learn_steps})
    res["fp32_local"].update({"tau_detail": det32, "tau_sweeps": sw32, "plaquette_mean_err": pl32})
    res["fp64_local"].update({"note": "the same Markov chain as fp32_local (FP64 arithmetic), so its tau_int"})
    out["samplers"] = res
    out["winner"] = max(res, key=lambda k: res[k]["ess_per_s"])
    out["learned_vs_fp64_local"] = res["fp32_learned"]["ess_per_s"] / res["fp64_local"]["ess_per_s"]
    out["learned_vs_fp32_local"] = res["fp32_learned"]["ess_per_s"] / res["fp32_local"]["ess_per_s"]
    d = res["fp32_learned"]["plaquette_mean_err"][0] - pl32[0]
    out["plaquette_difference_sigma"] = d / np.hypot(res["fp32_learned"]["plaquette_mean_err"][1], pl32[1])
    print(json.dumps(out), flush=True)


def observable_bytes(p, prec):
    """Algorithmic bytes of W that one call of the electric and of the
    fermionic kernel reads per chain: per pair, the B x r block between each
    link's source site and the link (electric) and the B x B block between the
    two sites of each site or link item (fermionic); B = 8 n_v, r = 4 n_v."""
    b = 8 if prec == 0 else 4
    per_pair = p.K * b + p.K * (p.K - 1) // 2 * 2 * b
    B, r = 8 * p.n_v, 4 * p.n_v
    return p.n_links * B * r * per_pair, (p.V + p.n_links) * B * B * per_pair


def run_observables(args):
    """Time the per-configuration observables of Secs. 5.2 and 5.3 and the
    derivatives built from the chains' inverses on the workload's chains (not
    part of the sampling step): K calls each after W warm-up calls, CUDA events
    on the launching stream, device buffers; bytes are the W elements each
    call reads (fermion4 reads three site-pair blocks per link and pair, the
    site score the diagonal site blocks, the link score the link blocks)."""
    import torch
    import ggf_inputs as gi
    from paper_2412_01737_gb300 import GGF
    p, chains, prec, refresh, delay, label = problem_for(args.workload)
    # the output buffers come on top of the inverses: 64 chains unless asked
    chains = args.chains or min(chains, 64)
    ctx = GGF(0)
    ctx.init_problem(p)
    ctx.chains_init(gi.random_links(p, chains, seed=BASE_SEED), precision=prec, refresh_every=refresh,
                    seed=BASE_SEED, delay=delay)
    ctx.sample(1 + args.burn)
    from paper_2412_01737_gb300.ggf import PAIRS_ELECTRIC
    dev = dict(dtype=torch.float64, device="cuda")
    P, B, r = p.K * (p.K + 1) // 2, 8 * p.n_v, 4 * p.n_v
    el = torch.zeros((chains, p.n_links, 2), **dev)
    fs = torch.zeros((chains, p.V, 2), **dev)
    fl = torch.zeros((chains, p.n_links, 2, 2, 2), **dev)
    f4 = torch.zeros((chains, p.n_links, 2), **dev)
    ep = torch.zeros((chains, p.n_links, p.K, p.K, 2), **dev)
    sc = torch.zeros((chains, p.V, B, B), **dev)
    ls = torch.zeros((chains, P, p.n_links, r, r, 2), **dev)
    calls = {"electric": lambda: ctx.chains_electric(out=el),
             "fermion": lambda: ctx.chains_fermion(site=fs, link=fl),
             "fermion4": lambda: ctx.chains_fermion4(out=f4),
             "electric_pairs": lambda: ctx.chains_pairs(PAIRS_ELECTRIC, out=ep),
             "site_score": lambda: ctx.chains_score(out=sc),
             "link_score": lambda: ctx.chains_link_score(out=ls)}
    from paper_2412_01737_gb300.ggf import PAIRS_FIELD, PAIRS_FOUR
    fp4 = torch.zeros((chains, p.n_links, p.K, p.K, 2), **dev)
    calls["four_pairs"] = lambda: ctx.chains_pairs(PAIRS_FOUR, out=fp4)
    if p.group == gi.U1:
        calls["electric_field"] = lambda: ctx.chains_electric_field(out=el)
        calls["field_pairs"] = lambda: ctx.chains_pairs(PAIRS_FIELD, out=ep)
    if p.group in (gi.Z2, gi.U1):
        calls["link_terms"] = lambda: ctx.chains_link_terms(p.q_phys, out=el)
    eb, fb = observable_bytes(p, prec)
    esz = 8 if prec == 0 else 4
    per_pair = p.K * esz + p.K * (p.K - 1) // 2 * 2 * esz
    read_bytes = {"electric": eb, "electric_pairs": eb, "electric_field": eb, "field_pairs": eb, "fermion": fb,
                  "four_pairs": p.n_links * 3 * B * B * per_pair,
                  "link_terms": p.n_links * B * B * per_pair,
                  "fermion4": p.n_links * 3 * B * B * per_pair,
                  "site_score": p.V * B * B * per_pair,
                  "link_score": p.n_links * r * r * per_pair}
    peak = load_peaks().get("hbm_gbs")
    out = {"metric": "observable_kernel_time", "unit": "ms per call (all chains)", "workload": args.workload,
           "config": {"workload": label, "chains": chains}, "steps": args.steps, "warmup": args.warmup}
    stream = torch.cuda.current_stream()
    for name, fn in calls.items():
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            fn()
        t1.record(stream)
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1) / args.steps
        byts = read_bytes[name] * chains
        gbs = byts / (ms * 1e-3) / 1e9
        out[name] = {"ms": ms, "bytes": byts, "achieved_gbs": gbs, "peak_gbs": peak,
                     "frac": gbs / peak if peak else None, "bound": "latency (scattered small blocks)"}
    print(json.dumps(out), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--burn", type=int, default=30,
                    help="thermalisation sweeps from the cold start (untimed, discarded)")
    ap.add_argument("--tau-sweeps", type=int, default=5,
                    help="untimed sweeps recorded (with warm-up and timed ones) for the run's own tau_int")
    ap.add_argument("--tau-chains", type=int, default=16, help="chains of the tau_int calibration run")
    ap.add_argument("--tau-burn", type=int, default=100, help="thermalisation sweeps of the calibration run")
    ap.add_argument("--tau-run", type=int, default=200,
                    help="recorded sweeps of the calibration run (0: no calibration run)")
    ap.add_argument("--prof-sweeps", type=int, default=9,
                    help="sweeps of the separate profiled pass (kernel shares, roofline)")
    ap.add_argument("--impl", default="ggf", choices=["ggf", "reference"])
    ap.add_argument("--workload", default="cfg3", choices=sorted(WORKLOADS) + ["cfg5"])
    ap.add_argument("--chains", type=int, default=0)
    ap.add_argument("--delay", type=int, default=0, help="override the workload's batch size (links per flush)")
    ap.add_argument("--refresh", type=int, default=0, help="override the workload's refresh cadence (accepts)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--burn-train", type=int, default=4, help="cfg4: local sweeps before collecting training data")
    ap.add_argument("--train-sweeps", type=int, default=6, help="cfg4: local sweeps whose configurations train the net")
    ap.add_argument("--train-steps", type=int, default=300, help="cfg4: Adam steps")
    ap.add_argument("--compare", action="store_true",
                    help="ESS/s of the plain FP64, plain FP32 and learned-proposal samplers (16x16 U(1), K=4)")
    ap.add_argument("--learn-chains", type=int, default=32, help="--compare: chains of the learned-proposal run")
    ap.add_argument("--learn-steps", type=int, default=100, help="--compare: recorded learned-proposal steps")
    ap.add_argument("--observables", action="store_true",
                    help="time the electric and fermionic observable kernels instead of sampling")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    elif args.observables:
        run_observables(args)
    elif args.workload == "cfg5":
        run_cfg5(args)
    elif args.compare:
        run_compare(args)
    else:
        run_ggf(args)


if __name__ == "__main__":
    main()
