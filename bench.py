"""Benchmark of the GB300 initiator-FCIQMC projector iteration.

One step = one full projector iteration (spawning, death, annihilation with
the initiator rule, semi-stochastic projection, shift update, E_proj
reduction) over a resident walker list.  Default workload: the 50-orbital,
10+10-electron synthetic ab initio system (200 Cholesky vectors, uniform
generator, initiator threshold 3, deterministic space of 1e4 determinants)
at about 1e8 walkers.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]
                  [--workload abinitio50|abinitio24|batch|serving]
"""
import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

METRIC = "spawn attempts/s + annihilated walkers/s; p50/p99 time-to-sigma(E)<1 mEh"
# tau: the prescribed 1e-3 gives tau * sum_j |H_ref,j| = 2.41 for this
# Hamiltonian (sum = 2412.4 Eh), beyond which no shift can hold the walker
# number; 0.5 / 2412.4 rounded down gives 2e-4.
TAU = 2e-4
TARGET = 6.25e5
E2E_STEPS = 40


def workload_params(seed_offset=0, workload="abinitio50", generator="uniform"):
    sysd, prm = _workload_params(seed_offset, workload)
    prm["generator"] = 1 if generator == "pchb" else 0
    return sysd, prm


def _workload_params(seed_offset=0, workload="abinitio50"):
    if workload == "abinitio50":
        # 50 orbitals, 10+10 electrons, 200 Cholesky vectors: sum_j |H_ref,j| = 39309 Eh,
        # so tau = 0.5 / 39309 rounded down = 1.25e-5 (the prescribed 5e-4 gives 19.7)
        sysd, prm = workloads.config_abinitio_50()
        prm = dict(prm, tau=1.25e-5, target_walkers=1e8, initial_walkers=1e6, shift_damping=1.0, shift_interval=2,
                   seed=prm["seed"] + seed_offset, semistoch_size=10000, semistoch_start=100)
        return sysd, prm
    sysd, prm = workloads.config_abinitio_24()
    prm = dict(prm, tau=TAU, target_walkers=TARGET, initial_walkers=TARGET, shift_damping=1.0, shift_interval=2,
               seed=prm["seed"] + seed_offset)
    return sysd, prm


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows if len(r) >= 9 for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def oracle_rate(sysd, prm, state, shift, iters):
    """The CPU oracle, as it stands, on a bounded sample of the workload:
    `iters` iterations from the given (sampled) state, one host core."""
    import oracle
    s = oracle.system_from_workload(sysd)
    r = oracle.Run(s, **prm)
    if state is not None:
        r.import_state(state["alpha"], state["beta"], state["c"], shift["iteration"], shift["S"], shift["vary"],
                       shift["shift_start"], shift["cnt"], shift["nw_last"])
    t = time.perf_counter()
    r.step(iters)
    el = time.perf_counter() - t
    st = r.stats()
    att = float(np.sum(st["attempts"][-iters:]))
    ann = float(np.sum(st["annihilated"][-iters:]))
    return att / el, ann / el, att, el


def kernels_code_hash():
    """SHA-256 of the kernel source's code: kernels.cu with // comments,
    trailing blanks and empty lines removed (a comment edit leaves it)."""
    import hashlib
    import re
    out = []
    with open(os.path.join(ROOT, "paper_2006_14956_gb300", "csrc", "kernels.cu"), encoding="utf-8") as f:
        for line in f:
            line = re.sub(r"//.*$", "", line.rstrip("\n")).rstrip()
            if line:
                out.append(line)
    return hashlib.sha256("\n".join(out).encode()).hexdigest()


def _oracle_job(job):
    sysd, prm, state, shift, iters = job
    return oracle_rate(sysd, prm, state, shift, iters)[2:]


def oracle_pool_rate(jobs):
    """The CPU oracle over all host cores: one process per job (spawned, not
    forked, so that no child inherits a CUDA context), attempts over the
    wall time of the whole pool."""
    import multiprocessing as mp
    cores = min(os.cpu_count() or 1, len(jobs))
    t = time.perf_counter()
    with mp.get_context("spawn").Pool(cores) as pool:
        out = pool.map(_oracle_job, jobs, chunksize=1)
    el = time.perf_counter() - t
    att = float(sum(a for a, _ in out))
    return att / el, att, el, cores


def key_sample(state, every):
    """The determinants whose key hash is 0 mod `every` (a uniform sample that
    always holds the same determinants of a given list)."""
    h = (state["alpha"] * np.uint64(0x9E3779B97F4A7C15)) ^ (state["beta"] * np.uint64(0xC2B2AE3D27D4EB4F))
    h ^= h >> np.uint64(29)
    sel = (h % np.uint64(every)) == 0
    return {k: v[sel] for k, v in state.items()}


def aggregate_ranks(t_dev, attempts, annihilated, dist, device):
    """Replicas (one independent run per rank): the job's time is the slowest
    rank's, its work the sum over ranks."""
    import torch
    tt = torch.tensor([t_dev, attempts, annihilated], dtype=torch.float64, device=device)
    tmax = tt[0:1].clone()
    dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(tt, op=dist.ReduceOp.SUM)
    return float(tmax[0]), float(tt[1]), float(tt[2])


def run_reference(args, rank, world):
    """--impl reference: the oracle on the host cores (rank 0 only), on the
    benchmark's workload from a bounded walker population."""
    if rank != 0:
        return None
    sysd, prm = workload_params(workload=args.workload if args.workload.startswith("abinitio") else "abinitio50",
                                generator=args.generator)
    # bounded sample: the same system and parameters (semi-stochastic space
    # off) from at most 2e5 walkers (one oracle iteration ~1 s), fewer when
    # many steps are asked, so that the whole run stays near a minute or two
    walkers = float(min(2e5, max(1e4, 1.2e7 / (args.steps + args.warmup))))
    prm = dict(prm, initial_walkers=walkers, target_walkers=walkers, semistoch_size=0)
    import oracle
    r = oracle.Run(oracle.system_from_workload(sysd), **prm)
    r.step(args.warmup)
    t = time.perf_counter()
    r.step(args.steps)
    el = time.perf_counter() - t
    st = r.stats()
    att = float(np.sum(st["attempts"][-args.steps:]))
    ann = float(np.sum(st["annihilated"][-args.steps:]))
    value = att / el
    return {"metric": METRIC, "value": value, "unit": "spawn attempts/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "annihilated_per_s": ann / el,
            "config": {"workload": WORKLOAD_NAMES[args.workload if args.workload in WORKLOAD_NAMES else "abinitio50"]
                       + ", oracle sample", "tau": prm["tau"], "initiator_threshold": 3, "walkers": walkers,
                       "semistoch": "off in the sample"},
            "cpu_baseline": {"value": value, "unit": "spawn attempts/s", "cores": 1, "kind": "oracle",
                             "sample": "%d oracle iterations from %.3g walkers (semi-stochastic space off)" %
                                       (args.steps, walkers)},
            "e2e": {"value": value, "unit": "spawn attempts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


KERNEL_NAMES = {"k_spawn": "k_spawn_draw + k_spawn_eval (split spawning)",
                "k_annihilate": "k_annihilate_staged + k_annihilate_big"}

WORKLOAD_NAMES = {
    "abinitio50": "abinitio-50orb-10a10b (synthetic: 200 Cholesky vectors, seed 4), D = 1e4, ~1e8 walkers",
    "abinitio24": "abinitio-24orb-6a6b (synthetic: 96 Cholesky vectors, seed 2), ~1e6 walkers",
}


def run_batch(args):
    """64 uneven 2D Hubbard runs (3x4, 4x4, 4x5 at half filling, U/t in {2,4,8},
    walker targets 1e4..1e6, tau 0.005, initiator threshold 3): every iteration
    of all runs in one batched launch, against the same runs stepped one at a
    time.  Attempts/s over the timed iterations of both."""
    import torch
    import paper_2006_14956_gb300 as fq
    runs = workloads.batched_hubbard_instances(64)
    runs = [(s, dict(p, shift_damping=0.5, shift_interval=5)) for s, p in runs]
    hs = [fq.fciqmc_create(s, p) for s, p in runs]
    fq.fciqmc_step_batch(hs, 300)                         # growth, untimed
    tuned = fq.fciqmc_autotune(hs, 20)                    # launch geometry, untimed
    fq.fciqmc_step_batch(hs, args.warmup)
    n0 = [fq.fciqmc_iter_stats_count(h) for h in hs]
    torch.cuda.synchronize()
    t = time.perf_counter()
    fq.fciqmc_step_batch(hs, args.steps)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t
    att_b = sum(float(np.sum(fq.fciqmc_iter_stats_get(h)["attempts"][n0[i]:])) for i, h in enumerate(hs))
    # the same states, one run at a time
    seq = []
    for (s, p), h in zip(runs, hs):
        st, sh = fq.fciqmc_export_state(h), fq.fciqmc_export_shift(h)
        g = fq.fciqmc_create(s, p)
        fq.fciqmc_import_state(g, st["alpha"], st["beta"], st["c"], sh["iteration"], sh["S"], sh["vary"],
                               sh["shift_start"], sh["cnt"], sh["nw_last"])
        seq.append(g)
    for g in seq:
        fq.fciqmc_step(g, args.warmup)
    m0 = [fq.fciqmc_iter_stats_count(g) for g in seq]
    torch.cuda.synchronize()
    t = time.perf_counter()
    for g in seq:
        fq.fciqmc_step(g, args.steps)
    torch.cuda.synchronize()
    ts = time.perf_counter() - t
    att_s = sum(float(np.sum(fq.fciqmc_iter_stats_get(g)["attempts"][m0[i]:])) for i, g in enumerate(seq))
    walkers = [float(fq.fciqmc_iter_stats_get(h)["nw"][-1]) for h in hs]
    # CPU baseline: the oracle on every run's final state, 2 iterations each, all host cores
    jobs = []
    for (s, p), g in zip(runs, seq):
        st, sh = fq.fciqmc_export_state(g), fq.fciqmc_export_shift(g)
        jobs.append((s, p, {k: st[k] for k in ("alpha", "beta", "c")}, sh, 2))
    del hs, seq
    o_rate, o_att, o_el, cores = oracle_pool_rate(jobs)
    return {"metric": METRIC, "value": att_b / tb, "unit": "spawn attempts/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tb / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "64 batched 2D Hubbard runs (3x4/4x4/4x5, U/t 2/4/8, targets 1e4..1e6)",
                       "tau": 0.005, "initiator_threshold": 3, "walkers_total": sum(walkers),
                       "walkers_min": min(walkers), "walkers_max": max(walkers)},
            "sequential": {"value": att_s / ts, "ms_per_step": ts / args.steps * 1e3},
            "autotuned": tuned,
            "batched_over_sequential": (att_b / tb) / (att_s / ts),
            "cpu_baseline": {"value": o_rate, "unit": "spawn attempts/s", "cores": cores, "kind": "oracle",
                             "sample": "2 oracle iterations of each of the 64 runs from its final state, one "
                                       "process per run over %d host cores (%.3g attempts, %.1f s)" %
                                       (cores, o_att, o_el)}}


def run_batch_to_sigma(args):
    """The batched set run to sigma(E_proj) < 1 mEh: the 64 Hubbard runs of
    run_batch submitted together to a server that steps every admitted run
    in one launch per kernel (max_active 64), against the same 64 run one at
    a time (max_active 1).  Each run retires at the first 50-iteration check
    with sigma < 1 mEh after 200 post-equilibration samples, or at
    --max-iters.  A run is bit-identical alone and in the batch, so both
    sides do the same iterations and the ratio of wall times is the ratio of
    throughputs; the identity is checked run by run."""
    import paper_2006_14956_gb300 as fq
    runs = workloads.batched_hubbard_instances(64)
    runs = [(s, dict(p, shift_damping=0.5, shift_interval=5)) for s, p in runs]
    res = {}
    for mode, active in (("batched", 64), ("sequential", 1)):
        srv = fq.fciqmc_server_create(100 << 30, max_active=active)
        ids = [fq.fciqmc_server_submit(srv, s, p, target_sigma=1e-3, max_iters=args.max_iters) for s, p in runs]
        t0 = time.perf_counter()
        while fq.fciqmc_server_tick(srv, 50) > 0:
            pass
        wall = time.perf_counter() - t0
        st = [fq.fciqmc_server_poll(srv, i) for i in ids]
        res[mode] = {"wall_s": wall, "status": st}
        del srv
    sb, ss = res["batched"]["status"], res["sequential"]["status"]
    # bit-identical: iterations, attempts, the energy and its error (every
    # statistics row is exact, E_num included)
    def close(x, y):
        return (np.isnan(x) and np.isnan(y)) or x == y
    same = all(a["iterations"] == b["iterations"] and a["attempts"] == b["attempts"] and close(a["energy"], b["energy"])
               and close(a["sigma"], b["sigma"]) for a, b in zip(sb, ss))
    att = float(sum(a["attempts"] for a in sb))
    tb, ts = res["batched"]["wall_s"], res["sequential"]["wall_s"]
    conv = sum(1 for a in sb if a["state_name"] == "converged")
    iters = [a["iterations"] for a in sb]
    return {"metric": METRIC, "value": att / tb, "unit": "spawn attempts/s", "n_gpus": 1, "steps": len(runs),
            "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "64 2D Hubbard runs (3x4/4x4/4x5, U/t 2/4/8, targets 1e4..1e6) each to "
                                   "sigma(E_proj) < 1 mEh", "tau": 0.005, "initiator_threshold": 3,
                       "max_iters": args.max_iters, "check_every": 50},
            "batched_wall_s": tb, "sequential_wall_s": ts, "batched_over_sequential": ts / tb,
            "sequential_attempts_per_s": att / ts, "converged": conv, "runs": len(runs),
            "iterations_min": min(iters), "iterations_max": max(iters), "iterations_sum": int(sum(iters)),
            "identical_alone_and_batched": bool(same),
            "sigma_mEh_not_converged": sorted(round(1e3 * a["sigma"], 2) for a in sb
                                              if a["state_name"] != "converged" and np.isfinite(a["sigma"]))}


def run_serving(args):
    """Poisson arrivals (20/s) of mixed FCIQMC requests (1D/2D Hubbard and
    synthetic ab initio systems, walker targets 1e4..1e7), each run until the
    blocking error of its energy is below 1 mEh (or an iteration cap).  Each
    request is submitted when it arrives, with its arrival time; the server
    admits it at its next scheduling round (every `--tick` iterations of the
    running batch).  Latency = completion - arrival.  Reports p50/p99 over the
    requests that reached the target, by system kind, with the count and the
    errors reached by the others, and the throughput of the whole stream."""
    import paper_2006_14956_gb300 as fq
    reqs = workloads.serving_requests(args.requests, rate=20.0, seed=5)
    # the client's own preparation (integral generation) happens before the clock starts
    prepared = []
    for r in reqs:
        sysd = r["system"]
        if sysd["kind"] == "abinitio":
            h1, eri = workloads.synthetic_abinitio(sysd["norb"], sysd["n_chol"], sysd["integral_seed"])
            sysd = dict(sysd, h1=h1, eri=eri, ecore=0.0)
        # a trial space (Sec. IV) gives E_Trial, whose error is far below E_proj's
        # when the reference carries little weight
        nt = args.trial_size if sysd["kind"] == "hubbard" else args.trial_size_abinitio
        prm = dict(tau=0.0, target_walkers=r["target_walkers"], initial_walkers=min(r["target_walkers"], 1e3),
                   initiator_threshold=3.0, seed=r["seed"], shift_damping=0.5, shift_interval=5,
                   trial_size=nt, trial_start=50)
        prepared.append((r, sysd, prm))
    srv = fq.fciqmc_server_create(200 << 30, max_active=64)
    t0 = fq.fciqmc_server_clock(srv)
    pending = list(prepared)
    ids = {}
    active = 0
    while pending or active:
        now = fq.fciqmc_server_clock(srv) - t0
        while pending and pending[0][0]["arrival"] <= now:
            r, sysd, prm = pending.pop(0)
            ids[r["id"]] = fq.fciqmc_server_submit(srv, sysd, prm, target_sigma=1e-3, max_iters=args.max_iters,
                                                   t_arrival=t0 + r["arrival"])
        active = fq.fciqmc_server_tick(srv, args.tick) if ids else 0
        if not active and pending:
            time.sleep(max(0.0, pending[0][0]["arrival"] - (fq.fciqmc_server_clock(srv) - t0)))
    t_end = fq.fciqmc_server_clock(srv) - t0
    st = [fq.fciqmc_server_poll(srv, ids[r["id"]]) for r in reqs]
    att = float(sum(s["attempts"] for s in st))
    kinds = {"hubbard": [], "abinitio": []}
    for s, r in zip(st, reqs):
        kinds[r["system"]["kind"]].append(s)

    def summary(group):
        conv = [s for s in group if s["state_name"] == "converged"]
        lat = np.array([s["t_done"] - s["t_arrival"] for s in conv])
        wait = np.array([s["t_start"] - s["t_arrival"] for s in group if s["t_start"] > 0])
        return {"requests": len(group), "converged": len(conv),
                "p50_s": float(np.percentile(lat, 50)) if lat.size else None,
                "p99_s": float(np.percentile(lat, 99)) if lat.size else None,
                "by_trial_estimator": sum(1 for s in conv if s["estimator"] == 1),
                "admission_wait_p50_s": float(np.percentile(wait, 50)) if wait.size else None,
                "sigma_mEh_not_converged": sorted(round(1e3 * s["sigma"], 2) for s in group
                                                  if s["state_name"] != "converged" and np.isfinite(s["sigma"])),
                "failed": sum(1 for s in group if s["state_name"] == "failed")}

    allc = [s for s in st if s["state_name"] == "converged"]
    lat = np.array([s["t_done"] - s["t_arrival"] for s in allc])
    p50 = float(np.percentile(lat, 50)) if lat.size else None
    return {"metric": METRIC, "value": p50, "unit": "s (p50 time from arrival to sigma(E) < 1 mEh)",
            "higher_is_better": False, "n_gpus": 1, "steps": len(reqs), "warmup": 0, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "p50_s": p50, "p99_s": float(np.percentile(lat, 99)) if lat.size else None,
            "converged": len(allc), "requests": len(reqs),
            "by_kind": {k: summary(v) for k, v in kinds.items()},
            "requests_per_s": len(reqs) / t_end, "attempts_per_s": att / t_end, "wall_s": t_end,
            "config": {"workload": "serving stream: Poisson 20/s, 1D/2D Hubbard 8-18 sites and ab initio 16-40 "
                                   "orbitals, targets 1e4..1e7, to sigma(E) < 1 mEh (E_proj or E_Trial, N_T = %d "
                                   "Hubbard, %d ab initio)" % (args.trial_size, args.trial_size_abinitio),
                       "max_iters": args.max_iters, "tick_iters": args.tick,
                       "tau": "0.5/sum_j|H_ref,j| per request"}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed iterations (default: 2000 for abinitio50, 200 for abinitio24, 100 for batch)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="abinitio50",
                    choices=["abinitio50", "abinitio24", "batch", "batch-sigma", "serving"])
    ap.add_argument("--target", type=float, default=0.0,
                    help="walker target in place of the workload's (smaller cases for profiling)")
    ap.add_argument("--equil", type=int, default=200,
                    help="untimed iterations after E_proj's equilibration start (shift start + 500)")
    ap.add_argument("--generator", default="uniform", choices=["uniform", "pchb"],
                    help="double excitations: uniform, or pre-computed heat-bath alias tables")
    ap.add_argument("--requests", type=int, default=200)
    ap.add_argument("--max-iters", type=int, default=20000)
    ap.add_argument("--tick", type=int, default=10, help="serving: iterations per scheduling round")
    ap.add_argument("--trial-size", type=int, default=32, help="serving: trial-space size of Hubbard requests")
    ap.add_argument("--trial-size-abinitio", type=int, default=256,
                    help="serving: trial-space size of ab initio requests")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.steps is None:
        args.steps = {"abinitio50": 2000, "batch": 100}.get(args.workload, 200)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out), flush=True)
        return
    if args.workload in ("batch", "batch-sigma", "serving"):
        import torch
        torch.cuda.set_device(local)
        out = {"batch": run_batch, "batch-sigma": run_batch_to_sigma, "serving": run_serving}[args.workload](args)
        if rank == 0:
            print(json.dumps(out), flush=True)
        return

    import torch
    import paper_2006_14956_gb300 as fq
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    sysd, prm = workload_params(seed_offset=rank, workload=args.workload, generator=args.generator)
    if args.target:  # a smaller list of the same workload (profiling captures)
        prm = dict(prm, target_walkers=args.target, initial_walkers=min(prm["initial_walkers"], args.target / 100.0))
    big = args.workload == "abinitio50"
    h = fq.fciqmc_create(sysd, prm)
    # growth and equilibration, untimed: until E_proj has `--equil` samples
    # after its equilibration start (the shift's start + 500 iterations)
    n_grow = 0
    while True:
        fq.fciqmc_step(h, 50)
        n_grow += 50
        en = fq.fciqmc_energy(h)
        if en["n_samples"] >= args.equil or n_grow >= 5000:
            break
    fq.fciqmc_step(h, args.warmup)                       # warm-up steps
    stream = torch.cuda.ExternalStream(fq.fciqmc_stream(h))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2
    n_before = fq.fciqmc_iter_stats_get(h)["iteration"].size

    # ---- timed region: K single iterations, L2 flushed before each, device events on the run's stream
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            for k in range(args.steps):
                flush.fill_(k & 0xff)
                starts[k].record(stream)
                fq.fciqmc_step_async(h, 1)
                ends[k].record(stream)
        fq.fciqmc_sync(h)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if dist:
        dist.barrier()
    dev_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    t_dev = sum(dev_ms) / 1e3
    launches_per_iter = fq.fciqmc_graph_kernels(h)
    st = fq.fciqmc_iter_stats_get(h)
    sel = slice(n_before, n_before + args.steps)
    attempts = float(np.sum(st["attempts"][sel]))
    annihilated = float(np.sum(st["annihilated"][sel]))
    ndet_mean = float(np.mean(st["ndet"][sel]))
    spawns_mean = float(np.mean(st["spawns"][sel]))
    attempts_mean = attempts / args.steps  # this rank's
    nw_mean = float(np.mean(st["nw"][sel]))
    if dist:
        t_dev, attempts, annihilated = aggregate_ranks(t_dev, attempts, annihilated, dist, "cuda")
    value = attempts / t_dev
    en = fq.fciqmc_energy(h)

    # ---- per-kernel device times for the roofline (events around each launch)
    fq.fciqmc_set_profiling(h, True)
    kprof_iters = min(args.steps, 100)
    n0 = fq.fciqmc_iter_stats_get(h)["iteration"].size
    fq.fciqmc_step(h, kprof_iters)
    fq.fciqmc_set_profiling(h, False)
    kt = fq.fciqmc_kernel_times(h)
    st = fq.fciqmc_iter_stats_get(h)
    nd = st["ndet"]
    n_in = nd[n0 - 1:n0 - 1 + kprof_iters].astype(np.float64)
    n_out = nd[n0:n0 + kprof_iters].astype(np.float64)
    n_sp = st["spawns"][n0:n0 + kprof_iters].astype(np.float64)
    # algorithmic bytes per launch: the spawning kernel reads the list (key + C,
    # 24 B per determinant) and writes the spawns (key + w, 24 B each); the
    # annihilation kernel reads the old list and the spawns and writes the new
    # list (24 B per determinant)
    alg = {"k_spawn": float(np.mean(24.0 * (n_in + n_sp))),
           "k_annihilate": float(np.mean(24.0 * (n_in + n_sp + n_out)))}
    tms = {"k_spawn": kt["spawn"], "k_annihilate": kt["annihilate"]}
    b_iter = float(np.mean(24.0 * n_in + 24.0 * n_out + 48.0 * n_sp))
    if big:
        nnz = fq.fciqmc_semistoch_info(h)["nnz"]
        b_iter += 12.0 * nnz + 16.0 * 1e4
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
        peak, peak_src = float(peaks["hbm_gbs"]), "measured"
    except Exception:
        peak, peak_src = 6800.0, "fallback"
    traffic_rec = {}
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic_%s.json" % args.workload)) as f:
            tr = json.load(f)
        # counters apply only to the kernels and the workload they were captured on
        if (tr.get("kernels_code_sha256") == kernels_code_hash() and
                tr.get("bench_args") == {"workload": args.workload, "generator": args.generator}):
            traffic_rec = tr["kernels"]
    except Exception:
        pass

    # issue ceiling: every SM sub-partition issues at most one warp instruction per clock
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    clk_sum = clk.summary()
    sm_hz = (clk_sum.get("sm_mhz") or clk_sum.get("sm_max_mhz") or 2070.0) * 1e6
    issue_peak = 4.0 * n_sm * sm_hz

    def roof(k):
        ach = alg[k] / (tms[k] * 1e-3) / 1e9
        rec = traffic_rec.get(k) or {}
        # DRAM bytes and warp instructions were counted on a smaller list; both
        # scale with the records a launch processes
        units = float(np.mean(n_in + n_sp))
        tr_b = rec["dram_bytes_per_unit"] * units if "dram_bytes_per_unit" in rec else rec.get("dram_bytes_per_launch")
        out = {"kernel": k, "kernels": KERNEL_NAMES[k], "achieved": ach, "frac": ach / peak, "traffic": tr_b,
               "alg_bytes_per_launch": alg[k], "launch_ms": tms[k]}
        if "inst_per_unit" in rec:
            inst = rec["inst_per_unit"] * units
            out["issue"] = {"bound": "issue", "warp_instructions_per_launch": inst,
                            "achieved": inst / (tms[k] * 1e-3), "peak": issue_peak,
                            "unit": "warp instructions/s", "frac": inst / (tms[k] * 1e-3) / issue_peak,
                            "peak_source": "4 per SM per clock x %d SMs x the median SM clock under load" % n_sm}
        return out

    # the device's nominal HBM bandwidth (double data rate x memory clock x bus width), stated beside the
    # measured copy bandwidth the fractions use
    try:
        mclk, mbus = fq.fciqmc_device_memory(local)
    except fq.FciqmcError:
        mclk, mbus = 0, 0
    nominal = 2.0 * mclk * 1e3 * mbus / 8.0 / 1e9 if mclk and mbus else None
    dominant = max(tms, key=tms.get)  # the kernel with the longest launches
    other = "k_annihilate" if dominant == "k_spawn" else "k_spawn"
    roofline = {"bound": "hbm", "peak": peak, "peak_source": peak_src + " hbm_gbs", "unit": "GB/s",
                "peak_nominal_device": nominal,
                "peak_nominal_source": "2 x peak memory clock x bus width (CUDA device attributes)", **roof(dominant),
                "iteration_frac": b_iter / (t_dev / args.steps) / 1e9 / peak, "other": roof(other)}

    # ---- end to end through the public API: restart from a pinned host checkpoint
    state = fq.fciqmc_export_state(h)
    shift = fq.fciqmc_export_shift(h)
    keep = ("alpha", "beta", "c")
    pinned = {k: torch.from_numpy(np.ascontiguousarray(state[k])).pin_memory() for k in keep}
    host_state = {k: v.numpy() for k, v in pinned.items()}
    # the job's output buffers: pinned host memory allocated before the job
    # (a checkpointing user keeps them), room for 25 % more determinants
    cap_out = int(state["c"].size * 1.25) + 4096
    pin_out = {"alpha": torch.empty(cap_out, dtype=torch.int64, pin_memory=True),
               "beta": torch.empty(cap_out, dtype=torch.int64, pin_memory=True),
               "c": torch.empty(cap_out, dtype=torch.float64, pin_memory=True),
               "hdiag": torch.empty(cap_out, dtype=torch.float64, pin_memory=True),
               "flags": torch.empty(cap_out, dtype=torch.int32, pin_memory=True)}
    out_bufs = {k: (v.numpy().view(np.uint64) if k in ("alpha", "beta") else v.numpy()) for k, v in pin_out.items()}
    # the restarted run selects its deterministic space from the imported list
    prm2 = dict(prm, semistoch_start=shift["iteration"] - shift["shift_start"]) if big else prm
    del h
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h2 = fq.fciqmc_create(sysd, prm2)
    t1 = time.perf_counter()
    fq.fciqmc_import_state(h2, host_state["alpha"], host_state["beta"], host_state["c"], shift["iteration"],
                           shift["S"], shift["vary"], shift["shift_start"], shift["cnt"], shift["nw_last"])
    t2 = time.perf_counter()
    fq.fciqmc_step(h2, E2E_STEPS)
    t3 = time.perf_counter()
    out_state = fq.fciqmc_export_state(h2, out=out_bufs)
    en2 = fq.fciqmc_energy(h2)
    e2e_el = time.perf_counter() - t0
    e2e_phases = {"create": t1 - t0, "import": t2 - t1, "steps": t3 - t2, "export_energy": t0 + e2e_el - t3}
    st2 = fq.fciqmc_iter_stats_get(h2)
    e2e_att = float(np.sum(st2["attempts"][-E2E_STEPS:]))
    # integrals and the checkpoint's keys and amplitudes in; the final list and statistics out
    h2d = sysd["h1"].nbytes + sysd["eri"].nbytes + sum(host_state[k].nbytes for k in keep)
    d2h = sum(v.nbytes for v in out_state.values()) + E2E_STEPS * ctypes.sizeof(fq.fciqmc_iter_stats)
    assert np.isfinite(en2["nw"])
    del h2, pinned, host_state, out_state, out_bufs, pin_out

    # ---- CPU baseline: the oracle on a key-hash sample of the same state, bounded
    cpu = None
    if rank == 0:
        every = 16 if big else 1
        sample = key_sample({k: state[k] for k in keep}, every) if every > 1 else {k: state[k] for k in keep}
        iters = 3 if big else 1
        o_att_rate, o_ann_rate, o_att, o_el = oracle_rate(sysd, dict(prm, semistoch_size=0), sample, shift, iters)
        cpu = {"value": o_att_rate, "unit": "spawn attempts/s", "cores": 1, "kind": "oracle",
               "sample": "%d oracle iteration(s) (%.3g attempts, %.1f s) from %s of the GPU state at %.3g walkers "
                         "(semi-stochastic space off)" %
                         (iters, o_att, o_el, ("a 1/%d key-hash sample (%d determinants)" % (every, sample["c"].size))
                          if every > 1 else "all", nw_mean)}
    del state

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "spawn attempts/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_dev / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "annihilated_per_s": annihilated / t_dev,
            "config": {"workload": WORKLOAD_NAMES[args.workload],
                       "generator": ("uniform" if args.generator == "uniform" else
                                     "pre-computed heat-bath doubles") + ", p_single 0.1",
                       "initiator_threshold": 3, "tau": prm["tau"],
                       "tau_note": ("prescribed 5e-4 exceeds 1/sum_j|H_ref,j| (39309 Eh): walker number uncontrollable"
                                    if big else
                                    "prescribed 1e-3 exceeds 1/sum_j|H_ref,j| (2412 Eh): walker number uncontrollable"),
                       "semistoch_size": prm.get("semistoch_size", 0),
                       "walkers_mean": nw_mean, "dets_mean": ndet_mean, "spawns_mean": spawns_mean,
                       "attempts_mean": attempts_mean, "l2": "flushed (256 MB write) between steps",
                       "untimed_iterations_before": n_grow + args.warmup,
                       "parallelism": "replicas" if world > 1 else "single"},
            "roofline": roofline,
            "kernel_ms": kt,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_att / e2e_el, "unit": "spawn attempts/s", "h2d_bytes_per_step": h2d / E2E_STEPS,
                    "d2h_bytes_per_step": d2h / E2E_STEPS,
                    "job": "create + import the %.3g-determinant checkpoint from pinned host memory + %d steps + "
                           "export into pinned host memory + energy" % (ndet_mean, E2E_STEPS),
                    "phases_s": e2e_phases},
            "gpu_launches": args.steps * launches_per_iter,
            "gpu_launches_per_step": launches_per_iter,
            "wall_s_timed": wall,
            "clocks": clk.summary(),
            "energy": {"e_proj_mean": en["e_proj_mean"], "e_proj_sigma": en["e_proj_sigma"],
                       "e_proj_samples": en["n_samples"], "shift_mean": en["shift_mean"],
                       "shift_sigma": en["shift_sigma"], "eref": en["eref"]},
        }
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
