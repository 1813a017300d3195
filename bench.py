"""Benchmark of the SIDM scattering step on one B300 (or N independent replicas).

Headline workload: isolated Hernquist halo, N = 2^20, N_ngb = 64 +- 5,
constant sigma/m = 1, open boundaries, FP64, power-of-two timestep bins with
~10 % of the particles active per finest step (step s of a 100-step cycle
uses the active set of finest step s).  One bench step = one complete
scattering step (keys, sort, structure, h_SI search, pairs + draws + Eq. 18,
kicks) on the step's active set.  Metric: particle updates (active
particles) per second.

The default run also measures, as sub-objects of its one JSON line:
  c2_eq18_bins  the same halo with bins from its own Eq. 18 limits (no bin
                clipped, so no pair reaches P = 1);
  c3_precision  NFW 2^23 with the Yukawa-like cross-section: the FP32-split
                form against the FP64 plain form, step by step;
  c4_batch      512 Hernquist haloes of uneven size stepped together, against
                the plain per-halo loop (graph-replayed too);
  c5_serving    halo requests served with continuous batching: p50/p99
                latency at the offered rate and at fractions of capacity.

    python bench.py [--steps K] [--warmup W] [--impl ours|reference] [--no-extras]

Under torchrun (N > 1) every rank runs its own halo replica on its own GPU
(independent problems, no data-path collective): value = all ranks'
updates / the slowest rank's time ("scaling": "weak"); the sub-objects are
measured at N = 1 only.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SIDM particle-updates/s (search+scatter)"
UNIT = "particle-updates/s"
CYCLE = 100

# Algorithmic HBM bytes of the step (FP64 state; what the method must move
# once), per particle (N) and per active particle (A):
#   build (keys, sort, structure): 24 B position read, 12 B key + index
#     written, 4 radix passes x 24 B, 2 x 60 B permutation, ~8 B cells
#     = 260 B x N;
#   neighbour search + pair/scatter kernels: own position and velocity read,
#     h and the Eq. 18 limit written = 64 B x A, plus the neighbour data
#     reached from HBM once, 48 B x N;
#   kicks ~100 B per accepted pair (not counted).
BUILD_BYTES_N = 260.0
NEIGHBOUR_SCATTER_BYTES = (48.0, 64.0)      # (per N, per A)
STEP_BYTES = (BUILD_BYTES_N + 48.0, 64.0)   # 308 B x N + 64 B x A

# DRAM read + write of the neighbour-search and pair kernels (search_kernel,
# pairs_kernel, pairs_walk_kernel, pairs_exact_kernel, limits_kernel) per
# step of the headline workload, from an ncu capture of this bench's own
# timed steps (10 graph-replayed steps, tuned shapes, L2 flushed between
# steps): 16.16 + 36.47 + 0.44 + 10.63 + 9.44 MB.  The velocity permutation
# that shares their phase time (40.8 MB) is a build term of the byte model.
# None once those kernels change and until they are captured again.
NEIGHBOUR_SCATTER_TRAFFIC = 73.14e6

# Warp instructions the search kernel issues per query on this workload, from
# an ncu capture of the bench's first timed launch (smsp__inst_executed.sum /
# queries: 206.6 M / 51,520), and the B300's issue rate: one warp instruction
# per scheduler per clock, 4 schedulers per SM, 148 SMs, 2032 MHz maximum.
SEARCH_INST_PER_QUERY = 4010.0
ISSUE_PEAK = 148 * 4 * 2032e6          # warp instructions per second


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6400.0)), "measured"
    return 6400.0, "fallback"


def _workload(seed_offset=0, n=1 << 20):
    """The bench halo of one replica: rank r steps the Hernquist halo of
    seed 1 + r (replicas only, no data-path collective)."""
    from paper_2607_05504_b300 import inputs as I
    w = I.hernquist_2pow20(seed=1 + seed_offset, n=n)
    masks = np.stack([I.active_at_step(w["bins"], s) for s in range(CYCLE)])
    return w, masks


def reduce_over_ranks(t_ms, updates, device):
    """Whole-job figures of a replicas run: the slowest rank's time and the
    updates of all ranks (two all-reduces of host-side scalars)."""
    import torch
    import torch.distributed as D
    tt = torch.tensor([t_ms, float(updates)], dtype=torch.float64, device=device)
    mx = tt.clone()
    D.all_reduce(mx, op=D.ReduceOp.MAX)
    D.all_reduce(tt, op=D.ReduceOp.SUM)
    return float(mx[0]), float(tt[1])


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="sidm_clocks_", suffix=".csv")
        os.close(fd)

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self) -> dict:
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
            os.remove(self.path)
        except Exception:
            return out
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except Exception:
                continue
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(smax), samples=len(sm))
        out["reasons"] = sorted(reasons)
        return out


def run_reference(args) -> None:
    """The oracle as it stands, on the host cores, on the same workload: each
    step runs the full oracle step on a bounded sample of the step's active set."""
    import oracle
    oracle.build()
    w, masks = _workload()
    p, bins = w["particles"], w["bins"]
    cap = 1 << 14
    rng = np.random.default_rng(0)

    def sample(s):
        a = masks[s].copy()
        idx = np.nonzero(a)[0]
        if idx.size > cap:
            a[:] = 0
            a[rng.choice(idx, cap, replace=False)] = 1
        return a

    vel = p.vel.copy()
    for k in range(args.warmup):
        s = k % CYCLE
        oracle.step(p.pos, vel, p.mass, p.ids, sample(s), bins, w["dt_max"], n_ngb=64, seed=0, step=s)
    upd, t0 = 0, time.perf_counter()
    for k in range(args.steps):
        s = (args.warmup + k) % CYCLE
        a = sample(s)
        r = oracle.step(p.pos, vel, p.mass, p.ids, a, bins, w["dt_max"], n_ngb=64, seed=0, step=s)
        vel = r["vel"]
        upd += int(a.sum())
    dt = time.perf_counter() - t0
    v = upd / dt
    cpu = host_cpu()
    cores = cpu["nproc"]
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": "hernquist-2^20 (N_ngb 64, sigma/m 1, ~10% active, 100-step bin cycle)",
                       "l2": "host run"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"full oracle step per bench step, active set capped at {cap} "
                                       "(seeded subset) of the step's active particles",
                             "cpu_model": cpu["model"], "nproc": cores},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def host_cpu() -> dict:
    """The host's CPU model and the cores this process may use."""
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    try:
        usable = len(os.sched_getaffinity(0))
    except AttributeError:
        usable = os.cpu_count()
    return {"model": model, "nproc": usable, "logical_cpus": os.cpu_count()}


def cpu_baseline(w, masks, budget_s=10.0, budget_1core_s=8.0) -> dict:
    """The oracle as it stands on the host cores: all cores on finest steps
    1, 2, ... of the cycle for about budget_s, then one core on steps from 1
    for about budget_1core_s (at least one whole step each)."""
    import oracle
    oracle.build()
    p, bins = w["particles"], w["bins"]
    cpu = host_cpu()

    def run(n_threads, budget):
        upd, t0, k = 0, time.perf_counter(), 0
        vel = p.vel.copy()
        while k < CYCLE - 1 and (k == 0 or (time.perf_counter() - t0) < budget):
            s = 1 + k
            r = oracle.step(p.pos, vel, p.mass, p.ids, masks[s], bins, w["dt_max"], n_ngb=64,
                            seed=0, step=s, n_threads=n_threads)
            vel = r["vel"]
            upd += int(masks[s].sum())
            k += 1
        return upd, time.perf_counter() - t0, k

    u_all, t_all, k_all = run(0, budget_s)
    u_one, t_one, k_one = run(1, budget_1core_s)
    return {"value": u_all / t_all, "unit": UNIT, "cores": cpu["nproc"], "kind": "oracle",
            "sample": f"finest steps 1..{k_all} of the 100-step cycle ({u_all} active updates, "
                      f"{t_all:.1f} s, all {cpu['nproc']} cores)",
            "one_core": {"value": u_one / t_one, "unit": UNIT, "cores": 1,
                         "sample": f"finest steps 1..{k_one} ({u_one} active updates, "
                                   f"{t_one:.1f} s, one OpenMP thread)"},
            "cpu_model": cpu["model"], "nproc": cpu["nproc"]}


def _setup_stream(local=0):
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    return torch, dev, stream


def _pair_keys(ctx) -> np.ndarray:
    """Accepted pairs of the context's last step as sorted (a << 32 | b) keys."""
    from paper_2607_05504_b300 import sidm
    total = sidm.sidm_get_pairs(ctx.handle, None, None, 0)
    ab = np.zeros((max(total, 1), 2), np.uint32)
    ords = np.zeros(max(total, 1), np.uint64)
    sidm.sidm_get_pairs(ctx.handle, ab, ords, total)
    return np.sort((ab[:total, 0].astype(np.uint64) << np.uint64(32)) | ab[:total, 1])


def batch_run(n_halos=512, steps=10, warmup=3, workers=0, precision=None, plain=True) -> dict:
    """c4: independent Hernquist haloes (N log-uniform in [2^12, 2^18],
    sigma/m log-uniform in [0.1, 10], own seeds, bins and step counters)
    stepped together (one sidm_step_haloes per tick, graph-replayed, launch
    shapes autotuned), against the plain per-halo form on the same haloes and
    ticks: one context per halo, one sidm_step per halo, graph-replayed with
    the same launch shapes.  Both forms run the same precision."""
    from paper_2607_05504_b300 import inputs as I
    from paper_2607_05504_b300 import sidm
    torch, dev, stream = _setup_stream()
    prec = sidm.FP32_SPLIT if precision is None else precision
    t0 = time.perf_counter()
    haloes = I.hernquist_batch(n_halos, workers=workers)
    t_gen = time.perf_counter() - t0
    p, off, bins = I.pack(haloes)
    n = p.n
    ticks = warmup + steps

    def masks_for(s):
        return np.concatenate([I.active_at_step(h["bins"], s) for h in haloes])

    cyc = [masks_for(s) for s in range(ticks)]
    n_active = [int(cyc[s].sum()) for s in range(ticks)]
    ctx = sidm.Context(n_ngb=64, box=0.0, stream=stream.cuda_stream, n_max=n, use_graph=True,
                       precision=prec)
    ctx.set_particles(torch.from_numpy(p.pos).to(dev), torch.from_numpy(p.vel).to(dev),
                      torch.from_numpy(p.ids.view(np.int32)).to(dev),
                      mass=torch.from_numpy(p.mass).to(dev))
    ctx.set_haloes(off)
    bins_d = torch.from_numpy(bins).to(dev)
    masks_d = [torch.from_numpy(m).to(dev) for m in cyc]

    def params(s):
        return [sidm.HaloParams(h["dt_max"], sidm.SigmaModel(0, h["sigma0"], 1.0), h["seed"], s)
                for h in haloes]

    prm = [params(s) for s in range(ticks)]
    for s in range(warmup):
        sidm.sidm_step_haloes(ctx.handle, masks_d[s], bins_d, prm[s], None)
    tuning = ctx.autotune(prm[warmup], masks_d[warmup], bins_d, reps=1)
    sidm.sidm_step_haloes(ctx.handle, masks_d[warmup - 1], bins_d, prm[warmup - 1], None)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")      # a profiler can keep to the timed ticks
    e0.record(stream)
    for s in range(warmup, ticks):
        sidm.sidm_step_haloes(ctx.handle, masks_d[s], bins_d, prm[s], None)
    e1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    t_batch = e0.elapsed_time(e1) * 1e-3
    graph_state = ctx.graph_state
    ctx.close()
    del masks_d
    torch.cuda.empty_cache()
    upd = sum(n_active[warmup:])
    if not plain:
        return {"value": upd / t_batch, "unit": UNIT, "ms_per_tick": 1e3 * t_batch / steps,
                "ticks": steps, "n": n, "n_halos": n_halos, "graph": graph_state,
                "tuning": tuning, "plain_per_halo": None}
    # plain per-halo form: a context per halo, stepped one after another
    plain = []
    for h in haloes:
        hp = h["particles"]
        c = sidm.Context(n_ngb=64, box=0.0, stream=stream.cuda_stream, n_max=hp.n, use_graph=True,
                         precision=prec)
        c.set_particles(torch.from_numpy(hp.pos).to(dev), torch.from_numpy(hp.vel).to(dev),
                        torch.from_numpy(hp.ids.view(np.int32)).to(dev),
                        mass=torch.from_numpy(hp.mass).to(dev))
        c.set_tuning(**tuning)
        mk = [torch.from_numpy(I.active_at_step(h["bins"], s)).to(dev) for s in range(ticks)]
        plain.append((c, mk, torch.from_numpy(h["bins"]).to(dev),
                      sidm.SigmaModel(0, h["sigma0"], 1.0)))
    for s in range(warmup):
        for (c, mk, hb, sg), h in zip(plain, haloes):
            c.step_counter = s
            sidm.sidm_step(c.handle, mk[s], hb, h["dt_max"], sg, h["seed"], None)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for s in range(warmup, ticks):
        for (c, mk, hb, sg), h in zip(plain, haloes):
            c.step_counter = s
            sidm.sidm_step(c.handle, mk[s], hb, h["dt_max"], sg, h["seed"], None)
    b.record(stream)
    torch.cuda.synchronize()
    t_plain = a.elapsed_time(b) * 1e-3
    plain_graphs = sum(1 for c, *_ in plain if c.graph_state == 1)
    for c, *_ in plain:
        c.close()
    del plain
    torch.cuda.empty_cache()
    return {"value": upd / t_batch, "unit": UNIT, "ms_per_tick": 1e3 * t_batch / steps,
            "ticks": steps, "warmup": warmup,
            "workload": f"{n_halos} Hernquist haloes, N log-uniform in [2^12, 2^18] (sum {n}), "
                        "sigma/m log-uniform in [0.1, 10], own seeds, bins and step counters, "
                        "N_ngb 64",
            "precision": "fp32_split" if prec == sidm.FP32_SPLIT else "fp64_plain",
            "n": n, "n_halos": n_halos, "mean_active": upd / steps,
            "form": "one multi-halo step per tick (sidm_step_haloes), graph-replayed",
            "graph": graph_state, "tuning": tuning,
            "plain_per_halo": {"value": upd / t_plain, "unit": UNIT,
                               "ms_per_tick": 1e3 * t_plain / steps,
                               "graphs": plain_graphs,
                               "note": "same haloes and ticks, one context and one sidm_step per "
                                       "halo, graph-replayed, the batch's launch shapes"},
            "speedup_vs_plain": t_plain / t_batch,
            "timing": "CUDA events on the launch stream around all ticks; inputs resident",
            "input_generation_s": round(t_gen, 1)}


def precision_run(log2_n=23, steps=10) -> dict:
    """c3: NFW halo (c = 10, r_s = 1, N = 2^log2_n), Yukawa-like sigma0/m = 1
    with w = v_c(r_s), N_ngb 64, power-of-two bins: the FP32-split form
    against the FP64 plain form, step by step from the same state (the FP64
    form's).  Reports both forms' throughput (CUDA events, one step at a time),
    the accepted-pair mismatch |A32 xor A64| / |A64|, and the split form's
    relative energy / momentum change per step, against its own start and
    against the FP64 form's result."""
    from paper_2607_05504_b300 import inputs as I
    from paper_2607_05504_b300 import sidm
    torch, dev, stream = _setup_stream()
    p = I.nfw_halo(1 << log2_n, 2)
    w = p.meta["v_c_rs"]
    bins, dt = I.timestep_bins(p, I.nfw_density, 1.0, 64)
    ctxs = {k: sidm.Context(n_ngb=64, stream=stream.cuda_stream, n_max=p.n, precision=v,
                            use_graph=True)
            for k, v in (("fp64", sidm.FP64_PLAIN), ("split", sidm.FP32_SPLIT))}
    pos, vel = torch.from_numpy(p.pos).to(dev), torch.from_numpy(p.vel).to(dev)
    ids, mass = torch.from_numpy(p.ids.view(np.int32)).to(dev), torch.from_numpy(p.mass).to(dev)
    for c in ctxs.values():
        c.set_particles(pos, vel, ids, mass=mass)
    bins_d = torch.from_numpy(bins).to(dev)
    sg = sidm.SigmaModel(sidm.SIGMA_YUKAWA, 1.0, w)
    # launch shapes of each form tuned on step 1's active set (the state is
    # restored), then warm-up: both forms' graphs captured on that set
    act1 = torch.from_numpy(I.active_at_step(bins, 1)).to(dev)
    tunings = {}
    for k, c in ctxs.items():
        c.step_counter = 1
        tunings[k] = c.autotune([sidm.HaloParams(dt, sg, 7, 1)], act1, bins_d, reps=3)
    for c in ctxs.values():
        c.step_counter = 1
        sidm.sidm_step(c.handle, act1, bins_d, dt, sg, 7, None)
        c.set_velocities(vel)
    torch.cuda.synchronize()
    t = {"fp64": 0.0, "split": 0.0}
    n64 = nx = upd = 0
    d_e, d_p, d_e64 = 0.0, 0.0, 0.0
    m64 = mass.to(torch.float64)
    vcur = vel.clone()
    vout = {k: torch.empty_like(vel) for k in ctxs}

    def energy_momentum(v):
        e = 0.5 * float(torch.sum(m64 * torch.sum(v * v, 1)).item())
        pm = torch.sum(m64[:, None] * v, 0).cpu().numpy()
        return e, pm

    pscale = float((m64[:, None] * vel.abs()).sum().item())
    for s in range(steps):
        act = torch.from_numpy(I.active_at_step(bins, s)).to(dev)
        keys = {}
        for k, c in ctxs.items():
            c.set_velocities(vcur)
            c.step_counter = s
            c.sync()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sidm.sidm_step(c.handle, act, bins_d, dt, sg, 7, None)
            b.record(stream)
            b.synchronize()
            t[k] += a.elapsed_time(b) * 1e-3
            keys[k] = _pair_keys(c)
            sidm.sidm_get_particles(c.handle, vout[k])
        upd += int(act.sum().item())
        n64 += keys["fp64"].size
        nx += np.setxor1d(keys["fp64"], keys["split"], assume_unique=True).size
        e0, p0 = energy_momentum(vcur)
        e32, p32 = energy_momentum(vout["split"])
        e64, _ = energy_momentum(vout["fp64"])
        d_e = max(d_e, abs(e32 - e0) / e0)
        d_e64 = max(d_e64, abs(e32 - e64) / e0)
        d_p = max(d_p, float(np.max(np.abs(p32 - p0))) / pscale)
        vcur.copy_(vout["fp64"])
    for c in ctxs.values():
        c.close()
    torch.cuda.empty_cache()
    return {"value": upd / t["split"], "unit": UNIT, "steps": steps,
            "workload": f"NFW c=10 N=2^{log2_n}, Yukawa sigma0/m=1 w=v_c(r_s), N_ngb 64, "
                        "power-of-two bins, finest steps 0..{}".format(steps - 1),
            "n": p.n, "mean_active": upd / steps,
            "fp64_plain": {"value": upd / t["fp64"], "unit": UNIT},
            "speedup_split_vs_fp64": t["fp64"] / t["split"],
            "tuning": tunings,
            "pair_mismatch": {"rate": nx / max(n64, 1), "pairs_fp64": int(n64),
                              "differing": int(nx), "target": 1e-5},
            "drift_per_step": {"energy_rel": d_e, "energy_rel_vs_fp64": d_e64,
                               "momentum_rel": d_p, "target_energy": 1e-10},
            "timing": "CUDA events around each step (graph-replayed), both forms from the "
                      "same state; energies from the returned velocities (FP64 sums)"}


def serving_run(requests=32, log2_nmax=21.0, max_steps=1000, budget_gb=120.0,
                offered_rate=200.0, fracs=(0.5, 0.9)) -> dict:
    """c5: Poisson streams of halo requests served with continuous batching
    under a device-memory budget.  First the saturated throughput (every
    request present at t = 0), which gives the capacity in requests/s; then
    Poisson arrivals at the offered rate and at fractions of capacity, each
    with p50/p99 latency.  A rate is stable when its offered work is at most
    the measured capacity (load <= 1) and the last third of the requests
    waits no longer than 1.5x the first third (no backlog).  The load test
    is needed because a finite stream whose requests all fit the budget at
    once shows an overload only as longer shared-time latencies, not as a
    growing queue."""
    import dataclasses
    from paper_2607_05504_b300 import serving as S
    torch, dev, stream = _setup_stream()
    t0 = time.perf_counter()
    base = S.request_stream(requests, rate=1.0, seed=3, log2_n=(12.0, log2_nmax),
                            steps=(10, max_steps), pool=0)
    t_gen = time.perf_counter() - t0
    unit_arrivals = [r.arrival for r in base]
    budget = budget_gb * 1e9

    def serve(rate):
        reqs = [dataclasses.replace(r, arrival=(0.0 if rate is None else a / rate), steps_done=0,
                                    admitted=None, finished=None, result_vel=None)
                for r, a in zip(base, unit_arrivals)]
        eng = S.GpuEngine(budget_bytes=budget, stream=stream)
        rep = S.Server(eng, S.Scheduler(budget, eng.bytes_per_particle)).run(reqs)
        eng.close()
        lat = [r.latency for r in sorted(reqs, key=lambda r: r.arrival)]
        third = max(len(lat) // 3, 1)
        growth = float(np.mean(lat[-third:]) / max(np.mean(lat[:third]), 1e-9))
        return rep, growth

    serve(None)                                  # first pass: host code and graphs warm
    sat, _ = serve(None)
    work = sat.updates / len(base)               # active-particle updates per request
    cap_rate = sat.throughput / work             # requests/s the device sustains
    rows = []
    for frac, rate in [(None, offered_rate)] + [(f, f * cap_rate) for f in fracs]:
        rep, growth = serve(rate)
        rows.append({"rate_per_s": rate, "load": (rate / cap_rate), "throughput": rep.throughput,
                     "p50_s": rep.percentile(50), "p99_s": rep.percentile(99),
                     "backlog_growth": growth,
                     "stable": rate <= cap_rate and growth <= 1.5})
    stable = [x for x in rows[1:] if x["stable"]]
    torch.cuda.empty_cache()
    return {"value": sat.throughput, "unit": UNIT,
            "workload": "halo requests: Hernquist or NFW, constant or Yukawa sigma, N log-uniform "
                        f"in [2^12, 2^{log2_nmax:g}], steps log-uniform in [10, {max_steps}], "
                        f"{requests} requests, {budget_gb:g} GB budget",
            "saturation": {"throughput": sat.throughput, "requests_per_s": cap_rate,
                           "p50_s": sat.percentile(50), "p99_s": sat.percentile(99),
                           "wall_s": sat.wall, "ticks": sat.ticks},
            "offered": rows[0], "sweep": rows[1:],
            "stable_rate_per_s": stable[-1]["rate_per_s"] if stable else None,
            "timing": "host clock from each request's arrival to its result on the host",
            "input_generation_s": round(t_gen, 1)}


def eq18_run(w, tuning, steps=20, warmup=5, local=0) -> dict:
    """The headline halo with bins from its own Eq. 18 limits (Sec. 4.4): an
    all-active step gives every particle's limit, each particle takes the
    smallest bin whose step lies below its limit (no clipping), and dt_max is
    set for a mean active fraction of 0.10 over the 100-step cycle.  Times
    the same cycle steps as the headline, and counts pairs at P >= 1."""
    from paper_2607_05504_b300 import inputs as I
    from paper_2607_05504_b300 import sidm
    torch, dev, stream = _setup_stream(local)
    p = w["particles"]
    n = p.n
    pos_d, vel_d = torch.from_numpy(p.pos).to(dev), torch.from_numpy(p.vel).to(dev)
    ids_d, mass_d = torch.from_numpy(p.ids.view(np.int32)).to(dev), torch.from_numpy(p.mass).to(dev)
    sg = sidm.SigmaModel(sidm.SIGMA_CONST, 1.0, 1.0)
    lc = sidm.Context(n_ngb=64, box=0.0, stream=stream.cuda_stream, device=local, n_max=n)
    lc.set_particles(pos_d, vel_d, ids_d, mass=mass_d)
    # every particle active; the limits do not depend on the step's dt, so
    # the headline's bins keep the step's probabilities in range
    sidm.sidm_step(lc.handle, None, torch.from_numpy(w["bins"]).to(dev), w["dt_max"], sg, 0, None)
    lim = torch.empty(n, dtype=torch.float64, device=dev)
    sidm.sidm_timestep_limits(lc.handle, lim)
    lc.close()
    bins, dt_max = I.eq18_bins(lim.cpu().numpy())
    masks = np.stack([I.active_at_step(bins, s) for s in range(CYCLE)])
    n_act = [int(m.sum()) for m in masks]
    masks_d = torch.from_numpy(masks).to(dev)
    bins_d = torch.from_numpy(bins).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    ctx = sidm.Context(n_ngb=64, box=0.0, stream=stream.cuda_stream, device=local, n_max=n,
                       use_graph=True)
    ctx.set_particles(pos_d, vel_d, ids_d, mass=mass_d)
    ctx.set_tuning(**tuning)
    for k in range(warmup):
        sidm.sidm_step(ctx.handle, masks_d[k % CYCLE], bins_d, dt_max, sg, 0, None)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    torch.cuda.synchronize()
    upd = 0
    for k in range(steps):
        s = (warmup + k) % CYCLE
        flush.zero_()
        ev[k][0].record(stream)
        sidm.sidm_step(ctx.handle, masks_d[s], bins_d, dt_max, sg, 0, None)
        ev[k][1].record(stream)
        upd += n_act[s]
    torch.cuda.synchronize()
    t_ms = sum(a.elapsed_time(b) for a, b in ev)
    ctx.close()
    # pair statistics of the same steps (untimed, from the same start state)
    sc = sidm.Context(n_ngb=64, box=0.0, stream=stream.cuda_stream, device=local, n_max=n)
    sc.set_particles(pos_d, vel_d, ids_d, mass=mass_d)
    pge1 = acc = mmax = 0
    for k in range(warmup + steps):
        st = sc.step(dt_max, masks_d[k % CYCLE], bins_d, seed=0)
        if k >= warmup:
            pge1 += st["n_p_ge_1"]
            acc += st["n_accepted"]
            mmax = max(mmax, st["max_multiplicity"])
    sc.close()
    del flush
    torch.cuda.empty_cache()
    return {"value": upd / (t_ms * 1e-3), "unit": UNIT, "ms_per_step": t_ms / steps,
            "steps": steps, "warmup": warmup, "mean_active": upd / steps,
            "bins": int(bins.max()) + 1, "dt_max": dt_max,
            "mean_active_fraction_cycle": float(np.mean(n_act)) / n,
            "n_p_ge_1": int(pge1), "n_accepted": int(acc), "max_multiplicity": int(mmax),
            "workload": "hernquist-2^20 with bins from its own step-0 Eq. 18 limits (smallest bin "
                        "below each limit, none clipped), dt_max set for 10 % mean activity",
            "timing": "as the headline: CUDA events per step, L2 flushed between steps"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="hernquist",
                    choices=["hernquist", "batch", "serving", "precision"])
    ap.add_argument("--log2-n", type=int, default=23)
    ap.add_argument("--n-halos", type=int, default=512)
    ap.add_argument("--requests", type=int, default=48)
    ap.add_argument("--log2-nmax", type=float, default=21.0)
    ap.add_argument("--max-steps", type=int, default=1000)
    ap.add_argument("--budget-gb", type=float, default=120.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--reuse-every", type=int, default=8,
                    help="also time the steps with the tree rebuilt every k steps (0: skip)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the c2-Eq.18, c3, c4 and c5 sub-objects of the default run")
    ap.add_argument("--no-plain", action="store_true",
                    help="--workload batch: skip the per-halo comparison loop")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    workers = max(1, min(16, (host_cpu()["nproc"] or 1)))
    if args.impl == "ours" and args.workload != "hernquist":
        if args.workload == "batch":
            d = batch_run(args.n_halos, args.steps, args.warmup, workers=workers,
                          plain=not args.no_plain)
        elif args.workload == "precision":
            d = precision_run(args.log2_n, args.steps)
        else:
            d = serving_run(args.requests, args.log2_nmax, args.max_steps, args.budget_gb)
        line = {"metric": METRIC, "value": d["value"], "unit": UNIT, "n_gpus": 1,
                "steps": d.get("steps", d.get("ticks", 0)), "warmup": args.warmup,
                "ms_per_step": d.get("ms_per_tick", d.get("ms_per_step")),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": {"workload": d.get("workload", args.workload)}, args.workload: d}
        print(json.dumps(line), flush=True)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return

    import torch
    from paper_2607_05504_b300 import sidm

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    w, masks = _workload(seed_offset=rank)
    p, bins = w["particles"], w["bins"]
    n = p.n
    dev = torch.device("cuda", local)
    # a non-default stream shared by torch and the library: the events that
    # time the steps are recorded on the stream the library launches on
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    masks_d = torch.from_numpy(masks).to(dev)
    bins_d = torch.from_numpy(bins).to(dev)
    pos_d = torch.from_numpy(p.pos).to(dev)
    vel_d = torch.from_numpy(p.vel).to(dev)
    ids_d = torch.from_numpy(p.ids.view(np.int32)).to(dev)
    mass_d = torch.from_numpy(p.mass).to(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > 126 MB L2

    ctx = sidm.Context(n_ngb=64, box=0.0, stream=stream.cuda_stream, device=local, n_max=n,
                       use_graph=True)
    ctx.set_particles(pos_d, vel_d, ids_d, mass=mass_d)
    sg = sidm.SigmaModel(sidm.SIGMA_CONST, 1.0, 1.0)

    # active counts per cycle step, taken before any timed region: host
    # bookkeeping inside the loop could let the device wait for the host
    n_active = [int(m.sum()) for m in masks]

    def step(k):
        s = k % CYCLE
        sidm.sidm_step(ctx.handle, masks_d[s], bins_d, w["dt_max"], sg, 0, None)
        return n_active[s]

    for k in range(args.warmup):
        step(k)
    # launch shapes: timed on the first timed step's active set (the state is restored)
    s_tune = args.warmup % CYCLE
    tuning = ctx.autotune([sidm.HaloParams(w["dt_max"], sg, 0, ctx.step_counter)],
                          masks_d[s_tune], bins_d, reps=3)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    upd = 0
    l0 = ctx.kernel_launches
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        # an NVTX range marks the timed steps (a profiler can keep to them)
        torch.cuda.nvtx.range_push("timed")
        for k in range(args.steps):
            flush.zero_()                       # L2 flush between timed steps (untimed)
            ev[k][0].record(stream)
            upd += step(args.warmup + k)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    launches = ctx.kernel_launches - l0
    ctx_graph_state = ctx.graph_state
    # the whole 100-step cycle, step 0 (every particle active) included
    cev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(CYCLE)]
    torch.cuda.synchronize()
    for s in range(CYCLE):
        flush.zero_()
        cev[s][0].record(stream)
        step(s)
        cev[s][1].record(stream)
    torch.cuda.synchronize()
    cyc_ms = [a.elapsed_time(b) for a, b in cev]
    full_cycle = {"value": sum(n_active) / (sum(cyc_ms) * 1e-3), "unit": UNIT,
                  "ms_per_step": sum(cyc_ms) / CYCLE, "step0_ms": cyc_ms[0],
                  "step0_active": n_active[0],
                  "note": "finest steps 0..99 of the bin cycle, the same context and shapes, "
                          "L2 flushed between steps"}
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_ms = sum(step_ms)
    srt = sorted(range(len(step_ms)), key=lambda i: step_ms[i])
    step_dist = {"median": step_ms[srt[len(srt) // 2]], "max": step_ms[srt[-1]],
                 "slowest": [[(args.warmup + i) % CYCLE, round(step_ms[i], 3)] for i in srt[-3:]],
                 "note": "finest step index in the cycle: the all-active step 0 is the slowest"}
    if dist:
        t_all, upd_all = reduce_over_ranks(t_ms, upd, dev)
        dist.barrier()
    else:
        t_all, upd_all = t_ms, float(upd)
    value = upd_all / (t_all * 1e-3)

    # ---- the same steps with the tree kept between full rebuilds (every 8 steps);
    # positions do not move in this workload, so the kept order stays ideal
    reuse = None
    if args.reuse_every > 1:
        rctx = sidm.Context(n_ngb=64, box=0.0, stream=stream.cuda_stream, device=local, n_max=n,
                            use_graph=True, rebuild_every=args.reuse_every)
        rctx.set_particles(pos_d, vel_d, ids_d, mass=mass_d)
        rctx.set_tuning(**tuning)
        for k in range(args.warmup):
            sidm.sidm_step(rctx.handle, masks_d[k % CYCLE], bins_d, w["dt_max"], sg, 0, None)
        rev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.zero_()
            rev[k][0].record(stream)
            sidm.sidm_step(rctx.handle, masks_d[(args.warmup + k) % CYCLE], bins_d, w["dt_max"],
                           sg, 0, None)
            rev[k][1].record(stream)
        torch.cuda.synchronize()
        rctx.close()
        r_ms = sum(a.elapsed_time(b) for a, b in rev)
        reuse = {"rebuild_every": args.reuse_every, "value": upd / (r_ms * 1e-3),
                 "ms_per_step": r_ms / args.steps,
                 "note": "key order kept between full rebuilds, boxes refitted; positions fixed "
                         "in this workload"}

    # ---- the opt-in search hint (each search starts from the particle's last
    # h): the same steps, and steps with the positions drifted between them
    hint = None
    if args.reuse_every > 1:
        # a gravity-like step between SIDM calls: 1e-3 of the halo's
        # dynamical time (G = M = a = 1), a few per cent of the central h
        # at the central speeds
        dt_f = 1e-3

        def timed_steps(search_hint, drift):
            hctx = sidm.Context(n_ngb=64, box=0.0, stream=stream.cuda_stream, device=local,
                                n_max=n, use_graph=True, search_hint=search_hint)
            hpos = pos_d.clone()
            hctx.set_particles(hpos, vel_d, ids_d, mass=mass_d)
            hctx.set_tuning(**tuning)
            hev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.steps)]
            for k in range(args.warmup + args.steps):
                if drift and k > 0:
                    # drift x += v dt_f before each step (harness work, untimed)
                    hpos.add_(vel_d, alpha=dt_f)
                    hctx.set_positions(hpos)
                flush.zero_()
                t = k - args.warmup
                if t >= 0:
                    hev[t][0].record(stream)
                sidm.sidm_step(hctx.handle, masks_d[k % CYCLE], bins_d, w["dt_max"], sg, 0, None)
                if t >= 0:
                    hev[t][1].record(stream)
            torch.cuda.synchronize()
            hctx.close()
            ms = sum(a.elapsed_time(b) for a, b in hev)
            return {"value": upd / (ms * 1e-3), "ms_per_step": ms / args.steps}

        hint = {"static": timed_steps(True, False),
                "drifting": {"plain": timed_steps(False, True), "hint": timed_steps(True, True),
                             "dt": dt_f},
                "note": "search_hint = 1: each search gathers first within 9/8 of the "
                        "particle's last h (results unchanged); 'static' repeats the headline's "
                        "steps, 'drifting' moves every particle by v dt (dt = 1e-3, a "
                        "gravity-like step) before each step, untimed, for the plain form and the "
                        "hinted form. "
                        "The headline is the plain form, which carries no h between steps"}

    # ---- roofline: phase times of the same steps, CUDA events on the library's stream
    pctx = sidm.Context(n_ngb=64, box=0.0, stream=stream.cuda_stream, device=local, n_max=n,
                        profile=True)
    pctx.set_particles(pos_d, vel_d, ids_d, mass=mass_d)
    pctx.set_tuning(**tuning)          # the launch shapes of the timed steps
    phase_sum = {k: 0.0 for k in sidm.PHASES}
    n_act_sum = 0
    reps = min(args.steps, CYCLE)
    for k in range(reps):
        flush.zero_()
        s = (args.warmup + k) % CYCLE
        sidm.sidm_step(pctx.handle, masks_d[s], bins_d, w["dt_max"], sg, 0, None)
        for name, ms in pctx.phase_times().items():
            phase_sum[name] += ms
        n_act_sum += int(masks[s].sum())
    pctx.close()
    hbm_peak, peak_kind = _peaks()
    ph = {k: v / reps for k, v in phase_sum.items()}
    a_mean = n_act_sum / reps
    # the neighbour-search and pair/scatter kernels (the dominant share of
    # the step): 48 B x N + 64 B x A over their summed phase time
    ns_bytes = NEIGHBOUR_SCATTER_BYTES[0] * n + NEIGHBOUR_SCATTER_BYTES[1] * a_mean
    ns_ms = ph["search"] + ph["pairs"]
    achieved = ns_bytes / (ns_ms * 1e-3) / 1e9
    step_bytes = STEP_BYTES[0] * n + STEP_BYTES[1] * a_mean
    step_ms = sum(ph.values())
    build_ms = ph["keys"] + ph["sort"] + ph["structure"]
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": NEIGHBOUR_SCATTER_TRAFFIC,
                "kernel": "search + pairs (search_kernel, pairs_kernel, pairs_walk_kernel, "
                          "pairs_exact_kernel, limits_kernel; the phase time also holds the "
                          "0.018 ms velocity permutation)",
                "traffic_note": "dram__bytes_read.sum + dram__bytes_write.sum per step of "
                                "these kernels, from an ncu capture of this bench's timed steps",
                "algorithmic_bytes": ns_bytes,
                "bytes_model": "48 B x N + 64 B x A (N particles, A active per step)",
                "peak_kind": peak_kind,
                "search_only": {"achieved": ns_bytes / (ph["search"] * 1e-3) / 1e9,
                                "frac": ns_bytes / (ph["search"] * 1e-3) / 1e9 / hbm_peak},
                # the search's binding resource is instruction issue, not HBM
                "search_issue": {"bound": "issue",
                                 "achieved": SEARCH_INST_PER_QUERY * a_mean / (ph["search"] * 1e-3),
                                 "peak": ISSUE_PEAK, "unit": "warp instructions/s",
                                 "frac": SEARCH_INST_PER_QUERY * a_mean / (ph["search"] * 1e-3)
                                 / ISSUE_PEAK,
                                 "note": "ncu warp instructions per query x active queries per "
                                         "step / live search time, against 148 SMs x 4 "
                                         "schedulers x 2032 MHz"},
                "build": {"bytes": BUILD_BYTES_N * n, "ms": build_ms,
                          "achieved": BUILD_BYTES_N * n / (build_ms * 1e-3) / 1e9,
                          "frac": BUILD_BYTES_N * n / (build_ms * 1e-3) / 1e9 / hbm_peak},
                "step": {"bytes": step_bytes, "bytes_model": "308 B x N + 64 B x A",
                         "ms": step_ms, "achieved": step_bytes / (step_ms * 1e-3) / 1e9,
                         "frac": step_bytes / (step_ms * 1e-3) / 1e9 / hbm_peak},
                "phase_ms_per_step": ph,
                "phase_share": {k: v / step_ms for k, v in ph.items()},
                "timing": "CUDA events between phases on the library's stream, the timed steps "
                          "repeated in a profiling context (same launch shapes, L2 flushed)"}

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
        pos_h, vel_h, ids_h, mass_h = pin(p.pos), pin(p.vel), pin(p.ids), pin(p.mass)
        masks_h = [pin(masks[s]) for s in range(CYCLE)]
        bins_h = pin(bins)
        out_v = pin(np.empty((n, 3)))
        # a simulation's use: particles loaded once, then per step the new
        # positions and velocities, the active mask and the bins go in and
        # the velocities come back (graph replay, the tuned launch shapes)
        ectx = sidm.Context(n_ngb=64, box=0.0, device=local, n_max=n, use_graph=True)
        ectx.set_particles(pos_h, vel_h, ids_h, mass=mass_h)
        ectx.set_tuning(**tuning)
        K2 = min(args.steps, 20)
        for k in range(2):
            sidm.sidm_step(ectx.handle, masks_h[1 + k], bins_h, w["dt_max"], sg, 0, None)
        sidm.sidm_get_particles(ectx.handle, out_v)
        # (a) the result read back whole
        eu, t0 = 0, time.perf_counter()
        for k in range(K2):
            s = (args.warmup + k) % CYCLE
            sidm.sidm_set_positions(ectx.handle, pos_h)
            sidm.sidm_set_velocities(ectx.handle, vel_h)
            sidm.sidm_step(ectx.handle, masks_h[s], bins_h, w["dt_max"], sg, 0, None)
            sidm.sidm_get_particles(ectx.handle, out_v)   # waits for the step
            eu += n_active[s]
        et_full = time.perf_counter() - t0
        # (b) the host holds the simulation's velocities in one pinned array:
        # they go in each step, and the kicks write every velocity they change
        # straight back into it (sidm_set_velocity_mirror); the step's result
        # is on the host once the stream is done
        def host_loop(host_v, readback):
            eu_, t0_ = 0, time.perf_counter()
            for k in range(K2):
                s = (args.warmup + k) % CYCLE
                sidm.sidm_set_positions(ectx.handle, pos_h)
                sidm.sidm_set_velocities(ectx.handle, host_v)
                sidm.sidm_step(ectx.handle, masks_h[s], bins_h, w["dt_max"], sg, 0, None)
                readback(host_v)                                 # waits for the step
                eu_ += n_active[s]
            return eu_, time.perf_counter() - t0_

        step0 = ectx.step_counter
        host_v = pin(vel_h.copy())
        ectx.set_velocity_mirror(host_v)
        for k in range(2):                                     # warm-up, untimed
            sidm.sidm_step(ectx.handle, masks_h[1 + k], bins_h, w["dt_max"], sg, 0, None)
        sidm.sidm_sync(ectx.handle)
        ectx.step_counter = step0
        host_v[:] = vel_h
        eu2, et = host_loop(host_v, lambda hv: sidm.sidm_sync(ectx.handle))
        ectx.set_velocity_mirror(None)
        # (c) the same through sidm_update_velocities after each step (the
        # changed particles written by one kernel after the step)
        host_u = pin(vel_h.copy())
        for k in range(2):                                     # warm-up, untimed
            sidm.sidm_step(ectx.handle, masks_h[1 + k], bins_h, w["dt_max"], sg, 0, None)
            sidm.sidm_update_velocities(ectx.handle, host_u)
        ectx.step_counter = step0
        host_u[:] = vel_h
        eu3, et3 = host_loop(host_u, lambda hv: sidm.sidm_update_velocities(ectx.handle, hv))
        # the same steps again, untimed, from the same step counter: the
        # particles that crossed the bus, and the host array they give
        ectx.step_counter = step0
        host_c = vel_h.copy()
        idx_h = np.empty(n, np.int32)
        chg_h = np.empty((n, 3))
        nchg = 0
        for k in range(K2):
            s = (args.warmup + k) % CYCLE
            sidm.sidm_set_positions(ectx.handle, pos_h)
            sidm.sidm_set_velocities(ectx.handle, host_c)
            sidm.sidm_step(ectx.handle, masks_h[s], bins_h, w["dt_max"], sg, 0, None)
            m = sidm.sidm_get_changed(ectx.handle, idx_h, chg_h)
            host_c[idx_h[:m]] = chg_h[:m]
            nchg += m
        ectx.close()
        e2e = {"value": eu2 / et, "unit": UNIT,
               "h2d_bytes_per_step": int(n * (24 + 24) + n + n),
               "d2h_bytes_per_step": int(4 + 24 * nchg / K2),
               "readback": "sidm_set_velocity_mirror: the kicks write the final velocity of "
                           "every particle the step changes into the host's pinned velocity "
                           "array, which is uploaded from and kept current in place",
               "replay_identical": bool(np.array_equal(host_c, host_v) and
                                        np.array_equal(host_c, host_u)),
               "update_velocities": {"value": eu3 / et3,
                                     "readback": "sidm_update_velocities after each step: one "
                                                 "kernel writes the changed particles into the "
                                                 "pinned array"},
               "full_readback": {"value": eu / et_full, "d2h_bytes_per_step": int(4 + n * 24),
                                 "readback": "all velocities (sidm_get_particles)"}}

    cb = None
    if rank == 0 and not args.no_cpu_baseline:
        cb = cpu_baseline(w, masks)

    ctx.close()
    del flush
    torch.cuda.empty_cache()

    # ---- the other configurations, each bounded in time (N = 1 only)
    extras = {}
    if rank == 0 and world == 1 and not args.no_extras:
        def guarded(name, fn):
            t0 = time.perf_counter()
            try:
                d = fn()
            except Exception as e:            # reported in the line, never hidden
                d = {"error": f"{type(e).__name__}: {e}"}
            d["wall_s"] = round(time.perf_counter() - t0, 1)
            extras[name] = d
            torch.cuda.synchronize()
            torch.cuda.empty_cache()

        guarded("c2_eq18_bins", lambda: eq18_run(w, tuning, args.steps, args.warmup, local))
        guarded("c3_precision", lambda: precision_run(23, 10))
        guarded("c4_batch", lambda: batch_run(512, 10, 3, workers=workers))
        guarded("c5_serving", lambda: serving_run(32, 21.0, 1000, 120.0))
    vs_plain = None
    if extras:
        vs_plain = {"c3_split_over_fp64": extras["c3_precision"].get("speedup_split_vs_fp64"),
                    "c4_batch_over_per_halo": extras["c4_batch"].get("speedup_vs_plain"),
                    "c5_saturation_over_c2": (extras["c5_serving"].get("value", 0.0) / value
                                              if "value" in extras["c5_serving"] else None)}
    if hint:
        if vs_plain is None:
            vs_plain = {}
        vs_plain["search_hint_over_plain_drifting"] = (hint["drifting"]["hint"]["value"] /
                                                      hint["drifting"]["plain"]["value"])
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": t_all / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "hernquist-2^20 (N_ngb 64, sigma/m 1, open, ~10% active "
                                       "per finest step, 100-step bin cycle)",
                           "n": n, "mean_active": upd / args.steps,
                           "parallelism": f"replicas{world}" if world > 1 else "single",
                           "l2": "flushed between timed steps (256 MB write)",
                           "bins": "8 power-of-two levels from a local collision-time estimate, "
                                   "clipped at the finest: ~800 pairs per step reach P >= 1 in "
                                   "the centre (a stress case for the kick ordering; "
                                   "c2_eq18_bins has every particle below its Eq. 18 limit)"},
                "roofline": roofline, "cpu_baseline": cb, "e2e": e2e,
                "gpu_launches": launches, "clocks": clk.summary(),
                "launch": {"graph": ctx_graph_state, "tuning": tuning}, "step_ms": step_dist,
                "tree_reuse": reuse, "search_hint": hint, "full_cycle": full_cycle,
                "vs_plain_form": vs_plain,
                **extras}
        print(json.dumps(line), flush=True)
    if dist:
        import torch.distributed as D
        D.destroy_process_group()


if __name__ == "__main__":
    main()
