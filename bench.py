"""Benchmark of the SIDM scattering step on one B300 (or N independent replicas).

Workload: isolated Hernquist halo, N = 2^20, N_ngb = 64 +- 5, constant
sigma/m = 1, open boundaries, FP64, power-of-two timestep bins with ~10 % of
the particles active per finest step (step s of a 100-step cycle uses the
active set of finest step s).  One bench step = one complete scattering step
(keys, sort, structure, h_SI search, pairs + draws + Eq. 18, kicks) on the
step's active set.  Metric: particle updates (active particles) per second.

    python bench.py [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs its own halo replica on its own GPU
(independent problems, no data-path collective): value = all ranks'
updates / the slowest rank's time ("scaling": "weak").
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SIDM particle-updates/s (search+scatter)"
UNIT = "particle-updates/s"
CYCLE = 100

# Algorithmic HBM bytes of each phase, per particle (n) and per active
# particle (a): the data the phase must read and write once (FP64 state,
# 4-byte ids/indices, 1-byte flags).
PHASE_BYTES = {
    "keys": (56.0, 0.0),        # bbox read 24, keys read 24, key+index write 8
    "sort": (68.0, 0.0),        # one histogram read 4 + 4 passes x (read 8 + write 8)
    "structure": (190.0, 0.0),  # gather 66 read, key-order state 97 written, leaf boxes ~27
    "search": (16.0, 56.0),     # FP32 positions once; own state 40 read, h 16 written
    "pairs": (0.0, 92.0),       # own state 84 read, Eq. 18 limit 8 written
    "resolve": (0.0, 0.0),      # per accepted pair, reported separately
}


SEARCH_DRAM_BYTES = 6.573568e6 + 1.042432e6   # dram read + write of the captured launch
SEARCH_DRAM_QUERIES = 51520


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
        self.path = os.path.join(ROOT, "gpurun_out" if os.path.isdir(os.path.join(ROOT, "gpurun_out")) else ".",
                                 f".clocks_{os.getpid()}.csv")

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
    cores = os.cpu_count()
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": "hernquist-2^20 (N_ngb 64, sigma/m 1, ~10% active, 100-step bin cycle)",
                       "l2": "host run"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"full oracle step per bench step, active set capped at {cap} "
                                       "(seeded subset) of the step's active particles"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(w, masks, budget_s=12.0) -> dict:
    import oracle
    oracle.build()
    p, bins = w["particles"], w["bins"]
    upd, t0, k = 0, time.perf_counter(), 0
    vel = p.vel.copy()
    while k < CYCLE - 1 and (time.perf_counter() - t0) < budget_s:
        s = 1 + k
        r = oracle.step(p.pos, vel, p.mass, p.ids, masks[s], bins, w["dt_max"], n_ngb=64, seed=0, step=s)
        vel = r["vel"]
        upd += int(masks[s].sum())
        k += 1
    dt = time.perf_counter() - t0
    return {"value": upd / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"finest steps 1..{k} of the 100-step cycle ({upd} active updates, {dt:.1f} s)"}


def run_batch(args) -> None:
    """512 independent Hernquist haloes (N log-uniform in [2^12, 2^18], sigma/m
    log-uniform in [0.1, 10], own seeds, bins and step counters) stepped
    together (one sidm_step_haloes per step), against the plain per-halo form
    (one sidm_step per halo) on the same haloes and steps."""
    import torch
    from paper_2607_05504_b300 import inputs as I
    from paper_2607_05504_b300 import sidm
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    haloes = I.hernquist_batch(args.n_halos)
    p, off, bins = I.pack(haloes)
    n = p.n
    bmax = [int(h["bins"].max()) for h in haloes]

    def masks_for(s):
        return np.concatenate([I.active_at_step(h["bins"], s) for h in haloes])

    steps = args.steps
    cyc = [masks_for(s) for s in range(args.warmup + steps)]
    ctx = sidm.Context(n_ngb=64, box=0.0, stream=stream.cuda_stream, n_max=n, use_graph=True)
    ctx.set_particles(torch.from_numpy(p.pos).to(dev), torch.from_numpy(p.vel).to(dev),
                      torch.from_numpy(p.ids.view(np.int32)).to(dev),
                      mass=torch.from_numpy(p.mass).to(dev))
    ctx.set_haloes(off)
    bins_d = torch.from_numpy(bins).to(dev)
    masks_d = [torch.from_numpy(m).to(dev) for m in cyc]

    def params(s):
        return [sidm.HaloParams(h["dt_max"], sidm.SigmaModel(0, h["sigma0"], 1.0), h["seed"], s)
                for h in haloes]

    prm = [params(s) for s in range(args.warmup + steps)]
    for s in range(args.warmup):
        sidm.sidm_step_haloes(ctx.handle, masks_d[s], bins_d, prm[s], None)
    tuning = ctx.autotune(prm[args.warmup], masks_d[args.warmup], bins_d, reps=1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    upd = 0
    n_active = [int(cyc[args.warmup + k].sum()) for k in range(steps)]   # host bookkeeping, untimed
    e0.record(stream)
    for k in range(steps):
        s = args.warmup + k
        sidm.sidm_step_haloes(ctx.handle, masks_d[s], bins_d, prm[s], None)
    e1.record(stream)
    upd = sum(n_active)
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) * 1e-3
    graph_state = ctx.graph_state
    ctx.close()
    # plain per-halo form: one context, each halo loaded then stepped alone
    pc = sidm.Context(n_ngb=64, box=0.0, stream=stream.cuda_stream, n_max=int(np.diff(off).max()))
    dev_h = [(torch.from_numpy(h["particles"].pos).to(dev), torch.from_numpy(h["particles"].vel).to(dev),
              torch.from_numpy(h["particles"].ids.view(np.int32)).to(dev),
              torch.from_numpy(h["particles"].mass).to(dev), torch.from_numpy(h["bins"]).to(dev))
             for h in haloes]
    t_plain, upd_plain = 0.0, 0
    for k in range(min(steps, 3)):
        s = args.warmup + k
        for j, h in enumerate(haloes):
            pos, vel, ids, mass, hb = dev_h[j]
            pc.set_particles(pos, vel, ids, mass=mass)
            mk = torch.from_numpy(I.active_at_step(h["bins"], s)).to(dev)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pc.step_counter = s
            sidm.sidm_step(pc.handle, mk, hb, h["dt_max"], sidm.SigmaModel(0, h["sigma0"], 1.0),
                           h["seed"], None)
            b.record(stream)
            b.synchronize()
            t_plain += a.elapsed_time(b) * 1e-3
            upd_plain += int(mk.sum().item())
    pc.close()
    line = {"metric": METRIC, "value": upd / t_batch, "unit": UNIT, "n_gpus": 1, "steps": steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_batch / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"batch of {args.n_halos} Hernquist haloes, N log-uniform in "
                                   "[2^12, 2^18], sigma/m log-uniform in [0.1, 10], N_ngb 64",
                       "n": n, "n_halos": args.n_halos, "mean_active": upd / steps},
            "launch": {"graph": graph_state, "tuning": tuning,
                       "form": "one multi-halo step per tick (sidm_step_haloes)"},
            "plain_per_halo": {"value": upd_plain / t_plain, "unit": UNIT,
                               "steps": min(steps, 3),
                               "note": "same haloes, one sidm_step per halo (kernel time only)"}}
    print(json.dumps(line), flush=True)


def run_precision(args) -> None:
    """NFW halo (c = 10, r_s = 1, N = 2^23), Yukawa-like sigma0/m = 1 with w =
    v_c(r_s), N_ngb 64, power-of-two bins: the FP32-split form against the
    FP64 plain form, step by step from the same state.  Reports both forms'
    throughput, the accepted-pair mismatch |A32 xor A64| / |A64| and the
    split form's relative energy / momentum change per step."""
    import torch
    from paper_2607_05504_b300 import inputs as I
    from paper_2607_05504_b300 import sidm
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    p = I.nfw_halo(1 << args.log2_n, 2)
    w = p.meta["v_c_rs"]
    bins, dt = I.timestep_bins(p, I.nfw_density, 1.0, 64)
    ctxs = {k: sidm.Context(n_ngb=64, stream=stream.cuda_stream, n_max=p.n, precision=v)
            for k, v in (("fp64", sidm.FP64_PLAIN), ("split", sidm.FP32_SPLIT))}
    pos, vel = torch.from_numpy(p.pos).to(dev), torch.from_numpy(p.vel).to(dev)
    ids, mass = torch.from_numpy(p.ids.view(np.int32)).to(dev), torch.from_numpy(p.mass).to(dev)
    for c in ctxs.values():
        c.set_particles(pos, vel, ids, mass=mass)
    bins_d = torch.from_numpy(bins).to(dev)
    sg = sidm.SigmaModel(sidm.SIGMA_YUKAWA, 1.0, w)
    t = {"fp64": 0.0, "split": 0.0}
    n64 = nx = upd = 0
    drift_e, drift_p = 0.0, 0.0
    vcur = torch.empty_like(vel)
    for s in range(args.steps):
        act = torch.from_numpy(I.active_at_step(bins, s)).to(dev)
        res = {}
        for k, c in ctxs.items():
            c.step_counter = s
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            sidm.sidm_step(c.handle, act, bins_d, dt, sg, 7, None)
            b.record(stream)
            b.synchronize()
            t[k] += a.elapsed_time(b) * 1e-3
            st = sidm.StepStats()
            res[k] = set(map(tuple, c.pairs()[0].tolist()))
        upd += int(act.sum().item())
        n64 += len(res["fp64"])
        nx += len(res["fp64"] ^ res["split"])
        # conservation of the split step: recompute with statistics
        sidm.sidm_get_particles(ctxs["fp64"].handle, vcur)
        c = ctxs["split"]
        c.set_velocities(vcur)
        c.step_counter = s
        st = c.step(dt, act, bins_d, sigma0=1.0, sigma_kind=sidm.SIGMA_YUKAWA, w=w, seed=7)
        drift_e = max(drift_e, abs(st["e_after"] - st["e_before"]) / st["e_before"])
        pscale = float((mass[:, None] * vcur.abs()).sum().item())
        drift_p = max(drift_p, float(np.max(np.abs(np.subtract(st["p_after"], st["p_before"])))) / pscale)
        c.set_velocities(vcur)
    for c in ctxs.values():
        c.close()
    line = {"metric": METRIC, "value": upd / t["split"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": 0, "ms_per_step": 1e3 * t["split"] / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64",
            "data": "synthetic",
            "config": {"workload": f"NFW c=10 N=2^{args.log2_n}, Yukawa sigma0/m=1 w=v_c(r_s), "
                                   "N_ngb 64, FP32-split vs FP64 plain", "n": p.n},
            "fp64_plain": {"value": upd / t["fp64"], "unit": UNIT},
            "pair_mismatch": {"rate": nx / max(n64, 1), "pairs_fp64": n64, "differing": nx},
            "drift_per_step": {"energy_rel": drift_e, "momentum_rel": drift_p}}
    print(json.dumps(line), flush=True)


def run_serving(args) -> None:
    """Poisson streams of halo requests served with continuous batching under
    a device-memory budget.  First the saturated throughput (every request
    present at t = 0), which gives the capacity in requests/s; then Poisson
    arrivals at fractions of that capacity, each with p50/p99 latency.  A rate
    is stable when the last third of the requests waits no longer than 1.5x
    the first third (no backlog builds up)."""
    import dataclasses
    import torch
    from paper_2607_05504_b300 import inputs as I
    from paper_2607_05504_b300 import serving as S
    torch.cuda.set_device(0)
    base = S.request_stream(args.requests, rate=1.0, seed=3, log2_n=(12.0, args.log2_nmax),
                            steps=(10, args.max_steps))
    unit_arrivals = [r.arrival for r in base]
    budget = args.budget_gb * 1e9
    per_particle = 700.0

    def serve(rate):
        reqs = [dataclasses.replace(r, arrival=(0.0 if rate is None else a / rate), steps_done=0,
                                    admitted=None, finished=None, result_vel=None)
                for r, a in zip(base, unit_arrivals)]
        eng = S.GpuEngine(capacity=int(budget / per_particle))
        rep = S.Server(eng, S.Scheduler(budget, per_particle)).run(reqs)
        eng.close()
        lat = [r.latency for r in sorted(reqs, key=lambda r: r.arrival)]
        third = max(len(lat) // 3, 1)
        growth = float(np.mean(lat[-third:]) / max(np.mean(lat[:third]), 1e-9))
        return rep, growth

    sat, _ = serve(None)
    work = sat.updates / len(base)               # active-particle updates per request
    cap_rate = sat.throughput / work             # requests/s the device sustains
    sweep = []
    for frac in (0.25, 0.5, 0.75, 0.9):
        rate = frac * cap_rate
        rep, growth = serve(rate)
        sweep.append({"rate_per_s": rate, "load": frac, "throughput": rep.throughput,
                      "p50_s": rep.percentile(50), "p99_s": rep.percentile(99),
                      "backlog_growth": growth, "stable": growth <= 1.5})
    stable = [x for x in sweep if x["stable"]]
    op = stable[-1] if stable else sweep[0]
    line = {"metric": METRIC, "value": sat.throughput, "unit": UNIT, "n_gpus": 1,
            "steps": sat.ticks, "warmup": 0, "ms_per_step": 1e3 * sat.wall / max(sat.ticks, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "serving: halo requests (Hernquist/NFW, const/Yukawa sigma), "
                                   f"N log-uniform in [2^12, 2^{args.log2_nmax:g}], steps "
                                   f"log-uniform in [10, {args.max_steps}]",
                       "requests": args.requests, "hbm_budget_gb": args.budget_gb},
            "saturation": {"throughput": sat.throughput, "requests_per_s": cap_rate,
                           "p50_s": sat.percentile(50), "p99_s": sat.percentile(99),
                           "wall_s": sat.wall},
            "stable_rate_per_s": op["rate_per_s"] if stable else None,
            "latency_s": {"rate_per_s": op["rate_per_s"], "p50": op["p50_s"], "p99": op["p99_s"]},
            "sweep": sweep}
    print(json.dumps(line), flush=True)


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
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "ours" and args.workload == "batch":
        return run_batch(args)
    if args.impl == "ours" and args.workload == "serving":
        return run_serving(args)
    if args.impl == "ours" and args.workload == "precision":
        return run_precision(args)

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
    dom = max(phase_sum, key=phase_sum.get)
    per_n, per_a = PHASE_BYTES[dom]
    bytes_per_step = per_n * n + per_a * (n_act_sum / reps)
    avg_ms = phase_sum[dom] / reps
    achieved = bytes_per_step / (avg_ms * 1e-3) / 1e9
    # DRAM bytes of the search kernel from one ncu capture of the current
    # kernel (7.57 MB on a launch of 51,520 queries of this workload),
    # scaled to this run's mean queries per step
    traffic = (SEARCH_DRAM_BYTES * (n_act_sum / reps) / SEARCH_DRAM_QUERIES
               if dom == "search" else None)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": traffic,
                "traffic_note": "bytes per launch, scaled by queries from a 51,520-query capture",
                "kernel": dom,
                "peak_kind": peak_kind,
                "phase_ms_per_step": {k: v / reps for k, v in phase_sum.items()},
                "phase_share": {k: v / sum(phase_sum.values()) for k, v in phase_sum.items()}}

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
        # (b) only the particles the step changed come back; the host applies
        # them to its own copy of the velocities (inside the timed region)
        host_v = vel_h.copy()
        sidm.sidm_update_velocities(ectx.handle, host_v)   # allocates its pinned staging once
        eu2, nchg, t0 = 0, 0, time.perf_counter()
        for k in range(K2):
            s = (args.warmup + k) % CYCLE
            sidm.sidm_set_positions(ectx.handle, pos_h)
            sidm.sidm_set_velocities(ectx.handle, vel_h)
            sidm.sidm_step(ectx.handle, masks_h[s], bins_h, w["dt_max"], sg, 0, None)
            sidm.sidm_update_velocities(ectx.handle, host_v)   # waits for the step
            eu2 += n_active[s]
        et = time.perf_counter() - t0
        # bytes of the changed-only read-back: the same steps again, untimed
        idx_h = np.empty(n, np.int32)
        chg_h = np.empty((n, 3))
        nchg = 0
        for k in range(K2):
            s = (args.warmup + k) % CYCLE
            sidm.sidm_step(ectx.handle, masks_h[s], bins_h, w["dt_max"], sg, 0, None)
            nchg += sidm.sidm_get_changed(ectx.handle, idx_h, chg_h)
        ectx.close()
        e2e = {"value": eu / et_full, "unit": UNIT,
               "h2d_bytes_per_step": int(n * (24 + 24) + n + n),
               "d2h_bytes_per_step": int(n * 24),
               "readback": "all velocities (sidm_get_particles)",
               "changed_readback": {"value": eu2 / et, "d2h_bytes_per_step": int(8 + 28 * nchg / K2),
                                    "note": "sidm_update_velocities: only the particles the step "
                                            "changed cross the bus and are written into a host "
                                            "copy of the velocities"}}

    cb = None
    if rank == 0 and not args.no_cpu_baseline:
        cb = cpu_baseline(w, masks)

    ctx.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": t_all / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "hernquist-2^20 (N_ngb 64, sigma/m 1, open, ~10% active "
                                       "per finest step, 100-step bin cycle)",
                           "n": n, "mean_active": upd / args.steps,
                           "parallelism": f"replicas{world}" if world > 1 else "single",
                           "l2": "flushed between timed steps (256 MB write)"},
                "roofline": roofline, "cpu_baseline": cb, "e2e": e2e,
                "gpu_launches": launches, "clocks": clk.summary(),
                "launch": {"graph": ctx_graph_state, "tuning": tuning}, "step_ms": step_dist,
                "tree_reuse": reuse}
        print(json.dumps(line), flush=True)
    if dist:
        import torch.distributed as D
        D.destroy_process_group()


if __name__ == "__main__":
    main()
