"""Benchmark: checkerboard Metropolis sweeps of the 2D Ising model on GB300.

Workload (one step): `--sweeps` checkerboard sweeps of each of three 2D
Ising spin-1/2 lattices, L = 4096 periodic, J = 1, h = 0, T in
{2.0, 2.269185, 3.0}, random +-1 start (seed 7), int8 spins, advanced
through the C ABI of liblattice.so.  One spin update = one site visited in
one sweep.

Prints ONE JSON line (rank 0):
  value      spin updates per ns over all GPUs, inputs resident in HBM
  roofline   the dominant kernel (one-launch tiled sweep) against measured
             HBM bandwidth, with algorithmic bytes = 2 B per site per sweep
             (one int8 read + one int8 write), plus its issue-rate roofline
  e2e        same metric through the C ABI with pinned host buffers: upload
             of the three lattices, the sweeps, and the read-back of the
             per-sweep E/M counters inside the timed region
  cpu_baseline  the CPU oracle (single thread) on a bounded sample
`--impl reference` times the CPU oracle instead (the reference arm).
Multi-GPU (torchrun): independent replicas, one per GPU (weak scaling).
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

L = 4096
TEMPS = (2.0, 2.269185, 3.0)
SEED = 7
WORKLOAD = ("2D Ising spin-1/2, L=4096 periodic, J=1, h=0, T in {2.0, 2.269185, 3.0}, "
            "random +-1 start (seed 7), int8 and bit-packed spin layouts")
LAYOUTS = ("int8", "bitpacked")
METRIC = "spin updates/ns"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


def max_over_ranks(x: float, device=None) -> float:
    """Max of a per-rank float over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(updates_per_rank: float, world: int, max_seconds: float) -> float:
    """Whole-job updates per ns of `world` independent replicas (weak scaling)."""
    return world * updates_per_rank / (max_seconds * 1e9)


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons in the background."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in getattr(self, "out", "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_oracle_sample(seconds_target=12.0, max_sweeps_per_T=3):
    """Time the CPU oracle (as it stands, single thread) on L=4096 sweeps."""
    import oracle
    done = 0
    t_total = 0.0
    n_T = 0
    for T in TEMPS:
        lat = oracle.Lattice(2, L, 1, oracle.ISING, 1.0, 0.0, T, seed=SEED, init=oracle.INIT_RANDOM)
        n_T += 1
        for _ in range(max_sweeps_per_T):
            t0 = time.perf_counter()
            lat.sweep(1)
            t_total += time.perf_counter() - t0
            done += 1
            if t_total > seconds_target:
                break
        if t_total > seconds_target:
            break
    ups = done * L * L / t_total / 1e9
    return {"value": ups, "unit": "updates/ns", "cores": 1, "kind": "oracle",
            "sample": "%d single-threaded oracle sweeps of L=4096 lattices over %d temperature(s), "
                      "%.1f s (init excluded)" % (done, n_T, t_total)}


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    import oracle
    oracle.build()
    # each step: one oracle sweep of each of the three lattices (a bounded
    # sample of the same workload; the full sweep count would take hours).
    lats = [oracle.Lattice(2, L, 1, oracle.ISING, 1.0, 0.0, T, seed=SEED, init=oracle.INIT_RANDOM)
            for T in TEMPS]
    for _ in range(args.warmup):
        for lat in lats:
            lat.sweep(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for lat in lats:
            lat.sweep(1)
    dt = time.perf_counter() - t0
    ups = args.steps * len(TEMPS) * L * L / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": ups, "unit": "updates/ns",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int8", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sweeps_per_step": 1, "lattices": len(TEMPS)},
            "cpu_baseline": {"value": ups, "unit": "updates/ns", "cores": 1, "kind": "oracle",
                             "sample": "%d steps x 3 lattices x 1 sweep, single-threaded CPU oracle"
                                       % args.steps},
            "e2e": {"value": ups, "unit": "updates/ns", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_gpu(args):
    import torch
    import paper_1209_0296_gb300 as lt

    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    S = args.sweeps

    lats = {lay: [lt.Lattice(2, L, 1, lt.ISING, 1.0, 0.0, T, seed=SEED, init=lt.INIT_RANDOM,
                             layout=lt.INT8 if lay == "int8" else lt.BITPACKED, stream=stream)
                  for T in TEMPS] for lay in LAYOUTS}
    int8_kernel = {"auto": lt.KERNEL_AUTO, "wide": lt.KERNEL_WIDE, "tiled": lt.KERNEL_TILED}[args.int8_kernel]
    for g in lats["int8"]:
        g.set_kernel(int8_kernel, 0, args.tile_h, args.graph)
    all_lats = lats["int8"] + lats["bitpacked"]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # 256 MiB > 129 MB L2

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.fill_(1)
            for g in all_lats:
                g.sweep(S)
        stream.synchronize()
        barrier()
        # events: [start, after the int8 lattices, after the bit-packed lattices] per step
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
        with Clocks(local) as clk:
            for k in range(args.steps):
                flush.fill_(k & 255)          # evict the lattices from L2 (outside the timed pair)
                ev[k][0].record(stream)
                for g in lats["int8"]:
                    g.sweep(S)
                ev[k][1].record(stream)
                for g in lats["bitpacked"]:
                    g.sweep(S)
                ev[k][2].record(stream)
            stream.synchronize()
        barrier()
    ms_int8 = sum(e[0].elapsed_time(e[1]) for e in ev)
    ms_bits = sum(e[1].elapsed_time(e[2]) for e in ev)
    total_ms = max_over_ranks(ms_int8 + ms_bits, dev)
    n_lat = len(all_lats)
    updates = world * args.steps * n_lat * S * L * L
    value = replica_value(args.steps * n_lat * S * L * L, world, total_ms * 1e-3)

    # Kernel launches per step: per int8 lattice, S sweeps (one launch each
    # for the tiled kernel, two for the wide one); per bit-packed lattice two
    # launches per sweep; plus one counter-advance kernel per graph replay
    # and per direct remainder.
    kinfo = lats["int8"][0].get_kernel()
    gk = kinfo["sweeps_per_graph"]
    gkb = lats["bitpacked"][0].get_kernel()["sweeps_per_graph"]
    per_sweep = 1 if kinfo["kernel"] == lt.KERNEL_TILED else 2
    adv = lambda g_: S // g_ + (1 if S % g_ else 0)
    launches = args.steps * len(TEMPS) * (per_sweep * S + adv(gk) + 2 * S + adv(gkb))
    sweep_launches = args.steps * len(TEMPS) * (per_sweep + 2) * S
    # average duration of one sweep of one lattice (all its launches, the
    # tiny advance kernels and launch gaps: this under-reports kernel rates)
    avg_kernel_us = ms_int8 * 1e3 / (args.steps * len(TEMPS) * S)
    avg_bits_us = ms_bits * 1e3 / (args.steps * len(TEMPS) * S)
    hbm, _, peak_kind = peaks()
    alg_bytes = 2.0 * L * L  # one int8 read + one int8 write per site per sweep
    achieved = alg_bytes / (avg_kernel_us * 1e-6) / 1e9
    kname = {lt.KERNEL_TILED: "tiled", lt.KERNEL_WIDE: "wide", lt.KERNEL_GENERIC: "generic"}.get(
        kinfo["kernel"], "?")
    prof = load_profile_numbers(kname)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": prof.get("traffic_bytes_per_sweep"),
                "kernel": "k_sweep_tiled<Ising>" if kname == "tiled" else "k_wide_pipe<colour 0, colour 1>",
                "peak_kind": peak_kind + " (copy bandwidth)",
                "bytes_per_sweep": alg_bytes,
                "avg_sweep_us": avg_kernel_us}
    bprof = load_profile_numbers("bitpacked")
    bbytes = 0.25 * L * L  # one bit read + one bit written per site per sweep
    bach = bbytes / (avg_bits_us * 1e-6) / 1e9
    roofline_bits = {"bound": "hbm", "achieved": bach, "peak": hbm, "unit": "GB/s", "frac": bach / hbm,
                     "traffic": bprof.get("traffic_bytes_per_sweep"), "kernel": "k_bits_pipe<colour 0, colour 1>",
                     "bytes_per_sweep": bbytes, "avg_sweep_us": avg_bits_us,
                     "updates_per_ns": L * L / (avg_bits_us * 1e3)}
    sm_clk = (clk.summary().get("sm_mhz") or 2070.0) * 1e6
    issue_peak = 152 * 4 * sm_clk   # warp instructions per second: 152 SMs x 4 schedulers x clock

    def issue(pr, us):
        # instruction-issue roofline from the committed ncu count of the same kernel
        if not pr.get("warp_inst_per_sweep"):
            return None
        rate = pr["warp_inst_per_sweep"] / (us * 1e-6)
        return {"bound": "alu", "achieved": rate / 1e12, "peak": issue_peak / 1e12, "unit": "Twarp-inst/s",
                "frac": rate / issue_peak, "inst_per_site": pr["warp_inst_per_sweep"] * 32 / (L * L),
                "peak_kind": "152 SMs x 4 schedulers x 1 warp-instruction per cycle at the sampled SM clock"}

    roofline["issue"] = issue(prof, avg_kernel_us)
    roofline_bits["issue"] = issue(bprof, avg_bits_us)
    if not args.no_other:
        roofline["hbm_sized"] = hbm_sized_run(dev, hbm)

    # ---- end to end through the C ABI with pinned host buffers ----------
    e2e = None
    if not args.no_e2e:
        host_in = [torch.empty(L * L, dtype=torch.int8, pin_memory=True) for _ in all_lats]
        rng = np.random.default_rng(1000 + rank)
        for h in host_in:
            h.numpy()[:] = np.where(rng.random(L * L) < 0.5, 1, -1).astype(np.int8)
        series = {k: np.zeros(S, dtype=np.int64) for k in ("bond", "mag")}

        def e2e_step():
            for g, h in zip(all_lats, host_in):
                g.set_spins_ptr(h.data_ptr())
                g.sweep(S)
                first = g.sweeps() - S
                g.series_into(first, S, series["bond"], series["mag"])

        for _ in range(max(1, args.warmup)):
            e2e_step()
        torch.cuda.synchronize(dev)
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize(dev)
        dt = max_over_ranks(time.perf_counter() - t0, dev)
        e2e = {"value": updates / (dt * 1e9), "unit": "updates/ns",
               "h2d_bytes_per_step": n_lat * L * L,
               "d2h_bytes_per_step": n_lat * S * 2 * 8}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_oracle_sample()
    extra = {}
    if rank == 0 and world == 1 and not args.no_serving:
        extra["batched"] = batched_bench()
        extra["served"] = served_bench()
    if rank == 0 and world == 1 and not args.no_other:
        extra["other_configs"] = other_configs(dev)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "updates/ns", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int8", "data": "synthetic",
                "config": {"workload": WORKLOAD, "lattices": n_lat, "sweeps_per_step": S,
                           "layouts": list(LAYOUTS),
                           "int8_kernel": kname + (" (autotuned)" if args.int8_kernel == "auto" else " (fixed)"),
                           "int8_updates_per_ns": len(TEMPS) * S * L * L * args.steps / (ms_int8 * 1e6),
                           "tile": [256, kinfo["tile_h"]] if kname == "tiled" else None,
                           "sweeps_per_graph": gk, "sweeps_per_graph_tuned": args.graph == 0,
                           "parallelism": "replicas" if world > 1 else "single GPU",
                           "l2": "flushed between steps (256 MiB write outside the timed events)"},
                "hbm_roofline_pct": 100.0 * roofline["frac"],
                "rows": {"int8": {"updates_per_ns": len(TEMPS) * S * L * L * args.steps / (ms_int8 * 1e6),
                                  "hbm_frac": roofline["frac"],
                                  "issue_frac": (roofline["issue"] or {}).get("frac")},
                         "bitpacked": {"updates_per_ns": len(TEMPS) * S * L * L * args.steps / (ms_bits * 1e6),
                                       "hbm_frac": roofline_bits["frac"],
                                       "issue_frac": (roofline_bits["issue"] or {}).get("frac")}},
                "roofline": roofline, "roofline_bitpacked": roofline_bits,
                "gpu_launches": launches, "sweep_launches": sweep_launches,
                "clocks": clk.summary()}
        if e2e is not None:
            line["e2e"] = e2e
        if cpu is not None:
            line["cpu_baseline"] = cpu
        line.update(extra)
        print(json.dumps(line), flush=True)
    for g in all_lats:
        g.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_profile(args):
    """A short, untimed run of the dominant kernel for ncu captures."""
    import torch
    import paper_1209_0296_gb300 as lt
    torch.cuda.set_device(0)
    if args.profile_model == "ne":
        c = 0.42 if args.profile_dynamics != "checkerboard" else 0.3
        g = lt.Lattice(2, args.profile_L, 1, lt.NE, 0.0, 0.0, c, seed=21, init=lt.INIT_EQUILIBRIUM)
    elif args.profile_model == "potts":   # q = 3 Potts at T_c = 1 / ln(1 + sqrt 3), random start (seed 7)
        import math
        g = lt.Lattice(2, args.profile_L, 2, lt.POTTS, 1.0, 0.0, 1.0 / math.log(1.0 + math.sqrt(3.0)), seed=7,
                       init=lt.INIT_RANDOM)
    elif args.profile_model == "rfim":   # random-field Ising, h = J, T = 2, eta from default_rng(6)
        import numpy as np
        g = lt.Lattice(2, args.profile_L, 1, lt.ISING, 1.0, 1.0, 2.0, seed=7, init=lt.INIT_RANDOM)
        g.set_fields(np.where(np.random.default_rng(6).random(args.profile_L ** 2) < 0.5, -1, 1).astype(np.int8))
    elif args.profile_model == "ising3d":   # 3D spin-1 at T = 2 + 7 * 2/15, random start (seed 11)
        g = lt.Lattice(3, args.profile_L, 2, lt.ISING, 1.0, 0.0, 2.0 + 7 * 2.0 / 15, seed=11,
                       init=lt.INIT_RANDOM)
    else:
        g = lt.Lattice(2, args.profile_L, 1, lt.ISING, 1.0, 0.0, TEMPS[0], seed=SEED,
                       init=lt.INIT_RANDOM,
                       layout=lt.BITPACKED if args.profile_layout == "bitpacked" else lt.INT8)
    kern = {"auto": lt.KERNEL_AUTO, "tiled": lt.KERNEL_TILED, "wide": lt.KERNEL_WIDE,
            "generic": lt.KERNEL_GENERIC, "resident": lt.KERNEL_RESIDENT}[args.profile_kernel]
    if args.profile_layout == "bitpacked":
        kern = lt.KERNEL_AUTO
    g.set_kernel(kern, 0, args.tile_h, 1 << 30)  # direct launches, no graphs
    if args.profile_dynamics != "checkerboard":
        g.set_dynamics(lt.DYNAMICS_RANDOM_SITE if args.profile_dynamics == "random-site"
                       else lt.DYNAMICS_RANDOM_SITE_BALANCED, args.profile_tile, args.profile_lambda)
    g.sweep(args.profile)
    g.synchronize()
    print("profile run: %d sweeps of L=%d (%s), kernel %s" % (args.profile, args.profile_L,
                                                           args.profile_model, g.get_kernel()))


def _lat_of(lt, r, stream=None):
    return lt.Lattice(r["dims"], r["L"], r["two_S"], r["model"], r["J"], r["h"], r["T_or_c"],
                      seed=r["seed"], init=r["init"], stream=stream)


def _warm_tuner(lt, reqs):
    """Run the autotuner once per lattice shape on throw-away lattices (one
    sweep call long enough for every candidate kernel and graph size) so
    the plain arm is timed with its tuned kernels, as in a long-running job."""
    seen = set()
    for r in reqs:
        key = (r["model"], r["dims"], r["two_S"], r["L"])
        if key in seen:
            continue
        seen.add(key)
        g = _lat_of(lt, r)
        g.sweep(600)
        g.close()


def batched_bench(n_lat=64, sweeps=200):
    """The same mixed lattices (served-mix sizes and models) advanced (a) by
    the batched engine and (b) one lattice after another with its own
    launches: updates/ns of each, and a bit-exactness check of (a) vs (b)."""
    import torch
    import paper_1209_0296_gb300 as lt
    from paper_1209_0296_gb300.workloads import served_mix
    reqs = served_mix(n=n_lat, seed=99)
    for r in reqs:
        r["sweeps"] = sweeps
    upd = sum(r["L"] ** 2 for r in reqs) * sweeps
    _warm_tuner(lt, reqs)
    # plain
    lats = [_lat_of(lt, r) for r in reqs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for g in lats:
        g.sweep(sweeps)
        g.synchronize()
    t_plain = time.perf_counter() - t0
    plain_spins = [g.get_spins() for g in lats[:4]]
    for g in lats:
        g.close()
    # batched
    lats = [_lat_of(lt, r) for r in reqs]
    # tune the batch engine for this composition first (a long throw-away
    # run), as a long-running job would have
    warm = [_lat_of(lt, r) for r in reqs]
    b = lt.Batch()
    for g in warm:
        b.add(g, 256)
    b.run()
    b.synchronize()
    for g in warm:
        g.close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for g in lats:
        b.add(g, sweeps)
    b.run()
    b.synchronize()
    t_batch = time.perf_counter() - t0
    tuning = b.tuning()
    exact = all(np.array_equal(g.get_spins(), ps) for g, ps in zip(lats[:4], plain_spins))
    for g in lats:
        g.close()
    b.close()
    return {"workload": "%d lattices of the served mix (2D Ising/North-East, L 32..4096), %d sweeps each"
                        % (n_lat, sweeps),
            "batched": upd / t_batch / 1e9, "plain": upd / t_plain / 1e9, "unit": "updates/ns",
            "speedup": t_plain / t_batch, "bit_exact_vs_plain": exact, "batch_tuning": tuning}


def _run_served(lt, reqs, chunk=64):
    """Serve the requests (arrival times in seconds from the start) through
    the continuous-batching server: per-request latencies (completion -
    arrival), the span from the first arrival to the last completion, all
    statuses OK, and the fraction of the wall time the GPU ran rounds."""
    srv = lt.Server(hbm_budget_bytes=32 << 30, max_slots=1024, chunk_sweeps=chunk)
    t0 = srv.clock()
    ids = []
    for r in reqs:
        while srv.clock() - t0 < r["arrival"]:
            pass
        ids.append(srv.submit(dims=r["dims"], L=r["L"], two_S=r["two_S"], model=r["model"],
                              J=r["J"], h=r["h"], T_or_c=r["T_or_c"], seed=r["seed"],
                              init=r["init"], sweeps=r["sweeps"]))
    srv.drain(0.0)
    res = [srv.poll(i) for i in ids]
    st = srv.stats()
    srv.close()
    lat = np.array([q["t_done"] - q["t_submit"] for q in res])
    span = max(q["t_done"] for q in res) - min(q["t_submit"] for q in res)
    ok = all(q["status"] == 0 for q in res)
    return lat, span, ok, st["busy_s"] / max(st["wall_s"] - t0, 1e-9)


def _run_plain(lt, reqs):
    """The same requests one after another, each lattice with its own
    launches (the plain arm): latencies and span."""
    t0 = time.perf_counter()
    lat = []
    for r in reqs:
        while time.perf_counter() - t0 < r["arrival"]:
            pass
        g = _lat_of(lt, r)
        g.sweep(r["sweeps"])
        g.synchronize()
        lat.append(time.perf_counter() - t0 - r["arrival"])
        g.close()
    return np.array(lat), time.perf_counter() - t0


def _pct(a):
    return {"p50_ms": float(np.percentile(a, 50) * 1e3), "p99_ms": float(np.percentile(a, 99) * 1e3)}


def served_bench(n_req=256, sweep_scale=0.01, arms=("served", "plain", "served_load_0.7", "plain_load_0.7")):
    """Requests of the served mix arriving as a Poisson process: served by
    the continuous-batching server, and (plain) one after another with one
    lattice's own launches each.  Latency = completion - arrival."""
    import paper_1209_0296_gb300 as lt
    from paper_1209_0296_gb300.workloads import served_mix, offered_updates
    base = served_mix(n=n_req, seed=99, gap_ms=2.0 * sweep_scale, sweep_scale=sweep_scale)
    upd = offered_updates(base)
    _warm_tuner(lt, base)
    scaled = "first %d requests" % n_req if n_req < 4096 else "all 4096 requests"
    out = {"workload": "%s of the served mix (default_rng(99)), sweeps x%g, gaps x%g"
                       % (scaled, sweep_scale, sweep_scale), "offered_updates": upd,
           "reduced": n_req < 4096 or sweep_scale != 1.0}
    lat, span, ok, busy = _run_served(lt, base)
    out["served"] = dict(_pct(lat), throughput=upd / span / 1e9, all_ok=ok, gpu_busy_frac=busy, span_s=span)
    if "plain" in arms:
        plat, pspan = _run_plain(lt, base)
        out["plain"] = dict(_pct(plat), throughput=upd / pspan / 1e9, span_s=pspan)
    arrival_span = base[-1]["arrival"]
    out["offered_load"] = upd / arrival_span / 1e9 / out["served"]["throughput"]
    # the same requests at an offered load of about 0.7 of the served throughput
    scale = (upd / (0.7 * out["served"]["throughput"] * 1e9)) / arrival_span
    slow = [dict(r, arrival=r["arrival"] * scale) for r in base]
    if "served_load_0.7" in arms:
        lat2, span2, ok2, busy2 = _run_served(lt, slow)
        out["served_load_0.7"] = dict(_pct(lat2), throughput=upd / span2 / 1e9, all_ok=ok2,
                                      gpu_busy_frac=busy2, span_s=span2)
    if "plain_load_0.7" in arms:
        plat2, pspan2 = _run_plain(lt, slow)
        out["plain_load_0.7"] = dict(_pct(plat2), throughput=upd / pspan2 / 1e9, span_s=pspan2)
    out["unit"] = "updates/ns"
    return out


def _timed_sweeps(torch, stream, lats, n, flush):
    """Device time (s) of n sweeps of each lattice, L2 flushed first."""
    with torch.cuda.stream(stream):
        for g in lats:
            g.sweep(2)                 # warm: tuner, graphs
        flush.fill_(3)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for g in lats:
            g.sweep(n)
        e1.record(stream)
        e1.synchronize()
    return e0.elapsed_time(e1) * 1e-3


def other_configs(dev):
    """The other named workloads at their full lattice sizes, for context
    (each a short timed run; the parity tests cover their bits)."""
    import torch
    import paper_1209_0296_gb300 as lt
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    hbm, _, _ = peaks()
    out = {}
    names = {lt.KERNEL_TILED: "tiled", lt.KERNEL_WIDE: "wide", lt.KERNEL_GENERIC: "generic",
             lt.KERNEL_RESIDENT: "resident"}

    # L = 64, cold start, T = 2.269185, seed 1234, 1000 sweeps
    g = lt.Lattice(2, 64, 1, lt.ISING, 1.0, 0.0, 2.269185, seed=1234, init=lt.INIT_COLD, stream=stream)
    g.sweep(100)
    t = _timed_sweeps(torch, stream, [g], 1000, flush)
    out["L64_cold_1000_sweeps"] = {"us_per_sweep": t / 1000 * 1e6, "updates_per_ns": 64 * 64 * 1000 / t / 1e9,
                                   "kernel": names.get(g.get_kernel()["kernel"], "?")}
    g.close()

    # 3D spin-1, L = 256, 16 temperatures in [2, 4], random start (seed 11)
    Ts = [2.0 + k * 2.0 / 15 for k in range(16)]
    lats = [lt.Lattice(3, 256, 2, lt.ISING, 1.0, 0.0, T, seed=11, init=lt.INIT_RANDOM, stream=stream) for T in Ts]
    n = 20
    t_solo = _timed_sweeps(torch, stream, lats[:1], n, flush)
    b = lt.Batch(stream=stream)
    for gg in lats:
        b.add(gg, 2)
    b.run()
    flush.fill_(4)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for gg in lats:
        b.add(gg, n)
    b.run()
    e1.record(stream)
    e1.synchronize()
    t_b = e0.elapsed_time(e1) * 1e-3
    N3 = 256 ** 3
    out["3d_spin1_L256_16T"] = {"solo_updates_per_ns": N3 * n / t_solo / 1e9,
                                "batched_updates_per_ns": 16 * N3 * n / t_b / 1e9,
                                "solo_alg_GBps": 2.0 * N3 * n / t_solo / 1e9, "sweeps": n,
                                "kernel": names.get(lats[0].get_kernel()["kernel"], "?")}
    b.close()
    for gg in lats:
        gg.close()

    # North-East, L = 8192, c in {0.05, 0.1, 0.2, 0.3}, equilibrium start (seed 21)
    lats = [lt.Lattice(2, 8192, 1, lt.NE, 0.0, 0.0, c, seed=21, init=lt.INIT_EQUILIBRIUM, stream=stream)
            for c in (0.05, 0.1, 0.2, 0.3)]
    n = 20
    t = _timed_sweeps(torch, stream, lats, n, flush)
    N4 = 8192 * 8192
    out["NE_L8192_4c"] = {"updates_per_ns": 4 * N4 * n / t / 1e9,
                          "alg_GBps": 2.25 * 4 * N4 * n / t / 1e9, "hbm_frac": 2.25 * 4 * N4 * n / t / 1e9 / hbm,
                          "sweeps": n, "kernel": names.get(lats[0].get_kernel()["kernel"], "?")}
    for gg in lats:
        gg.close()

    # the paper's own North-East algorithm (random sub-lattices and sites):
    # L = 8192, c = 0.42, 32x32 sub-lattices, 16 picks per round
    g = lt.Lattice(2, 8192, 1, lt.NE, 0.0, 0.0, 0.42, seed=21, init=lt.INIT_EQUILIBRIUM, stream=stream)
    g.set_dynamics(lt.DYNAMICS_RANDOM_SITE, 32, 16)
    n = 3
    t = _timed_sweeps(torch, stream, [g], n, flush)
    out["NE_L8192_random_site_b32_lambda16"] = {"updates_per_ns": N4 * n / t / 1e9, "sweeps": n,
                                                "us_per_sweep": t / n * 1e6}
    g.close()

    # its balance-preserving variant (single-colour rounds, four launches)
    g = lt.Lattice(2, 8192, 1, lt.NE, 0.0, 0.0, 0.42, seed=21, init=lt.INIT_EQUILIBRIUM, stream=stream)
    g.set_dynamics(lt.DYNAMICS_RANDOM_SITE_BALANCED, 32, 16)
    n = 3
    t = _timed_sweeps(torch, stream, [g], n, flush)
    out["NE_L8192_random_site_balanced_b32_lambda16"] = {"updates_per_ns": N4 * n / t / 1e9, "sweeps": n,
                                                         "us_per_sweep": t / n * 1e6}
    g.close()

    # a +-J spin glass (Eq. 1 with random bond signs, half negative), L = 4096
    g = lt.Lattice(2, 4096, 1, lt.ISING, 1.0, 0.0, 1.0, seed=7, init=lt.INIT_RANDOM, stream=stream)
    g.set_couplings(np.where(np.random.default_rng(5).random(2 * 4096 * 4096) < 0.5, -1, 1).astype(np.int8))
    n = 20
    t = _timed_sweeps(torch, stream, [g], n, flush)
    out["spin_glass_pmJ_L4096"] = {"updates_per_ns": 4096 * 4096 * n / t / 1e9, "sweeps": n,
                                   "alg_GBps": 3.0 * 4096 * 4096 * n / t / 1e9,
                                   "kernel": names.get(g.get_kernel()["kernel"], "?")}
    g.close()

    # the random-field Ising model (Eq. 1 with B_i = h * eta_i, eta_i = +-1
    # at random), L = 4096, h = J, T = 2
    g = lt.Lattice(2, 4096, 1, lt.ISING, 1.0, 1.0, 2.0, seed=7, init=lt.INIT_RANDOM, stream=stream)
    g.set_fields(np.where(np.random.default_rng(6).random(4096 * 4096) < 0.5, -1, 1).astype(np.int8))
    n = 20
    t = _timed_sweeps(torch, stream, [g], n, flush)
    out["random_field_ising_L4096"] = {"updates_per_ns": 4096 * 4096 * n / t / 1e9, "sweeps": n,
                                       "alg_GBps": 3.0 * 4096 * 4096 * n / t / 1e9,
                                       "kernel": names.get(g.get_kernel()["kernel"], "?")}
    g.close()

    # the q = 3 Potts model at its critical point, L = 4096
    import math
    g = lt.Lattice(2, 4096, 2, lt.POTTS, 1.0, 0.0, 1.0 / math.log(1.0 + math.sqrt(3.0)), seed=7,
                   init=lt.INIT_RANDOM, stream=stream)
    n = 10
    t = _timed_sweeps(torch, stream, [g], n, flush)
    out["potts_q3_L4096_Tc"] = {"updates_per_ns": 4096 * 4096 * n / t / 1e9, "sweeps": n,
                                "kernel": names.get(g.get_kernel()["kernel"], "?")}
    g.close()

    return out


def hbm_sized_run(dev, hbm, L5=32768, n=100):
    """The int8 sweep on one 2D Ising lattice far larger than L2 (L = 32768:
    1 GiB per buffer, random start, T = 2.269185), n timed sweeps: the kernel
    against HBM rather than L2."""
    import torch
    import paper_1209_0296_gb300 as lt
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    g = lt.Lattice(2, L5, 1, lt.ISING, 1.0, 0.0, 2.269185, seed=7, init=lt.INIT_RANDOM, stream=stream)
    t = _timed_sweeps(torch, stream, [g], n, flush)
    N5 = L5 * L5
    ach = 2.0 * N5 * n / t / 1e9
    out = {"workload": "2D Ising spin-1/2, L=%d, T=2.269185, random start (seed 7), int8" % L5,
           "sweeps": n, "updates_per_ns": N5 * n / t / 1e9, "achieved": ach, "peak": hbm, "unit": "GB/s",
           "frac": ach / hbm, "bytes_per_sweep": 2.0 * N5, "avg_sweep_us": t / n * 1e6,
           "kernel": {lt.KERNEL_WIDE: "k_wide_pipe<colour 0, colour 1>", lt.KERNEL_TILED: "k_sweep_tiled<Ising>"}.get(
               g.get_kernel()["kernel"], "?")}
    g.close()
    return out


def load_profile_numbers(kname):
    """Per-sweep DRAM traffic and instruction count of the chosen kernel,
    from the committed ncu summary (empty when absent)."""
    path = os.path.join(ROOT, "profiles", "%s_sweep_ising_L4096.txt" % kname)
    out = {}
    try:
        with open(path) as f:
            for line in f:
                line = line.strip()
                if not line or line.startswith("#") or ":" not in line:
                    continue
                k, v = line.split(":", 1)
                try:
                    out[k.strip()] = float(v)
                except ValueError:
                    out[k.strip()] = v.strip()
    except OSError:
        pass
    if out.get("kernel_matches_build") == "no":
        out["traffic_bytes_per_launch"] = None
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--sweeps", type=int, default=1000, help="sweeps per lattice per step")
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--tile-h", type=int, default=0)
    ap.add_argument("--int8-kernel", default="auto", choices=["auto", "wide", "tiled"],
                    help="int8 sweep kernel (auto = the library's autotuner; a fixed choice keeps "
                         "a profiled run on the kernel the plain run picks)")
    ap.add_argument("--graph", type=int, default=0, help="sweeps per CUDA graph (0 = default)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the batched and served measurements")
    ap.add_argument("--no-other", action="store_true", help="skip the timings of the other named workloads")
    ap.add_argument("--served-full", default="", metavar="ARMS",
                    help="no headline: serve the whole served-mix workload (all 4096 requests, unscaled sweeps "
                         "and gaps) through the arms named, comma-separated from served, plain, "
                         "served_load_0.7, plain_load_0.7; prints one JSON line")
    ap.add_argument("--profile", type=int, default=0, metavar="N",
                    help="no timing: run N sweeps of the T=2.0 lattice (a short run for ncu)")
    ap.add_argument("--profile-L", type=int, default=L)
    ap.add_argument("--profile-model", default="ising", choices=["ising", "ne", "ising3d", "potts", "rfim"])
    ap.add_argument("--profile-kernel", default="auto", choices=["auto", "tiled", "wide", "generic", "resident"])
    ap.add_argument("--profile-layout", default="int8", choices=["int8", "bitpacked"])
    ap.add_argument("--profile-dynamics", default="checkerboard", choices=["checkerboard", "random-site", "random-site-balanced"])
    ap.add_argument("--profile-tile", type=int, default=32, help="random-site sub-lattice side")
    ap.add_argument("--profile-lambda", type=int, default=16, help="random-site picks per round")
    args = ap.parse_args()
    if args.profile:
        run_profile(args)
        return
    if args.served_full:
        import torch
        torch.cuda.set_device(0)
        t0 = time.perf_counter()
        with Clocks(0) as clk:
            out = served_bench(n_req=4096, sweep_scale=1.0, arms=tuple(args.served_full.split(",")))
        out["wall_s"] = time.perf_counter() - t0
        out["clocks"] = clk.summary()
        print(json.dumps(out), flush=True)
        return
    if args.warmup < 3 and args.impl != "reference":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
