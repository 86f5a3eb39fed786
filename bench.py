"""Benchmark of the nucleon MD hot path on one B300 (or N replicas).

Default workload: the 409,600-nucleon run (Yp = 0.40, T = 0.5 MeV, start
density 0.080 fm^-3 with the box growing at xi = 7.5e-5 c/fm, FP32 pair
arithmetic / FP64 state, pair lists rebuilt within 10 steps with a 1 fm
skin, thermostat every 100 steps, energies every step, final cluster
analysis).  One timed "step" is one pass of the whole hot path: kick-drift,
rebuild decision (and rebuild when due), pair forces with energies, kick,
box growth and thermostat; the cluster analysis runs once at the end of the
timed region and its time is included.

Prints one JSON line (see the keys below).  Timing: CUDA events on the
library's stream around every step, with an L2 flush (a 256 MB write,
larger than the 126 MB L2) between timed steps, outside the events.

--impl reference times the FP64 CPU oracle on this host's cores on a bounded
sample of the same workload (forces on a contiguous range of targets against
all sources, plus their Verlet update).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

MEASURED = ROOT / "MEASURED_PEAKS.json"
TRAFFIC = ROOT / "profiles" / "force_split_409600_traffic.json"
PIPES = ROOT / "profiles" / "force_split_307200_pipes.json"
FORCE_SRC = ROOT / "paper_1412_8502_b300" / "csrc" / "k_force.cuh"

WORKLOADS = {
    "md409600": dict(N=409600, Yp=0.40, T=0.5, rho=0.080, seed=3, xi=7.5e-5,
                     desc="409,600 nucleons, Yp=0.40, T=0.5 MeV, rho 0.080 fm^-3 expanding at 7.5e-5 c/fm "
                          "(to 0.00125 over 20,000 steps), split FP32/FP64, 1 fm skin, rebuild <= 10 steps"),
    "md204800": dict(N=204800, Yp=0.40, T=0.5, rho=0.080, seed=6, xi=7.5e-5,
                     desc="204,800 nucleons, Yp=0.40, T=0.5 MeV, rho 0.080 fm^-3 expanding at 7.5e-5 c/fm"),
    "md307200": dict(N=307200, Yp=0.40, T=0.5, rho=0.080, seed=7, xi=7.5e-5,
                     desc="307,200 nucleons, Yp=0.40, T=0.5 MeV, rho 0.080 fm^-3 expanding at 7.5e-5 c/fm "
                          "(profiling size of the 409,600 workload: the same force-kernel path, no per-pair "
                          "wrap)"),
    "md51200": dict(N=51200, Yp=0.30, T=1.0, rho=0.080, seed=2, xi=7.5e-5,
                    desc="51,200 nucleons, Yp=0.30, T=1.0 MeV, rho 0.080 fm^-3 expanding at 7.5e-5 c/fm"),
    "md2000": dict(N=2000, Yp=0.30, T=1.0, rho=0.080, seed=1, xi=0.0,
                   desc="2,000 nucleons, Yp=0.30, T=1.0 MeV, rho 0.080 fm^-3, no expansion"),
}

# nominal algorithmic FP32 flops per in-range pair i<j, its force applied to both (FMA = 2 flops;
# the ex2 / rsqrt special-function operations are not counted)
FLOP_NUC, FLOP_COUL = 20.0, 30.0
SMS, FP32_LANES, SM_MAX_MHZ = 148, 128, 2032.0


def dist_env():
    from paper_1412_8502_b300 import replicas
    return replicas.dist_env()


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev: int):
        self.dev = dev
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                self.out = ""

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append(dict(sm=float(f[1]), smax=float(f[2]), hw=f[5], hwt=f[6], swt=f[7], pcap=f[8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = sorted(r["sm"] for r in rows)
        reasons = set()
        for r in rows:
            for k, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                            ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": rows[0]["smax"], "reasons": sorted(reasons),
                "samples": len(rows)}


def measured_peaks():
    if MEASURED.exists():
        return json.loads(MEASURED.read_text()), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


def force_traffic():
    """DRAM bytes per force launch from the committed ncu summary, if the
    force kernel source is unchanged since it was taken."""
    if not TRAFFIC.exists():
        return None
    d = json.loads(TRAFFIC.read_text())
    sha = hashlib.sha256(FORCE_SRC.read_bytes()).hexdigest()[:16]
    return d.get("dram_bytes_per_launch") if d.get("k_force_sha") == sha else None


def force_pipes():
    """Issue and pipe utilisation of the force kernel from the committed ncu
    summary, if the force kernel source is unchanged since it was taken."""
    if not PIPES.exists():
        return None
    d = json.loads(PIPES.read_text())
    sha = hashlib.sha256(FORCE_SRC.read_bytes()).hexdigest()[:16]
    if d.get("k_force_sha") != sha:
        return None
    keys = ("issue_active", "fma_pipe_active", "alu_pipe_active", "lsu_pipe_active", "xu_pipe_active",
            "fp64_pipe_active", "thread_inst_per_candidate", "thread_inst_per_in_range_pair")
    out = {k: d[k] for k in keys if k in d}
    out["source"] = "ncu, " + d.get("workload", "")
    return out


# ------------------------------------------------------------------ GPU arm
def run_gpu(args):
    import torch
    from paper_1412_8502_b300 import md, replicas

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    replicas.init("nccl")
    W = WORKLOADS[args.workload]
    N = W["N"]
    p = md.md_params_default()
    p.energy_every = 1
    p.T = W["T"]
    if args.lists == "verlet":          # the paper's per-particle neighbour lists, delta r = 4 fm
        p.list_kind = 1
        p.skin = 4.0
    if args.skin is not None:
        p.skin = args.skin
    if args.sort_bits is not None:
        p.sort_bits = args.sort_bits
    if args.plain_graph:                # profiling: ncu does not look inside graphs with conditional nodes
        p.cond_graph = 0
    sys_ = md.System(N, W["Yp"], W["rho"], W["T"], replicas.replica_seed(W["seed"], rank), p)
    stream = torch.cuda.Stream()
    sys_.set_stream(stream)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > L2

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            sys_.step(1, W["xi"])
        # the warm-up mirrors the timed region: steps, then one cluster
        # analysis (its first call allocates the system's cluster buffers);
        # the histograms land in page-locked host buffers reused by each call
        cl_out = (None, torch.zeros(N + 1, dtype=torch.int64, pin_memory=True).numpy(),
                  torch.zeros(sys_.Np + 1, dtype=torch.int64, pin_memory=True).numpy())
        sys_.clusters(labels=False, out=cl_out)
    torch.cuda.synchronize()
    # events only around the cell build, list build, force pass and kick inside
    # the timed region (an event node between every kernel slows the step)
    sys_.set_timing(2 if args.timing == "key" else 1)
    info0 = sys_.info()
    launches0, rebuilds0 = info0["launches"], info0["rebuilds"]
    K = args.steps
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K + 1)]
    pairs_nuc = pairs_coul = cand = 0
    replicas.barrier()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")
    with Clocks(local) as clk:
        for k in range(K):
            with torch.cuda.stream(stream):
                flush.zero_()
                evs[k][0].record(stream)
                sys_.step_async(1, W["xi"])      # no host round trip inside the step's events
                evs[k][1].record(stream)
            e = sys_.step_energy()
            pairs_nuc += e["pairs_nuc"]
            pairs_coul += e["pairs_coul"]
            cand += e["candidates"]
        with torch.cuda.stream(stream):
            flush.zero_()
            evs[K][0].record(stream)
            _, hA, hZ, cst = sys_.clusters(labels=False, out=cl_out)
            evs[K][1].record(stream)
        sys_.sync()                              # errors of the timed steps
        torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    step_ms = [a.elapsed_time(b) for a, b in evs[:K]]
    cl_ms = evs[K][0].elapsed_time(evs[K][1])
    total_ms = replicas.max_over_ranks(sum(step_ms) + cl_ms, device="cuda")
    info = sys_.info()
    launches = info["launches"] - launches0 + 6   # + the cluster kernels
    rebuilds = info["rebuilds"] - rebuilds0
    kt = sys_.kernel_times()
    # every kernel timed, on 10 further steps (outside the timed region)
    sys_.set_timing(1)
    with torch.cuda.stream(stream):
        sys_.step(10, W["xi"])
    torch.cuda.synchronize()
    kt_all = sys_.kernel_times()
    sys_.set_timing(False)

    # energy-criterion (MSTE) clusters of the final state, timed on their own
    # (after one untimed call: the first launch of a kernel loads its code)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        sys_.clusters_mste(labels=False)
        flush.zero_()
        ev0.record(stream)
        _, _, _, mst = sys_.clusters_mste(labels=False)
        ev1.record(stream)
    torch.cuda.synchronize()
    mste = {"ms": ev0.elapsed_time(ev1), "n_clusters": mst["n_clusters"], "n_big": mst["n_big"],
            "m_free_n": mst["m_free_n"], "distance_clusters_n_big": cst["n_big"],
            "note": "outside the timed region, second call; bound when V_ij + (M/4)|v_i - v_j|^2 < 0"}

    # end to end through the public API with pinned host buffers
    e2e = None
    if not args.no_e2e:
        # the integrator state (x, v and the cached forces f) makes the round
        # trip through pinned host memory every step
        xs, vs, fs = (torch.empty((N, 3), dtype=torch.float64, pin_memory=True).numpy() for _ in range(3))
        st = sys_.state(out=(xs, vs, fs))
        Ke = max(3, min(K, 20))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(Ke):
            sys_.set_state(xs, vs, st["L"], L_base=st["L_base"], t=st["t"], t_base=st["t_base"],
                           xi_dot=st["xi_dot"], step=st["step"], f=fs, L_F=st["L_F"])
            sys_.step(1, W["xi"])
            st = sys_.state(out=(xs, vs, fs))
            sys_.step_energy()
        wall = time.perf_counter() - t0
        e2e = {"value": N * Ke / wall, "unit": "nucleon-steps/s", "h2d_bytes_per_step": 3 * 24 * N,
               "d2h_bytes_per_step": 3 * 24 * N + 8 * 9, "steps": Ke,
               "note": "per step: md_set_state from pinned host x, v, f (restores the cached forces, no "
                       "force pass; the state goes into the current particle order and the rebuild rule "
                       "decides on the tiles); md_step; md_get_state of x, v, f to pinned host; md_step_energy"}

    # the same steps without the energy record (md_params.energy_every = 0,
    # the default), whose force passes are compiled for more resident blocks;
    # outside the timed region, same L2 flush between steps
    no_energy = None
    if not args.plain_graph:
        q = sys_.params
        q.energy_every = 0
        sys_.params = q
        with torch.cuda.stream(stream):
            sys_.step(3, W["xi"])
        torch.cuda.synchronize()
        Kn = max(3, min(K, 20))
        evn = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(Kn)]
        with torch.cuda.stream(stream):
            for a, b in evn:
                flush.zero_()
                a.record(stream)
                sys_.step_async(1, W["xi"])
                b.record(stream)
        sys_.sync()
        torch.cuda.synchronize()
        ms_ne = sum(a.elapsed_time(b) for a, b in evn) / Kn
        no_energy = {"value": N / (ms_ne * 1e-3), "unit": "nucleon-steps/s", "ms_per_step": ms_ne, "steps": Kn,
                     "note": "md_params.energy_every = 0 (the default): steps without the energy record, the "
                             "force passes compiled for 5 blocks per SM; after the timed region, no cluster "
                             "analysis; the headline keeps the energy record every step"}
        q.energy_every = 1
        sys_.params = q

    if rank != 0:
        replicas.finalize()
        return None

    force_ms, force_n = kt.get("force", (0, 0.0))[1], kt.get("force", (0, 0.0))[0]
    peaks, src = measured_peaks()
    flops = FLOP_NUC * pairs_nuc + FLOP_COUL * pairs_coul
    fp32_peak = SMS * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12          # TFLOP/s at max clock
    achieved = flops / (force_ms * 1e-3) / 1e12 if force_ms > 0 else None
    line = {
        "metric": "nucleon-steps/s",
        "value": world * N * K / (total_ms * 1e-3),
        "unit": "nucleon-steps/s",
        "n_gpus": world,
        "steps": K,
        "warmup": args.warmup,
        "ms_per_step": total_ms / K,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32 pair math / f64 state",
        "data": "synthetic: seeded uniform positions + 500 steepest-descent iterations, Maxwell velocities",
        "config": {"workload": W["desc"], "N": N, "Yp": W["Yp"], "T_MeV": W["T"], "rho_start": W["rho"],
                   "lists": "half tile-pair lists" if args.lists == "tiles" else "per-particle Verlet lists",
                   "graph": "plain nodes (profiling)" if args.plain_graph else "rebuild in conditional nodes",
                   "skin_fm": p.skin,
                   "xi_dot": W["xi"], "window": "first steps of the expansion (densest, slowest)",
                   "clusters": "one cluster analysis inside the timed region",
                   "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"bound": "alu", "kernel": "k_force_split", "achieved": achieved, "peak": fp32_peak,
                     "unit": "TFLOP/s", "frac": (achieved / fp32_peak) if achieved else None,
                     "traffic": force_traffic(),
                     "issue": force_pipes(),
                     "peak_note": "FP32 FMA issue peak 148 SM x 128 lanes x 2 flop x 2032 MHz (derived; "
                                  "MEASURED_PEAKS has no FP32 figure)",
                     "algorithmic": {"pairs_nuc_per_step": pairs_nuc / K, "pairs_coul_per_step": pairs_coul / K,
                                     "flop_per_pair": {"nuclear": FLOP_NUC, "coulomb": FLOP_COUL},
                                     "force_ms_per_launch": force_ms / max(force_n, 1),
                                     "candidate_pairs_per_step": cand / K,
                                     "candidate_efficiency": (pairs_nuc + pairs_coul) / max(cand, 1)}},
        "force_code": {"variant": info["force_code"], "tuner_trials": info["force_trials"],
                       "note": "split force-pass code in use: 4 long unrolled loops, 2 compact, 1 minimal, 3 minimal "
                               "in one-warp blocks; chosen on the device by timing all four every 500 steps from step "
                               "500 (bitwise the same results)"},
        "tiles": {"count": info["tiles"], "list_entries": info["list_entries"], "rebuilds": info["rebuilds"],
                  "halfext_mean_fm": info["tile_halfext_mean"], "halfext_max_fm": info["tile_halfext_max"],
                  "need_wrap": info["need_wrap"]},
        "lists": {"kind": args.lists, "skin_fm": p.skin, "rebuilds_in_timed_steps": rebuilds,
                  "steps_per_rebuild": K / max(rebuilds, 1),
                  "verlet_entries": info["verlet_entries"], "verlet_slots": info["verlet_slots"],
                  "verlet_capacity": info["verlet_capacity"]},
        "kernel_ms_per_step": {k: v[1] / 10.0 for k, v in kt_all.items()},
        "kernel_ms_note": "every kernel timed with CUDA events on 10 steps after the timed region; the timed "
                          "region itself times the cell build, list build, force pass and kick",
        "cell_build": cell_build_roofline(kt, rebuilds, N, info, peaks),
        "step_ms_p50": sorted(step_ms)[len(step_ms) // 2],
        "step_ms_p99": sorted(step_ms)[min(len(step_ms) - 1, int(math.ceil(0.99 * len(step_ms))) - 1)],
        "cluster_ms": cl_ms,
        "mste": mste,
        "clusters": {"n": cst["n_clusters"], "m_free_n": cst["m_free_n"]},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "peaks_source": src,
    }
    if e2e:
        line["e2e"] = e2e
    if no_energy:
        line["no_energy_record"] = no_energy
    # (not in the profiling mode --plain-graph, whose runs serve ncu captures)
    if not args.no_schedule and not args.plain_graph and world == 1 and args.precision == "split":
        line["schedule"] = run_schedule(args)
    if not args.no_batch and world == 1:
        line["batch"] = run_batch(args.batch_steps)
    if not args.no_serve and world == 1:
        line["serve"] = run_serve(args.serve_jobs, args.serve_steps, args.serve_rate)
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(W, args.cpu_seconds)
    replicas.finalize()
    return line


def cell_build_roofline(kt, rebuilds, N, info, peaks):
    """Spatial sort + tile build (hist, scan, scatter, move, tiles) per
    rebuild: algorithmic bytes / CUDA-event time.  In the step graph these
    kernels sit in a conditional node that runs only on rebuild steps; its
    event interval ("cell_build") is the time."""
    names = ("cell_build",) if "cell_build" in kt else ("hist", "scan", "scatter", "move", "tiles")
    ms = sum(kt.get(k, (0, 0.0))[1] for k in names)
    if rebuilds <= 0 or ms <= 0:
        return None
    bins = 2 * (1 << (3 * info["sort_bits"]))
    # per particle: hist 28 B (x, key), scatter 12 B, move 124 B (x, v, id read+write,
    # slot/key/bin lookups), tiles 68 B (x read, hi/lo and displacement write); per bin 12 B
    alg = 232.0 * N + 12.0 * bins
    per = ms / rebuilds
    gbs = alg / (per * 1e-3) / 1e9
    # the minimum a counting sort must move: read x (24 B) + type,
    # write a key (4 B), read x + key again and write the sorted x, local coordinates, type and
    # id (about 100 B per particle in all)
    minimal = 100.0 * N
    # DRAM bytes per rebuild measured by ncu on the 307,200 case (profiles/step_kernels_md307200_ncu.md:
    # hist 9.50, two scan passes 4.21, scatter 3.35, move 22.67, tiles 7.43 MB), scaled by N
    dram = 47.16e6 * N / 307200.0
    return {"bound": "hbm", "rebuilds": rebuilds, "ms_per_rebuild": per, "bytes_per_rebuild": alg,
            "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"],
            "frac_min_bytes": minimal / (per * 1e-3) / 1e9 / peaks["hbm_gbs"],
            "frac_ncu_dram_bytes": dram / (per * 1e-3) / 1e9 / peaks["hbm_gbs"],
            "note": "frac: the builder's own 232 B per particle + 12 B per bin; frac_min_bytes: the minimum "
                    "of about 100 B per particle; frac_ncu_dram_bytes: the DRAM bytes ncu measured for these "
                    "kernels (the rest of their traffic is served by L2). Six chained kernels of 4-16 us: "
                    "launch latency and the dependent gathers of the move bound it, not HBM bandwidth"}


# ------------------------------------------------------------------ batch / serve
def batch_jobs(seed=4):
    """Ensemble of the paper's Yp x T sweep (5 x 3 systems): N drawn from
    {4,000, 12,800, 25,600, 51,200}, density log-uniform in [0.00125, 0.080]
    fm^-3, no expansion."""
    import numpy as np
    rng = np.random.default_rng(seed)
    jobs = []
    for Yp in (0.05, 0.10, 0.20, 0.30, 0.40):
        for T in (0.5, 0.75, 1.0):
            N = int(rng.choice([4000, 12800, 25600, 51200]))
            rho = float(np.exp(rng.uniform(np.log(0.00125), np.log(0.080))))
            jobs.append(dict(N=N, Yp=Yp, rho=rho, T=T, seed=int(rng.integers(1 << 30)), xi_dot=0.0))
    return jobs


def run_batch(steps, cmp_steps=1000):
    """The 15-system ensemble (Yp x T sweep) stepped by ONE persistent kernel
    launch per step for all systems, its configured run of `steps` steps;
    then, from the state it reached, the same batch as a graph of separate
    kernels per step, and each system stepped alone, over cmp_steps steps
    each (the batch holds no expansion, so the work per step is stationary).
    Device time (CUDA-synchronised wall clock around the steps)."""
    import torch
    from paper_1412_8502_b300 import md
    jobs = batch_jobs()
    p = md.md_params_default()
    p.energy_every = 1
    ntot = sum(j["N"] for j in jobs)
    b = md.Batch(jobs, p)      # persistent = -1: one persistent launch per step for a batch
    p = b.autotune(10)         # project autotuner: skin x cell size (sort bits) x force-code variant
    tuned = {"skin_fm": p.skin, "sort_bits_sys0": p.sort_bits, "force_code": p.force_unroll}

    def timed(nsteps):
        b.step(3)
        torch.cuda.synchronize()
        l0 = b.systems[0].info()["launches"]
        t0 = time.perf_counter()
        b.step(nsteps)
        torch.cuda.synchronize()
        return time.perf_counter() - t0, (b.systems[0].info()["launches"] - l0) / nsteps

    tb, launches = timed(steps)
    q = b.systems[0].params
    q.persistent = 0
    b.systems[0].params = q
    cmp_steps = min(cmp_steps, steps)
    tg, launches_g = timed(cmp_steps)
    b.close()
    p.sort_bits = 0             # serial runs: same skin and code variant, sort resolution from each N
    p.r_C = 0.0                 # and the Coulomb cutoff from each box (min(40, L0/2))
    ts = 0.0
    for j in jobs:
        s = md.System(j["N"], j["Yp"], j["rho"], j["T"], j["seed"], p)
        s.step(3, 0.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s.step(cmp_steps, 0.0)
        torch.cuda.synchronize()
        ts += time.perf_counter() - t0
        s.close()
    batched = ntot * steps / tb
    serial = ntot * cmp_steps / ts
    return {"systems": len(jobs), "nucleons": ntot, "steps": steps, "tuned": tuned,
            "batched": batched, "serial": serial, "speedup": batched / serial,
            "batched_graph": ntot * cmp_steps / tg, "speedup_graph": (ntot * cmp_steps / tg) / serial,
            "unit": "nucleon-steps/s", "kernel_launches_per_step": launches,
            "kernel_launches_per_step_graph": launches_g, "compare_steps": cmp_steps,
            "accuracy": "each member bitwise equal to the same system stepped alone (tests)",
            "note": "15 systems (Yp x T sweep), N from {4000,12800,25600,51200}, rho log-uniform "
                    "[0.00125, 0.08], energies every step; batched = one persistent kernel launch per step "
                    "for all systems over the configured steps; batched_graph = the same batch as a graph of "
                    "separate kernels; serial = one system at a time (each its own graph); the comparisons "
                    "over compare_steps steps from the state the batched run reached"}


def serve_trace_jobs(rng, n_jobs, steps):
    """The serving workload's jobs: N log-uniform in [2,000, 409,600], Y_p and T
    from the sweep, density 0.080 falling to U[0.005, 0.02] fm^-3 over the steps."""
    import numpy as np
    jobs = []
    for _ in range(n_jobs):
        N = int(round(float(np.exp(rng.uniform(np.log(2000), np.log(args_serve_nmax))))))
        rho_f = float(rng.uniform(0.005, 0.02))
        xi = ((0.08 / rho_f) ** (1 / 3) - 1.0) / (2.0 * 2000)
        jobs.append(dict(N=N, Yp=float(rng.choice([0.05, 0.1, 0.2, 0.3, 0.4])), rho=0.08,
                         T=float(rng.choice([0.5, 0.75, 1.0])), seed=int(rng.integers(1 << 30)),
                         xi_dot=xi, steps=steps))
    return jobs


def run_serve_split(n_jobs, steps, seed=5):
    """Where the serving speed-up is bounded: the serving trace's four largest
    jobs and its other jobs, each set run one job at a time and submitted to
    the server at once (wall clock, CUDA-synchronised), and the creation
    (relaxation) and steps of the largest job apart."""
    import numpy as np
    import torch
    from paper_1412_8502_b300 import md
    jobs = serve_trace_jobs(np.random.default_rng(seed), n_jobs, steps)
    big = sorted(jobs, key=lambda j: -j["N"])[:4]
    small = [j for j in jobs if j not in big]
    p = md.md_params_default()

    def alone(js):
        t = 0.0
        for j in js:
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            s = md.System(j["N"], j["Yp"], j["rho"], j["T"], j["seed"], p)
            s.step(j["steps"], j["xi_dot"])
            s.energy()
            s.close()
            torch.cuda.synchronize()
            t += time.perf_counter() - t1
        return t

    def served(js):
        free, _ = torch.cuda.mem_get_info()
        sv = md.md_server_create(int(0.5 * free), p)
        t0 = time.perf_counter()
        for j in js:
            md.md_server_submit(sv, j)
        md.md_server_drain(sv, 1800.0)
        w = time.perf_counter() - t0
        md.md_server_destroy(sv)
        return w

    out = {"mode": "serve split", "big_N": [j["N"] for j in big], "big_alone_s": alone(big),
           "big_served_s": served(big), "small_N": sorted(j["N"] for j in small),
           "small_alone_s": alone(small), "small_served_s": served(small)}
    j = big[0]
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    s = md.System(j["N"], j["Yp"], j["rho"], j["T"], j["seed"], p)
    torch.cuda.synchronize()
    out["big0_create_s"] = time.perf_counter() - t1
    t1 = time.perf_counter()
    s.step(j["steps"], j["xi_dot"])
    torch.cuda.synchronize()
    out["big0_steps_s"] = time.perf_counter() - t1
    s.close()
    return out


def run_serve(n_jobs, steps, rate, seed=5):
    """Poisson stream of MD jobs into the server (continuous batching, HBM
    budget, device-resident state, interleaved steps); per-step latency from
    CUDA events on each job's stream.  Baseline: the same jobs on the same
    arrival trace served one at a time (FIFO), each job's duration measured
    by running it alone (create + relax + steps + energies + destroy)."""
    import numpy as np
    import torch
    from paper_1412_8502_b300 import md
    rng = np.random.default_rng(seed)
    jobs = serve_trace_jobs(rng, n_jobs, steps)
    gaps = rng.exponential(1.0 / rate, n_jobs)
    arrivals = np.concatenate([[0.0], np.cumsum(gaps[:-1])])
    p = md.md_params_default()
    free, total = torch.cuda.mem_get_info()
    sv = md.md_server_create(int(0.5 * free), p)
    t0 = time.perf_counter()
    for k, j in enumerate(jobs):
        wait = t0 + arrivals[k] - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        md.md_server_submit(sv, j)
    md.md_server_drain(sv, 1800.0)
    wall = time.perf_counter() - t0
    res = []
    while True:
        r = md.md_server_poll(sv)
        if r is None:
            break
        res.append(r)
    md.md_server_destroy(sv)
    ok = [r for r in res if r["status"] == 0]
    work = sum(r["N"] * r["steps"] for r in ok)
    lat = sorted(x for r in ok for x in (r["step_p50_ms"],))
    p99 = max(r["step_p99_ms"] for r in ok) if ok else None
    # one at a time: each job alone, then the FIFO schedule on the same arrivals
    dur = []
    for j in jobs:
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        s = md.System(j["N"], j["Yp"], j["rho"], j["T"], j["seed"], p)
        s.step(j["steps"], j["xi_dot"])
        s.energy()
        s.close()
        torch.cuda.synchronize()
        dur.append(time.perf_counter() - t1)
    t_free = 0.0
    for a, d in zip(arrivals, dur):
        t_free = max(a, t_free) + d
    serial_wall = t_free
    # per size class (the server's stream priorities): worst per-job p99 and median per-job p50
    classes = {"N<20k": (0, 20000), "20k<=N<100k": (20000, 100000), "N>=100k": (100000, 1 << 40)}
    by_class = {}
    for name, (lo, hi) in classes.items():
        rc = [r for r in ok if lo <= r["N"] < hi]
        if rc:
            p50s = sorted(r["step_p50_ms"] for r in rc)
            by_class[name] = {"jobs": len(rc), "step_p50_ms": round(p50s[len(p50s) // 2], 3),
                              "step_p99_ms": round(max(r["step_p99_ms"] for r in rc), 3)}
    return {"jobs": n_jobs, "completed": len(ok), "steps_per_job": steps, "arrival_rate_per_s": rate,
            "served": work / wall, "serial": work / serial_wall, "speedup": serial_wall / wall,
            "served_wall_s": wall, "serial_wall_s": serial_wall, "serial_busy_s": float(sum(dur)),
            "unit": "nucleon-steps/s (wall from the first arrival to the last completion, job creation and "
                    "relaxation included)",
            "step_p50_ms": lat[len(lat) // 2] if lat else None, "step_p99_ms": p99,
            "wait_ms_max": max(r["wait_ms"] for r in ok) if ok else None,
            "by_size_class": by_class,
            "job_N": [j["N"] for j in jobs],
            "job_step_p99_ms": {int(r["N"]): round(r["step_p99_ms"], 3) for r in ok},
            "job_run_s": {int(r["N"]): round(r["run_ms"] / 1e3, 3) for r in ok},
            "job_alone_s": {int(j["N"]): round(d, 3) for j, d in zip(jobs, dur)},
            "note": "N log-uniform in [2000, %d], Yp/T from the sweep, rho 0.080 -> U[0.005,0.02] over the job's "
                    "steps; p50 = median over jobs of each job's median step latency, p99 = max over jobs of "
                    "each job's 99th percentile; serial = the same arrival trace served one job at a time "
                    "(FIFO), job durations measured alone" % args_serve_nmax}


args_serve_nmax = 409600


# ------------------------------------------------------------------ full schedule
def run_full(args):
    """The workload's whole schedule (20,000 steps; for the expanding
    workloads rho 0.080 -> 0.00125) in chunks of 1,000 steps, each timed with
    CUDA events on the system's stream, and one cluster analysis after each
    chunk (outside the chunk's events): throughput per density window (first
    1,000 steps, whole run, last 1,000 steps) and the cluster statistics
    along the run.  Consecutive steps of one trajectory: L2 is not flushed."""
    import torch
    from paper_1412_8502_b300 import md

    torch.cuda.set_device(0)
    W = WORKLOADS[args.workload]
    N = W["N"]
    p = md.md_params_default()
    p.energy_every = 1
    p.T = W["T"]
    if args.precision == "fp64":
        p.precision = md.MD_PREC_FP64
    if args.force_unroll is not None:
        p.force_unroll = args.force_unroll
    if args.sort_bits is not None:
        p.sort_bits = args.sort_bits
    if args.skin is not None:
        p.skin = args.skin
    s = md.System(N, W["Yp"], W["rho"], W["T"], W["seed"], p)
    stream = torch.cuda.Stream()
    s.set_stream(stream)
    cl_out = (None, torch.zeros(N + 1, dtype=torch.int64, pin_memory=True).numpy(),
              torch.zeros(s.Np + 1, dtype=torch.int64, pin_memory=True).numpy())
    total = args.full_steps
    chunk = min(1000, total)
    rows = []
    with Clocks(0) as clk:
        for c in range(total // chunk):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                e0.record(stream)
                s.step(chunk, W["xi"])
                e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            en = s.energy()
            _, hA, hZ, cst = s.clusters(labels=False, out=cl_out)
            info = s.info()
            rows.append({"step": (c + 1) * chunk, "ms_per_step": round(ms / chunk, 4),
                         "rho": round(N / en["L"] ** 3, 6), "L_fm": round(en["L"], 3),
                         "E_per_nucleon_MeV": round((en["KE"] + en["PE_nuc"] + en["PE_coul"]) / N, 5),
                         "n_clusters": cst["n_clusters"], "n_big": cst["n_big"],
                         "A_mean": round(cst["A_mean"], 2), "Z_mean": round(cst["Z_mean"], 2),
                         "m_free_n": round(cst["m_free_n"], 5), "rebuilds": info["rebuilds"],
                         "force_code": info["force_code"]})
    if args.late_pass:                 # one energy force pass of the final state, for kernel profilers
        torch.cuda.nvtx.range_push("late")
        s.energy()
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    s.close()
    tot_ms = sum(r["ms_per_step"] * chunk for r in rows)
    first, last = rows[0], rows[-1]
    return {"metric": "nucleon-steps/s", "mode": "full schedule", "value": N * len(rows) * chunk / (tot_ms / 1e3),
            "unit": "nucleon-steps/s", "n_gpus": 1, "steps": len(rows) * chunk, "higher_is_better": True,
            "windows": {"first_chunk": N / (first["ms_per_step"] / 1e3), "whole_run": N * len(rows) * chunk /
                        (tot_ms / 1e3), "last_chunk": N / (last["ms_per_step"] / 1e3), "chunk_steps": chunk},
            "dtype": "f64" if args.precision == "fp64" else "f32 pair math / f64 state", "data": "synthetic",
            "config": {"workload": W["desc"], "N": N, "l2": "not flushed (consecutive steps of one trajectory)",
                       "clusters": "after every 1,000 steps, outside the timed chunks"},
            "chunks": rows, "clocks": clk.summary()}


def run_schedule(args):
    """The workload's whole 20,000-step schedule (for the 409,600 workload the
    expansion 0.080 -> 0.00125 fm^-3 into clusters), as run_full, summarised:
    throughput over the first 1,000 steps, the whole run and the last 1,000
    steps, and the state every 5,000 steps."""
    import copy
    a = copy.copy(args)
    a.full_steps = 20000
    a.late_pass = False
    r = run_full(a)
    keep = ("step", "ms_per_step", "rho", "n_clusters", "n_big", "A_mean", "Z_mean", "m_free_n", "rebuilds",
            "force_code")
    return {"steps": r["steps"], "unit": "nucleon-steps/s", "windows": r["windows"],
            "every_5000": [{k: c[k] for k in keep} for c in r["chunks"] if c["step"] % 5000 == 0],
            "clocks": r["clocks"],
            "note": "consecutive steps of one trajectory in 1,000-step chunks timed with CUDA events (L2 not "
                    "flushed); one cluster analysis after each chunk, outside the timed chunks; the headline "
                    "value is the dense start of this schedule with L2 flushed between steps"}


# ------------------------------------------------------------------ oracle
def cpu_baseline(W, seconds):
    """The FP64 oracle, as it stands, on this host's cores: forces on a
    contiguous range of targets against all N sources, plus their Verlet
    update, at the workload's start state (seeded uniform positions)."""
    import numpy as np
    import oracle

    N = W["N"]
    p = oracle.params(min(40.0, 0.5 * (N / W["rho"]) ** (1 / 3)))
    x, v, t, L = oracle.init(N, W["Yp"], W["rho"], W["T"], W["seed"], p)
    oracle.forces(x, t, L, p, 0, 64)              # start the thread pool
    n = 1024                                      # calibrate on enough targets for every core
    t0 = time.perf_counter()
    oracle.forces(x, t, L, p, 0, n)
    dt = time.perf_counter() - t0
    n = int(max(64, min(N, n * seconds / max(dt, 1e-6))))
    t0 = time.perf_counter()
    F, _ = oracle.forces(x, t, L, p, 0, n)
    h = 0.5 * 2.0 / 939.0
    vv = v[:n] + h * F[:n]
    xx = x[:n] + 2.0 * vv
    _ = xx.sum()
    dt = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": n / dt, "unit": "nucleon-steps/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} targets x {N} sources (brute-force FP64 pair sum + Verlet update), "
                      f"{dt:.1f} s, start density"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return None
    W = WORKLOADS[args.workload]
    per = max(2.0, args.cpu_seconds / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_baseline(W, per)
    vals = [cpu_baseline(W, per) for _ in range(args.steps)]
    v = sum(x["value"] for x in vals) / len(vals)
    return {"impl": "reference", "metric": "nucleon-steps/s", "value": v, "unit": "nucleon-steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * W["N"] / v,
            "ms_per_step_note": "projected: the time one whole step of all N nucleons would take at the rate "
                                "measured on the bounded samples (each sample step times a contiguous range "
                                "of targets against all N sources, see cpu_baseline.sample); no whole step ran",
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": W["desc"], "N": W["N"]},
            "cpu_baseline": {"value": v, "unit": "nucleon-steps/s", "cores": vals[0]["cores"], "kind": "oracle",
                             "sample": vals[0]["sample"]},
            "e2e": {"value": v, "unit": "nucleon-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="md409600", choices=list(WORKLOADS))
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--lists", default="tiles", choices=["tiles", "verlet"],
                    help="pair lists: half tile-pair lists (default) or per-particle Verlet lists (delta r = 4 fm)")
    ap.add_argument("--skin", type=float, default=None, help="pair-list skin / Verlet delta r, fm")
    ap.add_argument("--timing", default="key", choices=["key", "full"],
                    help="CUDA events inside the timed region: around the key kernels (default) or every kernel")
    ap.add_argument("--sort-bits", type=int, default=None, help="spatial-sort bits per axis (default: from N)")
    ap.add_argument("--plain-graph", action="store_true",
                    help="rebuild kernels as plain graph nodes instead of conditional ones (for kernel profilers)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-schedule", action="store_true", help="skip the whole 20,000-step schedule")
    ap.add_argument("--batch-steps", type=int, default=5000)
    ap.add_argument("--serve-jobs", type=int, default=12)
    ap.add_argument("--serve-steps", type=int, default=2000)
    ap.add_argument("--serve-rate", type=float, default=4.0)
    ap.add_argument("--serve-split", action="store_true",
                    help="time the serving trace's four largest jobs and the others apart, alone and served")
    ap.add_argument("--precision", default="split", choices=["split", "fp64"],
                    help="with --full-steps: split FP32/FP64 (default) or the FP64 mode")
    ap.add_argument("--force-unroll", type=int, default=None, choices=[0, 1, 2, 3, 4],
                    help="with --full-steps: fix the force-pass code variant (md_params.force_unroll)")
    ap.add_argument("--late-pass", action="store_true",
                    help="with --full-steps: one more force pass of the final state in an NVTX range 'late'")
    ap.add_argument("--full-steps", type=int, default=0,
                    help="run the workload's schedule for this many steps (20000: the whole expansion) in "
                         "1,000-step chunks and report throughput per density window instead")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.serve_split:
        line = run_serve_split(args.serve_jobs, args.serve_steps)
    elif args.full_steps:
        line = run_full(args)
    else:
        line = run_reference(args) if args.impl == "reference" else run_gpu(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
