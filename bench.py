#!/usr/bin/env python3
"""Throughput of the Pyramidal Gradient Matching hot path on GB300.

One step = the whole path (gradient pyramids of both images, pyramidal
matching in both directions, consistency and outlier filtering, region
removal and match export) over a batch of Sintel-shaped 1024x436 RGB pairs
with the paper's full version PGM-C (6-channel gradients, Table 2 colour
schedule, r = 7 / 5 patches, 4 / 6 iterations, W = 2, N = 2) on a 5-level
pyramid and a stride-3 seed lattice.  Inputs are resident in HBM when the
timed region starts; L2 is flushed (a 256 MB write) before every timed step.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle
(the plain C reference implementation of the method) on the host cores
instead.  Multi-GPU (torchrun): every rank matches its own pairs (replicas,
weak scaling, no collective on the data path).
"""
import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pairs/s and G candidate-evals/s at 1024×436 (bit-exact); served p50/p99 ms"
W_IMG, H_IMG = 1024, 436
PARAMS = dict(levels=5, seed_stride=3, patch_fwd=15, patch_bwd=11, color=1, descriptor=0,
              iters_coarse=4, iters_fine=6, refine_rounds=2, rs_W=2)
VARIANTS = {"PGM-CD": dict(color=1, descriptor=1), "PGM-G": dict(color=0, descriptor=0),
            "PGM-GD": dict(color=0, descriptor=1),
            # the checkerboard schedule at the iteration count above level 0
            # that meets the scan order's accuracy margins on this workload
            "PGM-C calibrated (iters_coarse 12)": dict(iters_coarse=12)}
# The paper's own matching times (Table 3, Sec. IV), quoted with the hardware
# it states: context beside this run's numbers, not a ratio (the paper matches
# every pixel of a 3-level pyramid of the real datasets).
PAPER_TIMINGS = {
    "source": "Table 3 (matching only, interpolation excluded)",
    "hardware": "Intel Pentium G3240 @ 3.1 GHz, 4 GB RAM, one thread, no GPU / OpenMP / SSE",
    "workload": "MPI Sintel and KITTI2012 training sets, dense per-pixel matching, L = 3",
    "s_per_pair": {"PGM-C": {"sintel": 3.49, "kitti2012": 4.55},
                   "PGM-G": {"sintel": 1.82, "kitti2012": 2.05},
                   "PGM-CD": {"sintel": 1.56, "kitti2012": 1.60},
                   "PGM-GD": {"sintel": 1.08, "kitti2012": 1.16},
                   "PGM-C3": {"sintel": 2.28, "kitti2012": 2.77},
                   "PGM-G3": {"sintel": 1.13, "kitti2012": 1.26}},
}
WORKLOAD = ("sintel-like 1024x436 RGB pairs (3-6 layered textured polygons, <=150 px motion), "
            "PGM-C: 6-ch Sobel-5 gradients, Table-2 colour schedule, L=5, seed stride 3, "
            "patch 15/11, iters 4/6, W=2, N=2")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=16, help="pairs per step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--cpu-pairs", type=int, default=0, help="oracle sample size in pairs (0: the step's pairs)")
    ap.add_argument("--tuning", default="",
                    help="fixed launch knobs 'SLACK,PAIRS[,TILE_W]' instead of autotuning them")
    ap.add_argument("--variant", default="", choices=[""] + list(VARIANTS),
                    help="time this variant's parameters instead of PGM-C (profiling runs)")
    ap.add_argument("--traffic-record", default="",
                    help="write the search kernel's DRAM traffic record from this ncu csv "
                         "(made by bench.TRAFFIC_CMD) and exit")
    ap.add_argument("--serve", type=int, default=300,
                    help="requests of the serving run (Poisson, 200/s); 0 skips it")
    return ap.parse_args()


# ------------------------------------------------------------ CPU oracle
def config_dict(batch, world):
    """The workload description both arms print (same pairs, same params)."""
    return {"workload": WORKLOAD, "pairs_per_step": batch, "image": "1024x436x3 uint8",
            "pair_seeds": "sintel_like_pair seeds 10*rank*B + 0..B-1",
            "l2": "GPU arm: flushed (256 MB write) before every timed step",
            "parallelism": "replicas" if world > 1 else "1 GPU"}


def _oracle_one(args):
    seed, prm, schedule = args
    import oracle as O
    from paper_1704_03217_gb300 import synth
    f1, f2, _ = synth.sintel_like_pair(seed, W_IMG, H_IMG)
    t0 = time.perf_counter()
    O.run_pair(prm, f1, f2, schedule, seed)
    return time.perf_counter() - t0


def oracle_rate(seeds, cores, schedule=0, prm=None):
    """Pairs/s of the oracle on the pairs of `seeds`, one pair per process,
    `cores` processes (schedule 0: checkerboard, 1: the paper's scan)."""
    from oracle import build as obuild
    obuild.build()
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        t0 = time.perf_counter()
        times = pool.map(_oracle_one, [(sd, prm or PARAMS, schedule) for sd in seeds])
        wall = time.perf_counter() - t0
    # pair generation runs inside the workers too: charge only the oracle time
    per_proc = max(sum(times[k::cores]) for k in range(cores))
    return len(seeds) / per_proc, per_proc, wall


def oracle_one_core(seed):
    """Pairs/s of one process on one pair, in the checkerboard schedule and
    in the paper's scan order (both run at once, one process each)."""
    from oracle import build as obuild
    obuild.build()
    ctx = mp.get_context("spawn")
    with ctx.Pool(2) as pool:
        t_cb, t_seq = pool.map(_oracle_one, [(seed, PARAMS, 0), (seed, PARAMS, 1)])
    return 1.0 / t_cb, 1.0 / t_seq


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    world = int(os.environ.get("WORLD_SIZE", "1"))
    cores = os.cpu_count() or 1
    seeds = rank_seeds(0, a.batch)
    procs = min(cores, len(seeds))
    for _ in range(a.warmup):
        oracle_rate(seeds[:procs], procs)
    secs = []
    for _ in range(a.steps):
        _, t, _ = oracle_rate(seeds, procs)
        secs.append(t)
    total = sum(secs)
    value = len(seeds) * a.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "pairs/s",
            "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * total / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": config_dict(a.batch, world),
            "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": procs, "kind": "oracle",
                             "sample": "the GPU arm's %d sintel-like pairs per step, one per "
                                       "process, checkerboard schedule" % len(seeds)},
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------- ncu traffic record
TRAFFIC_REC = os.path.join(ROOT, "profiles", "k_pm_r_traffic.json")
PM_SRC = os.path.join(ROOT, "paper_1704_03217_gb300", "csrc", "pm_row.cu")
DEVICE_MARK = "// Host side: launch configuration.  No device code below this line.\n"
# the capture the record is made from: DRAM counters of two level-0 search
# launches (forward and backward of the second iteration's first colour phase)
# of the first, eager step of an 8-pair run
TRAFFIC_PAIRS = 8
TRAFFIC_CMD = ("ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum "
               "--clock-control none --nvtx --nvtx-include \"pgm_match/level 0/\" "
               "-k regex:k_pm_r -s 4 -c 2 --csv --log-file k_pm_r_traffic.csv "
               "python bench.py --steps 1 --warmup 3 --batch %d --no-cpu-baseline --no-variants "
               "--serve 0 --tuning 2,32" % TRAFFIC_PAIRS)


def device_hash():
    import hashlib
    text = open(PM_SRC, encoding="utf-8").read()
    if DEVICE_MARK not in text:
        return None
    return hashlib.sha256(text.split(DEVICE_MARK)[0].encode("utf-8")).hexdigest()


def lattice_sizes(prm, w, h):
    """Seeds per level of a w x h image (stride sigma, offset sigma // 2)."""
    sig = prm["seed_stride"]
    c = sig // 2
    out = []
    for _ in range(prm["levels"]):
        out.append(((w - 1 - c) // sig + 1) * ((h - 1 - c) // sig + 1))
        w, h = (w + 1) // 2, (h + 1) // 2
    return out


def search_units(prm, w, h, pairs):
    """Seed-iterations of the search per step: every iteration of a visit at
    level l covers each of the n_l seeds of both directions once."""
    n = lattice_sizes(prm, w, h)
    return pairs * sum(2 * n[l] * (prm["iters_fine"] if l == 0 else prm["iters_coarse"])
                       for l in visit_levels(prm["levels"], prm.get("refine_rounds", 2)))


def write_traffic_record(csv_path):
    """profiles/k_pm_r_traffic.json from the capture TRAFFIC_CMD wrote."""
    import csv
    rows = list(csv.reader(open(csv_path)))
    start = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    hdr = rows[start]
    ii, ki, mi, vi = (hdr.index(k) for k in ("ID", "Kernel Name", "Metric Name", "Metric Value"))
    units_of = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9,
                "ns": 1e-3, "nsecond": 1e-3, "us": 1, "usecond": 1, "ms": 1e3, "msecond": 1e3}
    ui = hdr.index("Metric Unit")
    per = {}
    for r in rows[start + 1:]:
        if len(r) <= vi or "k_pm_r" not in r[ki]:
            continue
        v = float(r[vi].replace(",", "")) * units_of.get(r[ui], 1)
        per.setdefault(r[ii], {})[r[mi]] = v
    launches = len(per)
    rd = sum(x["dram__bytes_read.sum"] for x in per.values())
    wr = sum(x["dram__bytes_write.sum"] for x in per.values())
    us = sum(x["gpu__time_duration.sum"] for x in per.values())
    n0 = lattice_sizes(PARAMS, W_IMG, H_IMG)[0]
    units = launches * TRAFFIC_PAIRS * n0 / 2          # one colour of one direction each
    rec = {"kernel": "k_pm_r", "workload": WORKLOAD, "pairs": TRAFFIC_PAIRS, "level": 0,
           "launches": launches, "dram_read_bytes": rd, "dram_write_bytes": wr,
           "ncu_time_us": us, "seed_units": units, "bytes_per_seed_unit": (rd + wr) / units,
           "command": TRAFFIC_CMD,
           "note": "DRAM bytes of level-0 search launches per seed and iteration; bench.py "
                   "multiplies by its seed-iterations per step (all levels) and divides by its "
                   "search launches per step (coarse levels assumed to move as many bytes per "
                   "seed as level 0, an upper bound: their data sit in L2)",
           "device_sha256": device_hash(),
           "hash_note": "sha256 of pm_row.cu above the line " + json.dumps(DEVICE_MARK.strip())}
    with open(TRAFFIC_REC, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    return rec


def pm_traffic_per_launch(units, launches):
    """DRAM bytes per search launch: the committed record's bytes per seed
    unit times this step's `units` over its `launches`; None when the device
    code of the search kernel changed since the capture."""
    try:
        r = json.load(open(TRAFFIC_REC))
    except (OSError, ValueError):
        return None
    if r.get("device_sha256") != device_hash() or launches <= 0:
        return None
    return r["bytes_per_seed_unit"] * units / launches


# ------------------------------------------------- HBM-bound stages (a1-a3, a7-a9)
def visit_levels(levels, rounds):
    """Levels of the visits in order (reading R15): m, then (m-1, m) x N,
    then m-1 down to 0."""
    m = levels - 1
    if m == 0:
        return [0]
    seq = [m] + [m - 1, m] * rounds + list(range(m - 1, -1, -1))
    return seq


def hbm_stage_bytes(prm, w, h, pairs, matches_total):
    """Compulsory DRAM bytes per step of the stages around the search, for
    `pairs` pairs of w x h images (both images of a pair the same size):
      pyramid (a1-a3): each input image read once (3 B/px) and, per scheme and
        level, the descriptor and its split-byte copy written once
        (2 x 2C x 2 B/px);
      fields (a7-a9): per visit the consistency check reads both fields
        (5 B per seed: u and flags) and writes flags (1 B) in each direction,
        the transfer reads the source field (5 B per seed) and writes the
        destination field (13 B: u, cost, flags); the final filter reads the
        level-0 forward field (5 B per seed), writes its keep mask (1 B per
        seed) and the match rows (16 B each)."""
    L, sig = prm["levels"], prm["seed_stride"]
    C = 3 if prm["color"] == 1 else 1
    nsch = 2 if (C == 3 and prm.get("cs_sched", 0) == 0) else 1
    dims = [(w, h)]
    for _ in range(1, L):
        dims.append(((dims[-1][0] + 1) // 2, (dims[-1][1] + 1) // 2))
    px = sum(a * b for a, b in dims)
    pyr = 2 * pairs * (3 * w * h + nsch * 2 * (2 * C) * 2 * px)
    c = sig // 2
    n = [((a - 1 - c) // sig + 1) * ((b - 1 - c) // sig + 1) for a, b in dims]
    seq = visit_levels(L, prm.get("refine_rounds", 2))
    f = 0
    for v, l in enumerate(seq):
        f += 2 * n[l] * (5 + 5 + 1)                      # consistency, both directions
        if v > 0:
            f += 2 * (n[seq[v - 1]] * 5 + n[l] * 13)     # transfer, both directions
    f += n[0] * (5 + 1)                                  # final filter (per pair)
    return {"pyramid": pyr, "fields": pairs * f + 16 * matches_total}


def tc_steps(P, sigma):
    """K steps (pixel pairs) of the tensor-core initialisation for a P x P
    patch: the library's pairing (raster order, first later pixel also later
    in phase order, else a zero partner), restated to count MMAs."""
    used = [False] * (P * P)
    key = lambda i: ((((i // P) % sigma) * sigma + (i % P) % sigma), (i // P) // sigma,
                     (i % P) // sigma)
    n = 0
    for i in range(P * P):
        if used[i]:
            continue
        used[i] = True
        n += 1
        for j in range(i + 1, P * P):
            if not used[j] and key(j) > key(i):
                used[j] = True
                break
    return n


def init_tc_flops(prm, w, h, pairs):
    """Tensor-core initialisation per step: (executed, useful) fp16 FLOPs.
    Executed: every MMA issued (tiles of 128 flattened seeds x 160 flattened
    centres x 16, four split products per K step); useful: the four split
    products of the real (seed, centre) pairs over the six channels."""
    L, sig = prm["levels"], prm["seed_stride"]
    for _ in range(L - 1):
        w, h = (w + 1) // 2, (h + 1) // 2
    c = sig // 2
    nx, ny = (w - 1 - c) // sig + 1, (h - 1 - c) // sig + 1
    ex = us = 0
    for P in (prm["patch_fwd"], prm["patch_bwd"]):
        Wu = nx + (P - 1) // sig
        mt = -(-ny * Wu // 128)
        nt = -(-h * (w + P - 1) // 160)
        ex += mt * nt * tc_steps(P, sig) * 4 * 2 * 128 * 160 * 16
        us += nx * ny * w * h * P * P * 6 * 4 * 2
    return pairs * ex, pairs * us


def measured_tensor_peak():
    """Dense bf16 TFLOP/s, sustained (the fp16 rate is the same)."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
                     ["bf16_tflops_sustained"]), "measured (cuBLAS bf16, sustained)"
    except (OSError, ValueError, KeyError):
        return 1700.0, "fallback"


def measured_hbm_peak():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


# ------------------------------------------------------------- multi-rank
def rank_seeds(rank, batch):
    """Synthetic pair seeds of one rank: disjoint across ranks."""
    return [10 * rank * batch + k for k in range(batch)]


def max_over_ranks(value, world, device=None):
    """Max of a float over all ranks (timing only; no data-path collective)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu, self.p, self.path = gpu, None, None

    def start(self):
        try:
            self.path = "/tmp/pgm_clocks_%d.csv" % os.getpid()
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        self.p.wait()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in open(self.path):
            v = [x.strip() for x in ln.split(",")]
            if len(v) < 9:
                continue
            try:
                sm.append(float(v[1])); mx.append(float(v[2]))
            except ValueError:
                continue
            for nm, flag in zip(names, v[5:9]):
                if flag.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


# --------------------------------------------------------------- GPU arm
def optional_section(name, fn):
    """Run one of the line's supplementary measurements; an exception there is
    reported in its place (and on stderr) instead of ending the run, so that
    the headline numbers, measured before, are still printed."""
    try:
        return fn()
    except Exception as e:                        # reported, not hidden
        import traceback
        traceback.print_exc()
        return {"error": "%s: %s: %s" % (name, type(e).__name__, e)}


def run_ours(a):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        # the oracle leg runs first, before this process touches the GPU
        cores = os.cpu_count() or 1
        seeds = rank_seeds(0, a.cpu_pairs or a.batch)
        procs = min(cores, len(seeds))
        r, t, _ = oracle_rate(seeds, procs)
        one_cb, one_seq = oracle_one_core(seeds[0])
        cpu = {"value": r, "unit": "pairs/s", "cores": procs, "kind": "oracle",
               "sample": "the timed step's %d sintel-like 1024x436 PGM-C pairs, one per "
                         "process, %.1f s of oracle time per process" % (len(seeds), t),
               "one_core_pairs_per_s": one_cb, "one_core_scan_order_pairs_per_s": one_seq,
               "one_core_sample": "pair seed %d on one process, checkerboard schedule and the "
                                  "paper's scan order" % seeds[0]}

    from paper_1704_03217_gb300 import build as pbuild
    pbuild.build()
    from paper_1704_03217_gb300 import api, synth, _lib

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    B = a.batch
    P = dict(PARAMS, **VARIANTS.get(a.variant, {}))
    prm = api.Params(**P)
    pairs = [synth.sintel_like_pair(sd, W_IMG, H_IMG) for sd in rank_seeds(rank, B)]
    imgs1 = [torch.from_numpy(p[0]).to(dev) for p in pairs]
    imgs2 = [torch.from_numpy(p[1]).to(dev) for p in pairs]
    m = api.PairMatcher(prm, W_IMG, H_IMG, batch=B, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    sids = [rank * B + k for k in range(B)]

    # result-invariant launch knobs tuned on this workload, then the whole
    # step is captured once as a CUDA graph and replayed
    from paper_1704_03217_gb300 import tune
    if a.tuning:
        tune.set(*(int(x) for x in a.tuning.split(",")))
        tuned = tune.get()
    else:
        tuned, _ = tune.autotune(m, imgs1, imgs2, reps=2, slacks=(2, 4, 6), chunks=(16, 32),
                                 tiles=(4, 8, 16))
    per_step_launches = m.capture(imgs1, imgs2, sids)

    def step():
        m.replay()

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()

    # -------- device-timed region
    L = _lib.load()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(a.steps)]
    clocks = Clocks(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    for k in range(a.steps):
        flush.fill_(k & 0xff)                      # L2 flush, outside the events
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    launches = per_step_launches * a.steps
    clk = clocks.stop()
    ms = sum(s.elapsed_time(e) for s, e in ev)
    ms_max = max_over_ranks(ms, world, dev)
    value = world * B * a.steps / (ms_max * 1e-3)
    nominal = api.nominal_evals(prm, W_IMG, H_IMG, W_IMG, H_IMG)
    counts = [int(c) for c in m.count[:, 0].tolist()]

    # -------- end-to-end through the public API with host buffers: every step
    # copies its 2B images in from pinned host memory, matches them (graph
    # replay) and copies its matches back out; two steps are in flight (two
    # matchers, one H2D stream, the compute stream, one D2H stream), so the
    # copies of one step overlap the matching of the other, as in serving
    host1 = [torch.from_numpy(p[0]).pin_memory() for p in pairs]
    host2 = [torch.from_numpy(p[1]).pin_memory() for p in pairs]
    m2 = api.PairMatcher(prm, W_IMG, H_IMG, batch=B, device=dev)
    imgs1b = [torch.empty_like(x) for x in imgs1]
    imgs2b = [torch.empty_like(x) for x in imgs2]
    for i in range(B):
        imgs1b[i].copy_(imgs1[i])
        imgs2b[i].copy_(imgs2[i])
    m2.capture(imgs1b, imgs2b, sids)
    sets = [(m, imgs1, imgs2), (m2, imgs1b, imgs2b)]
    out_rows = [torch.empty(m.rows.shape, dtype=torch.int32).pin_memory() for _ in range(2)]
    out_cnt = [torch.empty(m.count.shape, dtype=torch.int32).pin_memory() for _ in range(2)]
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_done = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    e2e_steps = max(4, a.steps // 2)

    def e2e_run(nsteps):
        for k in range(nsteps):
            sset = k & 1
            mm, i1, i2 = sets[sset]
            if k >= 2:
                ev_out[sset].synchronize()            # the host has this set's last matches
            with torch.cuda.stream(s_in):
                if k >= 2:
                    s_in.wait_event(ev_done[sset])    # its last replay read the images
                for i in range(B):
                    i1[i].copy_(host1[i], non_blocking=True)
                    i2[i].copy_(host2[i], non_blocking=True)
                ev_in[sset].record(s_in)
            stream.wait_event(ev_in[sset])
            flush.fill_(k & 0xff)                     # L2 flush, inside the timed region
            mm.replay()
            ev_done[sset].record(stream)
            with torch.cuda.stream(s_out):
                s_out.wait_event(ev_done[sset])
                out_cnt[sset].copy_(mm.count, non_blocking=True)
                out_rows[sset].copy_(mm.rows, non_blocking=True)
                ev_out[sset].record(s_out)
        torch.cuda.synchronize()

    e2e_run(2)                                        # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_run(e2e_steps)
    e2e_t = time.perf_counter() - t0
    assert [int(c) for c in out_cnt[0][:, 0].tolist()] == counts   # same matches as the timed steps
    h2d = sum(x.numel() for x in host1) + sum(x.numel() for x in host2)
    d2h = out_rows[0].numel() * 4 + out_cnt[0].numel() * 4
    e2e = world * B * e2e_steps / max_over_ranks(e2e_t, world, dev)

    # -------- per-kernel times (profiling pass: eager launches, each kernel
    # class bracketed by events, both directions on one stream)
    import ctypes as C
    L.pgm_profile_enable(1)
    prof_steps = 2
    for _ in range(prof_steps):
        flush.fill_(1)
        m.enqueue(imgs1, imgs2, sids)
    torch.cuda.synchronize()
    kms = (C.c_double * 7)()
    kn = (C.c_int64 * 7)()
    L.pgm_profile_read(kms, kn)
    L.pgm_profile_enable(0)
    kernel_ms = {name: kms[i] / prof_steps for i, name in enumerate(_lib.K_CLASSES)}
    kernel_launches = {name: kn[i] // prof_steps for i, name in enumerate(_lib.K_CLASSES)}
    ev_counts = [w.evals() for w in m.ws]
    nch = 6 if P["color"] == 1 else 2
    el_pm = sum(e["pm"][0] * P["patch_fwd"] ** 2 * nch + e["pm"][1] * P["patch_bwd"] ** 2 * nch
                for e in ev_counts)                     # per step
    evals_step = {"pm": sum(sum(e["pm"]) for e in ev_counts),
                  "cost": sum(sum(e["cost"]) for e in ev_counts),
                  "init": sum(sum(e["init"]) for e in ev_counts),
                  "pm_global": sum(sum(e["pm_global"]) for e in ev_counts)}
    pm_launch_ms = kernel_ms["pm"] / max(1, kernel_launches["pm"])
    # the search's share of the timed (graph, overlapped) step: its share of
    # the serial kernel time applied to the timed step time
    serial_ms = sum(kernel_ms.values())
    pm_share = kernel_ms["pm"] / serial_ms if serial_ms > 0 else 0.0
    pm_step_ms = pm_share * ms_max / a.steps
    hb = hbm_stage_bytes(P, W_IMG, H_IMG, B, sum(counts))
    hpeak, hsrc = measured_hbm_peak()
    hbm_stages = {"peak_GBps": hpeak, "peak_source": hsrc + " (copy bandwidth)",
                  "note": "compulsory bytes per step over the stage's kernel time from the "
                          "profiling pass (definitions in bench.hbm_stage_bytes)"}
    for name, ms in (("pyramid", kernel_ms["pyramid"]),
                     ("fields", kernel_ms["consist"] + kernel_ms["transfer"] + kernel_ms["filter"])):
        gbs = hb[name] / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
        hbm_stages[name] = {"bytes_per_step": hb[name], "ms_per_step": ms, "GBps": gbs,
                            "frac": gbs / hpeak}
    el_per_launch = el_pm / max(1, kernel_launches["pm"])
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    sm_mhz = (clk or {}).get("sm_max_mhz") or 2070.0
    # integer multiply pipe: 64 lanes/clk/SM, one int16 x int16 element-MAC per lane-op
    peak_tmac = sms * 64 * sm_mhz * 1e6 / 1e12
    achieved_tmac = el_per_launch / (pm_launch_ms * 1e-3) / 1e12
    l1_gbs = 2 * el_per_launch / (pm_launch_ms * 1e-3) / 1e9
    l1_peak = sms * 128 * sm_mhz * 1e6 / 1e9
    traffic = (pm_traffic_per_launch(search_units(P, W_IMG, H_IMG, B), kernel_launches["pm"])
               if not a.variant else None)
    overlap_tmac = el_pm / (pm_step_ms * 1e-3) / 1e12 if pm_step_ms > 0 else 0.0
    init_roof = None
    if P["color"] == 1 and P["descriptor"] != 1 and kernel_ms["init"] > 0:
        ex, us = init_tc_flops(P, W_IMG, H_IMG, B)
        tpk, tsrc = measured_tensor_peak()
        sec = kernel_ms["init"] * 1e-3
        init_roof = {"kernel": "k_init_tc (exhaustive coarsest-level initialisation, tcgen05)",
                     "bound": "tensor", "achieved": ex / sec / 1e12, "peak": tpk,
                     "unit": "TFLOP/s (fp16 MMA)", "frac": ex / sec / 1e12 / tpk,
                     "peak_source": tsrc, "useful_TFLOPs": us / sec / 1e12,
                     "useful_frac": us / sec / 1e12 / tpk,
                     "element_Tmac_per_s": us / 8 / sec / 1e12,
                     "ms_per_step": kernel_ms["init"],
                     "launches_per_step": kernel_launches["init"],
                     "note": "achieved: every MMA issued (128 x 160 x 16 tiles, 8-channel "
                             "pixels, four split products per element); useful: the split "
                             "products of the real seed-centre pairs; element_Tmac_per_s: "
                             "int16 element MACs of Eq. 3's cross term per second; time of "
                             "the init class (clear, MMA and unpack launches)"}

    def run_variants():
        variants = {}
        for name, kw in VARIANTS.items():
            pv = prm.replace(**kw)
            mv = api.PairMatcher(pv, W_IMG, H_IMG, batch=B, device=dev)
            mv.capture(imgs1, imgs2, sids)
            for _ in range(2):
                mv.replay()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            tot = 0.0
            for k in range(max(3, a.steps // 4)):
                flush.fill_(k)
                e0.record(stream)
                mv.replay()
                e1.record(stream)
                torch.cuda.synchronize()
                tot += e0.elapsed_time(e1)
            variants[name] = {"pairs_per_s": B * max(3, a.steps // 4) / (tot * 1e-3),
                              "gcand_evals_per_s": api.nominal_evals(pv, W_IMG, H_IMG, W_IMG, H_IMG)
                              * B * max(3, a.steps // 4) / (tot * 1e-3) / 1e9}
            if kw.get("descriptor") == 1:
                variants[name]["roofline"] = bit_search_roofline(api, _lib, pv, mv, imgs1, imgs2,
                                                                 sids, flush, l1_peak)
            del mv
        variants["note"] = ("pairs/s of the same 16 pairs, whole step graph-replayed; "
                            "gcand_evals_per_s nominal")
        return variants

    variants = {}
    if not a.no_variants:
        variants = optional_section("variants", run_variants)

    workloads = None
    if not a.no_variants and rank == 0:
        workloads = optional_section(
            "workloads", lambda: run_workloads(api, prm, dev, flush, a.steps))

    batched = None
    if not a.no_variants and rank == 0:
        batched = optional_section("batched", lambda: run_batched(api, prm, dev))

    interp = None
    if not a.no_variants and rank == 0:
        interp = optional_section(
            "interpolation", lambda: run_interp(api, prm, m, dev, [p[2] for p in pairs]))

    serving = None
    if a.serve > 0 and rank == 0:
        serving = optional_section("serving", lambda: run_serving(api, prm, a.serve, dev))

    if rank == 0:
        cfg = config_dict(B, world)
        if a.variant:
            cfg["variant"] = dict(VARIANTS[a.variant], name=a.variant)
        line = {
            "metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms_max / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32", "data": "synthetic",
            "config": cfg,
            "launch": {"form": "whole step captured once as a CUDA graph, replayed",
                       "tuning": {"window_slack": tuned[0], "pairs_per_launch": tuned[1],
                                  "tile_w": tuned[2]}},
            "gcand_evals_per_s": nominal * value / 1e9,
            "gcand_evals_per_s_evaluated": (evals_step["pm"] + evals_step["cost"])
            * a.steps / (ms_max * 1e-3) / 1e9,
            "evals_note": "gcand_evals_per_s: nominal evaluations (every candidate of the "
                          "method's schedule) x pairs/s; _evaluated: candidates the kernels "
                          "scored (search + cost refresh), the rest being duplicates or "
                          "outside the image, skipped without changing a result",
            "nominal_evals_per_pair": nominal,
            "matches_per_pair": sum(counts) / len(counts),
            "e2e": {"value": e2e, "unit": "pairs/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches),
            "roofline": {"bound": "alu", "kernel": "k_pm_r (propagation + limited random search)",
                         "achieved": achieved_tmac, "peak": peak_tmac,
                         "unit": "Tmac/s (int16 x int16 element multiply-accumulates)",
                         "frac": achieved_tmac / peak_tmac, "traffic": traffic,
                         "peak_source": "derived: %d SMs x 64 integer-multiply lanes x %.0f MHz"
                                        % (sms, sm_mhz),
                         "l1_GBps": l1_gbs, "l1_peak_GBps": l1_peak, "l1_frac": l1_gbs / l1_peak,
                         "pm_ms_per_launch": pm_launch_ms,
                         "pm_launches_per_step": kernel_launches["pm"],
                         "pm_share_of_serial_kernel_time": pm_share,
                         "pm_ms_in_timed_step": pm_step_ms,
                         "frac_overlap_credited": overlap_tmac / peak_tmac,
                         "note": "achieved from per-launch event times of the profiling pass "
                                 "(directions serial); frac_overlap_credited divides by the "
                                 "search's share of the timed, overlapped step instead"},
            "init_roofline": init_roof,
            "hbm_stages": hbm_stages,
            "kernel_ms_per_step": kernel_ms, "kernel_launches_per_step": kernel_launches,
            "evals_per_step": evals_step,
            "variants": variants,
            "workloads": workloads,
            "batched": batched,
            "interpolation": interp,
            "serving": serving,
            "clocks": clk,
            "cpu_baseline": cpu,
            "paper_timings": PAPER_TIMINGS,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


# the other two single-pair workloads: method parameters as the oracle's
# accuracy margins use them (Sec. IV defaults where the workload fixes none)
C1_PARAMS = dict(levels=3, seed_stride=3, patch_fwd=8, patch_bwd=8, color=0, descriptor=0,
                 iters_coarse=6, iters_fine=6, refine_rounds=2, rs_W=2)
C3_PARAMS = dict(PARAMS)


def _replay_rate(mv, flush, stream, reps, pairs):
    """Pairs/s of a captured matcher: `reps` replays, L2 flushed before each."""
    import torch
    for _ in range(2):
        mv.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tot = 0.0
    for k in range(reps):
        flush.fill_(k)
        e0.record(stream)
        mv.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1)
    return pairs * reps / (tot * 1e-3), tot / reps


def run_workloads(api, prm, dev, flush, steps):
    """Throughput lines of the 256x192 gray noise-affine pair and the KITTI-
    shaped 1242x375 RGB pair, from resident device images, each whole batch
    captured as one CUDA graph; the gray pair also one pair per replay (the
    plain single-pair form)."""
    import torch
    from paper_1704_03217_gb300 import synth
    stream = torch.cuda.current_stream(dev)
    reps = max(3, steps // 4)
    out = {}
    # c1: 64 pairs per step, and one pair per graph replay
    pc1 = api.Params(**C1_PARAMS)
    pairs = [synth.config_pair("c1", sd) for sd in range(64)]
    i1 = [torch.from_numpy(p[0]).to(dev) for p in pairs]
    i2 = [torch.from_numpy(p[1]).to(dev) for p in pairs]
    mv = api.PairMatcher(pc1, 256, 192, batch=64, device=dev)
    mv.capture(i1, i2, list(range(64)))
    rate, ms = _replay_rate(mv, flush, stream, reps, 64)
    ms1 = api.PairMatcher(pc1, 256, 192, batch=1, device=dev)
    a1, a2 = i1[0].clone(), i2[0].clone()
    ms1.capture([a1], [a2], [0])
    ms1.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(64):
        a1.copy_(i1[k]); a2.copy_(i2[k])
        ms1.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    out["c1 256x192 gray noise-affine"] = {
        "params": C1_PARAMS, "pairs_per_step": 64, "ms_per_step": ms, "pairs_per_s": rate,
        "single_pair_pairs_per_s": 64 / (e0.elapsed_time(e1) * 1e-3),
        "gcand_evals_per_s": api.nominal_evals(pc1, 256, 192, 256, 192) * rate / 1e9}
    del mv, ms1
    # c3: 16 KITTI-shaped pairs, full-gradient and direction-only descriptors
    pairs = [synth.config_pair("c3", sd) for sd in range(16)]
    i1 = [torch.from_numpy(p[0]).to(dev) for p in pairs]
    i2 = [torch.from_numpy(p[1]).to(dev) for p in pairs]
    for name, kw in (("PGM-C", {}), ("PGM-CD", dict(descriptor=1))):
        pv = api.Params(**dict(C3_PARAMS, **kw))
        mv = api.PairMatcher(pv, 1242, 375, batch=16, device=dev)
        mv.capture(i1, i2, list(range(16)))
        rate, ms = _replay_rate(mv, flush, stream, reps, 16)
        out["c3 1242x375 RGB kitti-like " + name] = {
            "params": dict(C3_PARAMS, **kw), "pairs_per_step": 16, "ms_per_step": ms,
            "pairs_per_s": rate,
            "gcand_evals_per_s": api.nominal_evals(pv, 1242, 375, 1242, 375) * rate / 1e9}
        del mv
    out["note"] = "L2 flushed before every timed replay; gcand_evals_per_s nominal"
    return out


def bit_search_roofline(api, lib, pv, mv, imgs1, imgs2, sids, flush, l1_peak):
    """The bit-plane search kernels (direction descriptor) against the
    L1/shared roofline: per evaluated candidate the target patch's two
    bit-planes, P^2 2C / 4 bytes (P^2 2C values of 2 bits), over the search
    time per step from a profiling pass (CUDA events around every launch)."""
    import ctypes as C
    import torch
    L = lib.load()
    L.pgm_profile_enable(1)
    for _ in range(2):
        flush.fill_(2)
        mv.enqueue(imgs1, imgs2, sids)
    torch.cuda.synchronize()
    kms = (C.c_double * 7)()
    kn = (C.c_int64 * 7)()
    L.pgm_profile_read(kms, kn)
    L.pgm_profile_enable(0)
    ms = kms[lib.K_CLASSES.index("pm")] / 2
    nch = 6 if pv.color == 1 else 2
    ev = [w.evals() for w in mv.ws]
    nbytes = sum(e["pm"][0] * pv.patch_fwd ** 2 * nch / 4 + e["pm"][1] * pv.patch_bwd ** 2 * nch / 4
                 for e in ev)
    gbs = nbytes / (ms * 1e-3) / 1e9 if ms > 0 else 0.0
    return {"bound": "l1", "kernel": "k_pm_s / k_pm_b (bit-plane search)", "achieved": gbs,
            "peak": l1_peak, "unit": "GB/s (2-bit target-patch values read per evaluation)",
            "frac": gbs / l1_peak, "pm_ms_per_step": ms,
            "bytes_per_eval_fwd": pv.patch_fwd ** 2 * nch / 4,
            "bytes_per_eval_bwd": pv.patch_bwd ** 2 * nch / 4}


def run_batched(api, prm, dev, n=64, reps=3):
    """The mixed-size batch: n pairs of sizes drawn uniformly from 320x240,
    640x480, 1024x436, 1242x375 and 1920x1080, from resident device images,
    (a) in shared launches (batched pyramids, matching in launches of up to 32
    pairs, batched filter) captured once as a CUDA graph and replayed, and
    (b) in the plain form: each pair's two pyramids, its match and its filter
    launched one pair after the other.  Pairs/s from CUDA events over `reps`
    runs each; both forms must export the same matches.  The per-level
    iteration schedule of the shared form is then autotuned on the batch
    (tune.tune_schedule: fastest schedule whose accuracy against the pairs'
    ground truth stays within tune.MARGINS of the paper's schedule)."""
    import numpy as np
    import torch
    from paper_1704_03217_gb300 import evaluate, synth, tune
    rng = np.random.default_rng(77)
    pairs = []
    for _ in range(n):                       # RGB pairs for the colour descriptor
        w, h = synth.BATCH_SIZES[int(rng.integers(len(synth.BATCH_SIZES)))]
        pairs.append(synth.sintel_like_pair(int(rng.integers(1 << 30)), w, h,
                                            t_max=min(150.0, w / 8)))
    i1 = [torch.from_numpy(np.ascontiguousarray(p[0])).to(dev) for p in pairs]
    i2 = [torch.from_numpy(np.ascontiguousarray(p[1])).to(dev) for p in pairs]
    P1 = [api.Pyramid(prm, x.shape[1], x.shape[0], dev) for x in i1]
    P2 = [api.Pyramid(prm, x.shape[1], x.shape[0], dev) for x in i2]
    W = [api.Workspace(prm, q1.w, q1.h, q2.w, q2.h, dev) for q1, q2 in zip(P1, P2)]
    caps = [w.layout(0, 0)[0] * w.layout(0, 0)[1] for w in W]
    rows = [torch.empty((max(c, 1), 4), dtype=torch.int32, device=dev) for c in caps]
    cnt = [torch.zeros(1, dtype=torch.int32, device=dev) for _ in range(n)]
    sids = list(range(n))

    def shared(p):
        api.build_pyramids(p, i1 + i2, P1 + P2)
        api.match_batch(p, P1, P2, sids, W)
        api.filter_batch(p, W, rows, cnt)

    def plain(p):
        for k in range(n):
            P1[k].build(i1[k])
            P2[k].build(i2[k])
            api.match(p, P1[k], P2[k], sids[k], W[k])
            api.filter_into(p, W[k], rows[k], cnt[k])

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def graph_ms(p):
        shared(p)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            shared(p)
        return timed(g.replay)

    def accuracy(p):
        shared(p)
        torch.cuda.synchronize()
        acc = [evaluate.match_accuracy(rows[k][:int(cnt[k].item())].cpu().numpy(), pairs[k][2],
                                       caps[k]) for k in range(n)]
        return {m: float(np.mean([a[m] for a in acc])) for m in ("epe", "outliers_3px", "density")}

    t_shared = graph_ms(prm)
    got_shared = [int(c.item()) for c in cnt]
    t_plain = timed(lambda: plain(prm))
    got_plain = [int(c.item()) for c in cnt]
    assert got_shared == got_plain, "batched and single-pair matches differ"
    best, table = tune.tune_schedule(prm, graph_ms, accuracy)
    sizes = sorted({"%dx%d" % (p[0].shape[1], p[0].shape[0]) for p in pairs})
    ref = tuple(tune.SCHEDULES_L5[0])
    return {"pairs": n, "sizes": sizes, "data": "synthetic Sintel-like RGB pairs",
            "batched_ms": t_shared, "batched_pairs_per_s": n / (t_shared * 1e-3),
            "plain_ms": t_plain, "plain_pairs_per_s": n / (t_plain * 1e-3),
            "speedup": t_plain / t_shared,
            "schedule_tuning": {
                "paper_schedule": list(ref), "tuned_schedule": list(best),
                "margins": tune.MARGINS,
                "tuned_batched_pairs_per_s": n / (table[best]["ms"] * 1e-3),
                "tuned_speedup_vs_plain": t_plain / table[best]["ms"],
                "accuracy_paper": {k: table[ref][k] for k in ("epe", "outliers_3px", "density")},
                "accuracy_tuned": {k: table[best][k] for k in ("epe", "outliers_3px", "density")},
                "table": [dict(schedule=list(sch), **r) for sch, r in table.items()],
                "note": "levels listed from 0 (full resolution); accuracy of the exported "
                        "matches against the generator's flow; every schedule is bit-exact "
                        "with the oracle run at the same counts"}}


def run_interp(api, prm, m, dev, flows, reps=3):
    """Sparse-to-dense interpolation (pgm_interpolate) of the timed step's
    exported matches, pair by pair on the device: ms per 1024x436 pair from
    CUDA events (each call synchronises its stream while the relaxation runs)
    and the dense flow's end-point error against the generator's flow."""
    import numpy as np
    import torch
    ip = api.InterpParams()
    n = min(4, m.batch)
    ws = None
    for k in range(n):                         # warm-up, and the workspace
        _, ws = api.interpolate(prm, m.p1[k], m.rows[k], m.count[k], ip, ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        for k in range(n):
            flow, ws = api.interpolate(prm, m.p1[k], m.rows[k], m.count[k], ip, ws)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / (reps * n)
    epe = []
    for k in range(n):
        flow, ws = api.interpolate(prm, m.p1[k], m.rows[k], m.count[k], ip, ws)
        epe.append(np.hypot(*(flow.cpu().numpy() - flows[k]).transpose(2, 0, 1)))
    e = np.concatenate([x.ravel() for x in epe])
    return {"pairs": n, "k": ip.k, "ms_per_pair": ms, "mpix_per_s": W_IMG * H_IMG / (ms * 1e3),
            "epe_mean": float(e.mean()), "epe_median": float(np.median(e)),
            "outliers_3px": float((e > 3).mean()),
            "note": "k geodesic nearest matches, LA (matches above 2.2 % of the pixels); "
                    "median EPE is the typical pixel, the mean carries occluded regions"}


def run_serving(api, prm, n, dev):
    """Continuous batching of Poisson arrivals (mean 200 pairs/s) of pairs of
    640x480, 1280x720, 1920x1080 and 1024x436 (8 distinct pairs per size)
    under a 40 GB budget, next to the plain form (one pair per launch, one at
    a time) on the same requests; and the continuous form again under a
    budget of three 1920x1080 requests, where admission waits for memory."""
    import torch
    from paper_1704_03217_gb300 import serve
    out = {"offered_pairs_per_s": 200.0, "budget_gb": 40, "requests": n,
           "sizes": ["640x480", "1280x720", "1920x1080", "1024x436"], "distinct_pairs": 32}
    reqs0 = serve.poisson_requests(7, 200.0, n, pool=8)
    warm = serve.poisson_requests(8, 1e6, 4, pool=1)              # warm-up, not measured
    big = None
    for name, max_batch, streams, budget in (("continuous", 16, 3, 40 << 30), ("plain", 1, 1, 40 << 30),
                                             ("continuous, budget-bound", 16, 3, None)):
        reqs = [serve.Request(r.rid, r.arrival, r.img1, r.img2, stream_id=r.stream_id) for r in reqs0]
        ex = serve.GpuExecutor(prm, streams=streams, device=dev)
        if budget is None:
            big = max(ex.bytes_of(r) for r in reqs)
            budget = 3 * big
        serve.serve(warm, serve.Scheduler(budget, max_batch, ex.bytes_of), ex)
        torch.cuda.synchronize()
        sch = serve.Scheduler(budget, max_batch, ex.bytes_of)
        t0 = time.perf_counter()
        done = serve.serve(reqs, sch, ex)
        wall = time.perf_counter() - t0
        r = serve.summary(done, wall)
        r["max_batch"], r["streams"] = max_batch, streams
        r["budget_gb"] = budget / 2 ** 30
        r["peak_budget_gb"] = sch.peak / 2 ** 30
        out[name] = r
        del ex
    out["p50_ms"], out["p99_ms"] = out["continuous"]["p50_ms"], out["continuous"]["p99_ms"]
    return out


def main():
    a = parse()
    if a.traffic_record:
        print(json.dumps(write_traffic_record(a.traffic_record)))
        return 0
    if a.impl == "reference":
        return run_reference(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
