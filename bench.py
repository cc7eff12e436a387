#!/usr/bin/env python
"""Benchmark: pixels/s of DOPE ADMM to convergence on one GB300 (per rank).

Workload (default "ellipsoids256"): the 256x256x128 volume (D x H x W =
128 x 256 x 256, three nested ellipsoids, bias field, Rician-like noise),
6-connected contrast-sensitive Potts, 8x16x16 sub-regions (K = 4096),
lambda 3; one step = one solve to convergence (Algorithm 1, mu0 = 500,
mu_fact = 1.05, eps = 1e-3).  Inputs are synthetic (seeded), resident in HBM
for `value`; `e2e` goes through the C-ABI with pinned host buffers,
host<->device copies inside the timed region.  The L2 is flushed (a 256 MiB
write) before every timed step, outside the step's events.  The line also
carries the energy gap and the Dice coefficient against the global min-cut
(whole-volume BK), the oracle's own solve (cpu_baseline, oracle_match), and,
as sub-objects, the 512x512 RGB image line (lambda 1, 4, 16), the GPU
potentials and the serving comparison.

--impl reference times the oracle (the plain CPU implementation of the
method: BK per block + FP64 ADMM, OpenMP over blocks) on a bounded sample of
the same workload (reference_sample).
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

LAMBDAS = (1.0, 4.0, 16.0)
ARENA_BYTES = 0        # serving: the server's device arena (0: its default, 3/4 of the free memory)
METRIC = "pixels/sec to ADMM convergence"
PROFILES = os.path.join(ROOT, "profiles")
KERNEL_SRC = os.path.join(ROOT, "paper_1704_03116_gb300", "csrc", "dope_kernels.cuh")


def max_over_ranks(value, world, device="cuda"):
    """The largest value over the ranks (a job's time is its slowest rank's);
    the value itself for one process."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, seconds):
    """Whole-job throughput of `world` replicas that each processed
    units_per_rank in at most `seconds` (the slowest rank's time)."""
    return world * units_per_rank / seconds


def workload(name):
    from paper_1704_03116_gb300 import inputs
    if name == "ellipses512":
        d = inputs.ellipses_rgb(lam=1.0)
        return [dict(d, lam=lam) for lam in LAMBDAS], {
            "workload": "ellipses512x512_rgb_8conn_blocks32x32_lambda1,4,16", "grid": [512, 512],
            "connectivity": 8, "block": [32, 32], "lambdas": list(LAMBDAS), "mu0": 100.0,
            "mu_fact": 1.05, "eps": 1e-3}
    if name in ("ellipses512_size10", "ellipses512_size25"):
        # the paper's overlapping partitions: blocks grown by ~10% / 25% (Section 3);
        # 32x32 tiles grown by 2 / 4 pixels per side (36x36 / 40x40 blocks).  The
        # paper reports its 2-D results after a fixed 1 or 3 ADMM iterations
        # (Figure 2); with overlaps the literal iteration can cycle, so these
        # workloads run exactly 3 iterations.
        gr = 2 if name.endswith("10") else 4
        d = inputs.ellipses_rgb(lam=1.0)
        return [dict(d, lam=lam, grow=(gr, gr), max_iter=3) for lam in LAMBDAS], {
            "workload": f"ellipses512x512_rgb_8conn_blocks32x32_grow{gr}_lambda1,4,16_3iterations",
            "grid": [512, 512], "connectivity": 8, "block": [32, 32], "grow": [gr, gr],
            "lambdas": list(LAMBDAS), "mu0": 100.0, "mu_fact": 1.05, "eps": 1e-3, "max_iter": 3}
    if name in ("ellipses512_k5", "ellipses512_k7", "ellipses512_k9"):
        # Section 3's larger kernels: 5x5 / 7x7 / 9x9 square neighbourhoods
        ks = int(name[-1])
        conn = {5: 24, 7: 48, 9: 80}[ks]
        blk = (32, 32) if ks < 9 else (16, 32)       # 81-node kernels: smaller blocks fit shared memory
        d = inputs.ellipses_rgb(lam=1.0, conn=conn, block=blk)
        return [d], {"workload": f"ellipses512x512_rgb_kernel{ks}x{ks}_blocks{blk[0]}x{blk[1]}_lambda1",
                     "grid": [512, 512], "connectivity": conn, "block": list(blk), "lambdas": [1.0],
                     "mu0": 100.0, "mu_fact": 1.05, "eps": 1e-3}
    if name == "nonsubmodular1024":
        d = inputs.nonsubmodular_instance(size=1024)
        return [dict(d, lsa_steps=16)], {
            "workload": "nonsubmodular1024x1024_4conn_20pct_negative_blocks16x16_lsatr16",
            "grid": [1024, 1024], "connectivity": 4, "block": [16, 16], "lambdas": [1.0],
            "mu0": 100.0, "mu_fact": 1.05, "eps": 1e-3, "lsa_steps": 16}
    if name == "disk64":
        d = inputs.disk64()
        return [d], {"workload": "disk64x64_4conn_blocks16x16_lambda2", "grid": [64, 64],
                     "connectivity": 4, "block": [16, 16], "lambdas": [2.0], "mu0": 100.0,
                     "mu_fact": 1.05, "eps": 1e-3}
    if name == "ellipsoids256":
        d = inputs.ellipsoids3d()
        return [d], {"workload": "ellipsoids256x256x128_6conn_blocks16x16x8_lambda3",
                     "grid": [128, 256, 256], "connectivity": 6, "block": [8, 16, 16],
                     "lambdas": [3.0], "mu0": 500.0, "mu_fact": 1.05, "eps": 1e-3}
    raise SystemExit(f"unknown workload {name}")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def face_geometry(grid, block, conn):
    """(F, cross pairs per block): face pixels and (face pixel, cross edge)
    pairs of an interior block (used for the algorithmic byte counts)."""
    from paper_1704_03116_gb300.inputs import FWD_OFFSETS
    offs = FWD_OFFSETS[conn]
    b = tuple(block) if len(block) == 3 else (1,) + tuple(block)
    F = X = 0
    for z in range(b[0]):
        for y in range(b[1]):
            for x in range(b[2]):
                c = 0
                for (dz, dy, dx) in offs:
                    for s in (1, -1):
                        zz, yy, xx = z + s * dz, y + s * dy, x + s * dx
                        if not (0 <= zz < b[0] and 0 <= yy < b[1] and 0 <= xx < b[2]):
                            c += 1
                F += c > 0
                X += c
    return F, X


def algorithmic_bytes(n, k, F, X, nh):
    """Algorithmic HBM bytes of one launch of each hot kernel.
    Block solver, iteration >= 2: U 4 + Wl 4*nh + yhat read 1 + yhat write 1 per
    pixel, face y and a 16 per face pixel, neighbour face y 8 per cross pair.
    Block solver, iteration 1 (y = 1/2, a = 0): U, Wl, yhat write only.
    Face update: per face pixel own yhat 1, a 8, y and a written 16; per cross
    pair the neighbour's yhat 1 and the edge weight 4."""
    solve_first = n * (4 + 4 * nh + 1)
    solve_later = n * (4 + 4 * nh + 2) + k * F * 16 + k * X * 8
    update = k * F * (1 + 8 + 16) + k * X * (1 + 4)
    return solve_first, solve_later, update


def overlap_bytes(d):
    """Algorithmic HBM bytes of the overlapping-partition kernels, from the
    box nodes NB = sum_i q_i (every block copy of a pixel).  Block solve: per
    box node U 4 + Wl 4*nh + q 1 + y 8 + a 8 + yhat write 1.  Update (Eq. 10
    per pixel, Eq. 11 per box node): per pixel y write 8 + q 1 + Wl 4*nh, per
    box node yhat 1 + a 8 (gather) + yhat 1 + y 8 + a 8 + a write 8."""
    import oracle
    inst = oracle.quantise(d["grid"], d["conn"], d["block"], d["u"], d["wq"], d["lam"])
    grow = tuple(d.get("grow", (0,) * len(d["grid"])))
    ov = oracle.Overlap(inst, (0,) + grow if len(grow) == 2 else grow)
    nb = int(ov.q.sum())
    nh = d["conn"] // 2
    n = inst.n
    return nb * (22 + 4 * nh), n * (9 + 4 * nh) + nb * (9 + 25)


def kernel_traffic(kname, wname):
    """Per-launch DRAM bytes of the dominant kernel from the committed ncu
    summary of that kernel on that workload, or None when there is none or the
    kernel source changed since."""
    path = os.path.join(PROFILES, f"{kname}_{wname}.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    h = re.search(r"kernel_source_sha256:\s*([0-9a-f]+)", txt)
    if not m or not h:
        return None
    cur = hashlib.sha256(open(KERNEL_SRC, "rb").read()).hexdigest()
    return float(m.group(1)) if h.group(1) == cur else None


class Clocks:
    """nvidia-smi sampler running during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if not self.p:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def _oracle_solve(oracle, q, d):
    """The oracle's Algorithm 1 on one instance (overlapping partition if d has a grow)."""
    mi = d.get("max_iter", 1000)
    if d.get("lsa_steps"):
        return oracle.nsm_admm(q, d["mu0"], max_iter=mi, steps=d["lsa_steps"])
    if "grow" in d:
        g = tuple(d["grow"])
        return oracle.Overlap(q, (0,) + g if len(g) == 2 else g).admm(d["mu0"], max_iter=mi)
    return oracle.admm(q, d["mu0"], max_iter=mi)


def cpu_baseline(insts, gpu_labels=None):
    """The oracle (as it stands) on one full step of the workload: every
    instance's Algorithm 1 run, OpenMP over blocks on all host cores.  Also the
    gap of each oracle solve to the global minimum (whole-grid BK, the paper's
    sGC; serial LSA-TR on the whole grid for non-submodular blocks) and the
    Dice coefficient of the GPU's labels (else the oracle's) against it."""
    import oracle
    qs = [oracle.quantise(d["grid"], d["conn"], d["block"], d["u"], d["wq"], d["lam"], signed=bool(d.get("lsa_steps")))
          for d in insts]
    t0 = time.perf_counter()
    res = [_oracle_solve(oracle, q, d) for q, d in zip(qs, insts)]
    dt = time.perf_counter() - t0
    px = sum(q.n for q in qs)
    gaps, dscs = [], []
    for j, (q, r, d) in enumerate(zip(qs, res, insts)):
        if d.get("lsa_steps"):
            # non-submodular: against the serial LSA-TR on the whole grid (the paper's Table 3)
            lgc, egc = oracle.lsa_tr_global(q, steps=64)
        else:
            lgc, egc = oracle.global_mincut(q)
        gaps.append((r["energy"] - egc) / abs(egc))
        lab = gpu_labels[j] if gpu_labels is not None else r["labels"]
        dscs.append(dice(lab, lgc))
    return {"value": px / dt, "unit": "pixels/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"one full step ({len(qs)} solves, {px} pixels) in {dt:.2f} s",
            "oracle_iterations": [r["iterations"] for r in res]}, gaps, res, dscs


def reference_sample(name):
    """The bounded sample one step of the reference arm solves: the workload
    itself, or for the 256x256x128 volume (about 20-30 s of oracle time per
    solve) its middle slab of 16 x 256 x 256 voxels, two block layers (same
    blocks, lambda, mu0; n-links leaving the slab dropped): 1/8 of the volume,
    crossing all three ellipsoids, 15 iterations against the volume's 18."""
    from paper_1704_03116_gb300 import inputs
    insts, cfg = workload(name)
    if name == "ellipsoids256":
        d = insts[0]
        D = d["grid"][0]
        return [inputs.crop_instance(d, (D // 2 - 8, 0, 0), (16,) + tuple(d["grid"][1:]))], \
            "middle 16x256x256 slab of the volume (1/8), one oracle solve per step"
    return insts, "each step one solve of the workload, cycling over its lambdas"


def run_cpu_set(args):
    """The CPU timing set of the measurement plan, on this machine's host cores:
    for the 64x64 disk, the 512x512 RGB image (lambda 1, 4, 16), the 256x256x128
    volume and the 1024x1024 non-submodular grid, the wall time of one full
    step (every instance of the workload, inputs already in memory) of
      * the oracle (BK per block + FP64 ADMM) with OpenMP over blocks on all
        cores,
      * the same oracle on one thread,
      * the serial whole-grid solve the paper compares against (BK min-cut,
        its sGC; serial LSA-TR for the non-submodular grid), one thread;
    each the median of `--cpu-reps` runs.  Prints one JSON line."""
    import oracle
    out = {"nproc": os.cpu_count(), "threads_all": oracle.num_threads(), "reps": args.cpu_reps, "workloads": {}}
    all_threads = oracle.num_threads()
    for name in ("disk64", "ellipses512", "ellipsoids256", "nonsubmodular1024"):
        insts, cfg = workload(name)
        qs = [oracle.quantise(d["grid"], d["conn"], d["block"], d["u"], d["wq"], d["lam"],
                              signed=bool(d.get("lsa_steps"))) for d in insts]
        px = sum(q.n for q in qs)
        rec = {"workload": cfg["workload"], "pixels_per_step": px}

        def timed(fn):
            ts = []
            for _ in range(args.cpu_reps):
                t0 = time.perf_counter()
                fn()
                ts.append(time.perf_counter() - t0)
            return statistics.median(ts)

        for label, nthr in (("oracle_all_cores", all_threads), ("oracle_1_thread", 1)):
            oracle.set_threads(nthr)
            t = timed(lambda: [_oracle_solve(oracle, q, d) for q, d in zip(qs, insts)])
            rec[label] = {"s": t, "pixels_per_s": px / t, "threads": nthr}
        oracle.set_threads(1)
        if insts[0].get("lsa_steps"):
            t = timed(lambda: [oracle.lsa_tr_global(q, steps=64) for q in qs])
            rec["serial_lsa_tr_1_thread"] = {"s": t, "pixels_per_s": px / t}
        else:
            t = timed(lambda: [oracle.global_mincut(q) for q in qs])
            rec["serial_bk_1_thread"] = {"s": t, "pixels_per_s": px / t}
        oracle.set_threads(all_threads)
        out["workloads"][name] = rec
        print(json.dumps({name: rec}), file=sys.stderr, flush=True)
    print(json.dumps(out), flush=True)
    return 0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    _, cfg = workload(args.workload)
    insts, sample = reference_sample(args.workload)
    qs = [oracle.quantise(d["grid"], d["conn"], d["block"], d["u"], d["wq"], d["lam"], signed=bool(d.get("lsa_steps")))
          for d in insts]
    times, px = [], []
    for s in range(args.warmup + args.steps):
        j = s % len(qs)           # each step: one of the sample's solves
        t0 = time.perf_counter()
        _oracle_solve(oracle, qs[j], insts[j])
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
            px.append(qs[j].n)
    val = sum(px) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "pixels/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": val, "unit": "pixels/s", "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "pixels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _serve(dope, torch, reqs, dev_in, labels, mode, arrivals, warm, submit=None):
    """Run the request stream through a server; arrivals = None submits all
    at once (saturated).  submit(srv, r, inputs, labels, tag) queues one
    request (default: unaries and weights).  Returns per-request results and
    server stats."""
    if submit is None:
        def submit(srv, r, x, lab, tag):
            srv.submit(r["grid"], r["conn"], r["block"], r["lam"], x[0], x[1], lab, tag=tag)
    srv = dope.Server(mode=mode, hbm_bytes=ARENA_BYTES)
    for (x, lab, r) in warm:                          # first launches, tables
        submit(srv, r, x, lab, 0)
    got = 0
    while got < len(warm):
        got += len(srv.poll(timeout=1.0))
    res = {}
    t0 = srv.clock()
    for i, r in enumerate(reqs):
        if arrivals is not None:
            while True:
                for x in srv.poll(timeout=0.0):
                    res[x["tag"]] = x
                dt = t0 + arrivals[i] - srv.clock()
                if dt <= 0:
                    break
                time.sleep(min(dt, 0.001) if dt > 0.0002 else 0)
        submit(srv, r, dev_in[i], labels[i], i)
    deadline = time.time() + 600
    while len(res) < len(reqs) and time.time() < deadline:
        for x in srv.poll(timeout=0.5):
            res[x["tag"]] = x
    st = srv.stats()
    srv.close()
    torch.cuda.synchronize()
    return res, st, t0


def _summ(res, st, t0, reqs, arrivals):
    lat = sorted((res[i]["t_done"] - res[i]["t_submit"]) * 1e3 for i in res)
    done = max(res[i]["t_done"] for i in res) - t0
    px = sum(r["side"] * r["side"] for r in reqs)
    q = lambda p: lat[min(len(lat) - 1, int(round(p * (len(lat) - 1))))]
    return {"solves_per_s": round(len(res) / done, 2), "makespan_s": round(done, 3),
            "mpx_per_s": round(px / done / 1e6, 1), "p50_ms": round(q(0.5), 2), "p99_ms": round(q(0.99), 2),
            "mean_ms": round(sum(lat) / len(lat), 2),
            "queue_wait_p50_ms": round(sorted((res[i]["t_admit"] - res[i]["t_submit"]) * 1e3 for i in res)[len(res) // 2], 2),
            "gpu_busy_s": round(st["gpu_launch_s"], 3), "launches": st["launches"], "yields": st["yields"],
            "max_in_flight": st["max_in_flight"], "hbm_peak_gb": round(st["bytes_peak"] / 1e9, 2),
            "failed": sum(1 for i in res if res[i]["status"] != 0), "completed": len(res)}


_BASES = {}


def _serving_base(b):
    from paper_1704_03116_gb300 import inputs
    if b not in _BASES:
        _BASES[b] = inputs.serving_base(b)
    return _BASES[b]


def potentials_summary(reps=10):
    """Algorithm 1's first step on the GPU for a 2048 x 2048 RGB image (the
    serving stream's base image, 3 + 3 component mixtures, 8-connected
    contrast weights divided by the distance, sigma = mean contrast): device
    time of the data-term kernel and of the two contrast passes, L2 flushed
    before each repetition.  Algorithmic bytes per pixel: data term 12 read +
    4 written; contrast sum 12 read; contrast weights 12 read + 4 per offset
    written (neighbours' features come from cache)."""
    import torch
    from paper_1704_03116_gb300 import dope
    b = _serving_base(0)
    H, W = b["image"].shape[:2]
    n = H * W
    img = torch.from_numpy(np.ascontiguousarray(b["image"].reshape(-1, 3))).cuda()
    u = torch.empty(n, dtype=torch.float32, device="cuda")
    wq = torch.empty((4, n), dtype=torch.int32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(3):
        dope.dope_gmm_unaries(img, b["gmm_fg"], b["gmm_bg"], out=u)
        dope.dope_contrast_weights(img, (H, W), 8, channels=3, inv_dist=True, out=wq)
    tu, tw = [], []
    fg, bg = dope.gmm(*b["gmm_fg"]), dope.gmm(*b["gmm_bg"])
    for r in range(reps):
        flush.fill_(r & 0xFF)
        # keep the GPU busy while the host queues the timed launches, so the
        # events see device time only (no host marshalling in between)
        torch.cuda._sleep(2_000_000)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        dope.dope_gmm_unaries(img, fg, bg, out=u)
        e[1].record(stream)
        dope.dope_contrast_weights(img, (H, W), 8, channels=3, inv_dist=True, out=wq, read_sigma=False)
        e[2].record(stream)
        torch.cuda.synchronize()
        tu.append(e[0].elapsed_time(e[1]))
        tw.append(e[1].elapsed_time(e[2]))
    hbm, kind = peaks()
    bu, bw = 16 * n, (12 + 12 + 16) * n
    mu, mw = statistics.median(tu), statistics.median(tw)
    return {"workload": f"{H}x{W} RGB, 3+3 component mixtures, 8-conn contrast / distance, sigma = mean contrast",
            "unaries_us": 1e3 * mu, "weights_us": 1e3 * mw,
            "unaries_gbs": bu / (mu / 1e3) / 1e9, "weights_gbs": bw / (mw / 1e3) / 1e9,
            "frac": (bu + bw) / ((mu + mw) / 1e3) / 1e9 / hbm, "peak": hbm, "peak_kind": f"{kind} hbm_gbs",
            "pixels_per_s": n / ((mu + mw) / 1e3), "bytes_per_pixel": 56, "reps": reps,
            "l2": "flushed before every repetition (256 MiB write)"}


def serving_summary(requests, rate, saturated=True):
    """Serving stream: requests (RGB contrast-Potts crops, side U[128,2048],
    4/8-conn 50/50, lambda U[1,16]) arrive as a Poisson process at `rate`;
    the batched server (continuous batching) against the same server solving
    one request at a time through the single-problem path, and both again with
    every request queued at once (capacity).  Returns (summary, launches)."""
    import torch
    from paper_1704_03116_gb300 import inputs
    from paper_1704_03116_gb300 import dope
    n = requests
    reqs = inputs.serving_requests(n, rate=rate)
    arrivals = [r["arrival"] for r in reqs]
    bases = [_serving_base(b) for b in range(2)]
    dbase = [(torch.from_numpy(b["u"]).cuda(), torch.from_numpy(b["wq"]).cuda()) for b in bases]
    dev_in = []
    for r in reqs:
        U, WQ = dbase[r["base"]]
        s_, y0, x0, nh = r["side"], r["y0"], r["x0"], r["conn"] // 2
        u = U[y0:y0 + s_, x0:x0 + s_].contiguous().reshape(-1)
        w = WQ[:nh, y0:y0 + s_, x0:x0 + s_].clone()
        w[0, :, -1] = 0
        w[1, -1, :] = 0
        if nh == 4:
            w[2, -1, :] = 0
            w[2, :, -1] = 0
            w[3, -1, :] = 0
            w[3, :, 0] = 0
        dev_in.append((u, w.reshape(nh, -1)))
    labels = [torch.zeros(r["side"] * r["side"], dtype=torch.uint8, device="cuda") for r in reqs]
    keep = [torch.empty_like(l) for l in labels]
    warm = []
    for k in range(3):
        r = dict(reqs[k], lam=2.0)
        warm.append((dev_in[k], torch.zeros_like(labels[k]), r))
    torch.cuda.synchronize()
    out = {}
    res_b, st_b, t0b = _serve(dope, torch, reqs, dev_in, labels, 0, arrivals, warm)
    out["batched"] = _summ(res_b, st_b, t0b, reqs, arrivals)
    for a, b in zip(keep, labels):
        a.copy_(b)
    res_1, st_1, t01 = _serve(dope, torch, reqs, dev_in, labels, 1, arrivals, warm)
    out["one_at_a_time"] = _summ(res_1, st_1, t01, reqs, arrivals)
    same = all(res_b[i]["energy_int"] == res_1[i]["energy_int"] and
               res_b[i]["iterations"] == res_1[i]["iterations"] for i in range(n))
    same = same and all(torch.equal(a, b) for a, b in zip(keep, labels))
    if saturated:
        res_bs, st_bs, t0bs = _serve(dope, torch, reqs, dev_in, labels, 0, None, warm)
        out["batched_saturated"] = _summ(res_bs, st_bs, t0bs, reqs, None)
        res_1s, st_1s, t01s = _serve(dope, torch, reqs, dev_in, labels, 1, None, warm)
        out["one_at_a_time_saturated"] = _summ(res_1s, st_1s, t01s, reqs, None)
        # batching only as wide as the backlog (server mode 2), both ways
        res_a, st_a, t0a = _serve(dope, torch, reqs, dev_in, labels, 2, arrivals, warm)
        out["adaptive"] = _summ(res_a, st_a, t0a, reqs, arrivals)
        res_as, st_as, t0as = _serve(dope, torch, reqs, dev_in, labels, 2, None, warm)
        out["adaptive_saturated"] = _summ(res_as, st_as, t0as, reqs, None)
        same = same and all(res_a[i]["energy_int"] == res_1[i]["energy_int"] and
                            res_a[i]["iterations"] == res_1[i]["iterations"] for i in range(n))
        # the same stream given as RGB crops: the server computes the
        # potentials on the GPU (the bases' mixtures; sigma fixed to the base
        # image's, so a crop's weights mean what they mean in the full image)
        imgs = [torch.from_numpy(np.ascontiguousarray(b["image"])).cuda() for b in bases]
        gm = [(dope.gmm(*b["gmm_fg"]), dope.gmm(*b["gmm_bg"]), float(b["sigma"])) for b in bases]
        img_in = [imgs[r["base"]][r["y0"]:r["y0"] + r["side"], r["x0"]:r["x0"] + r["side"]].contiguous()
                  for r in reqs]
        del dev_in

        def submit_img(srv, r, x, lab, tag):
            fg, bg, sig = gm[r["base"]]
            srv.submit_image(r["grid"], r["conn"], r["block"], r["lam"], x, fg, bg, lab, sigma=sig,
                             inv_dist=True, tag=tag)
        warm_i = [(img_in[k], w[1], w[2]) for k, w in enumerate(warm)]
        torch.cuda.synchronize()
        res_bi, st_bi, t0bi = _serve(dope, torch, reqs, img_in, labels, 0, None, warm_i, submit_img)
        out["batched_saturated_from_image"] = dict(_summ(res_bi, st_bi, t0bi, reqs, None),
                                                   inputs="device-resident RGB crops, 12 B/px; "
                                                          "potentials computed by the server")
    out["results_identical_across_modes"] = bool(same)
    out["iterations_mean"] = round(sum(res_b[i]["iterations"] for i in range(n)) / n, 1)
    out["config"] = {"workload": "serving stream: RGB contrast-Potts crops of two seeded 2048x2048 ellipse "
                                 "images, side U[128,2048], 4/8-conn 50/50, lambda U[1,16], blocks 32x32",
                     "requests": n, "rate_per_s": rate, "inputs": "device-resident"}
    return out, int(2 * st_b["launches"] + 5 * n)


def run_serving(args):
    """bench.py --workload serving: the serving comparison as its own line."""
    import torch
    from paper_1704_03116_gb300 import _build
    _build.build()
    torch.cuda.set_device(0)
    clk = Clocks(0)
    clk.start()
    out, launches = serving_summary(args.requests, args.rate, not args.no_saturated)
    clocks = clk.stop()
    line = {"metric": "solves/sec of a Poisson request stream to ADMM convergence (p50/p99 latency)",
            "value": out["batched"]["solves_per_s"], "unit": "solves/s", "n_gpus": 1, "steps": 1,
            "warmup": 1, "ms_per_step": round(out["batched"]["makespan_s"] * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(out.pop("config"),
                                                l2="inputs larger than L2 (1.5 Mpx mean per request)"),
            "serving": out, "clocks": clocks, "gpu_launches": launches}
    print(json.dumps(line))


def measure(name, args, world, local, with_e2e=True):
    """Time one workload on this rank: `value` (device-resident inputs), the
    per-solve latencies, the dominant kernel's roofline, the block solver's
    counters and (with_e2e) the end-to-end figures through the C-ABI.
    Returns (line fields, the workload's instances, the last labels per
    instance on the host)."""
    import torch
    from paper_1704_03116_gb300 import dope

    insts, cfg = workload(name)
    ctxs = []
    overlap = "grow" in insts[0] or insts[0]["conn"] not in (4, 8, 6)
    notconv = "grow" in insts[0]
    for d in insts:
        g = dope.Dope(d["grid"], d["conn"], d["block"], d["lam"], mu0=d["mu0"], grow=d.get("grow"),
                      max_iter=d.get("max_iter"), lsa_steps=d.get("lsa_steps"))
        g.set_unaries(torch.from_numpy(d["u"]).cuda())
        g.set_weights(torch.from_numpy(d["wq"]).cuda())
        ctxs.append(g)
    n_px = sum(g.n for g in ctxs)
    labels = [torch.empty(g.n, dtype=torch.uint8, device="cuda") for g in ctxs]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        for g, lab in zip(ctxs, labels):
            g.solve(lab, allow_notconv=notconv)
    torch.cuda.synchronize()

    # ---- device-resident timed region -----------------------------------
    for g in ctxs:
        g.set_profiling(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps * len(ctxs))]
    clocks = Clocks(local)
    launches, iters, energies = 0, [], []
    work = {"pulses_total": 0, "free_nodes_total": 0, "bfs_levels_total": 0, "blocks_solved": 0,
            "blocks_updated": 0}
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    wall0 = time.perf_counter()
    step_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
    for s in range(args.steps):
        flush.fill_(s & 0xFF)
        # the step's solves queued back to back (dope_solve_begin), then
        # collected (dope_solve_end); one event pair around the whole step and
        # one around each solve (its device time, for the latency figures)
        step_ev[s][0].record(stream)
        for j, (g, lab) in enumerate(zip(ctxs, labels)):
            a, b = ev[s * len(ctxs) + j]
            a.record(stream)
            g.solve_begin(lab, stream=stream.cuda_stream)
            b.record(stream)
        step_ev[s][1].record(stream)
        for g in ctxs:
            _, E, it = g.solve_end(stream=stream.cuda_stream, allow_notconv=notconv)
            st = g.stats()
            launches += st["kernel_launches"]
            for key in work:
                work[key] += int(st.get(key, 0))
            iters.append(it)
            energies.append(E)
    torch.cuda.synchronize()
    barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    lat = [a.elapsed_time(b) for a, b in ev]
    step_ms = [a.elapsed_time(b) for a, b in step_ev]
    t_local = sum(step_ms) / 1e3
    t_max = max_over_ranks(t_local, world)
    value = job_rate(n_px * args.steps, world, t_max)
    profs = [g.profile() for g in ctxs]
    kinds = [g.stats()["solver_kernel"] for g in ctxs]
    for g in ctxs:
        g.set_profiling(False)
    host_labels = [lab.cpu().numpy() for lab in labels]

    # ---- roofline of the dominant kernel --------------------------------
    hbm, peak_kind = peaks()
    nh = insts[0]["conn"] // 2
    F, X = (0, 0) if overlap else face_geometry(insts[0]["grid"], insts[0]["block"], insts[0]["conn"])
    n1, k1 = ctxs[0].n, ctxs[0].nblocks
    sf, sl, up = algorithmic_bytes(n1, k1, F, X, nh)
    solve_ms = sum(p["ms"][0] for p in profs)
    solve_n = sum(p["launches"][0] for p in profs)
    first_n = sum(p["first_iteration_launches"] for p in profs)
    upd_ms = sum(p["ms"][1] for p in profs)
    upd_n = sum(p["launches"][1] for p in profs)
    iters_n = sum(p["iterations"] for p in profs)
    model = "per pixel-iteration figure x pixel-iterations (every pixel's bytes once per iteration)"
    processed = None
    if overlap:
        sb, ub = overlap_bytes(insts[0])
        if solve_ms >= upd_ms:
            kname, kms, kn, kbytes = "k_ov_solve", solve_ms, solve_n, solve_n * sb
        else:
            kname, kms, kn, kbytes = "k_ov_update", upd_ms, upd_n, upd_n * ub
        share = {"k_ov_solve": solve_ms / (solve_ms + upd_ms), "k_ov_y+k_ov_a": upd_ms / (solve_ms + upd_ms)}
    elif upd_n == 0:
        # persistent mode: one launch runs every iteration of a solve (the
        # resident kernel when every block fits on the GPU at once)
        kname = "k_admm_resident" if kinds[0] == 2 else "k_admm_persistent"
        kms, kn = solve_ms, solve_n
        kbytes = first_n * sf + (iters_n - first_n) * sl + iters_n * up
        if kname == "k_admm_persistent" and work["blocks_solved"]:
            # worklists: the launch's first iteration does every block, later
            # ones the blocks on the lists; the bytes of the blocks it processed
            sfb, slb, upb = sf / k1, sl / k1, up / k1
            pbytes = kn * k1 * (sfb + upb) + work["blocks_solved"] * slb + work["blocks_updated"] * upb
            processed = {"bytes_per_launch": pbytes / max(kn, 1),
                         "achieved_gbs": pbytes / (kms / 1e3) / 1e9,
                         "model": "iteration 1 every block, later ordinary iterations the blocks on the "
                                  "worklists (per block: solve %.0f B, update %.0f B); iterations inside "
                                  "run-ahead windows not counted" % (slb, upb)}
        share = {kname: 1.0}
        if kname == "k_admm_persistent":
            # a solve that reaches frozen labels is two launches back to back
            # (the plain form, then the windowed form from the hand-off); one
            # "launch" here is one solve, both timed together
            model += "; one launch = one solve (plain and windowed forms of k_admm_persistent)"
    elif solve_ms >= upd_ms:
        kname = "k_nsm_solve" if insts[0].get("lsa_steps") else "k_block_solve"
        kms, kn = solve_ms, solve_n
        kbytes = first_n * sf + (solve_n - first_n) * sl
        share = {"k_block_solve": solve_ms / (solve_ms + upd_ms), "k_face_update": upd_ms / (solve_ms + upd_ms)}
    else:
        kname, kms, kn = "k_face_update", upd_ms, upd_n
        kbytes = upd_n * up
        share = {"k_block_solve": solve_ms / (solve_ms + upd_ms), "k_face_update": upd_ms / (solve_ms + upd_ms)}
    achieved = kbytes / (kms / 1e3) / 1e9
    roof = {"kernel": kname, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "peak_kind": f"{peak_kind} hbm_gbs",
            "traffic": kernel_traffic(kname, name),
            "algorithmic_bytes_per_launch": kbytes / max(kn, 1), "bytes_model": model,
            "avg_launch_us": 1e3 * kms / max(kn, 1), "launches": kn, "iterations_covered": iters_n,
            "time_share": share}
    if processed:
        roof["blocks_processed"] = processed

    out = {"metric": METRIC if "grow" not in insts[0] else
           "pixels/sec of 3 ADMM iterations (overlapping partition, Figure 2 protocol)",
           "value": value, "unit": "pixels/s", "ms_per_step": statistics.mean(step_ms),
           "config": dict(cfg, l2="flushed before every step (256 MiB write)",
                          parallelism="replicas" if world > 1 else "single"),
           "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "solves": len(lat)},
           "iterations": sorted(set(iters)), "energies": sorted(set(energies)),
           "converged": [bool(g.stats()["converged"]) for g in ctxs],
           "pixel_iterations_per_s": sum(g.n * it for g, it in zip(ctxs * args.steps, iters)) / max(t_local, 1e-12),
           "wall_s": wall, "gpu_launches": launches, "roofline": roof, "clocks": clk,
           # the block solver's work (its own counters): push-relabel pulses, nodes
           # left for push-relabel after folding, BFS levels -- per solve and per
           # second; block solves / updates run from the persistent kernel's worklists
           "solver": {"pulses_per_solve": work["pulses_total"] / max(len(iters), 1),
                      "free_nodes_per_solve": work["free_nodes_total"] / max(len(iters), 1),
                      "bfs_levels_per_solve": work["bfs_levels_total"] / max(len(iters), 1),
                      "pulses_per_s": work["pulses_total"] / max(t_local, 1e-12),
                      "worklist_block_solves_per_solve": work["blocks_solved"] / max(len(iters), 1),
                      "worklist_block_updates_per_solve": work["blocks_updated"] / max(len(iters), 1),
                      "blocks": k1}}
    last_E = energies[-len(ctxs):]
    if not with_e2e:
        return out, insts, host_labels, last_E

    # ---- end to end through the C-ABI with pinned host buffers ---------
    up_s = torch.cuda.Stream()
    hu = [torch.from_numpy(d["u"]).pin_memory() for d in insts]
    hw = [torch.from_numpy(np.ascontiguousarray(d["wq"])).pin_memory() for d in insts]
    hl = [torch.empty(g.n, dtype=torch.uint8).pin_memory() for g in ctxs]
    e2e_ms = []
    barrier()
    for s in range(args.steps):
        flush.fill_((s + 1) & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        # every solve of the step queued, then one wait per solve; inputs go
        # up on their own stream, each solve ordered after its upload
        for g, u, w, lab in zip(ctxs, hu, hw, hl):
            g.set_inputs(u.numpy(), w.numpy(), stream=up_s.cuda_stream)
            ev_up = torch.cuda.Event()
            ev_up.record(up_s)
            stream.wait_event(ev_up)
            g.solve_begin(lab.numpy(), stream=stream.cuda_stream)
        for g in ctxs:
            g.solve_end(stream=stream.cuda_stream, allow_notconv=notconv)
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    barrier()
    e2e_t = max_over_ranks(sum(e2e_ms) / 1e3, world)
    h2d = sum(d["u"].nbytes + d["wq"].nbytes for d in insts)
    d2h = sum(g.n for g in ctxs) + 8 * len(ctxs)
    out["e2e"] = {"value": job_rate(n_px * args.steps, world, e2e_t), "unit": "pixels/s",
                  "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": statistics.mean(e2e_ms)}

    # ---- end to end from the image: potentials on the GPU (Algorithm 1's
    # first step), then the solve; pinned image in, labels out --------------
    if all("image" in d and "gmm_fg" in d and "inv_dist" in d for d in insts) and not overlap:
        hi = [torch.from_numpy(np.ascontiguousarray(d["image"], np.float32)).pin_memory() for d in insts]
        img_ms = []
        barrier()
        for s in range(args.steps):
            flush.fill_((s + 7) & 0xFF)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for g, d, im, lab in zip(ctxs, insts, hi, hl):
                g.set_image(im.numpy(), d["gmm_fg"], d["gmm_bg"], inv_dist=d["inv_dist"], read_sigma=False,
                            stream=up_s.cuda_stream)
                ev_up = torch.cuda.Event()
                ev_up.record(up_s)
                stream.wait_event(ev_up)
                g.solve_begin(lab.numpy(), stream=stream.cuda_stream)
            for g in ctxs:
                g.solve_end(stream=stream.cuda_stream, allow_notconv=notconv)
            torch.cuda.synchronize()
            img_ms.append(1e3 * (time.perf_counter() - t0))
        barrier()
        t_img = max_over_ranks(sum(img_ms) / 1e3, world)
        out["e2e_from_image"] = {"value": job_rate(n_px * args.steps, world, t_img), "unit": "pixels/s",
                                 "h2d_bytes_per_step": sum(im.numel() * 4 for im in hi),
                                 "d2h_bytes_per_step": d2h, "ms_per_step": statistics.mean(img_ms),
                                 "note": "image in; mixture data term and contrast weights computed on the GPU"}
    return out, insts, host_labels, last_E


def dice(a, b):
    """Dice similarity coefficient of the foreground (label 1) of two labellings."""
    a = np.asarray(a, bool)
    b = np.asarray(b, bool)
    s = int(a.sum()) + int(b.sum())
    return 1.0 if s == 0 else 2.0 * int((a & b).sum()) / s


def oracle_checks(out, insts, host_labels, last_E, with_cpu=True):
    """CPU side of a line: the oracle's Algorithm 1 on one full step (timed:
    cpu_baseline), the gap of every solve's energy to the global minimum (or
    to serial LSA-TR for non-submodular blocks), the Dice coefficient of the
    labels against the global minimiser (the paper's DSC against sGC), and
    whether the GPU energies match the oracle's."""
    cb, gaps, res, dscs = cpu_baseline(insts, host_labels)
    if with_cpu:
        out["cpu_baseline"] = cb
    key = "lsa_tr" if insts[0].get("lsa_steps") else "global_mincut"
    out["energy_gap_vs_serial_lsa_tr" if key == "lsa_tr" else "energy_gap_vs_global_mincut"] = gaps
    out["gap_target"] = 1e-3
    out["gap_within_target"] = [bool(x <= 1e-3) for x in gaps]
    out["dsc_vs_serial_lsa_tr" if key == "lsa_tr" else "dsc_vs_global_mincut"] = dscs
    out["oracle_match"] = all(abs(E * 1024 - r["energy"]) <= 1e-4 * abs(r["energy"])
                              for E, r in zip(last_E, res))
    out["oracle_labels_match"] = all(np.array_equal(l, r["labels"]) for l, r in zip(host_labels, res))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="dope", choices=["dope", "reference"])
    ap.add_argument("--workload", default="ellipsoids256")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--requests", type=int, default=1000, help="serving workload: requests")
    ap.add_argument("--rate", type=float, default=200.0, help="serving workload: arrivals per second")
    ap.add_argument("--no-saturated", action="store_true", help="serving workload: skip the capacity runs")
    ap.add_argument("--arena-gb", type=float, default=0.0,
                    help="serving: bound the server's device arena (GB; 0 = 3/4 of the free memory)")
    ap.add_argument("--no-serving", action="store_true",
                    help="default workload: skip the serving comparison added to its line")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload: only the headline (no 2-D line, potentials or serving)")
    ap.add_argument("--cpu-set", action="store_true",
                    help="time the oracle (all cores, one thread) and the serial whole-grid solve on the host")
    ap.add_argument("--cpu-reps", type=int, default=5, help="--cpu-set: runs per timing (median)")
    args = ap.parse_args()
    global ARENA_BYTES
    ARENA_BYTES = int(args.arena_gb * (1 << 30))
    if args.cpu_set:
        return run_cpu_set(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving":
        return run_serving(args)

    import torch
    import torch.distributed as dist
    from paper_1704_03116_gb300 import _build
    if int(os.environ.get("LOCAL_RANK", "0")) == 0:
        _build.build()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist.barrier()

    out, insts, host_labels, last_E = measure(args.workload, args, world, local)
    line = {"metric": out.pop("metric"), "value": out.pop("value"), "unit": out.pop("unit"), "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": out.pop("ms_per_step"),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "i32+f64",
            "data": "synthetic", "config": out.pop("config")}
    line.update(out)
    single = rank == 0 and world == 1
    if single and not args.no_cpu_baseline:
        oracle_checks(line, insts, host_labels, last_E)
    default = args.workload == "ellipsoids256" and not args.no_extras
    if single and default:
        # the 2-D colour-image workload (512 x 512 RGB, lambda 1, 4, 16) as its own object
        try:
            sub, si, sl, sE = measure("ellipses512", args, world, local, with_e2e=True)
            if not args.no_cpu_baseline:
                oracle_checks(sub, si, sl, sE)
            line["ellipses512"] = sub
        except Exception as e:  # the main line stands on its own
            line["ellipses512"] = {"error": f"{type(e).__name__}: {e}"}
    if single and (default or args.workload == "ellipses512"):
        try:
            line["potentials"] = potentials_summary()
        except Exception as e:  # the main line stands on its own
            line["potentials"] = {"error": f"{type(e).__name__}: {e}"}
    if single and (default or args.workload == "ellipses512") and not args.no_serving:
        # the serving target: batched vs one-at-a-time on the request stream
        try:
            srv, _ = serving_summary(args.requests, args.rate, not args.no_saturated)
            line["serving"] = srv
        except Exception as e:  # the main line stands on its own
            line["serving"] = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
