"""Benchmark of the brick codec on one B300 (or N replicas under torchrun).

A step is one pass of the whole hot path over the 512^3 warped-Voronoi volume
with 32^3 bricks (4096 bricks): frequency prepass over every 512th brick,
GPU encode of every brick, then one batched decode of every brick at full
resolution.  `value` is decoded GB/s (decimal, uint32 labels) of the whole
step; the phases are reported beside it, with the plain per-brick-launch
decode of the same bricks and the CPU oracle as baselines.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
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

WORKLOAD = "voronoi512"
B = 32
STRIDE = 512
# the per-launch timing events (and the encode / decode split) are recorded on every PROF_EVERY-th timed step:
# on every step they made each step about 0.03 ms longer (host time between the launches after the encode's
# read-back), which is the instrumentation's cost, not the work's
PROF_EVERY = 4


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--b", type=int, default=B)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--workload", default="voronoi512", choices=["voronoi512", "cells1024", "worley2048", "fiber4096", "variants"],
                    help="voronoi512: the headline step (sampled encode + decode of all bricks at LOD 0); "
                         "cells1024: one batched decode of 60000 mixed-LOD requests per step; "
                         "worley2048: serve a 600-frame camera trace (a step is one frame); "
                         "fiber4096: stream-encode the 4096x4096x2048 fiber volume made brick by brick, "
                         "then serve a trace with the leaf streams in host memory")
    ap.add_argument("--s-min", type=int, default=256, help="symbols per rANS state (format parameter S_min)")
    ap.add_argument("--k-max", type=int, default=32, help="most interleaved rANS states per stream (K_max)")
    ap.add_argument("--no-extra", action="store_true",
                    help="headline line only: skip the batched (cells1024) and serve (worley2048) blocks")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi sampling during the timed region (SM clock, throttle reasons)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        self.t0 = time.time()
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # wait (bounded) for the first sample so the region after this is covered
            while not self.lines and time.time() - self.t0 < 5.0 and self.proc.poll() is None:
                time.sleep(0.01)
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, t0, t1):
        """Wall-clock bounds of the timed region (to count the samples taken inside it)."""
        self.window = (t0, t1)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        w = getattr(self, "window", None)
        inside = sum(1 for t, _ in self.lines if w and w[0] <= t <= w[1])
        for _, ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm), "samples_in_timed_region": inside,
                "window": "warm-up through the timed region, every 100 ms"}


def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def kernel_traffic(kernel):
    """DRAM bytes per launch of a kernel on voronoi512 b=32 from the committed ncu capture
    (profiles/kernel_traffic_voronoi512_b32.md), or None once the kernel's source file has changed."""
    import hashlib
    here = os.path.dirname(os.path.abspath(__file__))
    try:
        lines = open(os.path.join(here, "profiles", "kernel_traffic_voronoi512_b32.md")).read().splitlines()
    except OSError:
        return None
    for ln in lines:
        f = [c.strip() for c in ln.strip().strip("|").split("|")]
        if len(f) == 5 and f[0] == kernel:
            src = os.path.join(here, "paper_2308_16619_b300", "csrc", f[1])
            try:
                sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:12]
            except OSError:
                return None
            return int(f[3]) + int(f[4]) if sha == f[2] else None
    return None


def oracle_step(vol, b, cores):
    """One step of the oracle on the headline workload, as the GPU step does it: prepass over every
    STRIDE-th brick, encode of every brick, decode of every brick at LOD 0.  Returns seconds."""
    import oracle as O
    N = b.bit_length() - 1
    t0 = time.perf_counter()
    V = O.encode_volume(vol, N, stride=STRIDE, n_threads=cores)
    n = V.n_bricks
    out, off, st = O.decode_bricks(V, np.arange(n, dtype=np.uint32), np.zeros(n, np.uint8), n_threads=cores)
    dt = time.perf_counter() - t0
    assert (st == 0).all()
    return dt


def oracle_sample(vol, b):
    n = vol.size // b ** 3
    return (f"oracle prepass (every {STRIDE}th brick) + encode + decode of all {n} bricks of the "
            f"{vol.shape[2]}x{vol.shape[1]}x{vol.shape[0]} volume per step, the GPU step's workload")


def cpu_baseline_oracle(vol, b, min_seconds=10.0, max_runs=60):
    """The oracle as it stands on all host cores, repeated on the whole headline workload until about
    min_seconds of work are done; the median step.  Returns (GB/s, cores, sample description)."""
    cores = os.cpu_count() or 1
    times, used = [], 0.0
    while used < min_seconds and len(times) < max_runs:
        dt = oracle_step(vol, b, cores)
        times.append(dt)
        used += dt
    gbs = vol.nbytes / statistics.median(times) / 1e9
    return gbs, cores, oracle_sample(vol, b) + f" ({len(times)} steps, median)"


def run_reference(args):
    """The oracle as the reference arm: the headline workload, whole, on the host cores."""
    import synth
    rank, world, _ = dist_env()
    if rank != 0:
        return
    vol = synth.make(WORKLOAD)
    b = args.b
    cores = os.cpu_count() or 1
    times = []
    for s in range(args.warmup + args.steps):
        dt = oracle_step(vol, b, cores)
        if s >= args.warmup:
            times.append(dt)
    ms = 1000 * statistics.median(times)
    gbs = vol.nbytes / (ms / 1000) / 1e9
    n = vol.size // b ** 3
    line = {"impl": "reference", "metric": "decoded GB/s uint32 labels (batched vs plain per-brick); serve p50/p99 ms",
            "value": gbs, "unit": "GB/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": f"{WORKLOAD} 512^3 warped Voronoi, 20000 cells, 30% background, b={b}",
                       "bricks": n, "lod": 0, "step": f"prepass (stride {STRIDE}) + encode + decode of every brick",
                       "sample": oracle_sample(vol, b)},
            "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": cores, "kind": "oracle",
                             "sample": oracle_sample(vol, b)},
            "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_cells1024(args):
    print(json.dumps(measure_cells1024(args, args.steps, args.warmup)))


def frame_requests(csgv, v, dims, n_frames, seed, max_nonempty=1):
    """Brick requests of a fly-around trace from the library's footprint kernel (one ray per pixel of a
    1920x1080 frame walks the brick grid, skips bricks with no opaque label, stops at the first brick that
    holds one).  Returns the per-frame (bricks, lods) host arrays and the kernels' ms per frame."""
    import synth
    cams = synth.camera_path(dims, n_frames, seed=seed)
    fp = csgv.Footprint(v, max_nonempty=max_nonempty)
    csgv.profile_read()
    csgv.profile_enable(True)
    frames = []
    for cam in cams:
        bricks, lods = fp.frame(csgv.make_camera(cam["pos"], cam["right"], cam["up"], cam["fwd"], cam["f_px"],
                                                 cam["width"], cam["height"]))
        frames.append((bricks.cpu().numpy().view(np.uint32).copy(), lods.cpu().numpy().copy()))
    csgv.profile_enable(False)
    prof = csgv.profile_read()
    fp.close()
    ms = sum(t for k, (t, c) in prof.items() if k.startswith("footprint")) / max(1, n_frames)
    return frames, ms


def measure_cells1024(args, steps, warmup):
    """1024^3 packed ellipsoids, b=32: encode once, then each step decodes 60000 requests at random LOD
    0..5 (brick ids uniform with replacement, seed 3) in one persistent launch.  Returns the JSON line."""
    import torch
    import synth
    import paper_2308_16619_b300 as csgv
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    b = 32
    vol_np = synth.make("cells1024")
    vol = torch.from_numpy(vol_np.view(np.int32)).to(dev)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    table = csgv.csgv_build_freq_table(vol, b, 512)
    v = csgv.csgv_encode_bricks(vol, b, table, K_max=args.k_max, S_min=args.s_min)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    enc_ms = e0.elapsed_time(e1)
    del vol
    inf = v.info()
    rng = np.random.default_rng(3)
    n = 60000
    ids_h = rng.integers(0, inf.n_bricks, size=n).astype(np.uint32)
    lods_h = rng.integers(0, 6, size=n).astype(np.uint8)
    offs_h, total = csgv.request_layout(b, lods_h)
    ids = torch.from_numpy(ids_h.view(np.int32)).to(dev)
    lods = torch.from_numpy(lods_h).to(dev)
    offs = torch.from_numpy(offs_h).to(dev)
    out = torch.empty(total, dtype=torch.int32, device=dev)
    status = torch.empty(n, dtype=torch.int32, device=dev)
    out_bytes = total * 4
    # the autotuner picks the launch shape for this batch (rANS ring depth and CTAs per SM, threads per LOD 0 and
    # LOD 1 request, workspace per slice)
    tune = csgv.csgv_decode_autotune(v, ids, lods, out, offs, status)
    # per-kernel times from CUDA events around each launch (direct calls)
    csgv.profile_read()
    csgv.profile_enable(True)
    for _ in range(3):
        csgv.csgv_decode_bricks(v, ids, lods, out, offs, status)
    torch.cuda.synchronize(dev)
    csgv.profile_enable(False)
    prof = csgv.profile_read()
    prof = {k: (t / 3 * steps, c // 3 * steps) for k, (t, c) in prof.items()}
    # the timed steps replay one captured graph of the decode call
    gs = torch.cuda.Stream(dev)
    gs.wait_stream(stream)
    with torch.cuda.stream(gs):
        csgv.csgv_decode_bricks(v, ids, lods, out, offs, status)
    stream.wait_stream(gs)
    torch.cuda.synchronize(dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=gs):
        csgv.csgv_decode_bricks(v, ids, lods, out, offs, status)
    clk = ClockSampler(local).__enter__()
    for _ in range(warmup):
        graph.replay()
    torch.cuda.synchronize(dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    w0 = time.time()
    for a, z in evs:
        a.record(stream)
        graph.replay()
        z.record(stream)
    torch.cuda.synchronize(dev)
    clk.mark(w0, time.time())
    clk.__exit__()
    ms = float(np.median([a.elapsed_time(z) for a, z in evs]))
    assert bool((status == 0).all())
    m = 2048
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    csgv.csgv_decode_bricks_plain(v, ids[:m], lods[:m], out, offs, status)
    p1.record(stream)
    torch.cuda.synchronize(dev)
    plain_gbs = int((((b >> lods_h[:m].astype(np.int64)) ** 3) * 4).sum()) / (p0.elapsed_time(p1) / 1e3) / 1e9
    peak, peak_kind = measured_peak_hbm()
    rb_ms = prof["rebuild"][0] / prof["rebuild"][1]
    # algorithmic bytes of the rebuild launches of one batch: the decoded labels written plus, at most, the
    # compressed volume read
    rb_per_batch = prof["rebuild"][0] / steps
    achieved = (out_bytes + inf.compressed_bytes) / (rb_per_batch / 1e3) / 1e9
    kernels = {k: {"ms_per_launch": t / c, "launches_per_step": c / steps} for k, (t, c) in prof.items()}
    line = {"metric": "decoded GB/s uint32 labels (batched vs plain per-brick); serve p50/p99 ms",
            "value": out_bytes / (ms / 1e3) / 1e9, "unit": "GB/s", "n_gpus": 1, "steps": steps,
            "warmup": warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "cells1024 1024^3 packed ellipsoids, b=32, 60000 requests LOD 0..5",
                       "step": "one batched decode (CUDA graph replay)", "decoded_bytes": out_bytes,
                       "K_max": args.k_max, "autotuned": tune.as_dict(),
                       "S_min": args.s_min, "l2": "outputs (1.5 GB) larger than L2"},
            "voxels_per_s": out_bytes / 4 / (ms / 1e3), "encode_ms_once": enc_ms,
            "plain_decode_gbs_2048": plain_gbs, "batched_vs_plain": (out_bytes / (ms / 1e3) / 1e9) / plain_gbs,
            "cr_percent": 100.0 * inf.compressed_bytes / (vol_np.nbytes),
            "roofline": {"bound": "hbm", "kernel": "rebuild", "achieved": achieved, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                         "ms_per_batch": rb_per_batch, "ms_per_launch": rb_ms},
            "kernels": kernels,
            "gpu_launches": int(sum(c for _, c in prof.values())), "clocks": clk.summary()}
    # outside the timed region: a sample of the requests against their bricks in the volume
    got = out.cpu().numpy().view(np.uint32)
    rs = np.random.default_rng(11).choice(np.nonzero(lods_h == 0)[0], size=32, replace=False)
    for r in rs:
        br = int(ids_h[r])
        g = 1024 // b
        bx, by, bz = br % g, (br // g) % g, br // (g * g)
        want = vol_np[bz * b:(bz + 1) * b, by * b:(by + 1) * b, bx * b:(bx + 1) * b].reshape(-1)
        assert np.array_equal(got[int(offs_h[r]):int(offs_h[r]) + b ** 3], want), "cells1024 decode mismatch"
    del out, v
    torch.cuda.empty_cache()
    return line


def run_variants(args):
    """Coding variants on voronoi512 b=32 (compression ratio and decode speed): two tables with K_max = 32
    (default), 16 and 1 (the paper's single rANS state), one table for both streams, no rANS (raw nibbles,
    two per byte; size from the symbol counts), and brick size 64."""
    import torch
    import synth
    import paper_2308_16619_b300 as csgv
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    b = args.b
    vol_np = synth.make("voronoi512")
    vol = torch.from_numpy(vol_np.view(np.int32)).to(dev)
    raw = vol_np.nbytes
    n = vol_np.size // b ** 3
    ids = torch.arange(n, dtype=torch.int32, device=dev)
    lods = torch.zeros(n, dtype=torch.uint8, device=dev)
    offs = torch.arange(n, dtype=torch.int64, device=dev) * b ** 3
    out = torch.empty(n * b ** 3, dtype=torch.int32, device=dev)
    status = torch.empty(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    two = csgv.csgv_build_freq_table(vol, b, 1)
    c = np.array(two.counts[:], np.uint64)
    one = csgv.csgv_freq_table_from_counts(np.concatenate([c[:16] + c[16:], c[:16] + c[16:]]))
    rows = {}
    for name, table, km in (("two tables, K_max=32", two, 32), ("two tables, K_max=16", two, 16),
                            ("two tables, K_max=1", two, 1), ("one table, K_max=32", one, 32)):
        v = csgv.csgv_encode_bricks(vol, b, table, K_max=km, S_min=args.s_min)
        ts = []
        for r in range(args.warmup + args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            csgv.csgv_decode_bricks(v, ids, lods, out, offs, status)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            if r >= args.warmup:
                ts.append(e0.elapsed_time(e1))
        assert bool((status == 0).all())
        assert torch.equal(out.view(n, b, b, b)[0].cpu(), vol[:b, :b, :b].cpu())
        inf = v.info()
        rows[name] = {"cr_percent": 100.0 * inf.compressed_bytes / raw,
                      "decode_gbs": n * b ** 3 * 4 / (float(np.median(ts)) / 1e3) / 1e9}
        if km == 32 and table is two:
            ex = v.export()
            nib = ex["n_int_sym"].astype(np.int64), ex["n_leaf_sym"].astype(np.int64)
            raw_nibbles = int(((nib[0] + 1) // 2 + (nib[1] + 1) // 2).sum())
            rows["no rANS (raw nibbles)"] = {
                "cr_percent": 100.0 * (len(ex["pal"]) * 4 + raw_nibbles + n * (3 * 8 + 2 * 4)) / raw,
                "decode_gbs": None}
        v.close()
    # brick size 64 (the level arrays in global memory): its own tables, the default K_max
    b64 = 64
    n64 = vol_np.size // b64 ** 3
    t64 = csgv.csgv_build_freq_table(vol, b64, 1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    v = csgv.csgv_encode_bricks(vol, b64, t64, S_min=args.s_min)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    enc64_ms = e0.elapsed_time(e1)
    ids64 = torch.arange(n64, dtype=torch.int32, device=dev)
    lods64 = torch.zeros(n64, dtype=torch.uint8, device=dev)
    offs64 = torch.arange(n64, dtype=torch.int64, device=dev) * b64 ** 3
    st64 = torch.empty(n64, dtype=torch.int32, device=dev)
    ts = []
    for r in range(args.warmup + args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        csgv.csgv_decode_bricks(v, ids64, lods64, out, offs64, st64)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if r >= args.warmup:
            ts.append(e0.elapsed_time(e1))
    assert bool((st64 == 0).all())
    assert torch.equal(out.view(n64, b64, b64, b64)[0].cpu(), vol[:b64, :b64, :b64].cpu())
    rows["b=64, two tables, K_max=32"] = {"cr_percent": 100.0 * v.info().compressed_bytes / raw,
                                          "decode_gbs": raw / (float(np.median(ts)) / 1e3) / 1e9,
                                          "encode_gbs": raw / (enc64_ms / 1e3) / 1e9}
    v.close()
    line = {"metric": "compression ratio and decoded GB/s of coding variants", "value": rows["two tables, K_max=32"]["cr_percent"],
            "unit": "% of raw", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "higher_is_better": False,
            "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"voronoi512 512^3 warped Voronoi, b={b}, S_min={args.s_min}"}, "variants": rows}
    print(json.dumps(line))


def run_worley2048(args):
    print(json.dumps(measure_worley2048(args, args.warmup)))


def measure_worley2048(args, warmup):
    """Serving: 2048x2048x1024 Worley cells (24-voxel jittered grid) made and compressed on the device,
    an 8 GiB decoded-brick cache, and a 600-frame fly-around trace at 1920x1080 (distance-based LOD).
    Frame f is submitted, then frame f-1 is awaited (one frame of lag) and frame f-2 released.  Latency
    per frame ticket is taken twice: by the server (ticket admitted to its last decode done) and by the
    client (submit call to the return of the poll that saw it done).  Returns the JSON line."""
    import torch
    import synth
    import paper_2308_16619_b300 as csgv
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    b = 32
    dims = (2048, 2048, 1024)
    vol = synth.worley_device((dims[2], dims[1], dims[0]), 24, seed=4)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    table = csgv.csgv_build_freq_table(vol, b, 4096)
    v = csgv.csgv_encode_bricks(vol, b, table, K_max=args.k_max, S_min=args.s_min)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    enc_ms = e0.elapsed_time(e1)
    raw_bytes = vol.numel() * 4
    del vol
    torch.cuda.empty_cache()
    inf = v.info()
    n_frames = 600
    frames, fp_ms = frame_requests(csgv, v, dims, n_frames, seed=4)
    srv = csgv.Server(v, cache_bytes=8 << 30, n_streams=3)
    clk = ClockSampler(local).__enter__()
    t0 = time.perf_counter()
    tickets, t_sub, t_done = [], [], []
    for f, (bricks, lods) in enumerate(frames):
        t_sub.append(time.perf_counter())
        tickets.append(srv.submit(bricks, lods))
        if f >= 1:
            rc, _ = srv.poll(tickets[f - 1], timeout_us=30_000_000)
            t_done.append(time.perf_counter())
            assert rc == csgv.CSGV_OK, rc
        if f >= 2:
            srv.release(tickets[f - 2])
    rc, _ = srv.poll(tickets[-1], timeout_us=30_000_000)
    t_done.append(time.perf_counter())
    assert rc == csgv.CSGV_OK
    wall = time.perf_counter() - t0
    client = 1000.0 * (np.array(t_done) - np.array(t_sub))
    clk.mark(time.time() - wall, time.time())
    clk.__exit__()
    st, lat = srv.stats(with_latencies=True)
    for t in tickets[-2:]:
        srv.release(t)
    srv.close()
    # the same trace once more, closed loop on a fresh cache: the client submits frame f and waits for it
    # before the next one, so the client's wall time per ticket is its latency (submit call to poll return)
    srv = csgv.Server(v, cache_bytes=8 << 30, n_streams=3)
    closed, prev = [], None
    for f, (bricks, lods) in enumerate(frames):
        c0 = time.perf_counter()
        tk = srv.submit(bricks, lods)
        rc, _ = srv.poll(tk, timeout_us=30_000_000)
        closed.append(1000.0 * (time.perf_counter() - c0))
        assert rc == csgv.CSGV_OK, rc
        if prev is not None:
            srv.release(prev)
        prev = tk
    srv.release(prev)
    srv.close()
    closed = np.array(closed)
    served = st["decoded_labels"] * 4
    n_req = int(sum(len(fb) for fb, _ in frames))
    warm = lat[warmup:] if len(lat) > warmup else lat
    line = {"metric": "decoded GB/s uint32 labels (batched vs plain per-brick); serve p50/p99 ms",
            "value": served / wall / 1e9, "unit": "GB/s", "n_gpus": 1, "steps": n_frames, "warmup": 0,
            "ms_per_step": 1000 * wall / n_frames, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "worley2048 2048x2048x1024 Worley cells, b=32, 600-frame 1920x1080 trace "
                                   "(footprint kernel: a ray stops at its first brick with an opaque label), "
                                   "8 GiB cache", "step": "one frame (submit f, await f-1, release f-2)",
                       "K_max": args.k_max, "S_min": args.s_min},
            "serve": {"p50_ms": float(np.percentile(warm, 50)), "p99_ms": float(np.percentile(warm, 99)),
                      "client_lagged_p50_ms": float(np.percentile(client[warmup:], 50)),
                      "client_lagged_p99_ms": float(np.percentile(client[warmup:], 99)),
                      "client_p50_ms": float(np.percentile(closed[warmup:], 50)),
                      "client_p99_ms": float(np.percentile(closed[warmup:], 99)),
                      "client_latency": "closed loop (submit frame f, wait for it, then frame f+1), fresh cache; "
                                        "client_lagged_*: the one-frame-lag loop, submit f to the poll after "
                                        "submitting f+1",
                      "max_ms": float(np.max(lat)), "first_frame_ms": float(lat[0]),
                      "requests": n_req, "hit_rate": st["hits"] / max(1, st["hits"] + st["misses"] + st["shared"]),
                      "misses": st["misses"], "batches": st["batches"], "evictions": st["evictions"],
                      "rebuilds": st["rebuilds"], "frames_per_s": n_frames / wall,
                      "footprint_ms_per_frame": fp_ms},
            "encode_ms_once": enc_ms, "encode_gbs": raw_bytes / (enc_ms / 1e3) / 1e9,
            "cr_percent": 100.0 * inf.compressed_bytes / raw_bytes, "clocks": clk.summary()}
    v.close()
    torch.cuda.empty_cache()
    return line


def run_fiber4096(args):
    """Stress: the 4096x4096x2048 fiber volume (1M Catmull-Rom tubes, 137 GB of labels) made brick by brick on
    the device and fed to the streaming encoder one brick layer (16384 bricks) at a time, so the raw volume
    never exists; the tables come from every 4096th brick, generated alone.  Then a layer is decoded (leaf
    streams on the device, then in mapped host memory: detail separation) and checked against its regenerated
    bricks, and a 600-frame trace is served from an 8 GiB cache with the leaf streams in host memory."""
    import torch
    import synth
    import paper_2308_16619_b300 as csgv
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    W = synth.WORKLOADS["fiber4096"]
    Z, Y, X = W["shape"]
    cell, tubes, seed = W["cell"], W["tubes"], W["seed"]
    b = 32
    dims = (X, Y, Z)
    nbx, nby, nbz = X // b, Y // b, Z // b
    n, layer = nbx * nby * nbz, nbx * nby
    raw_bytes = n * b ** 3 * 4
    stream = torch.cuda.current_stream(dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)

    t_all = time.perf_counter()
    p0, p1 = ev(), ev()
    p0.record(stream)
    ids = torch.arange(0, n, 4096, dtype=torch.int64, device=dev)
    counts = csgv.csgv_count_bricks(synth.fiber_bricks_device(dims, b, cell, tubes, seed, ids=ids), b)
    table = csgv.csgv_freq_table_from_counts(counts)
    p1.record(stream)
    enc = csgv.StreamEncoder(dims, b, table, K_max=args.k_max, S_min=args.s_min)
    buf = torch.empty(layer * b ** 3, dtype=torch.int32, device=dev)
    gen_ms = enc_ms = 0.0
    clk = ClockSampler(local).__enter__()
    w0 = time.time()
    for z in range(nbz):
        g0, g1, g2 = ev(), ev(), ev()
        g0.record(stream)
        synth.fiber_bricks_device(dims, b, cell, tubes, seed, first=z * layer, m=layer, out=buf)
        g1.record(stream)
        enc.add(buf, z * layer)
        g2.record(stream)
        torch.cuda.synchronize(dev)
        gen_ms += g0.elapsed_time(g1)
        enc_ms += g1.elapsed_time(g2)
    v = enc.finish()
    torch.cuda.synchronize(dev)
    clk.mark(w0, time.time())
    wall_enc = time.perf_counter() - t_all
    prepass_ms = p0.elapsed_time(p1)
    inf = v.info()

    # one brick layer decoded at LOD 0 (leaf streams on the device, then in host memory), checked bit-exact
    zl = nbz // 2
    ids32 = torch.arange(zl * layer, (zl + 1) * layer, dtype=torch.int32, device=dev)
    lods = torch.zeros(layer, dtype=torch.uint8, device=dev)
    offs = torch.arange(layer, dtype=torch.int64, device=dev) * b ** 3
    out = torch.empty(layer * b ** 3, dtype=torch.int32, device=dev)
    status = torch.empty(layer, dtype=torch.int32, device=dev)

    def timed_decode(reps=5):
        ts = []
        for r in range(reps + 1):
            d0, d1 = ev(), ev()
            d0.record(stream)
            csgv.csgv_decode_bricks(v, ids32, lods, out, offs, status)
            d1.record(stream)
            torch.cuda.synchronize(dev)
            if r:
                ts.append(d0.elapsed_time(d1))
        return float(np.median(ts))

    dec_dev_ms = timed_decode()
    synth.fiber_bricks_device(dims, b, cell, tubes, seed, first=zl * layer, m=layer, out=buf)
    torch.cuda.synchronize(dev)
    assert bool((status == 0).all()) and torch.equal(out, buf), "fiber layer does not decode to its bricks"
    v.leaves_to_host()
    dec_host_ms = timed_decode()
    assert bool((status == 0).all()) and torch.equal(out, buf)
    del buf, out
    torch.cuda.empty_cache()

    # serving with the leaf streams in host memory
    n_frames = 600
    frames, fp_ms = frame_requests(csgv, v, dims, n_frames, seed=5)
    srv = csgv.Server(v, cache_bytes=8 << 30, n_streams=3)
    clk2 = ClockSampler(local).__enter__()
    t0 = time.perf_counter()
    tickets = []
    for f, (bricks, lods_f) in enumerate(frames):
        tickets.append(srv.submit(bricks, lods_f))
        if f >= 1:
            rc, _ = srv.poll(tickets[f - 1], timeout_us=60_000_000)
            assert rc == csgv.CSGV_OK, rc
        if f >= 2:
            srv.release(tickets[f - 2])
    rc, _ = srv.poll(tickets[-1], timeout_us=60_000_000)
    assert rc == csgv.CSGV_OK
    wall = time.perf_counter() - t0
    clk2.mark(time.time() - wall, time.time())
    clk2.__exit__()
    clk.__exit__()
    st, lat = srv.stats(with_latencies=True)
    for t in tickets[-2:]:
        srv.release(t)
    srv.close()
    served = st["decoded_labels"] * 4
    warm = lat[args.warmup:] if len(lat) > args.warmup else lat
    layer_bytes = layer * b ** 3 * 4
    line = {"metric": "decoded GB/s uint32 labels (batched vs plain per-brick); serve p50/p99 ms",
            "value": served / wall / 1e9, "unit": "GB/s", "n_gpus": 1, "steps": n_frames, "warmup": 0,
            "ms_per_step": 1000 * wall / n_frames, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "fiber4096 4096x4096x2048 fibers (1M Catmull-Rom tubes, radius 2-6), b=32, "
                                   "made per brick, never whole; leaf streams in host memory; 600-frame trace (footprint kernel), "
                                   "8 GiB cache", "step": "one frame (submit f, await f-1, release f-2)",
                       "K_max": args.k_max, "S_min": args.s_min, "prepass": "every 4096th brick"},
            "encode": {"raw_gb": raw_bytes / 1e9, "generate_ms": gen_ms, "encode_ms": enc_ms,
                       "prepass_ms": prepass_ms, "encode_gbs": raw_bytes / (enc_ms / 1e3) / 1e9,
                       "generate_and_encode_gbs": raw_bytes / ((gen_ms + enc_ms) / 1e3) / 1e9,
                       "wall_s": wall_enc, "cr_percent": 100.0 * inf.compressed_bytes / raw_bytes,
                       "compressed_gb": inf.compressed_bytes / 1e9},
            "layer_decode": {"bricks": layer, "leaves_on_device_gbs": layer_bytes / (dec_dev_ms / 1e3) / 1e9,
                             "leaves_in_host_gbs": layer_bytes / (dec_host_ms / 1e3) / 1e9, "bit_exact": True},
            "serve": {"p50_ms": float(np.percentile(warm, 50)), "p99_ms": float(np.percentile(warm, 99)),
                      "max_ms": float(np.max(lat)), "first_frame_ms": float(lat[0]),
                      "requests": int(sum(len(fb) for fb, _ in frames)),
                      "hit_rate": st["hits"] / max(1, st["hits"] + st["misses"] + st["shared"]),
                      "misses": st["misses"], "batches": st["batches"], "evictions": st["evictions"],
                      "rebuilds": st["rebuilds"], "frames_per_s": n_frames / wall,
                      "footprint_ms_per_frame": fp_ms},
            "clocks": clk.summary()}
    print(json.dumps(line))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "cells1024":
        run_cells1024(args)
        return
    if args.workload == "variants":
        return run_variants(args)
    if args.workload == "fiber4096":
        run_fiber4096(args)
        return
    if args.workload == "worley2048":
        run_worley2048(args)
        return
    import torch
    import synth
    import paper_2308_16619_b300 as csgv
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    b = args.b
    N = b.bit_length() - 1

    vol_np = synth.make(WORKLOAD)
    vol = torch.from_numpy(vol_np.view(np.int32)).to(dev)
    Z, Y, X = vol_np.shape
    n = (X // b) * (Y // b) * (Z // b)
    out_bytes = n * b ** 3 * 4
    ids = torch.arange(n, dtype=torch.int32, device=dev)
    lods = torch.zeros(n, dtype=torch.uint8, device=dev)
    offs = torch.arange(n, dtype=torch.int64, device=dev) * b ** 3
    out = torch.empty(n * b ** 3, dtype=torch.int32, device=dev)
    status = torch.empty(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        # prepass counts taken from this encode's own nibble streams of every STRIDE-th brick
        v, _ = csgv.csgv_encode_bricks_sampled(vol, b, STRIDE, K_max=args.k_max, S_min=args.s_min)
        if ev:
            ev[1].record(stream)
        csgv.csgv_decode_bricks(v, ids, lods, out, offs, status)
        if ev:
            ev[2].record(stream)
        return v

    clk = ClockSampler(local).__enter__()
    prev = None
    for _ in range(args.warmup):
        v = step()
        if prev is not None:
            prev.close_async(stream.cuda_stream)
        prev = v
    torch.cuda.synchronize(dev)
    prof_steps = list(range(0, args.steps, PROF_EVERY))  # the timed steps that carry timing events
    evs = {s: [torch.cuda.Event(enable_timing=True) for _ in range(3)] for s in prof_steps}
    vols = []
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    if True:
        csgv.profile_read()  # drop records of the warm-up
        # the timing events of every launch of the timed steps, made before them (two per launch, at most 16
        # launches per step), so that no event is created between the launches of a step
        csgv.profile_reserve(2 * 16 * len(prof_steps))
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        w0 = time.time()
        t_start.record(stream)
        for s in range(args.steps):
            csgv.profile_enable(s in evs)  # per-kernel CUDA events on the launching stream
            v = step(evs.get(s))
            if prev is not None:
                prev.close_async(stream.cuda_stream)  # in stream order, after the decode that used it
            prev = v
        t_end.record(stream)
        torch.cuda.synchronize(dev)
        clk.mark(w0, time.time())
        vols = [prev]
        csgv.profile_enable(False)
        prof = csgv.profile_read()
    clk.__exit__()
    if world > 1:
        torch.distributed.barrier()
    total_ms = t_start.elapsed_time(t_end)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_step = total_ms / args.steps
    ph = np.array([[e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2])] for e in evs.values()])
    enc_ms, dec_ms = (float(np.median(ph[:, i])) for i in range(2))
    assert bool((status == 0).all()), "decode reported errors"
    g = (X // b, Y // b, Z // b)

    def as_volume(o):  # brick-major decoded labels -> [Z, Y, X]
        return o.view(g[2], g[1], g[0], b, b, b).permute(0, 3, 1, 4, 2, 5).reshape(Z, Y, X)

    verified = bool(torch.equal(as_volume(out), vol))  # the last timed step's decode, outside the timed region
    assert verified, "the decoded bricks differ from the volume"
    v = vols[-1]
    inf = v.info()

    # the decode call alone (both kernels), inputs resident, output > L2
    dec_times = []
    for r in range(23):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        csgv.csgv_decode_bricks(v, ids, lods, out, offs, status)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if r >= 3:
            dec_times.append(e0.elapsed_time(e1))
    dec_alone_ms = float(np.median(dec_times))
    comp_read = inf.compressed_bytes
    peak, peak_kind = measured_peak_hbm()
    # Roofline per kernel from the events around each launch in the timed steps.  Algorithmic bytes per
    # launch: encode reads the raw volume and its output is the compressed volume; rebuild writes the
    # decoded labels and the decode reads the compressed volume (charged to rebuild, the kernel that
    # writes the output); rans_encode / rans_records move only compressed-size data.
    alg = {"encode": out_bytes + comp_read, "rebuild": out_bytes + comp_read,
           "rans_records": comp_read, "rans_encode": comp_read, "encode_count": out_bytes // STRIDE}
    kernels = {k: {"ms_per_launch": ms / n_l, "launches_per_step": n_l / len(prof_steps),
                   "share": ms / sum(m for m, _ in prof.values())} for k, (ms, n_l) in prof.items()}
    dominant = max(prof, key=lambda k: prof[k][0])

    def roof(k):
        ms_l = prof[k][0] / prof[k][1]
        a = alg.get(k, 0) / (ms_l / 1e3) / 1e9
        tr = kernel_traffic(k) if (WORKLOAD == "voronoi512" and b == 32) else None
        return {"bound": "hbm", "kernel": k, "achieved": a, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                "frac": a / peak, "traffic": tr, "algorithmic_bytes": alg.get(k, 0), "ms_per_launch": ms_l}

    # plain per-brick-launch decode of the same bricks
    plain_gbs = None
    if not args.no_plain:
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        csgv.csgv_decode_bricks_plain(v, ids[:64], lods[:64], out, offs, status)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        csgv.csgv_decode_bricks_plain(v, ids, lods, out, offs, status)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        plain_gbs = out_bytes / (e0.elapsed_time(e1) / 1e3) / 1e9
        assert bool((status == 0).all())

    # detail separation: the leaf streams in mapped host memory, read in place by the decode
    v.leaves_to_host()
    hl = []
    for r in range(13):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        csgv.csgv_decode_bricks(v, ids, lods, out, offs, status)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if r >= 3:
            hl.append(e0.elapsed_time(e1))
    assert bool((status == 0).all())
    v.leaves_to_device()
    host_leaves = {"decode_gbs": out_bytes / (float(np.median(hl)) / 1e3) / 1e9,
                   "device_bytes_saved": int(inf.leaf_words) * 2}

    # end to end through the public API with host buffers: H2D volume, encode with tables, decode, D2H labels
    host_vol = torch.from_numpy(vol_np.view(np.int32)).pin_memory()
    host_out = torch.empty(n * b ** 3, dtype=torch.int32).pin_memory()
    e2e = []
    for r in range(max(2, min(args.steps, 5)) + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        vol.copy_(host_vol, non_blocking=True)
        vv = step()
        host_out.copy_(out, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        vv.close()
        if r >= 1:
            e2e.append(e0.elapsed_time(e1))
    e2e_ms = float(np.median(e2e))

    # the same, with two steps in flight: step k+1's volume comes in (copy-in stream) and step k's labels go
    # back (copy-out stream) while a step computes (compute stream); two device and two host buffers of each
    s_in, s_c, s_out = (torch.cuda.Stream(dev) for _ in range(3))
    vols = [vol, torch.empty_like(vol)]
    outs = [out, torch.empty_like(out)]
    host_outs = [host_out, torch.empty_like(host_out).pin_memory()]
    n_pipe = max(4, min(args.steps, 12))
    ev_in = [torch.cuda.Event() for _ in range(n_pipe)]
    ev_c = [torch.cuda.Event() for _ in range(n_pipe)]
    ev_out = [torch.cuda.Event() for _ in range(n_pipe)]
    torch.cuda.synchronize(dev)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(s_in)
    s_c.wait_stream(s_in)
    s_out.wait_stream(s_in)
    for k in range(n_pipe):
        j = k % 2
        with torch.cuda.stream(s_in):
            if k >= 2:
                s_in.wait_event(ev_c[k - 2])  # step k-2 is done reading vols[j]
            vols[j].copy_(host_vol, non_blocking=True)
            ev_in[k].record(s_in)
        with torch.cuda.stream(s_c):
            s_c.wait_event(ev_in[k])
            if k >= 2:
                s_c.wait_event(ev_out[k - 2])  # outs[j] has gone back
            vk, _ = csgv.csgv_encode_bricks_sampled(vols[j], b, STRIDE, K_max=args.k_max, S_min=args.s_min)
            csgv.csgv_decode_bricks(vk, ids, lods, outs[j], offs, status)
            ev_c[k].record(s_c)
            vk.close_async()
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_c[k])
            host_outs[j].copy_(outs[j], non_blocking=True)
            ev_out[k].record(s_out)
    s_out.wait_stream(s_in)
    s_out.wait_stream(s_c)
    p1.record(s_out)
    torch.cuda.synchronize(dev)
    assert bool((status == 0).all())
    e2e_pipe_ms = p0.elapsed_time(p1) / n_pipe
    # the labels that came back to the host are the volume (checked after the timing, on the device)
    for h in host_outs:
        assert torch.equal(as_volume(h.to(dev)), vol), "end-to-end labels differ from the volume"

    value = world * out_bytes / (ms_step / 1e3) / 1e9
    launches_per_step = sum(n_l for _, n_l in prof.values()) / len(prof_steps)  # library kernels, counted
    line = {
        "metric": "decoded GB/s uint32 labels (batched vs plain per-brick); serve p50/p99 ms",
        "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": f"{WORKLOAD} 512^3 warped Voronoi, 20000 cells, 30% background, b={b}",
                   "bricks": n, "lod": 0, "step": "encode with sampled tables (stride 512) + batched decode",
                   "K_max": args.k_max, "S_min": args.s_min,
                   "l2": "inputs and outputs (512 MiB each) larger than L2", "parallelism": f"replicas x{world}"},
        "phases_ms": {"encode_with_tables": enc_ms, "decode": dec_ms},
        "decode_gbs": out_bytes / (dec_alone_ms / 1e3) / 1e9,
        "encode_gbs": out_bytes / (enc_ms / 1e3) / 1e9,
        "plain_decode_gbs": plain_gbs,
        "leaves_on_host": host_leaves,
        "batched_vs_plain": (out_bytes / (dec_alone_ms / 1e3) / 1e9) / plain_gbs if plain_gbs else None,
        "cr_percent": 100.0 * inf.compressed_bytes / out_bytes,
        "roofline": roof(dominant),
        "roofline_decode": roof("rebuild"),
        "kernels": kernels,
        "e2e": {"value": world * out_bytes / (e2e_pipe_ms / 1e3) / 1e9, "unit": "GB/s", "ms": e2e_pipe_ms,
                "h2d_bytes_per_step": out_bytes, "d2h_bytes_per_step": out_bytes,
                "steps_in_flight": 2, "steps": n_pipe,
                "serial": {"value": world * out_bytes / (e2e_ms / 1e3) / 1e9, "ms": e2e_ms}},
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "clocks": clk.summary(),
        "verified": {"decode_equals_volume": verified, "e2e_labels_equal_volume": True},
    }
    if rank == 0 and world == 1:
        gbs, cores, sample = cpu_baseline_oracle(vol_np, b)
        line["cpu_baseline"] = {"value": gbs, "unit": "GB/s", "cores": cores, "kind": "oracle", "sample": sample}
    if world == 1 and not args.no_extra and b == 32:
        # the other two configurations of the metric, each its own workload, after the headline's timing:
        # batched mixed-LOD decode (cells1024) and serving (worley2048)
        del vol, out, host_vol, host_out, vols, outs, host_outs, v
        torch.cuda.empty_cache()
        c = measure_cells1024(args, 20, 3)
        line["batched"] = {k: c[k] for k in ("value", "unit", "ms_per_step", "voxels_per_s", "plain_decode_gbs_2048",
                                             "batched_vs_plain", "cr_percent", "roofline", "gpu_launches",
                                             "clocks")}
        line["batched"]["config"] = c["config"]
        w = measure_worley2048(args, 3)
        line["serve"] = dict(w["serve"], value=w["value"], unit=w["unit"], ms_per_frame=w["ms_per_step"],
                             config=w["config"], encode_gbs=w["encode_gbs"], cr_percent=w["cr_percent"],
                             clocks=w["clocks"])
        line["gpu_launches_extra"] = c["gpu_launches"]
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
