#!/usr/bin/env python3
"""Throughput of the frame-group enhancement hot path on one GB300 (or N replicas).

Workload: 1080p -> 4K 2x spatial SR with the sliding-window network of five
frames (conv 15->64, 10 residual blocks of 64 channels, conv 64->12,
PixelShuffle(2), bilinear skip), 10-bit 4:2:0 limited-range BT.709 input and
output.  One step = one pass of the whole path for one output frame: ingest
of the newest input frame into the device ring, tuple formation, the 22-layer
conv stack on the tensor cores (or SIMT for FP32), requantisation to 10-bit
4:2:0 planes.  Inputs are seeded synthetic frames resident in HBM; every layer
reads/writes 265 MB (64 channels x 1080p x BF16), far beyond the 129 MB L2, so
no L2 flush is needed between steps.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
instead (the reference arm: there is no reference implementation to run).
Secondary workloads report under their own keys: ``batched`` (24 streams),
``stvsr4x`` (deformable space-time SR), ``pyramid`` (the same with a
three-level feature-pyramid extract stage), ``modes`` (same-size and
vertical-2x scale modes) and ``serving``.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "output Mpix/s per GB300 at 1080p→4K 2x SR, BF16/FP8 vs FP32 at ±1 LSB; p99 latency"
W, H, S = 1920, 1080, 2
OUT_PIX = (W * S) * (H * S)
BODY_FLOP = 2.0 * W * H * 64 * 9 * 64          # one 64->64 3x3 conv at 1080p
ACT_BYTES = W * H * 64 * 2                     # one 64-channel BF16 activation at 1080p (265 MB)
# The trunk's 10 residual blocks run as one fused launch each (res_block_kernel: both
# convs, the middle tensor kept on chip).  Algorithmic DRAM bytes of a block launch: read
# x, write y (the residual re-read of x is an L2 hit; weights, 2 x 74 KB, are negligible).
BLOCK_BYTES = 2 * ACT_BYTES
H2D_BYTES = W * H * 2 + 2 * (W // 2) * (H // 2) * 2
D2H_BYTES = (W * S) * (H * S) * 2 + 2 * (W * S // 2) * (H * S // 2) * 2
NFRAMES = 12                                   # distinct resident input frames, cycled
# DRAM bytes (read + written) per block launch from one ncu capture of the block kernel at
# 1080p; None until the kernel as it stands has been captured
BLOCK_TRAFFIC = 501.1e6
BLOCK_TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum (278.7 + 222.4 MB) of the third "
                        "res_block_kernel launch of this bench's bf16 run with --steps 2, on the kernel as built")
WORKLOAD = ("1080p->4K 2x SR: sliding window T=5, conv 15->64, 10 residual blocks of 64 ch, conv 64->12, "
            "PixelShuffle(2), bilinear skip; 10-bit 4:2:0 limited BT.709 in and out")
DATA = "synthetic: seeded textured 10-bit 4:2:0 frames with global 0-4 px translation; random-init He-normal weights"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d["hbm_gbs"], d["bf16_tflops"], d.get("bf16_tflops_sustained", d["bf16_tflops"]), "measured"
    return 6800.0, 1900.0, 1700.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in out.strip().splitlines():
            t = [x.strip() for x in ln.split(",")]
            if len(t) < 7:
                continue
            try:
                sm.append(float(t[0]))
                mx.append(float(t[1]))
            except ValueError:
                continue
            for n, v in zip(names, t[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if os.environ.get("NVISR_BENCH_GLOO") is None else "gloo")
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def job_value(world, steps, pix_per_step, ms_max):
    """Whole-job output Mpix/s: the pixels every rank produced over the slowest rank's time."""
    return world * steps * pix_per_step / (ms_max * 1e-3) / 1e6


def allmax(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------- GPU arm

def gpu_frames(local):
    import torch
    frames = synth.frames_textured(synth.BASE_SEED + 2, NFRAMES, W, H, 10, "420", "limited")
    dev, pinned = [], []
    for f in frames:
        d, p = [], []
        for k in "YUV":
            a = np.ascontiguousarray(f[k]).view(np.int16)
            t = torch.from_numpy(a)
            p.append(t.pin_memory())
            d.append(t.to(f"cuda:{local}"))
        dev.append(tuple(d))
        pinned.append(tuple(p))
    return dev, pinned


def measure(nv, prec, steps, warmup, dev_frames, local, world, clocks=None, profile=False):
    """Device-timed push/pull loop of one precision.  With profile, per-kernel CUDA
    events are recorded as well (a separate pass: the headline is timed without them)."""
    import torch
    text, blob = synth.net_sr2x_t5()
    eng = nv.Engine(device=local)
    flt = eng.filter(text, blob, nv.fmt(W, H, 10), nv.fmt(W * S, H * S, 10), prec, S)
    out = (torch.empty((H * S, W * S), dtype=torch.int16, device=f"cuda:{local}"),
           torch.empty((H * S // 2, W * S // 2), dtype=torch.int16, device=f"cuda:{local}"),
           torch.empty((H * S // 2, W * S // 2), dtype=torch.int16, device=f"cuda:{local}"))
    pushed = [0]

    def push():
        st = flt.push(dev_frames[pushed[0] % NFRAMES])
        assert st == nv.Status.OK, st
        pushed[0] += 1

    pulled = [0]

    def pull():
        st, _ = flt.pull(out)
        assert st == nv.Status.OK, st
        pulled[0] += 1

    while flt.ready() == 0:  # output 0 needs frames 0..2 (FP8: the calibration tuples 0..3 too)
        push()
    # steady state keeps at most 4 frames ahead of the next output (7-slot ring, 5-frame tuples)
    while pushed[0] - pulled[0] > 4:
        pull()

    def step():
        push()
        pull()

    for _ in range(warmup):
        step()
    stream = torch.cuda.ExternalStream(eng.stream)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    if profile:
        flt.profile(True)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if clocks:
        clocks.start()
    t0.record(stream)
    for _ in range(steps):
        step()
    t1.record(stream)
    t1.synchronize()
    torch.cuda.synchronize()
    ck = clocks.stop() if clocks else None
    ms = t0.elapsed_time(t1)
    prof = None
    if profile:
        prof = flt.profile_read()
        flt.profile(False)
    barrier(world)
    ms_max = allmax(ms, world)
    eng.close()
    return ms_max, prof, ck


def measure_modes(nv, steps, warmup, dev_frames, local):
    """The scale modes besides 2 x 2 SR (Section 3.2's horizontal and vertical scale): a
    same-size enhancement (denoise, 1 x 1) and a vertical 2x (deinterlace, 1 x 2) network
    with the 1080p 2x SR network's trunk (T=5, 15->64, 10 residual blocks of 64), BF16, on the 1080p
    10-bit 4:2:0 frames; device-resident input and output, CUDA events on the engine
    stream around the timed push/pull loop."""
    import torch
    res = {}
    for name, (sx, sy) in (("denoise_1x1", (1, 1)), ("deinterlace_1x2", (1, 2))):
        text, blob = synth.net_tuple(synth.BASE_SEED + 2, frames=5, channels=64, nres=10, scale=(sx, sy))
        eng = nv.Engine(device=local)
        flt = eng.filter(text, blob, nv.fmt(W, H, 10), nv.fmt(W * sx, H * sy, 10), "bf16", (sx, sy))
        dev = f"cuda:{local}"
        out = (torch.empty((H * sy, W * sx), dtype=torch.int16, device=dev),
               torch.empty((H * sy // 2, W * sx // 2), dtype=torch.int16, device=dev),
               torch.empty((H * sy // 2, W * sx // 2), dtype=torch.int16, device=dev))
        k = [0]

        def push():
            assert flt.push(dev_frames[k[0] % NFRAMES]) == nv.Status.OK
            k[0] += 1

        while flt.ready() == 0:
            push()
        pulled = 0
        while k[0] - pulled > 4:
            assert flt.pull(out)[0] == nv.Status.OK
            pulled += 1

        def step():
            push()
            assert flt.pull(out)[0] == nv.Status.OK

        for _ in range(warmup):
            step()
        stream = torch.cuda.ExternalStream(eng.stream)
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(steps):
            step()
        t1.record(stream)
        t1.synchronize()
        ms = t0.elapsed_time(t1)
        eng.close()
        res[name] = {"metric": "output Mpix/s", "value": steps * W * sx * H * sy / (ms * 1e-3) / 1e6,
                     "ms_per_frame": ms / steps, "steps": steps, "input": f"{W}x{H}",
                     "output": f"{W * sx}x{H * sy}"}
    return res


def measure_stvsr(nv, steps, warmup, local, prec="bf16", pyramid=False):
    """Spatio-temporal SR with deformable alignment: 960x540 8-bit 4:2:0, two
    input frames -> two 3840x2160 outputs per run (the frame and the midpoint),
    BF16, device-resident input.  Reports output Mpix/s and the DCN kernel's
    time and achieved bytes (features + offsets/mask read, output written).
    pyramid: the network whose extract stage is a three-level feature pyramid,
    aligned at every level (its extract features are cached per frame)."""
    import torch
    w, h = 960, 540
    text, blob = synth.net_group_pyramid(synth.BASE_SEED + 3) if pyramid else synth.net_stvsr4x()
    frs = synth.frames_textured(synth.BASE_SEED + 3, 4, w, h, 8, "420", "limited")
    dev = f"cuda:{local}"
    frames = [tuple(torch.from_numpy(np.ascontiguousarray(f[c])).to(dev) for c in "YUV") for f in frs]
    eng = nv.Engine(device=local)
    flt = eng.filter(text, blob, nv.fmt(w, h, 8), nv.fmt(4 * w, 4 * h, 8), prec, 4)
    out = (torch.empty((4 * h, 4 * w), dtype=torch.uint8, device=dev),
           torch.empty((2 * h, 2 * w), dtype=torch.uint8, device=dev),
           torch.empty((2 * h, 2 * w), dtype=torch.uint8, device=dev))
    k = [0]

    def push():
        assert flt.push(frames[k[0] % 4]) == nv.Status.OK
        k[0] += 1

    def run():  # one input frame in, two outputs out
        push()
        for _ in range(2):
            st, _ = flt.pull(out)
            assert st == nv.Status.OK, st

    push()
    for _ in range(warmup):
        run()
    torch.cuda.synchronize()
    flt.profile(True)
    t0 = time.perf_counter()
    for _ in range(steps):
        run()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    prof = flt.profile_read()
    flt.profile(False)
    hits, misses = flt.cache_stats()
    eng.close()
    dcn_ms, dcn_n = prof["dcn"]
    # per DCN application: x (64 ch BF16) + offsets/mask (216 ch float32) read, y (64 ch BF16) written
    dcn_bytes = w * h * (64 * 2 + 216 * 4 + 64 * 2)
    net_text = ("extract pyramid 3->64, pool + 64->64 at 1/2 and 1/4 size (cached per frame); per level an "
                "offset/mask head 128->216 and a modulated deformable conv 64->64 (8 groups), coarse-to-fine 1x1 "
                "blends with the bilinear x2 of the level below" if pyramid else
                "extract 3->64 (cached per frame), offset/mask head 128->216, modulated deformable conv 64->64 "
                "(8 groups)")
    return {"workload": "960x540 8-bit 4:2:0 -> 2 x 3840x2160 per input frame: " + net_text + ", 1x1 blend, "
                        "6 residual blocks, two PixelShuffle(2) stages; BF16; device-resident input",
            "metric": "output Mpix/s", "value": steps * 2 * 16 * w * h / dt / 1e6, "steps": steps,
            "extract_cache": {"hits": hits, "misses": misses},
            "kernel_ms_per_run": {kk: round(v[0] / steps, 4) for kk, v in prof.items() if v[1]},
            "dcn": {"us_per_launch": dcn_ms / max(dcn_n, 1) * 1e3, "launches_per_run": dcn_n / steps,
                    "bytes_per_launch": dcn_bytes,
                    "achieved_gbs": dcn_bytes / (dcn_ms / max(dcn_n, 1) * 1e-3) / 1e9,
                    "gflop_per_launch": 2 * w * h * 64 * 576 / 1e9}}


# Batched multi-stream workload: 24 concurrent streams of the same network (BF16)
BATCH_STREAMS = ([(854, 480, 8, "420")] * 8 + [(1280, 720, 10, "420")] * 8 + [(1920, 1080, 8, "444")] * 8)
BATCH_OUT_PIX = sum(4 * w * h for w, h, _, _ in BATCH_STREAMS)


def measure_batched(nv, steps, warmup, local):
    """24 streams stepped together: one batch step (shared launches, CUDA graph)
    against the per-stream sequential engine step, both with device-resident
    input planes and device outputs.  Scene cuts: geometric gaps, p = 1/40."""
    import torch
    text, blob = synth.net_sr2x_t5()
    dev = f"cuda:{local}"
    clips = {}
    for key in set(BATCH_STREAMS):
        w, h, bits, sub = key
        frs = synth.frames_textured(synth.BASE_SEED + 4, 2, w, h, bits, sub, "limited")
        clips[key] = [tuple(torch.from_numpy(np.ascontiguousarray(f[c]).view(np.int16) if bits > 8
                                             else np.ascontiguousarray(f[c])).to(dev) for c in "YUV") for f in frs]
    rng = np.random.default_rng(synth.BASE_SEED + 4)
    total = warmup + steps + 8
    cuts = [rng.uniform(size=total) < 1.0 / 40 for _ in BATCH_STREAMS]

    def run(batched):
        eng = nv.Engine(device=local)
        flts, outs = [], []
        for w, h, bits, sub in BATCH_STREAMS:
            flts.append(eng.filter(text, blob, nv.fmt(w, h, bits, sub), nv.fmt(2 * w, 2 * h, bits, sub), "bf16", 2))
            dt = torch.int16 if bits > 8 else torch.uint8
            cw, ch = (w, h) if sub == "444" else (w // 2, h // 2)
            outs.append((torch.empty((2 * h, 2 * w), dtype=dt, device=dev),
                         torch.empty((2 * ch, 2 * cw), dtype=dt, device=dev),
                         torch.empty((2 * ch, 2 * cw), dtype=dt, device=dev)))
        bt = eng.batch(flts) if batched else None
        k = [0]

        def push_all():
            for i, (f, key) in enumerate(zip(flts, BATCH_STREAMS)):
                assert f.push(clips[key][k[0] % 2], cut=bool(cuts[i][k[0]]) and k[0] > 0) == nv.Status.OK
            k[0] += 1

        def step():
            push_all()
            n = bt.step() if batched else eng.step()
            for f, o in zip(flts, outs):
                st, _ = f.pull(o)
                assert st == nv.Status.OK, st
            return n

        push_all()
        push_all()
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            step()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        info = bt.info() if batched else None
        if bt:
            bt.close()
        eng.close()
        return dt, info

    dt_b, info = run(True)
    dt_s, _ = run(False)
    vb = steps * BATCH_OUT_PIX / dt_b / 1e6
    vs = steps * BATCH_OUT_PIX / dt_s / 1e6
    return {"workload": "24 streams, the 2x SR network (T=5, 10 residual blocks of 64) BF16: 8x 854x480 8-bit 4:2:0, 8x 1280x720 10-bit 4:2:0, "
                        "8x 1920x1080 8-bit 4:4:4; one output per stream per step; scene cuts p=1/40",
            "metric": "output Mpix/s", "value": vb, "sequential_value": vs, "speedup": vb / vs,
            "ms_per_step": dt_b / steps * 1e3, "sequential_ms_per_step": dt_s / steps * 1e3, "steps": steps,
            "warmup": warmup, "out_pix_per_step": BATCH_OUT_PIX, "cuda_graphs": info["graphs"],
            "rows_per_strip": info["rows_per_strip"],
            "baseline": "per-stream sequential launches (nvisr_engine_step)",
            "timing": "wall clock between device synchronisations (host launch work included)"}


SERVE_RES = [(854, 480), (1280, 720), (1920, 1080), (2560, 1440)]


def measure_serving(nv, seconds, rate, budget_gb, local, seed=synth.BASE_SEED + 5):
    """Serving loop: clips arrive as a Poisson process (rate per second) for
    `seconds`; each has log-uniform [30, 600] frames, a resolution from
    SERVE_RES, 8 or 10 bits 4:2:0, and runs the 2x tuple network or the 4x
    two-frame deformable network (50/50) in BF16, under an HBM budget.  Host
    input planes are pushed one frame per clip per server step; outputs are
    pulled into device planes.  Clips still running when the window closes
    count with the outputs they produced."""
    import torch
    rng = np.random.default_rng(seed)
    nets = {"sr2x": (synth.net_sr2x_t5(), 2), "stvsr": (synth.net_stvsr4x(), 4)}
    frames = {}
    outbuf = {}
    eng = nv.Engine(device=local, hbm_budget_bytes=int(budget_gb * 2 ** 30))
    srv = nv.Server(eng)
    dev = f"cuda:{local}"
    clips = {}
    out_pix = 0
    t0 = time.perf_counter()
    next_arrival = t0 + rng.exponential(1.0 / rate)
    submitted = 0
    steps = 0
    while time.perf_counter() - t0 < seconds:
        now = time.perf_counter()
        while next_arrival <= now:
            w, h = SERVE_RES[rng.integers(len(SERVE_RES))]
            bits = 8 if rng.uniform() < 0.5 else 10
            net = "sr2x" if rng.uniform() < 0.5 else "stvsr"
            n = int(round(np.exp(rng.uniform(np.log(30), np.log(600)))))
            (text, blob), sc = nets[net]
            key = (w, h, bits)
            if key not in frames:
                frames[key] = synth.frames_textured(seed, 2, w, h, bits, "420", "limited")
            okey = (sc * w, sc * h, bits)
            if okey not in outbuf:
                dt = torch.int16 if bits > 8 else torch.uint8
                outbuf[okey] = (torch.empty((sc * h, sc * w), dtype=dt, device=dev),
                                torch.empty((sc * h // 2, sc * w // 2), dtype=dt, device=dev),
                                torch.empty((sc * h // 2, sc * w // 2), dtype=dt, device=dev))
            cid = srv.submit(text, blob, nv.fmt(w, h, bits), nv.fmt(sc * w, sc * h, bits), "bf16", sc)
            clips[cid] = {"key": key, "okey": okey, "n": n, "next": 0, "flushed": False}
            submitted += 1
            next_arrival += rng.exponential(1.0 / rate)
        for cid, c in clips.items():
            if c["next"] < c["n"]:
                fr = frames[c["key"]][c["next"] % 2]
                if srv.push(cid, (fr["Y"], fr["U"], fr["V"])) == nv.Status.OK:
                    c["next"] += 1
            elif not c["flushed"] and srv.flush(cid) == nv.Status.OK:
                c["flushed"] = True
        srv.step()
        steps += 1
        done = []
        for cid, c in clips.items():
            while True:
                st, _ = srv.pull(cid, outbuf[c["okey"]])
                if st == nv.Status.OK:
                    out_pix += c["okey"][0] * c["okey"][1]
                    continue
                if st == nv.Status.EOS:
                    done.append(cid)
                break
        for cid in done:
            srv.close_clip(cid)
            del clips[cid]
    torch.cuda.synchronize()
    elapsed = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    eng.close()
    return {"workload": f"Poisson clip arrivals at {rate}/s for {seconds} s; 30-600 frames (log-uniform); "
                        "480p/720p/1080p/1440p, 8/10-bit 4:2:0; 2x tuple network or 4x deformable two-frame "
                        f"network (50/50), BF16; {budget_gb} GB HBM budget",
            "metric": "output Mpix/s", "value": out_pix / elapsed / 1e6, "seconds": elapsed,
            "latency_p50_ms": st["latency_p50_ms"], "latency_p99_ms": st["latency_p99_ms"],
            "queue_p50_ms": st["queue_p50_ms"], "queue_p99_ms": st["queue_p99_ms"],
            "submitted": submitted, "admitted": st["admitted"], "completed": st["completed"],
            "pending_at_end": st["pending"], "active_at_end": st["active"], "outputs": st["outputs"],
            "deferred_admissions": st["deferred_steps"], "server_steps": steps}


def measure_e2e(nv, prec, steps, pinned, local):
    """Host planes in, host planes out, through nvisr_push / nvisr_pull (copies inside)."""
    import torch
    text, blob = synth.net_sr2x_t5()
    eng = nv.Engine(device=local)
    flt = eng.filter(text, blob, nv.fmt(W, H, 10), nv.fmt(W * S, H * S, 10), prec, S)
    out = (torch.empty((H * S, W * S), dtype=torch.int16).pin_memory(),
           torch.empty((H * S // 2, W * S // 2), dtype=torch.int16).pin_memory(),
           torch.empty((H * S // 2, W * S // 2), dtype=torch.int16).pin_memory())
    k = [0]

    def push():
        assert flt.push(pinned[k[0] % NFRAMES]) == nv.Status.OK
        k[0] += 1

    while flt.ready() == 0:
        push()
    pulled = 0
    while k[0] - pulled > 4:
        assert flt.pull(out)[0] == nv.Status.OK
        pulled += 1
    lat = []
    for i in range(steps + 3):
        t = time.perf_counter()
        push()
        st, _ = flt.pull(out)
        assert st == nv.Status.OK
        pulled += 1
        if i >= 3:
            lat.append(time.perf_counter() - t)
    eng.close()
    total = sum(lat)
    lat_ms = sorted(x * 1e3 for x in lat)
    p = lambda q: lat_ms[min(len(lat_ms) - 1, int(round(q * (len(lat_ms) - 1))))]
    return total, p(0.5), p(0.99)


# ---------------------------------------------------------------------------- oracle arm

def oracle_sample(side_w, side_h, seed=synth.BASE_SEED + 2):
    """The oracle on a crop of the workload: 5 frames -> ingest -> network -> requantise 1 output."""
    import oracle
    frames = synth.frames_textured(seed, 5, side_w, side_h, 10, "420", "limited")
    flags = np.zeros(5, bool)
    text, blob = synth.net_sr2x_t5()
    fd = dict(bit_depth=10, subsampling="420", range="limited", chroma_loc="left")
    t = time.perf_counter()
    oracle.run_filter(frames, flags, text, blob, fd, fd, outputs=[2])
    dt = time.perf_counter() - t
    return dt, (2 * side_w) * (2 * side_h), oracle.oracle_threads()


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    oracle.oracle_threads()  # builds the C routines before timing
    side_w, side_h = 48, 48
    for _ in range(args.warmup):
        oracle_sample(side_w, side_h)
    total, px = 0.0, 0
    for _ in range(args.steps):
        dt, p, cores = oracle_sample(side_w, side_h)
        total += dt
        px += p
    val = px / total / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "Mpix/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": DATA, "config": {"workload": WORKLOAD, "input": f"{W}x{H}", "output": f"{W*S}x{H*S}",
                                     "parallelism": f"replicas{args.gpus}"},
            "cpu_baseline": {"value": val, "unit": "Mpix/s", "cores": cores, "kind": "oracle",
                             "sample": f"per step: one output of the full path on a {side_w}x{side_h} crop "
                                       f"of 5 frames ({2*side_w}x{2*side_h} output px)"},
            "e2e": {"value": val, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------- main

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precisions", default="bf16,fp16,fp8,fp32")
    ap.add_argument("--e2e-steps", type=int, default=30)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batched-steps", type=int, default=12, help="steps of the 24-stream batched run (0 = skip)")
    ap.add_argument("--stvsr-steps", type=int, default=20, help="runs of the deformable ST-SR network (0 = skip)")
    ap.add_argument("--serve-seconds", type=float, default=20.0, help="serving-loop window (0 = skip)")
    ap.add_argument("--modes-steps", type=int, default=30, help="frames of each 1x1 / 1x2 scale mode (0 = skip)")
    ap.add_argument("--serve-rate", type=float, default=6.0, help="clip arrivals per second")
    ap.add_argument("--serve-budget-gb", type=float, default=120.0)
    args = ap.parse_args()
    rank, world, local = dist_init()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    import paper_2308_03121_gb300 as nv
    torch.cuda.set_device(local)
    nv.load()
    hbm, bf16_burst, bf16_sust, peak_src = peaks()
    dev_frames, pinned = gpu_frames(local)
    results = {}
    clocks = Clocks(local)
    head = "bf16"
    precs = [p for p in args.precisions.split(",") if p]
    if head not in precs:
        precs.insert(0, head)
    errors = {}
    for prec in precs:
        steps = args.steps if prec != "fp32" else max(5, min(args.steps, 40))
        try:
            ms, _, ck = measure(nv, prec, steps, args.warmup, dev_frames, local, world,
                                clocks if prec == head else None)
            # per-kernel times come from a second, profiled pass
            psteps = max(3, min(steps, 50))
            pms, prof, _ = measure(nv, prec, psteps, args.warmup, dev_frames, local, world, profile=True)
        except Exception as e:  # a secondary precision failing must not hide the headline
            if prec == head:
                raise
            errors[prec] = repr(e)
            continue
        results[prec] = {"ms": ms, "steps": steps, "prof": prof, "psteps": psteps, "pms": pms, "clocks": ck,
                         "mpix_s": job_value(world, steps, OUT_PIX, ms)}
    r = results[head]
    prof = r["prof"]
    body_ms, body_n = prof["conv_body"]
    avg_body = body_ms / max(body_n, 1)
    # 20 trunk convolutions per step in body_n / psteps launches (10 fused blocks)
    convs = 20 * r["psteps"] / max(body_n, 1)
    achieved_tf = convs * BODY_FLOP / (avg_body * 1e-3) / 1e12
    achieved_gbs = convs / 2 * BLOCK_BYTES / (avg_body * 1e-3) / 1e9
    launches = round(sum(n for _, n in prof.values()) * r["steps"] / r["psteps"])
    e2e_total, p50, p99 = measure_e2e(nv, head, args.e2e_steps, pinned, local)
    stvsr = pyramid = None
    if args.stvsr_steps > 0:
        try:
            stvsr = measure_stvsr(nv, args.stvsr_steps, 3, local)
        except Exception as e:  # the secondary workload must not hide the headline
            errors["stvsr4x"] = repr(e)
        try:
            pyramid = measure_stvsr(nv, args.stvsr_steps, 3, local, pyramid=True)
        except Exception as e:  # the secondary workload must not hide the headline
            errors["pyramid"] = repr(e)
    modes = None
    if args.modes_steps > 0:
        try:
            modes = measure_modes(nv, args.modes_steps, 3, dev_frames, local)
        except Exception as e:  # the secondary workload must not hide the headline
            errors["modes"] = repr(e)
    serving = None
    if args.serve_seconds > 0:
        try:
            serving = measure_serving(nv, args.serve_seconds, args.serve_rate, args.serve_budget_gb, local)
        except Exception as e:  # the secondary workload must not hide the headline
            errors["serving"] = repr(e)
    batched = None
    if args.batched_steps > 0:
        try:
            batched = measure_batched(nv, args.batched_steps, 3, local)
        except Exception as e:  # the secondary workload must not hide the headline
            errors["batched"] = repr(e)
    e2e_val = world * args.e2e_steps * OUT_PIX / e2e_total / 1e6
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        dt, px, cores = oracle_sample(320, 192)
        cpu = {"value": px / dt / 1e6, "unit": "Mpix/s", "cores": cores, "kind": "oracle",
               "sample": f"one output of the full path (ingest, network, requantise) on a 320x192 crop of "
                         f"5 frames: {px} output px in {dt:.1f} s"}
    if rank != 0:
        return
    by_prec = {}
    for p, v in results.items():
        pr = v["prof"]
        by_prec[p] = {"value": v["mpix_s"], "ms_per_step": v["ms"] / v["steps"], "steps": v["steps"],
                      "kernel_ms_per_step": {k: round(ms / v["psteps"], 4) for k, (ms, n) in pr.items() if n},
                      "profiled_ms_per_step": v["pms"] / v["psteps"]}
    if "fp32" in results:
        for p in by_prec:
            by_prec[p]["speedup_vs_fp32"] = by_prec[p]["value"] / by_prec["fp32"]["value"]
    line = {
        "metric": METRIC, "value": r["mpix_s"], "unit": "Mpix/s", "n_gpus": world, "steps": r["steps"],
        "warmup": args.warmup, "ms_per_step": r["ms"] / r["steps"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": head, "data": DATA,
        "config": {"workload": WORKLOAD, "input": f"{W}x{H}", "output": f"{W*S}x{H*S}", "tuple": 5,
                   "l2": "inputs larger than L2: every conv layer streams 265 MB in and out (L2 129 MB)",
                   "parallelism": f"replicas{world}"},
        "frames_per_s": world * r["steps"] / (r["ms"] * 1e-3),
        # the body is a dense contraction: its bound is the tensor pipe (BF16, timed inside
        # a long step, so the sustained peak); its HBM fraction is given beside it
        "roofline": {"kernel": f"res_block_kernel (residual block of two 64->64 3x3 convs in one launch of 2-CTA "
                               f"clusters, BF16, {body_n / r['psteps']:g} launches/step)",
                     "bound": "tensor", "achieved": achieved_tf, "peak": bf16_sust, "unit": "TFLOP/s",
                     "frac": achieved_tf / bf16_sust, "peak_source": f"bf16_tflops_sustained of {peak_src}",
                     "algorithmic_flop_per_launch": convs * BODY_FLOP, "avg_launch_ms": avg_body,
                     "traffic": BLOCK_TRAFFIC, "traffic_source": BLOCK_TRAFFIC_SOURCE,
                     "hbm": {"achieved": achieved_gbs, "peak": hbm, "unit": "GB/s", "frac": achieved_gbs / hbm,
                             "peak_source": f"hbm_gbs of {peak_src}",
                             "algorithmic_bytes_per_launch": convs / 2 * BLOCK_BYTES}},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": "Mpix/s", "h2d_bytes_per_step": H2D_BYTES,
                "d2h_bytes_per_step": D2H_BYTES, "steps": args.e2e_steps},
        "latency_ms": {"p50": p50, "p99": p99, "what": "per-frame push->pull wall time, host planes"},
        "gpu_launches": launches,
        "clocks": r["clocks"],
        "precisions": by_prec,
        "batched": batched,
        "stvsr4x": stvsr,
        "pyramid": pyramid,
        "modes": modes,
        "serving": serving,
        "hbm_peak_gbs": hbm,
    }
    if errors:
        line["errors"] = errors
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
