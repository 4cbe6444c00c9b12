#!/usr/bin/env python
"""Benchmark of the pyramid-splatting mapping iteration on one GB300 (or N replicas).

Default workload (the batched mapping step): 8 keyframes of uneven size (4 x 1200x680 and
4 x 640x480 RGB-D-semantic frames of a seeded 6x5x3 m room with 20 boxes), each with its
3-level pyramid = 24 images, over 500k Gaussians sampled on the room's surfaces, C = 16
semantic features decoded to 32 classes.  One step = one full mapping iteration over every
image: EWA projection, tile lists, compositing, loss (L1 + D-SSIM RGB, masked depth L1,
cross-entropy), adjoint to every Gaussian parameter, Adam -- one persistent launch per
kernel, replayed as one CUDA graph.  L2 is flushed (a 256 MiB write) before every timed
step; the flush is outside each step's event pair.

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle instead (the
reference arm: a bounded pixel sample of the same workload per step, extrapolated).

--workload replica: one 1200x680 keyframe x 3 levels, 300k Gaussians.  --workload scannet:
one 640x480 keyframe x 4 levels (down to 80x60), 1M Gaussians, C = 40 class logits (no
decoder), depth noise 1 cm.
"""
from __future__ import annotations

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

METRIC = "fwd+bwd pyramid-splat iters/s"
UNIT = "iters/s"
WORKLOADS = {
    "replica": dict(workload="replica-like room, 1 keyframe x 3 pyramid levels (1200x680, 600x340, 300x170)",
                    gaussians=300_000, sem_features=16, classes=32, levels=3),
    "batched": dict(workload="replica-like room, 8 keyframes of uneven size (4 x 1200x680, 4 x 640x480) "
                             "x 3 pyramid levels = 24 images in one launch per kernel",
                    gaussians=500_000, sem_features=16, classes=32, levels=3),
    "scannet": dict(workload="scannet-like room, 1 keyframe x 4 pyramid levels (640x480 .. 80x60), "
                             "40 class logits, depth noise 1 cm",
                    gaussians=1_000_000, sem_features=40, classes=40, levels=4),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tile", default="16x16")
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--ppt", type=int, default=1, help="pixels per thread of the forward compositing kernel")
    ap.add_argument("--ppt-bwd", type=int, default=2, help="pixels per thread of the backward kernel")
    ap.add_argument("--batch-bwd", type=int, default=0, help="batch of the backward kernel (0: --batch)")
    ap.add_argument("--half-masks", action="store_true",
                    help="per-instance half masks in the tile lists (one adjoint warp per half of an 8x8 tile)")
    ap.add_argument("--half-tile-fwd", action="store_true",
                    help="with --half-masks: the forward also one warp per half tile")
    ap.add_argument("--workload", default="batched", choices=sorted(WORKLOADS))
    ap.add_argument("--gaussians", type=int, default=None, help="default: the workload's count")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="use --tile/--batch/--ppt as given")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU-baseline sample time")
    return ap.parse_args()


# ------------------------------------------------------------------------------------------
# workload
# ------------------------------------------------------------------------------------------

def build_inputs(workload, n_gauss, seed_offset=0):
    """(cameras, ray-cast level-0 frames, Gaussians, decoder or None) of a workload."""
    import synthetic
    w = WORKLOADS[workload]
    if workload == "scannet":
        room = synthetic.Room(n_classes=40, seed=3)
        cams = [room.trajectory(8, synthetic.SCANNET_LIKE, seed=7)[(1 + seed_offset) % 8]]
        frames = [room.raycast(c, depth_noise=0.01) for c in cams]
    else:
        room = synthetic.Room(n_classes=32, seed=3)
        traj = room.trajectory(8, synthetic.REPLICA_LIKE, seed=7)
        if workload == "batched":
            cams = traj[:4] + room.trajectory(4, synthetic.SCANNET_LIKE, seed=8)
        else:
            cams = [traj[(1 + seed_offset) % 8]]
        frames = [room.raycast(c) for c in cams]
    C = w["sem_features"]
    g = room.sample_gaussians(n_gauss, C, seed=4 + seed_offset, sem_mode="random")
    g["sem"] *= 0.5
    decoder = None
    if C != w["classes"]:
        rng = np.random.default_rng(11)
        decoder = rng.normal(size=(w["classes"], C)).astype(np.float32) * 0.3
    return cams, frames, g, decoder


# ------------------------------------------------------------------------------------------
# algorithmic traffic / flops model (per step)
# ------------------------------------------------------------------------------------------

def step_stats(r):
    """Counts measured from the last forward: visible records, instances, pixels, list
    entries examined up to the last contributor and contributors."""
    import torch
    torch.cuda.synchronize()
    rect = r.rect.view(-1, 2)
    n_vis = int((rect[:, 0] != rect[:, 1]).sum().item())
    K = r.instance_count()
    last = r.last.to(torch.int64)
    E = int(last.sum().item())
    contrib = int(r.n_contrib.to(torch.int64).sum().item())
    return dict(N=r.N, V=r.V, n_vis=n_vis, K=K, P=r.P, E=E, contrib=contrib, C=r.C)


def algorithmic_bytes(s):
    """HBM bytes one iteration must move (float32), by kernel:
    projection fwd 44 N V + 32 R + 8 R (params read per view-level, records + rects written),
    tile lists: compaction 8 R + 8 n_vis, depth sort 24 n_vis, emission 16 n_vis + 8 K,
    tile sort 24 K, ranges 8 K, raster fwd K_r (4 + 24 + 12 + 4C) + P (4 (4 + C) + 12),
    loss P (8 (4 + C) + 24), raster bwd P (4 (4 + C) + 12) + K_r (44 + 4 C) + 2 n_vis 32 +
    atomics, projection bwd n_vis (32 + 32) + N 44 + N 4 (10 + C) grads, Adam N (14 + C) 16."""
    N, V, nv, K, P, C = s["N"], s["V"], s["n_vis"], s["K"], s["P"], s["C"]
    R = N * V
    Kr = K  # instances read (upper bound: tiles stop early)
    b = {}
    b["project_fwd"] = 44 * N + (32 + 8) * R
    b["tile_lists"] = 8 * R + 8 * nv + 24 * nv + 16 * nv + 8 * K + 24 * K + 8 * K
    b["raster_fwd"] = Kr * (4 + 24 + 12 + 4 * C) + P * (4 * (4 + C) + 12)
    b["loss"] = P * (8 * (4 + C) + 24)
    b["raster_bwd"] = P * (4 * (4 + C) + 12) + Kr * (44 + 4 * C) + 2 * nv * 32
    b["project_bwd"] = nv * 64 + N * 44 + N * 4 * (10 + C)
    b["adam"] = N * (14 + C) * 16
    return b


def raster_flops_model(s):
    """Algorithmic flops of the compositing kernels by the per-entry model of the hot path: E
    list entries examined (pixel, entry pairs) times 15 + 2 (4 + C) in the forward and
    40 + 4 (4 + C) in the backward, as if every examined entry contributed."""
    E, C = s["E"], s["C"]
    nf = 4 + C
    return E * (15 + 2 * nf), E * (40 + 4 * nf)


def raster_flops(s):
    """Algorithmic flops of the method (independent of how the kernels map them): alpha
    evaluation ~13 per examined (pixel, entry) pair and 3 + 2 (4 + C) per contributor in
    the forward; the backward re-evaluates alpha (13), and per contributor spends 2 (4 + C)
    on g.f, (4 + C) on the feature gradients and ~25 on the geometric gradients."""
    E, c, C = s["E"], s["contrib"], s["C"]
    nf = 4 + C
    fwd = 13 * E + (3 + 2 * nf) * c
    bwd = 13 * E + (2 * nf + nf + 25) * c
    return fwd, bwd


# ------------------------------------------------------------------------------------------
# DRAM traffic of the dominant kernel, from a committed ncu summary
# ------------------------------------------------------------------------------------------

KERNEL_SOURCES = ["paper_2412_01217_gb300/csrc/raster_impl.cuh", "paper_2412_01217_gb300/csrc/raster.cuh",
                  "paper_2412_01217_gb300/csrc/sg_common.cuh"]


def _code_only(text):
    """Source text without comments and blank lines (a comment edit leaves the hash alone)."""
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(ln.rstrip() for ln in text.splitlines() if ln.strip())


def kernel_source_sha():
    """Hash of the compositing kernels' code (comments excluded), recorded beside every
    profile whose counters the benchmark reuses."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(_code_only(open(os.path.join(ROOT, f)).read()).encode())
    return h.hexdigest()[:16]


def profiled_traffic(kernel, units_now, workload="replica"):
    """dram__bytes_read.sum + dram__bytes_write.sum per launch from profiles/<kernel>_*.md
    (lines 'source_sha: ...', 'dram_bytes_per_launch: ...', 'units: ...'), scaled by the
    units processed if the capture ran a different case; None when the kernel sources
    changed since the capture."""
    import glob
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", f"{kernel}_{workload}_*.md"))):
        kv = {}
        for line in open(path):
            if ":" in line and line.strip().startswith(("source_sha", "dram_bytes_per_launch", "units")):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip().strip("`")
        if kv.get("source_sha") != kernel_source_sha() or "dram_bytes_per_launch" not in kv:
            continue
        b = float(kv["dram_bytes_per_launch"])
        u = float(kv.get("units", units_now) or units_now)
        return b * units_now / u if u else b
    return None


# ------------------------------------------------------------------------------------------
# clocks
# ------------------------------------------------------------------------------------------

# NVML clocks-event reason bits (nvml.h) reported by name
_NVML_REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
                 0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}


class NvmlClocks:
    """Reads the SM clock, its maximum and the active clocks-event reasons of one GPU through
    NVML (libnvidia-ml, read-only queries), fast enough to sample a short timed region every
    few milliseconds.  `ok` is False when NVML is not available."""

    def __init__(self, device_index=0):
        import ctypes
        self.ok = False
        try:
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                return
            h = ctypes.c_void_p()
            found = False
            try:  # match the CUDA device by UUID (NVML may number the GPUs differently)
                import torch
                u = str(torch.cuda.get_device_properties(device_index).uuid)
                u = u if u.startswith("GPU-") else "GPU-" + u
                found = nv.nvmlDeviceGetHandleByUUID(u.encode(), ctypes.byref(h)) == 0
            except Exception:
                found = False
            if not found and nv.nvmlDeviceGetHandleByIndex_v2(device_index, ctypes.byref(h)) != 0:
                return
            self.nv, self.h, self.ct = nv, h, ctypes
            mx = ctypes.c_uint()
            self.max_mhz = float(mx.value) if nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0 else None
            self.reasons_fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                getattr(nv, "nvmlDeviceGetCurrentClocksThrottleReasons")
            self.ok = self.sample() is not None
        except Exception:
            self.ok = False

    def sample(self):
        """(SM MHz, reason bits) now, or None."""
        ct = self.ct
        mhz, bits = ct.c_uint(), ct.c_ulonglong()
        if self.nv.nvmlDeviceGetClockInfo(self.h, 1, ct.byref(mhz)) != 0:
            return None
        if self.reasons_fn(self.h, ct.byref(bits)) != 0:
            bits.value = 0
        return float(mhz.value), int(bits.value)


class ClockSampler:
    """Samples the GPU's SM clock and throttle reasons during the timed region: NVML polled
    every 5 ms by a thread (so even a timed loop of a few tens of milliseconds has samples),
    else nvidia-smi every 100 ms.  Every sample carries the host time it was taken."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []
        self.samples = []  # (host time, MHz, [reason names]) from NVML
        self.nvml = NvmlClocks(index)
        self._stop = threading.Event()

    def start(self):
        if self.nvml.ok:
            def poll():
                while not self._stop.is_set():
                    r = self.nvml.sample()
                    if r is not None:
                        self.samples.append((time.time(), r[0], [n for b, n in _NVML_REASONS.items() if r[1] & b]))
                    time.sleep(0.005)
            self.t = threading.Thread(target=poll, daemon=True)
            self.t.start()
            return
        cmd = ["nvidia-smi", f"--id={self.index}",
               "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
               "--format=csv,noheader,nounits", "-lms", "100"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        # each sample is stamped with the host time it arrived (about its sampling time: the
        # tool flushes every line), so that the timed region's samples can be picked out
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def wait_first(self, timeout=5.0):
        """Block until the sampler has its first sample (NVML initialised, the poller in its
        steady loop), so that its start-up does not overlap the timed steps."""
        t0 = time.time()
        while not (self.lines or self.samples) and (self.proc is not None or self.nvml.ok) and \
                time.time() - t0 < timeout:
            time.sleep(0.02)

    def stop(self, t0=None, t1=None):
        """Median SM clock, maximum clock and the throttle reasons seen by the samples taken
        between host times t0 and t1 (the timed region); all samples if none fell inside."""
        if self.nvml.ok:
            self._stop.set()
            self.t.join(timeout=1.0)
            inside = [x for x in self.samples if t0 is not None and t0 <= x[0] <= t1]
            sel = inside if inside else self.samples
            if not sel:
                return None
            return {"sm_mhz": statistics.median(x[1] for x in sel), "sm_max_mhz": self.nvml.max_mhz,
                    "reasons": sorted({n for x in sel for n in x[2]}), "samples": len(sel),
                    "during_timed_region": bool(inside), "source": "NVML, polled every 5 ms"}
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=2)
        except Exception:
            self.proc.kill()
        lines = self.lines
        inside = [x for x in lines if t0 is not None and t0 <= x[0] <= t1]
        sel = inside if inside else lines
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for _, ln in sel:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm), "during_timed_region": bool(inside), "source": "nvidia-smi, every 100 ms"}


# ------------------------------------------------------------------------------------------
# CPU baseline (the oracle, as it stands)
# ------------------------------------------------------------------------------------------

def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=5).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu model")):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def oracle_sample_time(g, cams, levels, stride, seed=0):
    """Oracle forward + backward over every stride-th row and column of every level of every
    camera.  Returns (seconds, sampled pixels, total pixels)."""
    import oracle
    g64 = {k: np.asarray(v, np.float64) for k, v in g.items() if k != "label"}
    rng = np.random.default_rng(seed)
    t0 = time.perf_counter()
    n_s, n_t = 0, 0
    for oc in [lc for cam in cams for lc in oracle.level_cameras(cam, levels)]:
        ys, xs = np.meshgrid(np.arange(0, oc["H"], stride), np.arange(0, oc["W"], stride), indexing="ij")
        pix = np.stack([xs.ravel(), ys.ravel()], 1)
        f = oracle.render(g64, oc, pixels=pix)
        C = g64["sem"].shape[1]
        oracle.render_backward(g64, oc, rng.normal(size=(3, len(pix))), rng.normal(size=len(pix)),
                               rng.normal(size=(C, len(pix))), pixels=pix)
        n_s += len(pix)
        n_t += oc["W"] * oc["H"]
    return time.perf_counter() - t0, n_s, n_t


def cpu_baseline(g, cams, levels, target_s):
    """The oracle's cost of one full iteration, from two pixel samples: every call also pays a
    fixed cost (projecting all Gaussians), so t(n) = a + b n is fitted to a coarse sample and a
    fine one of about target_s seconds, and evaluated at the full pixel count."""
    import oracle
    oracle.build()
    s1 = 64
    t1, n1, nt = oracle_sample_time(g, cams, levels, s1)

    def fit(t2, n2):
        b = (t2 - t1) / max(1, n2 - n1)
        return max(0.0, t1 - b * n1), max(b, 1e-12)

    # first guess from the coarse sample's cost per pixel (an upper bound: it includes the
    # fixed cost), then one refit if the fine sample came out far below the target
    stride = min(s1 // 2, max(1, int(np.sqrt(nt * (t1 / max(1, n1)) / target_s))))
    t2, n2, _ = oracle_sample_time(g, cams, levels, stride)
    if t2 < 0.5 * target_s and stride > 1:
        a, b = fit(t2, n2)
        s2 = min(stride - 1, max(1, int(np.sqrt(nt * b / max(target_s - a, 0.1 * target_s)))))
        stride = s2
        t2, n2, _ = oracle_sample_time(g, cams, levels, stride)
    a, b = fit(t2, n2)
    full = a + b * nt
    return {"value": 1.0 / full, "unit": UNIT, "cores": oracle.num_threads(), "cpu_model": cpu_model(),
            "kind": "oracle",
            "sample": f"FP64 oracle forward+backward on every {stride}-th row and column of all {levels} levels "
                      f"({n2} of {nt} pixels, {t2:.1f} s) and every {s1}-th ({n1} pixels, {t1:.1f} s); "
                      f"fixed cost {a:.2f} s + {b * 1e3:.4f} ms per pixel, evaluated at all {nt} pixels",
            "seconds_per_iter": full}


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores, each step one bounded sample."""
    import oracle
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    oracle.build()
    W = WORKLOADS[args.workload]
    L = W["levels"]
    cams, frames, g, dec = build_inputs(args.workload, args.gaussians or W["gaussians"])
    # every call pays a fixed cost (projecting all Gaussians) besides its per-pixel cost:
    # t(n) = a + b n from two coarse samples, so that a step's small sample extrapolates
    # its per-pixel part only
    t1, n1, nt = oracle_sample_time(g, cams, L, 96)
    t2, n2, _ = oracle_sample_time(g, cams, L, 48)
    b = max((t2 - t1) / max(1, n2 - n1), 1e-12)
    a = max(0.0, t1 - b * n1)
    budget = 150.0 / max(1, args.steps + args.warmup)
    stride = max(8, int(np.sqrt(nt * b / max(0.25, budget - a))))
    for _ in range(args.warmup):
        oracle_sample_time(g, cams, L, stride)
    times = []
    for k in range(args.steps):
        t, ns, nt = oracle_sample_time(g, cams, L, stride, seed=k)
        times.append(a + max(t - a, 0.0) * nt / ns)
    per = float(np.mean(times))
    value = 1.0 / per
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(W, l2="n/a (CPU)"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "cpu_model": cpu_model(),
                             "kind": "oracle",
                             "sample": f"every {stride}-th row and column of all {L} levels per step ({ns} of {nt} px); "
                                       f"fixed cost {a:.2f} s per call (from samples at strides 96 and 48) "
                                       f"plus the sample's per-pixel time extrapolated to all pixels"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------
# Multi-rank aggregation (N independent replicas, one per GPU)
# ------------------------------------------------------------------------------------------

def max_over_ranks(seconds, device):
    """The slowest rank's time (every rank returns the same value); the local value when
    torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(seconds)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(steps, world, seconds):
    """Iterations per second of the whole job: every rank ran `steps` iterations of its own
    replica, and the job took the slowest rank's time."""
    return steps * world / seconds


# ------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------

def run_ours(args):
    import torch
    import torch.distributed as dist
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2412_01217_gb300 import (LossConfig, MappingStep, PyramidRasterizer, RenderConfig,
                                        build_pyramid, load_library, to_device_params)
    lib = load_library()
    tw, th = (int(x) for x in args.tile.split("x"))
    W = WORKLOADS[args.workload]
    L, C_sem, n_cls = W["levels"], W["sem_features"], W["classes"]
    n_gauss = args.gaussians or W["gaussians"]
    cams, frames, g, dec = build_inputs(args.workload, n_gauss, seed_offset=rank)
    fr = lambda key: [f[key] for f in frames]
    cfg = RenderConfig(tile_w=tw, tile_h=th, batch=args.batch, pixels_per_thread=args.ppt,
                       pixels_per_thread_bwd=args.ppt_bwd, batch_bwd=args.batch_bwd, half_masks=args.half_masks,
                       half_tile_fwd=args.half_tile_fwd)
    p = to_device_params(g, dev)
    decoder = torch.tensor(dec, device=dev) if dec is not None else None
    tune_table = None
    if not args.no_autotune:
        from paper_2412_01217_gb300.autotune import autotune
        probe = PyramidRasterizer(n_gauss, C_sem, cams, levels=L, cfg=cfg,
                                  loss_cfg=LossConfig(n_classes=n_cls), device=dev)
        gt0 = build_pyramid(probe, fr("rgb"), fr("depth"), fr("label"))
        del probe
        cfg, tune_table = autotune(p, cams, L, gt0, LossConfig(n_classes=n_cls), base=cfg, decoder=decoder,
                                   use_cache=False, log=lambda m: print("autotune:", m, file=sys.stderr))
        del gt0
        torch.cuda.empty_cache()
    r = PyramidRasterizer(n_gauss, C_sem, cams, levels=L, cfg=cfg,
                          loss_cfg=LossConfig(n_classes=n_cls), device=dev)
    gt = build_pyramid(r, fr("rgb"), fr("depth"), fr("label"))
    ms = MappingStep(r, p, gt, decoder=decoder)
    ms.step()
    torch.cuda.synchronize()
    r.check_status()
    stats = step_stats(r)

    # ---- capture the iteration with timing events around the two raster calls ------------
    ev = {k: torch.cuda.Event(enable_timing=True, external=True) for k in
          ("s0", "fwd0", "fwd1", "bwd0", "bwdr", "bwd1", "s1")}
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream(device=dev)
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        ms.step()
    torch.cuda.current_stream().wait_stream(side)
    from paper_2412_01217_gb300.splat import _ptr, _stream
    from paper_2412_01217_gb300._lib import call

    groups, n_groups = ms._adam_groups()

    def body(t):
        if ms.decoder_grad is not None:
            ms.decoder_grad.zero_()
        ev["s0"].record()
        r.project(p)
        r.build_lists()
        ev["fwd0"].record()
        r.rasterize(p)
        ev["fwd1"].record()
        r.loss(gt, decoder=decoder, decoder_grad=ms.decoder_grad)
        ev["bwd0"].record()
        r.backward(p, ms.grads, between=ev["bwdr"].record)
        ev["bwd1"].record()
        call("sg_adam_multi", groups, n_groups, 0.9, 0.999, 1e-15, t, 1, None, _stream())
        ev["s1"].record()

    n0 = lib.sg_kernel_launch_count()  # the launches captured into the step's graph
    with torch.cuda.graph(graph):
        body(2)
    launches_per_step = lib.sg_kernel_launch_count() - n0
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    for _ in range(args.warmup):
        flush.zero_()
        graph.replay()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    clocks.wait_first()
    time.sleep(0.2)
    step_ms, fwd_ms, bwd_ms, pre_ms, loss_ms, adam_ms, pbwd_ms = [], [], [], [], [], [], []
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    torch.cuda.synchronize()
    t_wall0 = time.time()
    for i in range(args.steps):
        flush.zero_()
        starts[i].record()
        graph.replay()
        ends[i].record()
        ends[i].synchronize()
        fwd_ms.append(ev["fwd0"].elapsed_time(ev["fwd1"]))
        bwd_ms.append(ev["bwd0"].elapsed_time(ev["bwdr"]))
        pbwd_ms.append(ev["bwdr"].elapsed_time(ev["bwd1"]))
        pre_ms.append(ev["s0"].elapsed_time(ev["fwd0"]))
        loss_ms.append(ev["fwd1"].elapsed_time(ev["bwd0"]))
        adam_ms.append(ev["bwd1"].elapsed_time(ev["s1"]))
    torch.cuda.synchronize()
    t_wall1 = time.time()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    clk = clocks.stop(t_wall0, t_wall1)
    total_s = sum(step_ms) / 1e3
    total_s = max_over_ranks(total_s, dev)
    value = whole_job_rate(args.steps, world, total_s)
    ms_per = total_s * 1e3 / args.steps

    # ---- end to end through the public API with host buffers ----------------------------
    e2e = None
    if not args.no_e2e:
        # A step's inputs are its keyframes (level-0 RGB, depth and labels from pinned host
        # memory) and its result the loss terms; the map (Gaussian parameters and Adam moments)
        # stays on the device between iterations, as a training loop keeps its weights.
        h_frames = [(torch.as_tensor(f["rgb"]).pin_memory(), torch.as_tensor(f["depth"]).pin_memory(),
                     torch.as_tensor(f["label"]).pin_memory()) for f in frames]
        h_terms = torch.empty(r.terms.numel(), dtype=torch.float32).pin_memory()
        from paper_2412_01217_gb300._lib import call as _call
        import ctypes as C

        # Input pipeline: a copy stream uploads the next step's keyframes into a device
        # staging area while the current step computes; each step waits for its upload, moves
        # it into the GT pyramid's level 0 and frees the staging area for the next upload.
        copy_st = torch.cuda.Stream()
        d_frames = [tuple(torch.empty(t.shape, dtype=t.dtype, device=dev) for t in f) for f in h_frames]
        ev_in, ev_free = torch.cuda.Event(), torch.cuda.Event()

        def upload(after=None):
            with torch.cuda.stream(copy_st):
                copy_st.wait_event(ev_free)  # (a no-op before the first record)
                if after is not None:
                    copy_st.wait_event(after)
                for d, h in zip(d_frames, h_frames):
                    for dt, ht in zip(d, h):
                        dt.copy_(ht, non_blocking=True)
                ev_in.record(copy_st)

        def e2e_step(last):
            main = torch.cuda.current_stream()
            main.wait_event(ev_in)
            for c, (d_rgb, d_depth, d_label) in enumerate(d_frames):  # level 0 of every keyframe
                v = c * L
                r.view_slice(gt["rgb"], v, 3).copy_(d_rgb, non_blocking=True)
                r.view_slice(gt["depth"], v, 1)[0].copy_(d_depth, non_blocking=True)
                r.view_slice(gt["label"], v, 1)[0].copy_(d_label, non_blocking=True)
            ev_free.record(main)
            if not last:
                upload()  # the next step's input, during this step's compute
            _call("sg_build_pyramid", _ptr(gt["rgb"]), _ptr(gt["depth"]), _ptr(gt["label"]), C.c_void_p(0), 0,
                  r.views_host, r.V, _stream())
            graph.replay()
            h_terms.copy_(r.terms, non_blocking=True)

        upload()
        for i in range(2):
            e2e_step(last=i == 1)
        torch.cuda.synchronize()
        es, ee = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        es.record()
        upload(after=es)  # every timed step's upload lies after the start event
        for i in range(args.steps):
            e2e_step(last=i == args.steps - 1)
        ee.record()
        torch.cuda.synchronize()
        e2e_s = es.elapsed_time(ee) / 1e3
        h2d = sum(t.numel() * t.element_size() for f in h_frames for t in f)
        d2h = h_terms.numel() * 4
        e2e_s = max_over_ranks(e2e_s, dev)
        e2e = {"value": whole_job_rate(args.steps, world, e2e_s), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h),
               "l2": "not flushed: the steps run back to back without a host wait, as a training loop "
                     "runs them (the device-timed loop above waits for every step and flushes L2 "
                     "before the next one)"}

    # ---- roofline of the dominant kernel ---------------------------------------------------
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak_tflops = sms * 128 * 2 * sm_max * 1e6 / 1e12
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    f_fwd, f_bwd = raster_flops_model(stats)
    c_fwd, c_bwd = raster_flops(stats)
    fwd_avg = float(np.mean(fwd_ms)) / 1e3
    bwd_avg = float(np.mean(bwd_ms)) / 1e3
    bytes_model = algorithmic_bytes(stats)
    step_bytes = sum(bytes_model.values())
    dominant = "raster_bwd" if bwd_avg >= fwd_avg else "raster_fwd"
    d_flops = f_bwd if dominant == "raster_bwd" else f_fwd
    d_strict = c_bwd if dominant == "raster_bwd" else c_fwd
    d_time = bwd_avg if dominant == "raster_bwd" else fwd_avg
    achieved = d_flops / d_time / 1e12
    roofline = {"bound": "alu", "kernel": dominant, "achieved": achieved, "peak": fp32_peak_tflops,
                "unit": "TFLOP/s", "frac": achieved / fp32_peak_tflops,
                "flops_per_launch": d_flops,
                "flops_model": "E x (40 + 4 (4 + C)) backward, E x (15 + 2 (4 + C)) forward; E = list entries "
                               "examined (per-pixel last summed)",
                "frac_per_contribution": d_strict / d_time / 1e12 / fp32_peak_tflops,
                "traffic": profiled_traffic(dominant, stats["E"], args.workload),
                "traffic_unit": "DRAM bytes per launch (ncu), scaled by list entries examined",
                "peak_source": f"derived: {sms} SMs x 128 FP32 lanes x 2 flop x {sm_max:.0f} MHz",
                "launch_ms": d_time * 1e3}
    evals = 2 * stats["E"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(W, tile=f"{cfg.tile_w}x{cfg.tile_h}", batch=cfg.batch,
                       pixels_per_thread=cfg.pixels_per_thread, pixels_per_thread_bwd=cfg.pixels_per_thread_bwd,
                       batch_bwd=cfg.batch_bwd or cfg.batch, half_masks=bool(cfg.half_masks), half_tile_fwd=bool(cfg.half_tile_fwd),
                       autotuned=not args.no_autotune, gaussians=n_gauss,
                       l2="flushed (256 MiB write) before every timed step", parallelism="replicas"),
        "gpu_launches": int(launches_per_step * args.steps),
        "launches_per_step": int(launches_per_step),
        "gaussian_pixel_evals_per_s": evals * value / world * world if world else evals * value,
        "hbm": {"algorithmic_bytes_per_step": int(step_bytes), "achieved_GBps": step_bytes / (ms_per / 1e3) / 1e9,
                "peak_GBps": hbm_peak, "frac": step_bytes / (ms_per / 1e3) / 1e9 / hbm_peak,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in peaks else "fallback 6800 GB/s"},
        "phases_ms": {"project+tile_lists": float(np.mean(pre_ms)), "raster_fwd": fwd_avg * 1e3,
                      "loss": float(np.mean(loss_ms)), "raster_bwd": bwd_avg * 1e3,
                      "project_bwd": float(np.mean(pbwd_ms)),
                      "adam": float(np.mean(adam_ms))},
        "counts": stats,
        "roofline": roofline,
        "clocks": clk,
        "e2e": e2e,
    }
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(g, cams, L, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
