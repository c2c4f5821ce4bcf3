#!/usr/bin/env python
"""Benchmark of the RPNN render hot path: RPNN shading queries/s on one GB300.

Workload (one step = one full render: camera rays + delta tracking + NEE, descriptor
gather, network, composite): a 256^3 FP32 cloud of thresholded 6-octave fBm noise
(30% non-zero voxels, peak extinction 50 per unit), 512 x 512 pixels, 1 sample per
pixel, random light direction, He-initialised network.  The network runs in BF16 on
the tensor cores (the FP32 CUDA-core form is timed beside it for the ratio).

Prints one JSON line.  --impl reference times the CPU oracle on the same workload.
Multi-GPU (torchrun): every rank renders its own view of the cloud (weak scaling, no
collective on the data path); the barrier and the max over ranks only frame timing.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RPNN shading queries/s on 1 GB300, BF16/FP8 vs FP32 GPU form at stated RMSE"
WORKLOAD = ("single cloud render: 256^3 FP32 fBm density (6 octaves, 30% non-zero, peak "
            "sigma_t 50/unit, albedo 0.99, HG g 0.85), 512x512, 1 spp, random light dir, "
            "RPNN at the paper's sizes (10 blocks x 2 + 3 layers, width 200), He-init weights")
FLOP_PER_QUERY = 2 * (10 * 226 * 200 + 9 * 200 * 200 + 10 * 200 * 200 + 2 * 200 * 200 + 200)
L2_FLUSH_BYTES = 256 << 20


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per shading query of the
# dominant kernels, from one ncu capture of the benchmark workload (178,675 queries; the
# summaries under profiles/ give the commands), with the SHA-256 prefixes of the sources the
# captured build was compiled from.  A kernel whose sources changed since reports null.
NCU_TRAFFIC = {
    "descriptor": {"bytes_per_query": (795.414272e6 + 5.620736e6) / 178675,
                   "sources": {"descriptor.cu": "05b2f345e006b04d", "desc_lookup.cuh": "96d43ff4040f8e82",
                               "volume.cu:k_pack": "f1b80b6358e59e22"}},
    "network": {"bytes_per_query": (886.175488e6 + 3.624960e6) / 178675,
                "sources": {"mlp_tc.cu": "57c21e9d2ae6b860", "tc_ptx.cuh": "294268ada12e7cd2",
                            "tc_net.cuh": "84cfe3d7ca7bea66"}},
    "network_fp8": {"bytes_per_query": (460.973824e6 + 1.656832e6) / 178675,
                    "sources": {"mlp_tc.cu": "57c21e9d2ae6b860", "tc_ptx.cuh": "294268ada12e7cd2",
                                "tc_net.cuh": "84cfe3d7ca7bea66"}},
}


def _source_digest(csrc, name):
    """SHA-256 prefix of a source file, or of one function in it ("file.cu:k_name": the text
    from that __global__ function's line up to the first line that is a lone closing brace)."""
    import hashlib
    fname, _, fn = name.partition(":")
    with open(os.path.join(csrc, fname), "rb") as f:
        data = f.read()
    if fn:
        text = data.decode()
        i = text.index("__global__ void " + fn + "(")
        j = text.index("\n}\n", i) + 3
        data = text[i:j].encode()
    return hashlib.sha256(data).hexdigest()[:16]


def traffic_per_launch(kernel, nq):
    """ncu-measured DRAM bytes for one launch over nq queries, or None once a source that
    determines the kernel's traffic has changed since the capture."""
    t = NCU_TRAFFIC.get(kernel)
    if t is None:
        return None
    csrc = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_1709_05418_gb300", "csrc")
    for name, digest in t["sources"].items():
        if _source_digest(csrc, name) != digest:
            return None
    return t["bytes_per_query"] * nq


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": d["hbm_gbs"], "bf16_tflops": d["bf16_tflops"],
                "bf16_tflops_sustained": d.get("bf16_tflops_sustained"),
                "sm_max_mhz": d.get("sm_max_mhz", 2070.0), "src": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0, "src": "fallback"}


def fp8_peak(dev):
    """Dense E4M3 tensor throughput of this GPU, measured here the way the BF16 peak is:
    a library GEMM (torch._scaled_mm, cuBLASLt) of 8192^3 with E4M3 operands, FP32
    accumulation and BF16 output, best of 10 launches timed with CUDA events.  Returns
    (TFLOP/s, source) or the nominal ratio (2 x BF16) when the call is unavailable."""
    import torch
    pk = peaks()
    try:
        n = 8192
        g = torch.Generator(device=dev).manual_seed(0)
        a = torch.randn(n, n, device=dev, generator=g).to(torch.float8_e4m3fn)
        b = torch.randn(n, n, device=dev, generator=g).to(torch.float8_e4m3fn).t()
        one = torch.ones((), device=dev, dtype=torch.float32)
        for _ in range(3):
            torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
        best = float("inf")
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch._scaled_mm(a, b, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        del a, b
        return 2.0 * n ** 3 / (best / 1e3) / 1e12, "measured here: torch._scaled_mm E4M3 8192^3, best of 10"
    except Exception as e:   # no FP8 GEMM in this torch build
        return 2 * pk["bf16_tflops"], f"{pk['src']} bf16 x 2 (nominal E4M3:BF16 ratio; E4M3 GEMM unavailable: {e})"


class _Nvml:
    """Read-only NVML queries through ctypes (SM clock, its maximum, the clock event
    reasons) for the GPU the process uses; None where the library or the device is not
    found.  Nothing is set."""
    SM = 1                                           # NVML_CLOCK_SM
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown"}

    @classmethod
    def open(cls, index):
        import ctypes
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return None
            h = ctypes.c_void_p()
            ok = False
            try:
                import torch
                pr = torch.cuda.get_device_properties(index)
                bus = "%08x:%02x:%02x.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
                ok = lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), ctypes.byref(h)) == 0
            except Exception:
                ok = False
            if not ok:
                vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
                ids = [t for t in vis.split(",") if t.strip()]
                nv = int(ids[index]) if index < len(ids) and ids[index].strip().isdigit() else index
                if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(nv), ctypes.byref(h)) != 0:
                    return None
            reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons", None)
            if reasons is None:
                return None
            o = cls()
            o.ct, o.lib, o.h, o.reasons = ctypes, lib, h, reasons
            return o if o.sample() else None
        except (OSError, AttributeError, ValueError):
            return None

    def sample(self):
        c, mx, r = self.ct.c_uint(), self.ct.c_uint(), self.ct.c_ulonglong()
        if (self.lib.nvmlDeviceGetClockInfo(self.h, self.SM, self.ct.byref(c)) != 0 or
                self.lib.nvmlDeviceGetMaxClockInfo(self.h, self.SM, self.ct.byref(mx)) != 0 or
                self.reasons(self.h, self.ct.byref(r)) != 0):
            return None
        return float(c.value), float(mx.value), [n for b, n in self.REASONS.items() if r.value & b]


class Clocks:
    """SM clock and clock event reasons sampled during the timed region: NVML every 2 ms
    from a thread (the timed regions last tens of milliseconds), else nvidia-smi every
    200 ms."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None
        self.nv = None
        self.thread = None
        self.record = None

    def start(self):
        self.nv = _Nvml.open(self.index)
        if self.nv is not None:
            import threading
            self.samples = []
            self.halt = threading.Event()

            def run():
                while True:
                    s = self.nv.sample()
                    if s:
                        self.samples.append(s)
                    if self.halt.wait(0.002):
                        break

            self.thread = threading.Thread(target=run, daemon=True)
            self.thread.start()
            return
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.p = None

    def stop(self):
        if self.thread is not None:
            self.halt.set()
            self.thread.join(timeout=5)
            self.thread = None
            if not self.samples:
                return None
            sm = [a for a, _, _ in self.samples]
            reasons = sorted({n for _, _, rs in self.samples for n in rs})
            return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(b for _, b, _ in self.samples),
                    "sm_mhz_min": min(sm), "samples": len(sm), "reasons": reasons,
                    "source": "NVML every 2 ms during the timed region"}
        if not self.p:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [t.strip() for t in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons), "source": "nvidia-smi every 200 ms"}


def clocks_rejected(clk):
    """A timed region that saw a hardware or thermal slowdown, or SM clocks well below their
    maximum with no reason given (a clock lock left by someone else)."""
    if not clk:
        return False
    if set(clk.get("reasons", [])) & {"hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"}:
        return True
    return not clk.get("reasons") and clk["sm_mhz"] < 0.85 * clk["sm_max_mhz"]


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("RPNN_BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend)
    return ws, rank, local


def max_over_ranks(x, ws, device):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, ws, device):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def calibration_sample(hit, n):
    """Indices of at most n shading points spread evenly over the image (every k-th hit in
    pixel order), so the FP8 scales see the whole range of the render's activations."""
    import torch
    idx = torch.nonzero(hit).squeeze(1)
    return idx[::max(1, idx.numel() // n)][:n]


def make_workload(rank, device=None):
    from paper_1709_05418_gb300 import workloads as W
    dens = W.fbm_cloud(256, seed=7, device=device)
    cam = W.camera(dens.shape, 512, 512, spp=1, seed=3 + rank, light_seed=4 + rank)
    params = W.he_init(seed=2)
    return dens, cam, params


def oracle_warm(v, shape):
    """Builds every FP64 pyramid level the oracle's descriptor reads (it builds them on first
    use), so no timed oracle step pays for them: one descriptor at the box centre."""
    centre = np.array(shape[::-1], np.float64) / max(shape) / 2
    v.descriptor(centre[None], np.array([[0.0, 0.0, 1.0]]), np.array([0.0, 1.0, 0.0]))


def oracle_pixels(dens, cam, params, npix, seed=0):
    """Oracle render of `npix` sampled pixels (untimed; for the image error)."""
    import oracle
    v = oracle.Volume(dens)
    pix = np.sort(np.random.default_rng(seed).choice(cam["width"] * cam["height"], npix, replace=False))
    vals = v.render_pixels(cam, pix, params=params.astype(np.float64), nthreads=os.cpu_count() or 1)
    v.close()
    return pix, vals


def oracle_rate(dens, cam, params, npix, steps, warmup, seed=123):
    """The CPU oracle's render rate on the benchmark workload: `warmup` + `steps` renders of
    `npix` random pixels each, on all host threads, after every pyramid level was built.
    Returns (queries per step, seconds per step, threads) of the timed steps."""
    import oracle
    v = oracle.Volume(dens)
    nthreads = os.cpu_count() or 1
    p64 = params.astype(np.float64)
    oracle_warm(v, dens.shape)
    rng = np.random.default_rng(seed)
    times, queries = [], []
    for i in range(warmup + steps):
        pix = np.sort(rng.choice(cam["width"] * cam["height"], npix, replace=False))
        hits = sum(1 for p in pix if v.primary(cam, int(p), 0)[0] == 1)
        t0 = time.perf_counter()
        v.render_pixels(cam, pix, params=p64, nthreads=nthreads)
        dt = time.perf_counter() - t0
        if i >= warmup:
            times.append(dt)
            queries.append(hits)
    v.close()
    return queries, times, nthreads


def cpu_baseline_subprocess(npix, steps, warmup):
    """The reference arm's own measurement (the CPU oracle, `bench.py --impl reference`) run
    in a fresh single-rank process, so the oracle's threads share the host with nothing the
    GPU run left behind; returns that line's cpu_baseline."""
    import subprocess
    env = {k: v for k, v in os.environ.items()
           if k not in ("RANK", "LOCAL_RANK", "WORLD_SIZE", "LOCAL_WORLD_SIZE", "MASTER_ADDR", "MASTER_PORT",
                        "GROUP_RANK", "ROLE_RANK", "TORCHELASTIC_RUN_ID")}
    cmd = [sys.executable, os.path.abspath(__file__), "--impl", "reference", "--steps", str(steps),
           "--warmup", str(warmup), "--ref-pixels", str(npix)]
    r = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=900)
    if r.returncode != 0:
        raise RuntimeError("CPU oracle run failed: " + r.stderr[-2000:])
    line = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])
    return line["cpu_baseline"]


BATCH_WORKLOAD = ("batched serving: 16 fBm clouds (seeds 200-215), edges log-uniform in [64, 512], FP16 "
                  "density, per-cloud shading-point targets log-uniform in [1k, 1M] (square images, 1 spp), "
                  "random light per cloud, one rpnn_render_batch call (CUDA graph), BF16 RPNN, He-init weights")


def make_batch_workload(device):
    """16 clouds of uneven size and query count; returns (densities FP16 on device, cameras)."""
    import torch
    from paper_1709_05418_gb300 import workloads as W
    rng = np.random.default_rng(2024)
    edges = np.exp(rng.uniform(np.log(64), np.log(512), 16)).round().astype(int)
    targets = np.exp(rng.uniform(np.log(1e3), np.log(1e6), 16))
    clouds, cams = [], []
    for i in range(16):
        n = int(edges[i])
        d = W.fbm_cloud(n, seed=200 + i, device=device)
        clouds.append(torch.from_numpy(d).to(device=device, dtype=torch.float16))
        # the cloud covers roughly a third of a 30-degree view at distance 1.7
        side = max(16, int(round(math.sqrt(targets[i] / 0.33))))
        cams.append(W.camera(d.shape, side, side, spp=1, seed=300 + i, light_seed=400 + i))
    return clouds, cams, edges


def run_batch(args, ws, rank, local):
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1709_05418_gb300 import api
    from paper_1709_05418_gb300 import workloads as W
    clouds, cams, edges = make_batch_workload(dev)
    ctx = api.Context()
    vols = []
    for d in clouds:
        v = ctx.load_volume(d)
        ctx.build_mips(v)
        vols.append(v)
    ctx.set_weights(torch.from_numpy(W.he_init(seed=2)).to(dev))
    jobs = [(v, c) for v, c in zip(vols, cams)]
    images, counts = ctx.render_batch(jobs, want_counts=True)
    nq = int(sum(counts))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        ctx.render_batch(jobs, images=images)
    ctx.sync_status()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = Clocks(local)
    clocks.start()
    torch.cuda.synchronize()
    barrier(ws)
    for e0, e1 in evs:
        flush.zero_()
        e0.record()
        ctx.render_batch(jobs, images=images)
        e1.record()
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    ctx.sync_status()
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), ws, dev)
    q_total = sum_over_ranks(float(nq) * args.steps, ws, dev)
    # end to end: the batch call plus the device->host copy of every image, per step
    host = [torch.empty(im.shape, dtype=torch.float32, pin_memory=True) for im in images]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.render_batch(jobs, images=images)
        for h, im in zip(host, images):
            h.copy_(im, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, ws, dev)
    d2h = int(sum(im.numel() * 4 for im in images))
    line = {
        "metric": METRIC, "value": q_total / (ms / 1e3), "unit": "queries/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD, "queries_per_step": nq, "queries_per_cloud": [int(c) for c in counts],
                   "edges": [int(e) for e in edges], "l2": "flushed: 256 MB write between timed steps"},
        "gpu_launches": 6 * args.steps,   # primary (all items), offsets, descriptor, network, scatter, composite
        "e2e": {"value": q_total / e2e_s, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": d2h},
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


def train_launches(tab, bf16, batch):
    """Kernels of one training step.  FP32: 23 forward GEMMs, the loss (2), 78 backward launches
    (GEMMs, bias-gradient sums, one mask), Adam and the BF16 render image.  BF16: the training
    weight image and descriptor conversion, the forward (one launch of the persistent
    tensor-core network in its training form), the loss (2), 4 output-layer backward launches,
    1 conversion, 74 backward GEMMs and sums, Adam and the render image.  Plus one reduction
    per split-K weight-gradient GEMM: the 200 x 200 shape runs 21 times a step (T1, T2, W2 x 10,
    W1 x 9), the 200 x 226 one 10 times, the 1 x 200 once."""
    n = 86 if bf16 else 105
    for e in tab:
        if e["splits"] <= 1 or e["K0"] != batch:
            continue
        tc = bool(e["flags"] & 256)
        if e["M"] == 1:
            n += 1
        elif tc == bf16:
            n += 21 if e["N"] == 200 else 10
    return n


TRAIN_WORKLOAD = ("training: fBm clouds (seeds 100-103, edges drawn from {128, 160, 192, 224, 256}, FP32 "
                  "density), labelled records (uniform direction, origin on the bounding-sphere disk, "
                  "uniform light; path-traced L_i until +-2% at 95% confidence, 64 paths at least, capped "
                  "as `records.rule` states), FP32 "
                  "descriptors; one step = forward with saved activations, log-MSE loss, backward, Adam "
                  "(lr 1e-3) on a minibatch of 4,096 records")


def run_train(args, ws, rank, local):
    """Label generation (records/s) and the training step (samples/s) of the network."""
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1709_05418_gb300 import api
    from paper_1709_05418_gb300 import workloads as W
    rng = np.random.default_rng(100 + rank)
    ctx = api.Context()
    desc_dtype = torch.bfloat16 if args.train_precision == "bf16" else torch.float32
    per_cloud = max(1, args.train_records // 4)
    gen_ms, pool_z, pool_t, npaths = 0.0, [], [], []
    for i in range(4):
        edge = int(rng.choice([128, 160, 192, 224, 256]))
        vol = ctx.load_volume(torch.from_numpy(W.fbm_cloud(edge, seed=100 + 4 * rank + i)).to(dev))
        ctx.build_mips(vol)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        x, d, wl, lab, npa = ctx.gen_records(vol, 0, per_cloud, 1000 + i, rel_ci=0.02, n_min=64,
                                             n_max=args.train_max_paths)
        e1.record()
        torch.cuda.synchronize()
        gen_ms += e0.elapsed_time(e1)
        print(f"cloud {i}: edge {edge}, {per_cloud} records in {e0.elapsed_time(e1):.0f} ms", file=sys.stderr, flush=True)
        # records kept as BF16 rows (4.8 KB each) for BF16 training, FP32 rows otherwise
        pool_z.append(ctx.extract_descriptors(vol, x, d, wl, dtype=desc_dtype))
        pool_t.append(lab)
        npaths.append(npa)
    ctx.sync_status()
    z = torch.cat(pool_z)
    t = torch.cat(pool_t)
    npa = torch.cat(npaths)
    nrec = z.shape[0]
    B = 4096
    nb = max(1, nrec // B)
    params = torch.from_numpy(W.he_init(seed=2)).to(dev)
    ctx.set_weights(params)
    ctx.set_autotune(not args.no_autotune)
    m = torch.zeros_like(params)
    v = torch.zeros_like(params)
    loss = torch.empty(1, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    batches = [(z[i * B:(i + 1) * B].contiguous(), t[i * B:(i + 1) * B].contiguous()) for i in range(nb)]
    step = 0

    def timed_steps(prec, steps):
        nonlocal step
        ctx.set_train_precision(prec)
        ctx.set_weights(params)
        for i in range(args.warmup):
            step += 1
            ctx.train_step(*batches[i % nb], params, m, v, step, loss=loss)
        ctx.sync_status()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        barrier(ws)
        for i, (e0, e1) in enumerate(evs):
            flush.zero_()
            step += 1
            e0.record()
            ctx.train_step(*batches[i % nb], params, m, v, step, loss=loss)
            e1.record()
        torch.cuda.synchronize()
        barrier(ws)
        ctx.sync_status()
        return max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), ws, dev)

    main_prec = api.BF16 if args.train_precision == "bf16" else api.F32
    other_prec = api.F32 if main_prec == api.BF16 else api.BF16
    ms_other = timed_steps(other_prec, max(3, args.steps // 2))
    clocks = Clocks(local)
    clocks.start()
    ms = timed_steps(main_prec, args.steps)
    clk = clocks.stop()
    total = sum_over_ranks(float(B) * args.steps, ws, dev)
    # end to end: each step's minibatch copied from pinned host memory, the loss read back
    hz = [bz.cpu().pin_memory() for bz, _ in batches]
    ht = [bt.cpu().pin_memory() for _, bt in batches]
    dz = torch.empty_like(batches[0][0])
    dt_ = torch.empty_like(batches[0][1])
    hl = torch.empty(1, dtype=torch.float64, pin_memory=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        step += 1
        dz.copy_(hz[i % nb], non_blocking=True)
        dt_.copy_(ht[i % nb], non_blocking=True)
        ctx.train_step(dz, dt_, params, m, v, step, loss=loss)
        hl.copy_(loss, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, ws, dev)
    pk = peaks()
    flop = 3 * FLOP_PER_QUERY * B
    ach = flop / (ms / args.steps / 1e3) / 1e12
    alu_peak = 152 * 128 * 2 * pk["sm_max_mhz"] * 1e6 / 1e12
    line = {
        "metric": "RPNN training samples/s on 1 GB300 (log-MSE + Adam, minibatch 4096)",
        "value": total / (ms / 1e3), "unit": "samples/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.train_precision, "data": "synthetic",
        "config": {"workload": TRAIN_WORKLOAD, "batch": B, "records": int(nrec),
                   "minibatches": f"{nb} distinct minibatches of the record pool, in turn",
                   "l2": "flushed: 256 MB write between timed steps"},
        "records": {"value": nrec / (gen_ms / 1e3), "unit": "records/s", "records": int(nrec),
                    "rule": f"+-2% at 95% confidence, 64..{args.train_max_paths} paths",
                    "mean_paths_per_record": float(npa.double().mean()),
                    "paths_per_s": float(npa.double().sum()) / (gen_ms / 1e3),
                    "capped_at_max_paths": int((npa >= args.train_max_paths).sum()),
                    "met_rule_fraction": float((npa < args.train_max_paths).double().mean()),
                    "desc_dtype": "bf16" if desc_dtype == torch.bfloat16 else "f32",
                    "kernel": "k_records: one warp per record, 32 paths per round, the rule tested at every "
                              "path count (FP32 prefix sums, Kahan-compensated totals)"},
        "gpu_launches": None,
        "e2e": {"value": total / e2e_s, "unit": "samples/s", "h2d_bytes_per_step": int(dz.numel() * dz.element_size() + dt_.numel() * 4),
                "d2h_bytes_per_step": 8},
        "roofline": ({"bound": "tensor", "achieved": ach, "peak": pk["bf16_tflops_sustained"] or pk["bf16_tflops"],
                      "unit": "TFLOP/s", "frac": ach / (pk["bf16_tflops_sustained"] or pk["bf16_tflops"]),
                      "traffic": None,
                      "kernel": "whole training step (BF16 tcgen05 GEMMs + FP32 epilogues, 3 x 2.5844 MFLOP per sample)",
                      "peak_src": pk["src"] + " BF16 sustained"}
                     if main_prec == api.BF16 else
                     {"bound": "alu", "achieved": ach, "peak": alu_peak, "unit": "TFLOP/s", "frac": ach / alu_peak,
                      "traffic": None,
                      "kernel": "whole training step (FP32 CUDA-core GEMMs, 3 x 2.5844 MFLOP per sample)",
                      "peak_src": "152 SMs x 128 FP32 lanes x 2 FLOP x max SM clock"}),
        "other_precision": {"dtype": "f32" if main_prec == api.BF16 else "bf16",
                            "value": float(B) * max(3, args.steps // 2) / (ms_other / 1e3), "unit": "samples/s",
                            "ms_per_step": ms_other / max(3, args.steps // 2)},
        "clocks": clk,
    }
    tab = ctx.autotune_table()
    line["gpu_launches"] = train_launches(tab, main_prec == api.BF16, B) * args.steps
    line["autotune"] = {"on": not args.no_autotune, "shapes": len(tab),
                        "tuned_us_sum": sum(e["us"] for e in tab),
                        "default_tile_us_sum": sum(e["default_us"] for e in tab),
                        "choices": [f'{e["M"]}x{e["N"]}x{e["K0"]}+{e["K1"]}: {e["tile_m"]}x{e["tile_n"]}x{e["tile_k"]}'
                                    f' split {e["splits"]} ({e["us"]:.1f} vs {e["default_us"]:.1f} us)' for e in tab]}
    if rank == 0 and not args.no_cpu:
        import oracle
        zn = z[:args.cpu_rows].reshape(-1, 10, api.DESC_STRIDE)[:, :, :226].double().cpu().numpy()
        tn = t[:args.cpu_rows].double().cpu().numpy()
        pc = params.double().cpu().numpy().copy()
        mc = np.zeros_like(pc); vc = np.zeros_like(pc)
        t0 = time.perf_counter()
        g = oracle.mlp_forward(pc, zn)
        _, dg = oracle.logmse_loss(g, tn)
        grad = oracle.mlp_backward(pc, zn, dg)
        oracle.adam(pc, mc, vc, grad, 1)
        dt = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": zn.shape[0] / dt, "unit": "samples/s", "cores": 1, "kind": "oracle",
                                "sample": f"one FP64 training step on {zn.shape[0]} records of the pool"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


RECORDS_WORKLOAD = ("training-record generation (Sec. 5.1): 32 fBm clouds (seeds 100-131, edges drawn from "
                    "{128, 160, 192, 224, 256}, FP32 density), records per cloud as `config.records_per_cloud`: "
                    "uniform direction, origin on the bounding-sphere disk, free flight by delta tracking, uniform "
                    "light; L_i path traced until the 95% half-width is within 2% of the mean (64 to 65,536 paths)")


def run_records(args, ws, rank, local):
    """Label generation at the training configuration's cloud mix and the paper's stopping
    rule: records/s, paths/s and the fraction of labels that met the rule before the cap."""
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1709_05418_gb300 import api
    from paper_1709_05418_gb300 import workloads as W
    rng = np.random.default_rng(2025)
    edges = rng.choice([128, 160, 192, 224, 256], size=32)
    ctx = api.Context()
    per = args.records_per_cloud
    n_max = args.records_max_paths
    gen_ms, nps = 0.0, []
    for i, edge in enumerate(edges):
        vol = ctx.load_volume(torch.from_numpy(W.fbm_cloud(int(edge), seed=100 + i, device=dev)).to(dev))
        ctx.build_mips(vol)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        _, _, _, lab, npa = ctx.gen_records(vol, 0, per, 1000 + i, rel_ci=0.02, n_min=64, n_max=n_max)
        e1.record()
        torch.cuda.synchronize()
        gen_ms += e0.elapsed_time(e1)
        nps.append(npa)
        ctx.sync_status()
    npa = torch.cat(nps).double()
    nrec = int(npa.numel())
    rate = nrec / (gen_ms / 1e3)
    met = float((npa < n_max).double().mean())
    line = {
        "metric": "RPNN training records/s on 1 GB300 (labels path traced until +-2% at 95% confidence)",
        "value": rate, "unit": "records/s", "n_gpus": ws, "steps": 1, "warmup": 0,
        "ms_per_step": gen_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": RECORDS_WORKLOAD, "records_per_cloud": per, "records": nrec,
                   "edges": [int(e) for e in edges]},
        "paths_per_s": float(npa.sum()) / (gen_ms / 1e3),
        "mean_paths_per_record": float(npa.mean()),
        "median_paths_per_record": float(npa.median()),
        "met_rule_fraction": met,
        "capped_at_max_paths": int((npa >= n_max).sum()),
        "seconds_for_2M_records": 2e6 / rate,
        "gpu_launches": 32,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


ENV_WORKLOAD = ("environment lighting: the single-cloud render (256^3 fBm, 512x512, 1 spp) under a sun and "
                "8 sky directions (seeded, upper hemisphere) standing in for a sun-sky model; every shading "
                "point gets one next-event estimate and one BF16 network prediction per direction")


def run_env(args, ws, rank, local):
    """Environment-lit render: shading queries x directions per second."""
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1709_05418_gb300 import api
    from paper_1709_05418_gb300 import workloads as W
    dens, cam, params = make_workload(rank, device=dev)
    ctx = api.Context()
    vol = ctx.load_volume(torch.from_numpy(dens).to(dev))
    ctx.build_mips(vol)
    ctx.set_weights(torch.from_numpy(params).to(dev))
    sky = [W.unit_sphere_dir(500 + i) for i in range(8)]
    dirs = np.array([cam["light_dir"]] + [s if s[1] > 0 else -s for s in sky], np.float32)
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    irr = np.array([1.0] + [0.1] * 8, np.float32)
    img, nq = ctx.render_env(vol, cam, dirs, irr, precision=api.BF16, want_count=True)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        ctx.render_env(vol, cam, dirs, irr, precision=api.BF16, image=img)
    ctx.sync_status()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = Clocks(local)
    clocks.start()
    torch.cuda.synchronize()
    barrier(ws)
    for e0, e1 in evs:
        flush.zero_()
        e0.record()
        ctx.render_env(vol, cam, dirs, irr, precision=api.BF16, image=img)
        e1.record()
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop()
    ctx.sync_status()
    ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), ws, dev)
    nl = dirs.shape[0]
    total = sum_over_ranks(float(nq) * nl * args.steps, ws, dev)
    host = torch.empty(img.shape, dtype=torch.float32, pin_memory=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.render_env(vol, cam, dirs, irr, precision=api.BF16, image=img)
        host.copy_(img, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, ws, dev)
    line = {
        "metric": "RPNN shading queries x light directions per second on 1 GB300 (environment lighting)",
        "value": total / (ms / 1e3), "unit": "queries*directions/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": ENV_WORKLOAD, "queries_per_step": int(nq), "directions": int(nl),
                   "l2": "flushed: 256 MB write between timed steps"},
        "gpu_launches": (1 + 1 + 2 * nl + nl + 1) * args.steps,   # primary, env NEE, descriptor+network per light, scatters, composite
        "e2e": {"value": total / e2e_s, "unit": "queries*directions/s", "h2d_bytes_per_step": int(dirs.nbytes + irr.nbytes),
                "d2h_bytes_per_step": int(img.numel() * 4)},
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


TTUV_WORKLOAD = ("time to unit variance (Sec. 6, Table 1): the 256^3 fBm cloud at 256x256, 1 spp, rendered "
                 "with 16 camera seeds by the RPNN (BF16, weights trained here on path-traced records of 4 "
                 "small fBm clouds) and by the library's plain path tracer; TTUV = seconds per render x mean "
                 "per-pixel variance over the seeds")


def run_ttuv(args, ws, rank, local):
    """TTUV of the RPNN render and of plain path tracing, and their ratio (the speedup
    measure of Table 1), with a network trained here briefly on synthetic records."""
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1709_05418_gb300 import api
    from paper_1709_05418_gb300 import workloads as W
    dens, cam, params = make_workload(rank, device=dev)
    cam = W.camera(dens.shape, 256, 256, spp=1, seed=3 + rank, light_seed=4 + rank)
    ctx = api.Context()
    # a network trained here first (untrained weights predict values far off the path
    # tracer's scale, which would make the variance comparison meaningless): path-traced
    # records from four small fBm clouds, BF16 training steps
    from paper_1709_05418_gb300 import train as T
    clouds = [W.fbm_cloud(64, seed=900 + i) for i in range(4)]
    desc, label = T.records(ctx, clouds, 4000, seed=77, rel_ci=0.05, n_min=32, n_max=1024)
    tr, va = T.split(desc, label)
    p = torch.from_numpy(W.he_init(seed=5)).to(dev)
    p.mul_(0.5)
    ctx.set_train_precision(api.BF16)
    ctx.set_weights(p)
    v0 = T.val_loss(ctx, *va)
    hist = T.fit(ctx, tr, va, p, steps=args.ttuv_train_steps, batch=1024, lr=1e-3,
                 eval_every=args.ttuv_train_steps)
    ctx.set_weights(p)
    vol = ctx.load_volume(torch.from_numpy(dens).to(dev))
    ctx.build_mips(vol)
    out = {}
    for name, prec, mode in (("rpnn", api.BF16, api.MODE_RPNN), ("path_tracing", api.F32, api.MODE_PATH)):
        imgs = []
        for s in range(args.warmup):
            ctx.render(vol, dict(cam, seed=10_000 + s), precision=prec, mode=mode)
        ctx.sync_status()
        ms = 0.0
        for s in range(16):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            img = ctx.render(vol, dict(cam, seed=20_000 + 7919 * s), precision=prec, mode=mode)
            e1.record()
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            imgs.append(img.double())
        ctx.sync_status()
        stack = torch.stack(imgs)
        var = float(stack.var(dim=0, unbiased=True).mean())
        sec = ms / 16 / 1e3
        out[name] = {"ms_per_render": sec * 1e3, "mean_pixel_variance": var, "ttuv": sec * var,
                     "mean_pixel_value": float(stack.mean())}
    line = {
        "metric": "time-to-unit-variance speedup of the RPNN render over plain path tracing on 1 GB300",
        "value": out["path_tracing"]["ttuv"] / out["rpnn"]["ttuv"], "unit": "x", "n_gpus": ws, "steps": 16,
        "warmup": args.warmup, "ms_per_step": out["rpnn"]["ms_per_render"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
        "config": {"workload": TTUV_WORKLOAD}, "rpnn": out["rpnn"], "path_tracing": out["path_tracing"],
        "training": {"records": int(desc.shape[0]), "steps": args.ttuv_train_steps, "val_loss_start": v0,
                     "val_loss_end": hist[-1][2]},
        "note": "variance and time on one view; the network is trained briefly on 4 small synthetic clouds, "
                "so its bias (which Table 1 reports beside the speedup) is not representative",
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


LARGE_WORKLOAD = ("large render: 1024^3 FP16 fBm density (seed 300, 6 octaves, 30% non-zero, peak sigma_t "
                  "50/unit), 1920x1080 at 4 spp, random light dir, descriptor/network stages in chunks of "
                  "1,048,576 queries, FP8 (E4M3, per-tensor scales) RPNN, He-init weights")


def run_large(args, ws, rank, local):
    """The large configuration: BF16 and FP8 renders of a 1024^3 FP16 cloud at 1920x1080x4,
    the FP8 one (the configuration's precision) as the line's value; error of both against
    the FP64 oracle on a seeded sample of pixels."""
    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1709_05418_gb300 import api
    from paper_1709_05418_gb300 import workloads as W
    dens = torch.from_numpy(W.fbm_cloud(1024, seed=300, device=dev)).to(device=dev, dtype=torch.float16)
    cam = W.camera(tuple(dens.shape), 1920, 1080, spp=4, seed=301 + rank, light_seed=302 + rank)
    params = W.he_init(seed=2)
    ctx = api.Context()
    vol = ctx.load_volume(dens)
    dens_host = dens.float().cpu().numpy() if (rank == 0 and not args.no_cpu) else None
    del dens
    ctx.build_mips(vol)
    ctx.set_weights(torch.from_numpy(params).to(dev))
    # FP8 scales from the FP32 network on 65,536 of this render's shading points
    hit, qx, qd, _ = ctx.trace_primary(vol, cam)
    sel = calibration_sample(hit, 65536)
    wl = torch.as_tensor(np.asarray(cam["light_dir"], np.float32), device=dev)
    ctx.calibrate_fp8(ctx.extract_descriptors(vol, qx[sel].contiguous(), qd[sel].contiguous(), wl))
    del hit, qx, qd, sel

    def timed(prec):
        rd = ctx.render_desc(cam, prec, api.MODE_RPNN)
        img = torch.empty((1080, 1920), dtype=torch.float32, device=dev)
        _, nq = ctx.render(vol, cam, desc=rd, image=img, want_count=True)
        for _ in range(args.warmup):
            ctx.render(vol, cam, desc=rd, image=img)
        ctx.sync_status()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        torch.cuda.synchronize()
        barrier(ws)
        ctx.set_profiling(True)
        for e0, e1 in evs:
            e0.record()
            ctx.render(vol, cam, desc=rd, image=img)
            e1.record()
        torch.cuda.synchronize()
        barrier(ws)
        ctx.set_profiling(False)
        prof = ctx.read_profile()
        ctx.sync_status()
        ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in evs), ws, dev)
        n = max(1, prof["renders"])
        return nq, ms, {k: prof[k] / n for k in ("primary", "descriptor", "network", "composite")}, img

    clocks = Clocks(local)
    clocks.start()
    nq, ms8, st8, img8 = timed(api.FP8)
    _, ms16, st16, img16 = timed(api.BF16)
    clk = clocks.stop()
    q_total = sum_over_ranks(float(nq) * args.steps, ws, dev)
    line = {
        "metric": METRIC, "value": q_total / (ms8 / 1e3), "unit": "queries/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms8 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "fp8e4m3", "data": "synthetic",
        "config": {"workload": LARGE_WORKLOAD, "queries_per_step": int(nq), "pixel_samples": 1920 * 1080 * 4,
                   "l2": "inputs larger than L2 (4.3 GB grid, descriptor chunks of 1,048,576 rows)",
                   "fp8_calibration": "per-tensor E4M3 scales from the FP32 network on 65,536 of the render's "
                                      "shading points, spread evenly over the image"},
        "stages_ms_per_step": st8,
        "stage_note": "chunked render: the descriptor stage includes the network chunks",
        "bf16_form": {"value": q_total / (ms16 / 1e3), "unit": "queries/s", "ms_per_step": ms16 / args.steps,
                      "stages_ms_per_step": st16},
        "clocks": clk,
    }
    if rank == 0 and not args.no_cpu:
        import oracle
        v = oracle.Volume(dens_host)
        npix = args.large_oracle_pixels
        pix = np.sort(np.random.default_rng(7).choice(1920 * 1080, npix, replace=False))
        oracle_warm(v, dens_host.shape)
        t0 = time.perf_counter()
        vals = v.render_pixels(cam, pix, params=params.astype(np.float64), nthreads=os.cpu_count() or 1)
        dt = time.perf_counter() - t0

        def rel(img):
            g = img.double().cpu().numpy().ravel()[pix]
            return float(np.sqrt(np.mean((g - vals) ** 2)) / max(np.sqrt(np.mean(vals ** 2)), 1e-30))

        line["error_vs_fp64_oracle"] = {"pixels": int(npix), "fp8_rel_rmse": rel(img8), "bf16_rel_rmse": rel(img16),
                                        "oracle_seconds": dt}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()


def run_reference(args, ws, rank):
    if rank != 0:
        return
    dens, cam, params = make_workload(0, device="cpu")
    npix = args.ref_pixels
    queries, times, nthreads = oracle_rate(dens, cam, params, npix, args.steps, args.warmup)
    T = sum(times)
    val = sum(queries) / T
    rates = sorted(q / t for q, t in zip(queries, times))
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "queries/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": f"{npix} random pixels of the 512x512 image per step"},
        "cpu_baseline": {"value": val, "unit": "queries/s", "cores": nthreads, "kind": "oracle",
                         "sample": f"{npix} random pixels per step x {args.steps} timed steps after "
                                   f"{args.warmup} warm-up steps, every FP64 pyramid level built first",
                         "per_step_median": rates[len(rates) // 2], "per_step_min": rates[0],
                         "per_step_max": rates[-1]},
        "e2e": {"value": val, "unit": "queries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["bf16", "f32"])
    ap.add_argument("--cpu-pixels", type=int, default=2048,
                    help="pixels the FP64 oracle renders for the image error")
    ap.add_argument("--ref-pixels", type=int, default=4096,
                    help="pixels the CPU oracle renders per timed step (reference arm and cpu_baseline)")
    ap.add_argument("--cpu-steps", type=int, default=10,
                    help="timed oracle steps of the cpu_baseline (a fresh reference-arm process)")
    ap.add_argument("--large-oracle-pixels", type=int, default=10000,
                    help="pixels the FP64 oracle renders for the large workload's error")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="default 64x64 tile for every FP32 CUDA-core GEMM (no tuning)")
    ap.add_argument("--ttuv-train-steps", type=int, default=600,
                    help="training steps of the network the TTUV workload renders with")
    ap.add_argument("--train-precision", default="bf16", choices=["bf16", "f32"],
                    help="arithmetic of the training workload's timed steps (the other is timed beside)")
    ap.add_argument("--train-records", type=int, default=8192,
                    help="labelled records generated (and timed) for the training workload")
    ap.add_argument("--train-max-paths", type=int, default=4096,
                    help="path cap of the records' stopping rule in the training workload")
    ap.add_argument("--cpu-rows", type=int, default=256,
                    help="records in the FP64 oracle's training step (training workload)")
    ap.add_argument("--records-per-cloud", type=int, default=2048,
                    help="records per cloud of the record-generation workload (32 clouds)")
    ap.add_argument("--records-max-paths", type=int, default=65536,
                    help="path cap of the record-generation workload's stopping rule")
    ap.add_argument("--workload", default="single",
                    choices=["single", "batch", "large", "train", "records", "env", "ttuv"],
                    help="single: the 256^3 / 512x512 render (default); batch: 16 clouds in one batched "
                         "call; large: 1024^3 FP16 cloud at 1920x1080x4")
    ap.add_argument("--profile-only", action="store_true",
                    help="one BF16, one FP32, one FP8 and one fused BF16 render of the workload, no timing "
                         "(for ncu captures)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    ws, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if args.workload == "batch":
        run_batch(args, ws, rank, local)
        return
    if args.workload == "large":
        run_large(args, ws, rank, local)
        return
    if args.workload == "train":
        run_train(args, ws, rank, local)
        return
    if args.workload == "records":
        run_records(args, ws, rank, local)
        return
    if args.workload == "env":
        run_env(args, ws, rank, local)
        return
    if args.workload == "ttuv":
        run_ttuv(args, ws, rank, local)
        return

    import torch
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_1709_05418_gb300 import api
    dens, cam, params = make_workload(rank, device=dev)
    ctx = api.Context()
    vol = ctx.load_volume(torch.from_numpy(dens).to(dev))
    ctx.build_mips(vol)
    ctx.set_weights(torch.from_numpy(params).to(dev))
    ctx.set_autotune(not args.no_autotune)
    info = ctx.get_volume_info(vol)
    # statistics + Gaussian pyramid + corner packing of the volume (per-volume preprocessing,
    # outside the render), rebuilt a few times with the L2 flushed in between
    fl = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    pyr_ms = []
    for _ in range(4):
        fl.zero_()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record()
        ctx.build_mips(vol)
        a1.record()
        torch.cuda.synchronize()
        pyr_ms.append(a0.elapsed_time(a1))
    del fl
    if args.profile_only:
        for p in (api.BF16, api.F32):
            ctx.render(vol, cam, precision=p)
        hit, qx, qd, _ = ctx.trace_primary(vol, cam)
        sel = calibration_sample(hit, 65536)
        wl = torch.as_tensor(np.asarray(cam["light_dir"], np.float32), device=dev)
        ctx.calibrate_fp8(ctx.extract_descriptors(vol, qx[sel].contiguous(), qd[sel].contiguous(), wl))
        ctx.render(vol, cam, precision=api.FP8)
        ctx.set_fused(True)                 # the descriptor gather fused into the network
        ctx.render(vol, cam, precision=api.BF16)
        ctx.set_fused(False)
        ctx.sync_status()
        torch.cuda.synchronize()
        ctx.close()
        return

    def timed(prec, steps, warmup, clocks=None):
        img = torch.empty((512, 512), dtype=torch.float32, device=dev)
        rd = ctx.render_desc(cam, prec, api.MODE_RPNN)
        _, nq = ctx.render(vol, cam, desc=rd, image=img, want_count=True)
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        for _ in range(warmup):
            ctx.render(vol, cam, desc=rd, image=img)
        ctx.sync_status()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        barrier(ws)
        torch.cuda.synchronize()
        if clocks is not None:
            clocks.start()
        ctx.set_profiling(True)
        for e0, e1 in evs:
            flush.zero_()                         # L2 flush between steps (outside the events)
            e0.record()
            ctx.render(vol, cam, desc=rd, image=img)
            e1.record()
        torch.cuda.synchronize()
        if clocks is not None:
            clocks.record = clocks.stop()
        barrier(ws)
        ctx.set_profiling(False)
        prof = ctx.read_profile()
        ms = sum(a.elapsed_time(b) for a, b in evs)
        ctx.sync_status()
        return nq, ms, prof, img

    prec = api.BF16 if args.precision == "bf16" else api.F32
    clocks = Clocks(local)
    try:
        nq, ms, prof, img = timed(prec, args.steps, args.warmup, clocks)
    except api.RPNNError as e:
        if prec != api.BF16 or e.code != -8:
            raise
        prec = api.F32                      # tensor-core network not built: report FP32
        nq, ms, prof, img = timed(prec, args.steps, args.warmup, clocks)
    clk = clocks.record
    if clocks_rejected(clk):
        # a throttled or clock-locked measurement is taken once more
        first = clk
        nq, ms, prof, img = timed(prec, args.steps, args.warmup, clocks)
        clk = dict(clocks.record or {}, remeasured_after={k: first.get(k) for k in ("sm_mhz", "reasons")})
    ms_max = max_over_ranks(ms, ws, dev)
    q_total = sum_over_ranks(float(nq) * args.steps, ws, dev)
    value = q_total / (ms_max / 1e3)
    per_step = ms_max / args.steps

    # FP32 CUDA-core form of the same render, for the ratio
    f32_form = None
    if prec == api.BF16:
        nq32, ms32, prof32, img32 = timed(api.F32, max(3, args.steps // 4), 3)
        f32_form = {"value": nq32 * max(3, args.steps // 4) / (ms32 / 1e3), "unit": "queries/s",
                    "ms_per_step": ms32 / max(3, args.steps // 4),
                    "network_ms_per_step": prof32["network"] / max(1, prof32["renders"])}
        f32_form["ratio"] = value / ws / f32_form["value"]
        # the ratio's denominator against its own roofline: the 23-launch FP32 CUDA-core GEMM
        # chain (autotuned tiles) on the FP32 pipe, 128 FMA lanes x 2 FLOP per SM per clock
        pk32 = peaks()
        alu_peak = 152 * 128 * 2 * pk32["sm_max_mhz"] * 1e6 / 1e12
        ach32 = nq32 * FLOP_PER_QUERY / (f32_form["network_ms_per_step"] / 1e3) / 1e12
        f32_form["network_roofline"] = {"bound": "alu", "achieved": ach32, "peak": alu_peak, "unit": "TFLOP/s",
                                        "frac": ach32 / alu_peak, "kernel": "k_gemm chain (23 launches)",
                                        "peak_src": "152 SMs x 128 FP32 lanes x 2 FLOP x max SM clock"}

    # the same BF16 render with the descriptor gather inside the network kernel (no
    # descriptor rows in HBM; rpnn_set_fused), beside the default separate kernels
    fused_form = None
    if prec == api.BF16:
        ctx.set_fused(True)
        nqf, msf, proff, imgf = timed(api.BF16, args.steps, 3)
        ctx.set_fused(False)
        nr = max(1, proff["renders"])
        fused_form = {"value": nqf * args.steps / (msf / 1e3), "unit": "queries/s", "ms_per_step": msf / args.steps,
                      "fused_kernel_ms_per_step": proff["network"] / nr,
                      "primary_ms_per_step": proff["primary"] / nr,
                      "image_equal_to_unfused": bool(torch.equal(imgf, img)),
                      "note": "k_rpnn_fused: 16 gather warps beside the network's 10; slower than the two "
                              "separate kernels on this GPU (the gather alone takes about twice the "
                              "standalone kernel's time inside it)"}
        del imgf

    # FP8 (E4M3) form of the same render: per-tensor scales calibrated on this render's own
    # shading points (FP32 descriptors of up to 65,536 of them), outside the timed region
    fp8_form, img8 = None, None
    if prec == api.BF16:
        hit, qx, qd, _ = ctx.trace_primary(vol, cam)
        sel = calibration_sample(hit, 65536)
        wl = torch.as_tensor(np.asarray(cam["light_dir"], np.float32), device=dev)
        ctx.calibrate_fp8(ctx.extract_descriptors(vol, qx[sel].contiguous(), qd[sel].contiguous(), wl))
        nq8, ms8, prof8, img8 = timed(api.FP8, args.steps, 3)
        fp8_form = {"value": nq8 * args.steps / (ms8 / 1e3),
                    "unit": "queries/s", "ms_per_step": ms8 / args.steps,
                    "network_ms_per_step": prof8["network"] / max(1, prof8["renders"]),
                    "descriptor_ms_per_step": prof8["descriptor"] / max(1, prof8["renders"]),
                    "calibration": "per-tensor E4M3 scales from the FP32 network on <= 65,536 of the render's "
                                   "own shading points, spread evenly over the image"}
        img8 = img8.clone()

    fp8_pk, fp8_src = fp8_peak(dev) if prec == api.BF16 else (None, None)

    # the network kernel alone at steady state: 1,048,576 rows (a chunk of the large render),
    # the render's own BF16 descriptors repeated, so the last partial wave of 128-row tiles
    # (9.19 tiles per SM on the render above) costs little
    net_1m, net8_1m = None, None
    if prec == api.BF16:
        hit, qx, qd, _ = ctx.trace_primary(vol, cam)
        idx = torch.nonzero(hit).squeeze(1)
        wl = torch.as_tensor(np.asarray(cam["light_dir"], np.float32), device=dev)
        zb = ctx.extract_descriptors(vol, qx[idx].contiguous(), qd[idx].contiguous(), wl, dtype=torch.bfloat16)
        rows = 1 << 20
        reps = -(-rows // zb.shape[0])
        z1m = zb.repeat(reps, 1, 1)[:rows].contiguous()
        del zb
        g1m = torch.empty(rows, dtype=torch.float32, device=dev)
        for _ in range(3):
            ctx.mlp_forward(z1m, precision=api.BF16, out=g1m)
        ctx.sync_status()
        evn = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
        flush1 = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        for e0, e1 in evn:
            flush1.zero_()
            e0.record()
            ctx.mlp_forward(z1m, precision=api.BF16, out=g1m)
            e1.record()
        torch.cuda.synchronize()
        ms1 = sum(a.elapsed_time(b) for a, b in evn) / len(evn)
        ach1 = rows * FLOP_PER_QUERY / (ms1 / 1e3) / 1e12
        pk1 = peaks()
        net_1m = {"rows": rows, "ms_per_launch": ms1, "bound": "tensor", "achieved": ach1,
                  "peak": pk1["bf16_tflops"], "unit": "TFLOP/s", "frac": ach1 / pk1["bf16_tflops"],
                  "peak_src": pk1["src"], "tiles_per_sm": rows / 128 / 152}
        del z1m
        if fp8_form:
            z8 = ctx.extract_descriptors(vol, qx[idx].contiguous(), qd[idx].contiguous(), wl, dtype=torch.uint8)
            z8m = z8.repeat(reps, 1, 1)[:rows].contiguous()
            del z8
            for _ in range(3):
                ctx.mlp_forward(z8m, precision=api.FP8, out=g1m)
            ctx.sync_status()
            for e0, e1 in evn:
                flush1.zero_()
                e0.record()
                ctx.mlp_forward(z8m, precision=api.FP8, out=g1m)
                e1.record()
            torch.cuda.synchronize()
            ms8 = sum(a.elapsed_time(b) for a, b in evn) / len(evn)
            ach8 = rows * FLOP_PER_QUERY / (ms8 / 1e3) / 1e12
            net8_1m = {
                "rows": rows, "ms_per_launch": ms8, "bound": "tensor", "achieved": ach8,
                "peak": fp8_pk, "unit": "TFLOP/s", "frac": ach8 / fp8_pk, "peak_src": fp8_src}
            del z8m
        del g1m, flush1

    # end to end through the public API: host-visible result every step
    host_img = torch.empty((512, 512), dtype=torch.float32, pin_memory=True)
    rd = ctx.render_desc(cam, prec, api.MODE_RPNN)
    gimg = torch.empty((512, 512), dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    barrier(ws)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.render(vol, cam, desc=rd, image=gimg)
        host_img.copy_(gimg, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, ws, dev)
    e2e = {"value": q_total / e2e_s, "unit": "queries/s", "h2d_bytes_per_step": 12,
           "d2h_bytes_per_step": 512 * 512 * 4}

    # roofline of the dominant stage
    pk = peaks()
    n = max(1, prof["renders"])
    stage_ms = {k: prof[k] / n for k in ("primary", "descriptor", "network", "composite")}
    dom = max(stage_ms, key=stage_ms.get)
    elem = 2 if prec == api.BF16 else 4
    pyr_bytes = sum((a + 1) * (b + 1) * (c + 1) * 32 for i, (a, b, c) in enumerate(info["dims"])
                    if i in set(info["mip_of_level"]))
    desc_bytes = nq * (2251 * elem + 24) + pyr_bytes
    if dom == "network" and prec == api.BF16:
        ach = nq * FLOP_PER_QUERY / (stage_ms["network"] / 1e3) / 1e12
        roof = {"bound": "tensor", "achieved": ach, "peak": pk["bf16_tflops"], "unit": "TFLOP/s"}
    elif dom == "network":
        alu_peak = 152 * 128 * 2 * pk["sm_max_mhz"] * 1e6 / 1e12
        ach = nq * FLOP_PER_QUERY / (stage_ms["network"] / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": ach, "peak": alu_peak, "unit": "TFLOP/s"}
    else:
        st = "descriptor" if dom == "descriptor" else dom
        ach = desc_bytes / (stage_ms[st] / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = traffic_per_launch(dom, nq) if prec == api.BF16 else None
    roof["traffic_unit"] = "bytes per launch (ncu dram read + write)"
    roof["kernel"] = dom
    roof["peak_src"] = pk["src"]
    # a1/a2: the FP32 grid read once and the packed pyramid levels written once
    nvox = int(np.prod(info["n"]))
    pyr_ms_med = float(np.median(pyr_ms[1:]))
    pyr_alg = nvox * 4 + pyr_bytes
    pyramid = {"ms": pyr_ms_med, "algorithmic_bytes": pyr_alg,
               "roofline": {"bound": "hbm", "achieved": pyr_alg / (pyr_ms_med / 1e3) / 1e9, "peak": pk["hbm_gbs"],
                            "unit": "GB/s", "frac": pyr_alg / (pyr_ms_med / 1e3) / 1e9 / pk["hbm_gbs"],
                            "peak_src": pk["src"]},
               "note": "statistics, separable Gaussian levels and corner-record packing; median of 3 rebuilds"}
    # the tensor-core network beside it (BF16 here, E4M3 in fp8_form): dense FLOPs per launch over
    # the CUDA-event time of the launch, against the measured BF16 burst peak (x2 for E4M3, the
    # nominal FP8:BF16 tensor ratio)
    if prec == api.BF16:
        ach = nq * FLOP_PER_QUERY / (stage_ms["network"] / 1e3) / 1e12
        line_net = {"bound": "tensor", "achieved": ach, "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
                    "frac": ach / pk["bf16_tflops"], "traffic": traffic_per_launch("network", nq),
                    "algorithmic_bytes": nq * (10 * 240 * 2), "kernel": "network", "peak_src": pk["src"]}
        if fp8_form:
            ms_net8 = fp8_form["network_ms_per_step"]
            ach8 = nq8 * FLOP_PER_QUERY / (ms_net8 / 1e3) / 1e12
            fp8_form["network_roofline"] = {
                "bound": "tensor", "achieved": ach8, "peak": fp8_pk, "unit": "TFLOP/s",
                "frac": ach8 / fp8_pk, "traffic": traffic_per_launch("network_fp8", nq8),
                "algorithmic_bytes": nq8 * (10 * 256), "kernel": "network", "peak_src": fp8_src}
            if net8_1m:
                fp8_form["network_roofline"]["steady_state_1m_rows"] = net8_1m

    line = {
        "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16" if prec == api.BF16 else "f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "queries_per_step": int(nq), "pixels": 512 * 512,
                   "l2": "flushed: 256 MB write between timed steps",
                   "mip_of_level": info["mip_of_level"]},
        "stages_ms_per_step": stage_ms,
        "primary_rays_per_s": 512 * 512 / (stage_ms["primary"] / 1e3),
        "pyramid_build": pyramid,
        # primary, descriptor, network, scatter, composite (BF16); the FP32 form runs the
        # descriptor and 23 GEMM launches
        "gpu_launches": (5 if prec == api.BF16 else 27) * args.steps,
        "e2e": e2e, "roofline": roof, "clocks": clk,
    }
    if prec == api.BF16:
        line["network_roofline"] = line_net
        if net_1m:
            line["network_roofline"]["steady_state_1m_rows"] = net_1m
    if f32_form:
        line["fp32_form"] = f32_form
    if fused_form:
        line["fused_form"] = fused_form
    if fp8_form:
        line["fp8_form"] = fp8_form
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline_subprocess(args.ref_pixels, args.cpu_steps, 3)
        pix, vals = oracle_pixels(dens, cam, params, args.cpu_pixels)
        got = img.double().cpu().numpy().ravel()[pix]
        err = float(np.sqrt(np.mean((got - vals) ** 2)) / max(np.sqrt(np.mean(vals ** 2)), 1e-30))
        line["error_vs_fp64_oracle"] = {"pixels": int(pix.size), "rel_rmse": err}
        if fp8_form:
            g8 = img8.double().cpu().numpy().ravel()[pix]
            fp8_form["error_vs_fp64_oracle"] = {
                "pixels": int(pix.size),
                "rel_rmse": float(np.sqrt(np.mean((g8 - vals) ** 2)) / max(np.sqrt(np.mean(vals ** 2)), 1e-30))}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
