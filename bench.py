"""Benchmark: Wavelet OIT build + resolve (+ composite) on one GB300 per rank.

One step = one pass of the hot path over one synthetic frame resident in
HBM: every fragment's absorbance step is projected onto its pixel's Haar
coefficients (stored in the coefficient buffer), the visibility is
reconstructed at every fragment, and the weighted resolve is composited over
the background.  Default workload: the 4K heavy-smoke frame
(3840x2160, lognormal fragments per pixel mean 24 cap 1024, ~199M fragments,
J = 5), FP32 coefficient storage, fused kernel wt_build_resolve.

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle
(the reference arm) on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "fragments/s build+resolve & % HBM roofline; served p50/p99 frame latency"
UNIT = "fragments/s"
WORKLOADS = {
    "heavy4k": "4K heavy smoke: 3840x2160, lognormal fragments/pixel (mean 24, cap 1024), "
               "5-slab depth mixture + 10% uniform, alpha U[.01,.4], J=5",
    "smoke1080": "1080p smoke: 1920x1080, 30% smoke pixels lognormal (mean 32, cap 512), "
                 "70% surface pixels U{0..4}, J=4",
    "plain64": "64x64, Poisson(4) capped at 16, alpha U[.05,.6], J=4",
}
DTYPE_NAME = {0: "f32", 1: "bf16", 2: "f16", 3: "se16"}
DTYPE_BYTES = {0: 4, 1: 2, 2: 2, 3: 2}


def coeff_bytes(P: int, C: int, dt: int) -> int:
    """Bytes of a frame's stored coefficients: P C values, plus one shared
    exponent byte per pixel for SE16."""
    return P * C * DTYPE_BYTES[dt] + (P if dt == 3 else 0)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# the sources the fused kernel is compiled from (its FP32 instantiation)
FUSED_SOURCES = ("wt_internal.h", "wt_tile.cuh", "wt_kernels.cuh", "wt_kernels_f32.cu")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2201_00094_gb300", "csrc")
    for name in FUSED_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode() + f.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, workload: str, dtype: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rows = json.load(f)
    except Exception:
        return None
    for r in rows:
        if r.get("kernel") == kernel and r.get("workload") == workload and r.get("dtype") == dtype:
            if r.get("source_hash") == kernel_source_hash():
                return r.get("dram_bytes_per_launch")
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def barrier(world):
    if world > 1:
        torch.distributed.barrier()


def _agg_device():
    # NCCL reduces CUDA tensors; gloo (the CPU tests) reduces host tensors
    return "cuda" if torch.distributed.get_backend() == "nccl" else "cpu"


def max_over_ranks(x: float, world: int) -> float:
    """Timing rule of the multi-GPU run: the slowest rank's time."""
    if world == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=_agg_device())
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int) -> float:
    """Work of the whole job: every rank renders its own frame (weak scaling)."""
    if world == 1:
        return x
    t = torch.tensor([x], dtype=torch.float64, device=_agg_device())
    torch.distributed.all_reduce(t)
    return float(t.item())


def rank_seed(seed: int, rank: int) -> int:
    """Each rank renders an independent frame: pixels never cross ranks, so the
    data path needs no collective."""
    return seed + rank


# ---------------------------------------------------------------- CPU oracle sample

def sample_tiles(fr, ntiles_sample: int, seed: int):
    """A seeded set of whole tiles and their fragments, renumbered to local
    pixel ids (tiles are independent, so this is an exact sub-problem)."""
    rng = np.random.default_rng(seed)
    tiles = np.sort(rng.choice(fr.ntiles, size=min(ntiles_sample, fr.ntiles), replace=False))
    off = fr.tile_offsets.cpu().numpy()
    idx = np.concatenate([np.arange(off[t], off[t + 1]) for t in tiles]).astype(np.int64)
    idx_t = torch.from_numpy(idx).to(fr.pixel.device)
    pix = fr.pixel[idx_t].cpu().numpy().astype(np.int64)
    uniq, local = np.unique(pix, return_inverse=True)
    cols = {k: getattr(fr, k)[idx_t].cpu().numpy() for k in ("z", "alpha", "r", "g", "b")}
    return tiles, uniq, local.astype(np.uint32), cols


def _oracle_frame(J, bg, sample):
    """The oracle's build + resolve + composite of one tile sample (FP64)."""
    import oracle
    _, uniq, local, c = sample
    coeff = oracle.build_coeffs(local, c["z"], c["alpha"], len(uniq), J)
    return oracle.resolve(local, c["z"], c["alpha"], (c["r"], c["g"], c["b"]), len(uniq), J, coeff, bg=bg)[0]


def run_oracle_sample(fr, ntiles_sample, seed):
    sample = sample_tiles(fr, ntiles_sample, seed)
    t0 = time.perf_counter()
    out = _oracle_frame(fr.J, fr.bg, sample)
    dt = time.perf_counter() - t0
    return dict(n=len(sample[2]), pixels=len(sample[1]), seconds=dt, out=out, pixel_ids=sample[1])


def run_oracle_threads(fr, ntiles_sample, threads, seed):
    """The oracle as it stands on `threads` host cores at once: every thread
    runs the single-threaded FP64 oracle on its own seeded sample of whole
    tiles (the oracle's C functions hold no global state, and ctypes releases
    the interpreter lock for the duration of each C call).  Samples are drawn
    before the clock starts; the wall time of all threads is timed."""
    from concurrent.futures import ThreadPoolExecutor
    samples = [sample_tiles(fr, ntiles_sample, seed + t) for t in range(threads)]
    with ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(lambda _: None, range(threads)))  # threads started before the clock
        t0 = time.perf_counter()
        list(ex.map(lambda smp: _oracle_frame(fr.J, fr.bg, smp), samples))
        dt = time.perf_counter() - t0
    return dict(n=sum(len(smp[2]) for smp in samples), pixels=sum(len(smp[1]) for smp in samples),
                seconds=dt, threads=threads)


def host_cpu() -> dict:
    """The host's logical core count and CPU model (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        import subprocess
        for line in subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model or "unknown"}


# ---------------------------------------------------------------- GPU arm

def run_wt(args):
    import paper_2201_00094_gb300 as wt

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=dev)
    # weak scaling (default): every rank renders its own independent frame;
    # --split rows: every rank holds the same frame and renders its own band of
    # tile rows of it (strong scaling), then the bands are gathered
    split = args.split == "rows"
    seed = args.seed if split else rank_seed(args.seed, rank)
    fr = synth.make(args.workload, seed=seed, device=dev, **size_kw(args))
    torch.cuda.synchronize()
    n, P, J = fr.n, fr.P, fr.J
    dt = {"f32": wt.F32, "bf16": wt.BF16, "f16": wt.F16, "se16": wt.SE16}[args.dtype]
    C = 1 << J
    frags = wt.make_frags(fr.pixel, fr.z, fr.alpha, fr.tile_offsets, fr.r, fr.g, fr.b)
    stream = torch.cuda.current_stream()

    def buffers(dtype):
        d = wt.make_desc(fr.width, fr.height, J, dtype, tile_w=fr.tile_w, tile_h=fr.tile_h)
        return wt.coeff_buffer(d, dev), torch.empty(P, 4, device=dev)

    coeff, out = buffers(dt)
    desc = wt.make_desc(fr.width, fr.height, J, dt, tile_w=fr.tile_w, tile_h=fr.tile_h)

    band = None
    if split:
        from paper_2201_00094_gb300 import shard
        ranges = shard.split_tile_rows(fr.tile_offsets.cpu().numpy(), desc, world)
        band = ranges[rank]

    # the two-pass method hands the build's near bounds and totals to the resolve
    zmin2 = torch.empty(P, device=dev) if args.path == "two_pass" else None
    total2 = torch.empty(P, device=dev) if args.path == "two_pass" else None

    def step_fused(d=desc, c=coeff, o=out):
        if band is not None:
            shard.build_resolve_band(d, frags, band, o, c, bg=fr.bg, stream=stream)
            if world > 1:
                shard.gather_bands(o, ranges, d, rank)
        elif args.path == "fused":
            wt.wt_build_resolve(d, frags, o, c, None, bg=fr.bg, stream=stream)
        else:
            wt.wt_build(d, frags, c, zmin2, stream=stream, total=total2)
            wt.wt_resolve_composite(d, frags, c, zmin2, o, bg=fr.bg, stream=stream, total=total2)

    K, W = args.steps, args.warmup
    for _ in range(W):
        step_fused()
    torch.cuda.synchronize()
    assert wt.wt_get_error(stream) == 0
    barrier(world)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(K)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        barrier(world)
        t_start.record(stream)
        for k in range(K):
            ev[k][0].record(stream)
            step_fused()
            ev[k][1].record(stream)
        t_end.record(stream)
        torch.cuda.synchronize()
        barrier(world)
    total_ms = max_over_ranks(t_start.elapsed_time(t_end), world)
    launch_ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    frags_all = float(n) if split else sum_over_ranks(float(n), world)
    value = frags_all * K / (total_ms / 1e3)

    # the dominant kernel's share of the frame: all of it, or this rank's band
    n_k, P_k = n, P
    if band is not None:
        offs = fr.tile_offsets.cpu().numpy()
        n_k = int(offs[band[0] + band[1]] - offs[band[0]])
        y0, y1 = shard.band_rows(band, desc)
        P_k = (y1 - y0) * fr.width
    cb = coeff_bytes(P_k, C, dt)
    # Algorithmic bytes of one frame of the method (two passes over the
    # fragments, coefficients written once and read once, RGBA written once):
    # 36 n + 2 P C s + 16 P.  The fused kernel's own minimum is 24 n + P C s + 16 P
    # (fragments read once, coefficients written once); both are reported.
    # (P C s is the coefficient storage, with SE16's exponent bytes.)
    method_bytes = n_k * 36 + 2 * cb + 16 * P_k
    fused_min_bytes = n_k * 24 + cb + 16 * P_k
    alg_bytes = method_bytes
    hbm, peak_kind = peaks()
    achieved = alg_bytes / (launch_ms / 1e3) / 1e9
    traffic = profiled_traffic("k_fused", args.workload, args.dtype) if args.path == "fused" else None

    # ---- variants (not part of `value`): two-pass path, single pass and 16-bit
    # storage.  Every (storage, path) is timed in REPEATS rounds interleaved
    # across the storage types, so that a drift of the clock or of the memory
    # system affects all of them alike; the median and the spread are reported.
    variants = {}
    if not args.no_variants and not args.no_mono_variants:
        REPEATS = 3
        runs = {}
        zmin_v, total_v = torch.empty(P, device=dev), torch.empty(P, device=dev)
        for name, d2 in (("f32", wt.F32), ("bf16", wt.BF16), ("f16", wt.F16), ("se16", wt.SE16)):
            dsc = wt.make_desc(fr.width, fr.height, J, d2, tile_w=fr.tile_w, tile_h=fr.tile_h)
            c2, o2 = buffers(d2)
            c3 = torch.empty_like(c2)
            cb2 = coeff_bytes(P, C, d2)

            # the three calls of §2.1 steps 2-4, the build's near bounds and
            # per-pixel totals handed to the resolve
            def two_pass(dsc=dsc, c2=c2, o2=o2):
                wt.wt_build(dsc, frags, c2, zmin_v, stream=stream, total=total_v)
                wt.wt_resolve_composite(dsc, frags, c2, zmin_v, o2, bg=fr.bg, stream=stream, total=total_v)

            def fused(dsc=dsc, c2=c2, o2=o2):
                wt.wt_build_resolve(dsc, frags, o2, c2, None, bg=fr.bg, stream=stream)

            # the single pass of §4 on an unchanged scene: frame t-1's
            # coefficients are this frame's (from the fused call)
            def single_pass(dsc=dsc, c2=c2, c3=c3, o2=o2):
                wt.wt_build_resolve_single_pass(dsc, frags, c2, o2, c3, bg=fr.bg, stream=stream)

            runs[name] = [(label, fn, byts) for label, fn, byts in (
                ("fused", fused, n * 24 + cb2 + 16 * P),
                ("two_pass", two_pass, n * 36 + 2 * cb2 + 16 * P + 16 * P),
                ("single_pass", single_pass, n * 24 + 2 * cb2 + 16 * P))]
            fused()
        times = {(nm, lb): [] for nm in runs for lb, _, _ in runs[nm]}
        reps = max(3, min(K, 20))
        for _ in range(REPEATS):
            for nm, lst in runs.items():
                for label, fn, byts in lst:
                    for _ in range(3):
                        fn()
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    for _ in range(reps):
                        fn()
                    b.record(stream)
                    torch.cuda.synchronize()
                    times[(nm, label)].append(a.elapsed_time(b) / reps)
        for nm, lst in runs.items():
            res = {}
            for label, fn, byts in lst:
                t = sorted(times[(nm, label)])
                ms = float(np.median(t))
                res[label] = {"ms": round(ms, 4), "ms_min_max": [round(t[0], 4), round(t[-1], 4)],
                              "fragments_per_s": n / (ms / 1e3), "alg_bytes": byts,
                              "alg_GBps": round(byts / (ms / 1e3) / 1e9, 1)}
            variants[nm] = res
        del runs

    # ---- coloured absorbance on the same frame (per-channel opacity alpha x (1, .8, .6)),
    # FP32 and E5B9G9R9 coefficient storage; the method's bytes as for the mono path:
    # per fragment pixel, z and three opacities in the build (20), the same plus r, g,
    # b in the resolve (32); the coefficients written and read once; the output
    if not args.no_variants:
        ac = [fr.alpha, (fr.alpha * 0.8).contiguous(), (fr.alpha * 0.6).contiguous()]
        o3 = torch.empty(P, 4, device=dev)
        col = {}
        for label, fmt, cbuf in (("f32", wt.RGB_F32, torch.empty(3, P, C, device=dev)),
                                 ("e5b9g9r9", wt.RGB_E5B9G9R9, torch.empty(P, C, device=dev, dtype=torch.int32))):
            def rgb_step(fmt=fmt, cbuf=cbuf):
                wt.wt_build_resolve_rgb(desc, frags, *ac, o3, cbuf, fmt, bg=fr.bg, stream=stream)
            for _ in range(3):
                rgb_step()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(10):
                rgb_step()
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / 10
            cbytes = cbuf.numel() * cbuf.element_size()
            col[label] = {"ms": round(ms, 4), "fragments_per_s": n / (ms / 1e3),
                          "coeff_bytes": cbytes, "method_bytes": n * 52 + 2 * cbytes + 16 * P,
                          "frac_method_bytes": round((n * 52 + 2 * cbytes + 16 * P) / (ms / 1e3) / 1e9 / hbm, 4)}
            del cbuf
        assert wt.wt_get_error(stream) == 0
        variants["coloured"] = col
        del ac, o3

    # ---- the chromatic-aberration composite (§3) over this frame's accumulators:
    # a background image and a smooth refraction-offset field of up to 8 pixels;
    # bytes per pixel: accumulators 20, offset 8, background 12 (read once), out 16
    if not args.no_variants:
        zm = torch.empty(P, device=dev)
        acc = torch.empty(P, 5, device=dev)
        wt.wt_build(desc, frags, coeff, zm, stream=stream)
        wt.wt_resolve(desc, frags, coeff, zm, acc, stream=stream)
        g = torch.Generator(device=dev)
        g.manual_seed(args.seed + 7)
        bg_img = torch.rand(P, 3, device=dev, generator=g)
        yy = torch.arange(fr.height, device=dev, dtype=torch.float32)[:, None].expand(fr.height, fr.width)
        xx = torch.arange(fr.width, device=dev, dtype=torch.float32)[None, :].expand(fr.height, fr.width)
        offset = torch.stack([8.0 * torch.sin(yy / 57.0), 8.0 * torch.cos(xx / 43.0)], dim=-1).reshape(P, 2)
        offset = offset.contiguous()
        o_ca = torch.empty(P, 4, device=dev)
        ca = {}
        for taps in (1, 5):
            def ca_step(taps=taps):
                wt.wt_composite_ca(desc, acc, bg_img, o_ca, offset, 0.5, taps, stream=stream)
            for _ in range(3):
                ca_step()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(20):
                ca_step()
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / 20
            ca[f"taps{taps}"] = {"ms": round(ms, 4), "pixels_per_s": P / (ms / 1e3), "alg_bytes": 56 * P,
                                 "frac_hbm": round(56 * P / (ms / 1e3) / 1e9 / hbm, 4)}
        assert wt.wt_get_error(stream) == 0
        variants["chromatic_aberration"] = ca
        del zm, acc, bg_img, offset, o_ca, xx, yy

    # ---- end to end through the C ABI from pinned host buffers
    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(wt, fr, desc, coeff, out, stream, K, world, frags_all)
    # ---- CPU baseline: the FP64 oracle on a bounded sample (rank 0, N = 1)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        res = run_oracle_sample(fr, args.cpu_tiles, seed=1234)
        got = out.cpu().numpy()[res["pixel_ids"]]
        host = host_cpu()
        threads = max(1, host["nproc"] or 1)
        par = run_oracle_threads(fr, args.cpu_tiles, threads, seed=5678)
        cpu = {"value": par["n"] / par["seconds"], "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": f"{threads} threads, each on its own {args.cpu_tiles} seeded random "
                         f"{fr.tile_w}x{fr.tile_h} tiles of the same frame ({par['pixels']} pixels, "
                         f"{par['n']} fragments in all), build + resolve + composite, FP64, "
                         f"{par['seconds']:.1f} s wall",
               "host": host,
               "single_thread": {"value": res["n"] / res["seconds"], "cores": 1,
                                 "sample": f"{args.cpu_tiles} tiles ({res['pixels']} pixels, {res['n']} "
                                           f"fragments), {res['seconds']:.1f} s"},
               "max_abs_err_gpu_vs_oracle_on_sample": float(np.abs(got - res["out"]).max())}
    preprocess = None
    if rank == 0 and world == 1 and not args.no_preprocess:
        preprocess = run_preprocess(wt, fr, desc, stream)
    particles = None
    if rank == 0 and world == 1 and not args.no_particles:
        particles = run_particles(wt, args, stream)
    backward = None
    if rank == 0 and world == 1 and not args.no_backward:
        del coeff, out
        torch.cuda.empty_cache()
        backward = run_backward(wt, args)
        coeff, out = None, None
    serving = None
    if rank == 0 and world == 1 and not args.no_serve:
        coeff = out = None
        torch.cuda.empty_cache()
        serving = serving_legs(args)
        serving["workload"] = (f"{args.serve_requests} requests from a pool of {SERVE_POOL} frames (sizes "
                               "{360p,720p,1080p,4K}, Poisson(lambda ~ U[2,32]) fragments/pixel per frame, "
                               "alpha U[.02,.6]), J=4, 40 GB cap, step 8192 tiles; open: Poisson arrivals "
                               "mean 2 ms; closed: 8 requests in flight; 5 interleaved repeats, median [min, max]")
        torch.cuda.empty_cache()
    kernel_name = "k_fused" if args.path == "fused" else "k_build + k_resolve"
    path_name = ("wt_build_resolve (fused kernel)" if args.path == "fused"
                 else "wt_build + wt_resolve_composite (two kernels)")
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": total_ms / K, "higher_is_better": True,
            "scaling": "strong" if split else "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOADS[args.workload], "name": args.workload,
                       "split": ("bands of tile rows of one frame, gathered with all_gather"
                                 if split else "one independent frame per rank"),
                       "fragments_per_gpu": n, "pixels": P, "J": J,
                       "coeff_storage": args.dtype, "path": path_name,
                       "size_override": args.size or None, "tile": args.tile,
                       "l2": f"inputs larger than L2 ({n * 24 / 1e9:.1f} GB of fragments)"},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm,
                         "unit": "GB/s", "frac": round(achieved / hbm, 4),
                         "traffic": traffic, "kernel": kernel_name,
                         "alg_bytes_per_launch": alg_bytes,
                         "alg_bytes_definition": "36 n + 2 P C s + 16 P (the method's two passes)",
                         "fused_min_bytes_per_launch": fused_min_bytes,
                         "frac_of_fused_min_bytes": round(fused_min_bytes / (launch_ms / 1e3) / 1e9 / hbm, 4),
                         "dram_frac_measured": (round(traffic / (launch_ms / 1e3) / 1e9 / hbm, 4)
                                                if traffic else None),
                         "launch_ms": round(launch_ms, 4),
                         "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_kind})"},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": K * (1 if args.path == "fused" else 2),
            "clocks": clk.summary(),
            "variants": variants,
            "preprocess": preprocess,
            "particles": particles,
            "backward": backward,
            "serving": serving,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_preprocess(wt, fr, desc, stream):
    """The steps before the build on the same frame: grouping the frame's
    fragments, put in a seeded random order, by tile (wt_bin), and the
    per-pixel depth bounds of §2.1 step 1 with the normalisation of depth into
    them (wt_depth_bounds, wt_normalize_depth).  Bytes per fragment: binning
    reads the pixel id twice and the six arrays once and writes them once
    (52 B; with two sort passes its intermediate stream adds 50 B of workspace
    traffic); bounds read pixel, z, alpha (12 B); normalisation reads pixel
    and z and writes z (12 B)."""
    dev = fr.pixel.device
    n, P = fr.n, fr.P
    g = torch.Generator(device=dev)
    g.manual_seed(4321)
    perm = torch.randperm(n, device=dev, generator=g)
    src = {k: getattr(fr, k)[perm].contiguous() for k in ("pixel", "z", "alpha", "r", "g", "b")}
    del perm
    out = {k: torch.empty_like(v) for k, v in src.items()}
    out["tile_offsets"] = torch.empty_like(fr.tile_offsets)
    ws = torch.empty(max(1, wt.wt_bin_workspace_bytes(desc, n)), dtype=torch.uint8, device=dev)
    zlo, zhi = torch.empty(P, device=dev), torch.empty(P, device=dev)
    zn = torch.empty(n, device=dev)

    def timed(fn, reps=10):
        for _ in range(3):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    bin_ms = timed(lambda: wt.wt_bin(desc, src["pixel"], src["z"], src["alpha"], src["r"], src["g"],
                                     src["b"], out=out, workspace=ws, stream=stream))
    frags = wt.make_frags(out["pixel"], out["z"], out["alpha"], out["tile_offsets"])
    bounds_ms = timed(lambda: wt.wt_depth_bounds(desc, frags, zlo, zhi, stream=stream))
    norm_ms = timed(lambda: wt.wt_normalize_depth(desc, frags, zlo, zhi, zn, stream=stream))
    assert wt.wt_get_error(stream) == 0
    assert torch.equal(out["tile_offsets"], fr.tile_offsets)
    hbm, _ = peaks()
    res = {}
    for name, ms, per in (("bin", bin_ms, 52), ("depth_bounds", bounds_ms, 12), ("normalize_depth", norm_ms, 12)):
        gbs = n * per / (ms / 1e3) / 1e9
        res[name] = {"ms": round(ms, 4), "fragments_per_s": n / (ms / 1e3), "alg_bytes_per_fragment": per,
                     "alg_GBps": round(gbs, 1), "frac_of_hbm_peak": round(gbs / hbm, 4)}
    res["input"] = "the bench frame's fragments in a seeded random order"
    del src, out, ws, zlo, zhi, zn
    torch.cuda.empty_cache()
    return res


def run_particles(wt, args, stream):
    """The whole device chain from particles to the composite on a 4K frame:
    1.1M smoke particles (centres uniform over the screen, radius U[2,12]
    pixels, depth from five Gaussian slabs, alpha U[.01,.4], colour U[0,1],
    seeded) rasterised into an unordered stream (wt_raster_count/_emit,
    ~200M fragments), grouped by tile (wt_bin) and built + resolved
    (wt_build_resolve), each step timed on its own."""
    dev = torch.device("cuda")
    W, H, N = 3840, 2160, 1_100_000
    tw, th = tile_of(args)
    g = torch.Generator(device=dev)
    g.manual_seed(args.seed + 99)
    u = lambda lo, hi: lo + (hi - lo) * torch.rand(N, generator=g, device=dev)
    slab = torch.randint(0, 5, (N,), generator=g, device=dev).float()
    pt = {"cx": u(0, W), "cy": u(0, H), "radius": u(2, 12),
          "z": (0.1 + 0.2 * slab + 0.03 * torch.randn(N, generator=g, device=dev)).clamp(0, 1),
          "alpha": u(0.01, 0.4), "r": u(0, 1), "g": u(0, 1), "b": u(0, 1)}
    desc = wt.make_desc(W, H, 5, wt.F32, tile_w=tw, tile_h=th)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    times = {"raster": [], "bin": [], "build_resolve": []}
    out = torch.empty(W * H, 4, device=dev)
    for rep in range(3):
        ev[0].record(stream)
        fr = wt.wt_raster(desc, **pt, stream=stream)
        ev[1].record(stream)
        b = wt.wt_bin(desc, fr["pixel"], fr["z"], fr["alpha"], fr["r"], fr["g"], fr["b"], stream=stream)
        ev[2].record(stream)
        frags = wt.make_frags(b["pixel"], b["z"], b["alpha"], b["tile_offsets"], b["r"], b["g"], b["b"])
        wt.wt_build_resolve(desc, frags, out, bg=(0.5, 0.5, 0.5), stream=stream)
        ev[3].record(stream)
        torch.cuda.synchronize()
        if rep:  # the first repetition warms up
            times["raster"].append(ev[0].elapsed_time(ev[1]))
            times["bin"].append(ev[1].elapsed_time(ev[2]))
            times["build_resolve"].append(ev[2].elapsed_time(ev[3]))
        n = int(fr["total"])
        del fr, b, frags
    assert wt.wt_get_error(stream) == 0
    res = {k: round(float(np.mean(v)), 4) for k, v in times.items()}
    tot = sum(res.values())
    del pt
    # glass panes: 100k quads (two triangles each) with sides U[8,40] px in random
    # orientations, a depth plane per pane, through the same chain
    Q = 100_000
    uq = lambda lo, hi: lo + (hi - lo) * torch.rand(Q, generator=g, device=dev)
    c = torch.stack([uq(0, W), uq(0, H)], 1)
    ang = uq(0, 6.2831853)
    su, sv = uq(8, 40), uq(8, 40)
    e1 = torch.stack([torch.cos(ang), torch.sin(ang)], 1) * su[:, None]
    e2 = torch.stack([-torch.sin(ang), torch.cos(ang)], 1) * sv[:, None]
    p0 = c - (e1 + e2) / 2
    corners = torch.stack([p0, p0 + e1, p0 + e1 + e2, p0 + e2], 1)  # [Q, 4, 2]
    zc = torch.rand(Q, 4, generator=g, device=dev)
    idx = torch.tensor([0, 1, 2, 0, 2, 3], device=dev)
    tv = corners[:, idx, :].reshape(-1, 2)
    tri = {"x": tv[:, 0].contiguous(), "y": tv[:, 1].contiguous(), "z": zc[:, idx].reshape(-1).contiguous(),
           "alpha": uq(0.05, 0.6).repeat_interleave(2), "r": torch.rand(2 * Q, generator=g, device=dev),
           "g": torch.rand(2 * Q, generator=g, device=dev), "b": torch.rand(2 * Q, generator=g, device=dev)}
    ptimes = {"raster_tri": [], "bin": [], "build_resolve": []}
    for rep in range(3):
        ev[0].record(stream)
        fr = wt.wt_raster_tri(desc, **tri, stream=stream)
        ev[1].record(stream)
        b = wt.wt_bin(desc, fr["pixel"], fr["z"], fr["alpha"], fr["r"], fr["g"], fr["b"], stream=stream)
        ev[2].record(stream)
        frags = wt.make_frags(b["pixel"], b["z"], b["alpha"], b["tile_offsets"], b["r"], b["g"], b["b"])
        wt.wt_build_resolve(desc, frags, out, bg=(0.5, 0.5, 0.5), stream=stream)
        ev[3].record(stream)
        torch.cuda.synchronize()
        if rep:
            ptimes["raster_tri"].append(ev[0].elapsed_time(ev[1]))
            ptimes["bin"].append(ev[1].elapsed_time(ev[2]))
            ptimes["build_resolve"].append(ev[2].elapsed_time(ev[3]))
        npanes = int(fr["total"])
        del fr, b, frags
    assert wt.wt_get_error(stream) == 0
    pres = {k: round(float(np.mean(v)), 4) for k, v in ptimes.items()}
    return {"workload": "3840x2160, 1.1M particles, radius U[2,12] px, 5 depth slabs, alpha U[.01,.4], J=5",
            "fragments": n, "ms": res, "total_ms": round(tot, 4),
            "fragments_per_s_whole_chain": n / (tot / 1e3),
            "note": "raster includes one read-back of the fragment total to size the arrays",
            "panes": {"workload": "100k glass quads (200k triangles), sides U[8,40] px, random orientation, "
                                  "depth plane per pane, alpha U[.05,.6]",
                      "fragments": npanes, "ms": pres, "total_ms": round(sum(pres.values()), 4)}}


def run_backward(wt, args):
    """Adjoint of build + resolve + composite (wt_backward) on the
    differentiation workload: 16 frames of 512x512 stacked as 512x8192 (pixels
    are independent), Poisson(32) fragments per pixel capped at 256,
    alpha U[.05,.5], J = 4, FP32, with a seeded dL/d(out).  The forward (fused)
    call on the same frame is timed beside it."""
    dev = torch.device("cuda")
    tw, th = tile_of(args)
    bw, bh = (int(x) for x in args.backward_size.lower().split("x"))
    fr = synth.uniform_frame(bw, bh, 32.0, 256, (0.05, 0.5), 4, args.seed, dev, name="diff512",
                             tile_w=tw, tile_h=th)
    n, P = fr.n, fr.P
    desc = wt.make_desc(fr.width, fr.height, fr.J, wt.F32, tile_w=fr.tile_w, tile_h=fr.tile_h)
    frags = wt.make_frags(fr.pixel, fr.z, fr.alpha, fr.tile_offsets, fr.r, fr.g, fr.b)
    g = torch.Generator(device=dev)
    g.manual_seed(args.seed + 17)
    grad_out = torch.rand(P, 4, device=dev, generator=g) - 0.5
    grad_alpha = torch.empty(n, device=dev)
    grad_rgb = torch.empty(3, n, device=dev)
    out = torch.empty(P, 4, device=dev)
    stream = torch.cuda.current_stream()

    def timed(fn, reps=10):
        for _ in range(3):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    # the forward as the autograd function runs it (it keeps the pixel sums,
    # 20 B per pixel, for the backward), and the backward with and without them
    accum = torch.empty(P, 5, device=dev)
    fwd_ms = timed(lambda: wt.wt_build_resolve(desc, frags, out, None, None, bg=fr.bg, stream=stream,
                                               accum=accum))
    bwd_ms = timed(lambda: wt.wt_backward(desc, frags, grad_out, grad_alpha, grad_rgb, bg=fr.bg,
                                          stream=stream, accum=accum))
    bwd_re_ms = timed(lambda: wt.wt_backward(desc, frags, grad_out, grad_alpha, grad_rgb, bg=fr.bg,
                                             stream=stream))
    assert wt.wt_get_error(stream) == 0
    stack = "16 x 512x512 stacked as 512x8192" if (bw, bh) == (512, 8192) else f"{bw}x{bh}"
    return {"workload": f"{stack}, Poisson(32) cap 256, alpha U[.05,.5], J=4, FP32",
            "fragments": n, "forward_ms": round(fwd_ms, 4), "backward_ms": round(bwd_ms, 4),
            "backward_ms_forward_sums_recomputed": round(bwd_re_ms, 4),
            "backward_fragments_per_s": n / (bwd_ms / 1e3),
            "backward_bytes_per_fragment": 24 + 16,
            "backward_GBps_of_fragment_io": round(n * 40 / (bwd_ms / 1e3) / 1e9, 1)}


def measure_e2e(wt, fr, desc, coeff, out, stream, K, world, frags_all, nchunks=8):
    """Same metric through the C ABI with the fragment stream copied from
    pinned host memory and the composite copied back, every step.  The frame
    goes up in `nchunks` ranges of whole tile rows: chunk c's arrays are copied
    on an upload stream while wt_build_resolve_tiles works on chunk c-1; the
    composite comes back in one copy at the end (concurrent downloads slowed
    the uploads).  The host link's own rate (the same bytes copied with
    nothing else running) is reported beside it."""
    dev = out.device
    P = fr.P
    host = {k: getattr(fr, k).cpu().pin_memory() for k in ("pixel", "z", "alpha", "r", "g", "b",
                                                             "tile_offsets")}
    out_host = torch.empty(P, 4, pin_memory=True)
    h2d = sum(t.numel() * t.element_size() for t in host.values())
    d2h = out_host.numel() * 4
    dev_bufs = {k: torch.empty_like(v, device=dev) for k, v in host.items()}
    frags_e2e = wt.make_frags(dev_bufs["pixel"], dev_bufs["z"], dev_bufs["alpha"],
                              dev_bufs["tile_offsets"], dev_bufs["r"], dev_bufs["g"], dev_bufs["b"])
    off = host["tile_offsets"].numpy()
    ntx = -(-fr.width // fr.tile_w)
    nty = -(-fr.height // fr.tile_h)
    rows = np.linspace(0, nty, min(nchunks, nty) + 1).round().astype(np.int64)
    chunks = []
    for r0, r1 in zip(rows[:-1], rows[1:]):
        if r1 > r0:
            t0, t1 = r0 * ntx, r1 * ntx
            chunks.append((int(t0), int(t1), int(off[t0]), int(off[t1])))
    up = torch.cuda.Stream(device=dev)
    arrays = ("pixel", "z", "alpha", "r", "g", "b")

    def step_e2e():
        up.wait_stream(stream)  # the previous step's kernels are done with the buffers
        with torch.cuda.stream(up):
            dev_bufs["tile_offsets"].copy_(host["tile_offsets"], non_blocking=True)
        for (t0, t1, f0, f1) in chunks:
            with torch.cuda.stream(up):
                for k in arrays:
                    dev_bufs[k][f0:f1].copy_(host[k][f0:f1], non_blocking=True)
            stream.wait_stream(up)
            wt.wt_build_resolve_tiles(desc, frags_e2e, t0, t1 - t0, out, coeff, stream=stream)
        out_host.copy_(out, non_blocking=True)  # after the last range, not against the uploads

    def copies_only():
        with torch.cuda.stream(up):
            for k in host:
                dev_bufs[k].copy_(host[k], non_blocking=True)
        stream.wait_stream(up)

    for _ in range(2):
        step_e2e()
    torch.cuda.synchronize()
    assert wt.wt_get_error(stream) == 0
    # the host link switches between a fast and a slow rate from one second to
    # the next, so the step is timed in three rounds, each beside a round of
    # the copies alone; the median round is reported, with the spread
    Ke = max(3, min(K, 10))
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rounds = []
    for _ in range(3):
        barrier(world)
        a.record(stream)
        for _ in range(Ke):
            step_e2e()
        b.record(stream)
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(a.elapsed_time(b) / Ke, world)
        a.record(stream)
        for _ in range(3):
            copies_only()
        b.record(stream)
        torch.cuda.synchronize()
        rounds.append((e2e_ms, a.elapsed_time(b) / 3))
    rounds.sort()
    e2e_ms, link_ms = rounds[1]
    return {"value": frags_all / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_ms, 3),
            "ms_per_step_rounds": [round(r[0], 3) for r in rounds], "chunks": len(chunks),
            "h2d_alone_ms": round(link_ms, 3), "h2d_alone_GBps": round(h2d / (link_ms / 1e3) / 1e9, 1),
            "h2d_alone_ms_rounds": [round(r[1], 3) for r in rounds]}


# ---------------------------------------------------------------- serving

SERVE_POOL = 96  # distinct pre-rendered frames, each with its own size and lambda


def serve_pool(args):
    """The frames the serving legs draw from: SERVE_POOL frames, each with its
    own resolution (uniform over the four sizes) and its own lambda ~ U[2, 32]
    (Poisson fragments per pixel), alpha U[.02, .6], J = 4 -- about 113 GB of
    fragments on the device.  Request i is served frame i mod SERVE_POOL, so
    every request's size and lambda are independent draws within a cycle of
    the pool; distinct frames for all 256 requests would need about 300 GB."""
    dev = torch.device("cuda")
    tw, th = tile_of(args)
    draws = synth.serve_request_params(SERVE_POOL, seed=args.seed + 17)
    pool = [synth.serve_frame(q["width"], q["height"], q["lam"], seed=q["seed"], device=dev, tile_w=tw, tile_h=th)
            for q in draws]
    torch.cuda.synchronize()
    return pool, [q["lam"] for q in draws]


def run_serving(args, dtype_name, pool, mode="open", outstanding=8):
    """Continuous-batching serving run of ``args.serve_requests`` requests, J = 4,
    40 GB cap, frames from the pool (serve_pool).

    mode "open": exponential inter-arrival times, mean 2 ms (the configuration's
    arrival process; the offered load is about a quarter of the service rate,
    so this leg is bound by the arrivals).  mode "closed": ``outstanding``
    requests are kept in flight, a new one submitted as soon as one finishes
    (offered load above the service rate: latency and throughput are those of
    the service).  Latency = GPU completion of a request's last tile (CUDA
    event) minus its submission time."""
    import paper_2201_00094_gb300 as wt
    dev = torch.device("cuda")
    dt = {"f32": wt.F32, "bf16": wt.BF16, "f16": wt.F16, "se16": wt.SE16}[dtype_name]
    reqs = synth.serve_request_params(args.serve_requests, seed=args.seed)
    tw, th = tile_of(args)
    srv = wt.Server(J=4, coeff_dtype=dt, max_slots=64, mem_cap_bytes=40 << 30, step_tiles=8192,
                    tile_w=tw, tile_h=th)
    pending = []
    lat, frags = [], 0

    def retire(block: bool):
        nonlocal frags
        while pending and (block or srv.query(pending[0][0]).state == 2):
            r0, n0 = pending.pop(0)
            assert srv.wait(r0, 120_000_000), "serving request timed out"
            info = srv.query(r0)
            lat.append((info.done_us - info.submit_us) / 1e3)
            frags += n0
            srv.release(r0)
            if block:
                return

    t_start = time.perf_counter()
    try:
        for i, rq in enumerate(reqs):
            fr = pool[i % len(pool)]
            if mode == "open":
                while (time.perf_counter() - t_start) * 1e3 < rq["arrival_ms"]:
                    pass
            else:
                while len(pending) >= outstanding:
                    retire(True)
            d = wt.make_desc(fr.width, fr.height, 4, dt, tile_w=fr.tile_w, tile_h=fr.tile_h)
            f = wt.make_frags(fr.pixel, fr.z, fr.alpha, fr.tile_offsets, fr.r, fr.g, fr.b)
            out = torch.empty(fr.P, 4, device=dev)
            rid = srv.submit(d, f, out, keep=fr)
            pending.append((rid, fr.n))
            retire(False)  # finished requests release their memory
        while pending:
            retire(True)
        makespan_s = time.perf_counter() - t_start
    finally:
        srv.close()
    lat = np.array(lat)
    return {"requests": len(lat), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "mean_ms": float(lat.mean()),
            "max_ms": float(lat.max()), "fragments": int(frags), "fragments_per_s": frags / makespan_s,
            "makespan_s": makespan_s}


def serving_legs(args, dtypes=("bf16", "se16", "f32"), repeats=5):
    """Both serving legs for each storage type, ``repeats`` runs each,
    interleaved across the types; per figure the median and the [min, max], and
    per 16-bit type the number of repeats in which it beat FP32 (the runs of one
    repeat follow each other, so they share the box's state)."""
    pool, lams = serve_pool(args)
    runs = {(m, d): [] for m in ("open", "closed") for d in dtypes}
    for _ in range(repeats):
        for m in ("open", "closed"):
            for d in dtypes:
                runs[(m, d)].append(run_serving(args, d, pool, m))
    res = {"pool": {"frames": len(pool), "fragments": int(sum(f.n for f in pool)),
                    "lambda_min_max": [round(min(lams), 2), round(max(lams), 2)]}}
    for (m, d), rs in runs.items():
        leg = res.setdefault(m, {})
        leg[d] = {}
        for key in ("p50_ms", "p99_ms", "fragments_per_s"):
            v = sorted(r[key] for r in rs)
            leg[d][key] = round(float(np.median(v)), 4) if key != "fragments_per_s" else float(np.median(v))
            leg[d][key + "_min_max"] = [round(v[0], 4), round(v[-1], 4)] if key != "fragments_per_s" \
                else [float(v[0]), float(v[-1])]
        leg[d]["requests"] = rs[0]["requests"]
        leg[d]["makespan_s"] = round(float(np.median([r["makespan_s"] for r in rs])), 4)
    for m in ("open", "closed"):
        base = runs.get((m, "f32"))
        if not base:
            continue
        for d in dtypes:
            if d == "f32":
                continue
            rs = runs[(m, d)]
            res[m][d]["repeats_beating_f32"] = {
                "p50": f"{sum(a['p50_ms'] < b['p50_ms'] for a, b in zip(rs, base))}/{len(rs)}",
                "p99": f"{sum(a['p99_ms'] < b['p99_ms'] for a, b in zip(rs, base))}/{len(rs)}",
                "fragments_per_s": f"{sum(a['fragments_per_s'] > b['fragments_per_s'] for a, b in zip(rs, base))}"
                                   f"/{len(rs)}"}
    del pool
    return res


# ---------------------------------------------------------------- reference arm

def run_reference(args):
    world, rank, local = dist_env()
    if rank != 0:
        return
    dev = torch.device("cuda", local) if torch.cuda.is_available() else torch.device("cpu")
    fr = synth.make(args.workload, seed=args.seed, device=dev, **size_kw(args))
    K, W = args.steps, args.warmup
    host = host_cpu()
    threads = max(1, host["nproc"] or 1)
    probe = run_oracle_sample(fr, 4, seed=99_999)
    per_tile = max(probe["seconds"] / 4, 1e-4)
    # every step runs `threads` samples of `tiles` tiles at once, one per core;
    # the whole run is sized to stay near --ref-seconds of wall time
    tiles = args.ref_tiles or max(1, int(args.ref_seconds / (K + W) / per_tile))
    for w in range(W):
        run_oracle_threads(fr, tiles, threads, seed=10_000 + 100 * w)
    tot_n, tot_s = 0, 0.0
    for k in range(K):
        r = run_oracle_threads(fr, tiles, threads, seed=100 * k)
        tot_n += r["n"]
        tot_s += r["seconds"]
    value = tot_n / tot_s
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": tot_s / K * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": WORKLOADS[args.workload], "name": args.workload,
                   "fragments_per_gpu": fr.n, "pixels": fr.P, "J": fr.J,
                   "coeff_storage": "f64", "path": "FP64 CPU oracle", "tile": args.tile},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "host": host,
                         "sample": f"per step {threads} threads at once, each on its own {tiles} seeded "
                                   f"random {fr.tile_w}x{fr.tile_h} tiles of the frame, build + resolve + "
                                   "composite, FP64 (the single-threaded oracle on every core)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def tile_of(args):
    tw, th = (int(x) for x in args.tile.lower().split("x"))
    return tw, th


def size_kw(args):
    tw, th = tile_of(args)
    kw = {"tile_w": tw, "tile_h": th}
    if args.size:
        w, h = (int(x) for x in args.size.lower().split("x"))
        kw.update(width=w, height=h)
    return kw


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="wt", choices=["wt", "reference"])
    ap.add_argument("--workload", default="heavy4k", choices=sorted(WORKLOADS))
    ap.add_argument("--tile", default="192x1",
                    help="screen tile WxH (one CTA each); row spans need no division, and at J = 5 "
                         "tiles of <= 192 pixels fit four CTAs per SM")
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16", "f16", "se16"])
    ap.add_argument("--split", default="none", choices=["none", "rows"],
                    help="rows: one frame split across the ranks by bands of tile rows (strong scaling)")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--size", default="", help="override the workload's WxH (profiling runs)")
    ap.add_argument("--cpu-tiles", type=int, default=96)
    ap.add_argument("--ref-tiles", type=int, default=0, help="tiles per step (0: sized by time)")
    ap.add_argument("--ref-seconds", type=float, default=120.0)
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-mono-variants", action="store_true",
                    help="time only the coloured variants (FP32 and E5B9G9R9 storage)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-backward", action="store_true")
    ap.add_argument("--backward-size", default="512x8192",
                    help="WxH of the differentiation frame (16 frames of 512x512 stacked; smaller for profiling)")
    ap.add_argument("--no-preprocess", action="store_true")
    ap.add_argument("--no-particles", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=256)
    ap.add_argument("--path", default="fused", choices=["fused", "two_pass"],
                    help="fused kernel (default) or wt_build + wt_resolve_composite")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_wt(args)


if __name__ == "__main__":
    main()
