"""Benchmark: filtered backprojection of one 2048^2 slice (2048 bins, 1800 angles) on GB300.

One step = the hot path over one synthetic slice: Shepp-Logan row filter (bp_filter)
followed by the direct pixel-driven R* (bp_backproject_direct), both through the C ABI.
Metric: backprojection pixel-angle updates per second (N^2 * n_theta per step), in G/s.

Prints ONE JSON line on rank 0.  `e2e` is the same metric through bp_fbp_host from pinned
host memory: the e2e steps run as one call over that many slices, each slice copied in and
its image copied out inside the timed region (the call overlaps the copies of neighbouring
slices with the kernels).  `--impl reference` times the FP64 CPU oracle instead.
Multi-GPU (torchrun): each rank backprojects its own independent slice (no data-path
collective); the barrier and max-over-ranks timing are the only cross-rank traffic.
"""
from __future__ import annotations

import argparse
import hashlib
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

FLOPS_PER_UPDATE = 7          # coordinate FMA (2) + fraction (1) + lerp sub and FMA (3) + accumulate (1)
FP32_LANES_PER_SM = 128       # FP32 FMA lanes per SM
L2_FLUSH_BYTES = 256 << 20    # > 129 MB L2
# shared-memory wavefront caps (128 B/clk/SM): the pair-table kernel reads 8 B per update,
# the 2 x 2-block kernel one 16-byte entry per 4 updates
SMEM_UPDATES_PER_CLK = {"bp_direct_tma_kernel": 16, "bp_direct_quad_sync_kernel": 32}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def _kernel_hash() -> str:
    h = hashlib.sha256()
    for fn in ("direct.cu", "direct_tile.cuh", "tma.cuh", "geometry.cuh", "f32x2.cuh"):
        with open(os.path.join(ROOT, "paper_1608_03589_gb300", "csrc", fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic_record(shape):
    """DRAM bytes per launch of the direct kernel from the committed ncu summary, if the
    kernel source is unchanged since that capture and it used the same launch shape; else None."""
    path = os.path.join(ROOT, "profiles", "bp_direct_kernel_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        if rec.get("kernel_hash") == _kernel_hash() and list(rec.get("launch_shape", [])) == list(shape):
            return rec
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines: list[str] = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self._t:
            self._t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def _gpu_id_for_smi(local_idx: int) -> str:
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        ids = [v.strip() for v in vis.split(",") if v.strip()]
        if local_idx < len(ids):
            return ids[local_idx]
    return str(local_idx)


def _dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def replica_slice(rank: int) -> int:
    """Slice of the workload a rank backprojects: replicas only, each rank its own slice (seed
    offset by the rank), no data exchanged between ranks."""
    return rank


def max_over_ranks(value: float, dist, device) -> float:
    """The job's time for a quantity each rank measured: the maximum over ranks (all-reduce MAX)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def throughput(updates_per_rank: int, world: int, steps: int, total_ms: float) -> float:
    """Whole-job G updates/s: the updates of all ranks over the slowest rank's time."""
    return updates_per_rank * world * steps / (total_ms / 1e3) / 1e9


# ----------------------------------------------------------------------------------------------- oracle arm
def run_reference(args, world, rank):
    """FP64 CPU oracle on the host cores: each step backprojects a bounded pixel sample and
    filters a bounded row sample of the same workload; throughput is extrapolated per update."""
    if rank != 0:
        return
    import oracle
    from paper_1608_03589_gb300 import synth

    wl = synth.LARGE
    g = wl.sinogram()
    q = oracle.filter_rows(g[:8], wl.det_spacing, oracle.SHEPP_LOGAN)  # warm the library
    q_full = g  # timing only: the per-pixel cost does not depend on the values
    n_pix, n_rows = 65536, 240  # about 30 ms of 16-core oracle work per step
    rng = np.random.default_rng(0)
    times, upd = [], 0
    for s in range(args.warmup + args.steps):
        pix = rng.choice(wl.N * wl.N, n_pix, replace=False)
        rows = rng.choice(wl.n_theta, n_rows, replace=False)
        t0 = time.perf_counter()
        oracle.filter_rows(g[rows], wl.det_spacing, oracle.SHEPP_LOGAN)
        t1 = time.perf_counter()
        oracle.bp_linear_points(q_full, wl.N, wl.theta, wl.det_spacing, pix)
        t2 = time.perf_counter()
        if s >= args.warmup:
            # this step's share of a full slice: n_pix / N^2 of the R* work and the same share of the filter
            t_filter_share = (t1 - t0) * (wl.n_theta / n_rows) * (n_pix / (wl.N * wl.N))
            times.append((t2 - t1) + t_filter_share)
            upd += n_pix * wl.n_theta
    total = sum(times)
    value = upd / total / 1e9
    cores = oracle.num_threads()
    sample = (f"per step: oracle R* at {n_pix} random pixels x {wl.n_theta} angles plus the oracle filter on "
              f"{n_rows} rows scaled to the same share of the slice; FP64, OpenMP")
    line = {
        "metric": "backprojection G pixel·angle updates/s at 2048²×1800; % of roofline",
        "impl": "reference", "value": value, "unit": "Gupdates/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "N": wl.N, "n_det": wl.n_det, "n_theta": wl.n_theta,
                   "filter": "shepp-logan", "step": "filter + direct R* (sampled)"},
        "cpu_baseline": {"value": value, "unit": "Gupdates/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "Gupdates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline():
    """The oracle as it stands on this host's cores: the whole filtered backprojection of the
    2048^2 x 1800 workload (oracle Shepp-Logan filter on all rows, oracle R* on all pixels)."""
    import oracle
    from paper_1608_03589_gb300 import synth

    wl = synth.LARGE
    g = wl.sinogram()
    t0 = time.perf_counter()
    q = oracle.filter_rows(g, wl.det_spacing, oracle.SHEPP_LOGAN)
    t1 = time.perf_counter()
    oracle.bp_linear(q, wl.N, wl.theta, wl.det_spacing)
    t2 = time.perf_counter()
    return {"value": wl.updates / (t2 - t0) / 1e9, "unit": "Gupdates/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"the full workload once: FP64 oracle Shepp-Logan filter on all {wl.n_theta} rows "
                      f"({t1 - t0:.1f} s) + oracle R* on all {wl.N}x{wl.N} pixels ({t2 - t1:.1f} s)"}


# ----------------------------------------------------------------------------------------------- other paths
def _timed(fn, stream, flush, reps):
    import torch
    fn()
    torch.cuda.synchronize()
    tot = 0.0
    for _ in range(reps):
        flush.zero_()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        fn()
        e.record(stream)
        torch.cuda.synchronize()
        tot += s.elapsed_time(e)
    return tot / reps


def other_paths(plan, q, img, flush, stream, dev, only=()):
    """Every other row of the path on its own workload, each timed with CUDA events."""
    import numpy as np
    import torch

    from paper_1608_03589_gb300 import autograd as ag
    from paper_1608_03589_gb300 import bp, synth

    wl = synth.LARGE
    out = {}

    def guard(name, fn):
        if only and name not in only:
            return
        try:
            out[name] = fn()
        except Exception as exc:  # reported, never hidden
            out[name] = {"unavailable": f"{type(exc).__name__}: {str(exc)[:160]}"}
        torch.cuda.empty_cache()

    # 2048^2 x 1800 slice: Fourier R*, R (direct and Fourier adjoint), BF16 storage
    def fourier():
        ms = _timed(lambda: plan.backproject_fourier(q, out=img), stream, flush, 10)
        plan.set_fourier_width(4)
        ms4 = _timed(lambda: plan.backproject_fourier(q, out=img), stream, flush, 10)
        plan.set_fourier_width(6)
        return {"ms": ms, "equiv_Gupdates_s": wl.updates / ms / 1e6, "kernel_width": 6,
                "width4_ms": ms4, "width4_equiv_Gupdates_s": wl.updates / ms4 / 1e6}
    guard("fourier_backprojection_2048", fourier)

    def fbp_fourier():
        tmp = torch.empty_like(q)
        fused = _timed(lambda: plan.fbp_fourier(q, "shepp-logan", out=img), stream, flush, 10)
        two = _timed(lambda: (plan.filter(q, "shepp-logan", out=tmp), plan.backproject_fourier(tmp, out=img)),
                     stream, flush, 10)
        return {"fused_ms": fused, "filter_then_fourier_ms": two, "equiv_Gupdates_s": wl.updates / fused / 1e6}
    guard("fbp_fourier_fused_2048", fbp_fourier)

    def bst():
        res = {}
        for os in (1, 4):
            ms = _timed(lambda: plan.backproject_bst(q, os, out=img), stream, flush, 10)
            res[f"oversampling_{os}"] = {"ms": ms, "equiv_Gupdates_s": wl.updates / ms / 1e6}
        return res
    guard("bst_interpolation_2048", bst)

    def bst_windowed():
        res = {}
        for os in (1, 4):
            ms = _timed(lambda: plan.backproject_bst_windowed(q, 6.0, os, out=img), stream, flush, 10)
            res[f"oversampling_{os}"] = {"ms": ms, "equiv_Gupdates_s": wl.updates / ms / 1e6, "beta": 6.0}
        return res
    guard("bst_windowed_2048", bst_windowed)

    def logpolar():
        ms = _timed(lambda: plan.backproject_logpolar(q, out=img), stream, flush, 5)
        return {"ms": ms, "equiv_Gupdates_s": wl.updates / ms / 1e6}
    guard("logpolar_2048", logpolar)

    def logpolar_partial():
        plan.backproject_logpolar_partial(q, 8, 0.25, out=img)  # workspace and pixel tables (untimed)
        ms = _timed(lambda: plan.backproject_logpolar_partial(q, 8, 0.25, out=img), stream, flush, 5)
        return {"ms": ms, "equiv_Gupdates_s": wl.updates / ms / 1e6, "sectors": 8, "a_r": 0.25}
    guard("logpolar_partial_2048", logpolar_partial)

    def radon():
        shape, _ = plan.autotune("radon", batch=1)
        ms = _timed(lambda: plan.radon(img, out=q), stream, flush, 5)
        return {"ms": ms, "Gupdates_s": wl.updates / ms / 1e6, "launch_shape": {"angles_per_cta": shape[0],
                                                                               "bands": shape[1]}}
    guard("radon_direct_2048", radon)

    def radon_f():
        ms = _timed(lambda: plan.radon(img, out=q, fourier=True), stream, flush, 10)
        return {"ms": ms, "equiv_Gupdates_s": wl.updates / ms / 1e6}
    guard("radon_fourier_2048", radon_f)

    def bf16():
        q16 = q.to(torch.bfloat16)
        shape, _ = plan.autotune("direct", torch.bfloat16, 1)
        ms = _timed(lambda: plan.backproject(q16, out=img), stream, flush, 10)
        return {"ms": ms, "Gupdates_s": wl.updates / ms / 1e6, "launch_shape": {"stage": shape[0],
                                                                               "angle_groups": shape[1]}}
    guard("direct_bf16_storage_2048", bf16)

    # 256^2 slice, 256 bins, 180 angles (16 pixel tiles): default launch shape vs autotuned
    def small():
        S = synth.SMALL
        ps = bp.Plan(S.N, S.n_det, S.theta, S.det_spacing)
        gs = torch.from_numpy(S.sinogram().astype(np.float32)).to(dev)
        qs = ps.filter(gs, "ramlak")
        ims = torch.empty((S.N, S.N), dtype=torch.float32, device=dev)
        res = {}
        for label, shp in (("one_cta_per_tile", (16, 1)), ("default", None)):
            if shp:
                ps.set_shape(shp, "direct", torch.float32, 1)
            else:
                ps = bp.Plan(S.N, S.n_det, S.theta, S.det_spacing)
            used = ps.get_shape("direct", torch.float32, 1)
            ms = _timed(lambda: ps.backproject(qs, out=ims), stream, flush, 20)
            res[label] = {"ms": ms, "Gupdates_s": S.updates / ms / 1e6, "launch_shape": list(used)}
        shape, _ = ps.autotune("direct", torch.float32, 1)
        ms = _timed(lambda: ps.backproject(qs, out=ims), stream, flush, 20)
        res["autotuned"] = {"ms": ms, "Gupdates_s": S.updates / ms / 1e6, "launch_shape": list(shape)}
        ps.close()
        return res
    guard("slice256_bins256_ang180_shapes", small)

    # volume: 256 slices of 2048^2 from BF16 sinograms, one batched launch replayed from a CUDA graph
    def volume():
        V = synth.VOLUME
        n = synth.VOLUME_SLICES
        vol = torch.empty((n, V.n_theta, V.n_det), dtype=torch.bfloat16, device=dev)
        chunk = 32
        tmp = torch.empty((chunk, V.n_theta, V.n_det), dtype=torch.float32, device=dev)
        for c0 in range(0, n, chunk):
            for i in range(chunk):
                e = synth.random_ellipses(V.n_ellipses, V.seed + c0 + i)
                tmp[i] = synth.ellipse_sinogram_torch(e, V.theta, V.n_det, V.det_spacing, dev).float()
            plan.filter(tmp, "shepp-logan", out=tmp)
            vol[c0:c0 + chunk] = tmp.to(torch.bfloat16)
        del tmp
        imgs = torch.empty((n, V.N, V.N), dtype=torch.float32, device=dev)
        plan.backproject(vol, out=imgs)
        s2 = torch.cuda.Stream(dev)
        s2.wait_stream(torch.cuda.current_stream(dev))
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s2):
            plan.backproject(vol, out=imgs)
        ms = _timed(graph.replay, stream, flush, 3)
        return {"slices": n, "ms": ms, "Gupdates_s": n * V.updates / ms / 1e6, "storage": "bf16",
                "launch": "one batched launch replayed from a CUDA graph"}
    guard("volume256_bf16_graph", volume)

    # differentiable reconstruction: 8 x 1024^2, 1024 bins, 720 angles, 50 GD iterations on ||Rf-g||^2 + 1e-3 TV
    def tv():
        N, nd, nt, B = 1024, 1024, 720, 8
        p2 = bp.Plan(N, nd, synth.uniform_theta(nt))
        g = torch.stack([synth.ellipse_sinogram_torch(synth.random_ellipses(30, 4000 + i), synth.uniform_theta(nt),
                                                      nd, 2.0 / nd, dev).float() for i in range(B)])
        p2.autotune("radon", batch=B)
        p2.autotune("direct", torch.float32, B)  # R^T runs the direct R* kernel
        step = 1.0 / (2.0 * ag.lipschitz_estimate(p2, (B, N, N), dev) + 1e-3 * 8.0 / 1e-3)
        ag.tv_reconstruct(g, p2, iters=2, step=step)
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        st = ag.tv_reconstruct(g, p2, iters=50, step=step)
        e.record(stream)
        torch.cuda.synchronize()
        ms = s.elapsed_time(e)
        p2.close()
        return {"batch": B, "iterations": 50, "ms": ms, "ms_per_iteration": ms / 50,
                "loss_first_last": [st.losses[0], st.losses[-1]],
                "Gupdates_s": 2 * 50 * B * N * N * nt / ms / 1e6}
    guard("tv_reconstruction_8x1024", tv)

    # uneven batch: 64 slices, widths in {512..4096}, 360-3000 angles, FP16, one persistent launch
    def mixed():
        geo = synth.mixed_batch_geometries()
        plans, sinos, imgs2 = [], [], []
        upd = 0
        for i, (N, nd, nt) in enumerate(geo):
            th = synth.uniform_theta(nt)
            pi = bp.Plan(N, nd, th)
            e = synth.random_ellipses(30, 5000 + i)
            g = synth.ellipse_sinogram_torch(e, th, nd, 2.0 / nd, dev).float()
            sinos.append(pi.filter(g, "shepp-logan").to(torch.float16))
            plans.append(pi)
            imgs2.append(torch.empty((N, N), dtype=torch.float32, device=dev))
            upd += N * N * nt
        ms = _timed(lambda: bp.backproject_batched(plans, sinos, imgs2), stream, flush, 3)
        for pi in plans:
            pi.close()
        return {"slices": len(geo), "updates": upd, "ms": ms, "Gupdates_s": upd / ms / 1e6, "storage": "fp16",
                "launch": "one persistent launch (dynamic tile queue)"}
    guard("mixed64_fp16_persistent", mixed)

    # single 8192^2 slice, 8192 bins, 6000 angles: direct and Fourier
    def big():
        N, nd, nt = 8192, 8192, 6000
        th = synth.uniform_theta(nt)
        pb = bp.Plan(N, nd, th)
        g = synth.ellipse_sinogram_torch(synth.random_ellipses(30, 5999), th, nd, 2.0 / nd, dev).float()
        qb = pb.filter(g, "shepp-logan")
        del g
        ib = torch.empty((N, N), dtype=torch.float32, device=dev)
        pb.autotune("direct", torch.float32, 1)
        msd = _timed(lambda: pb.backproject(qb, out=ib), stream, flush, 2)
        msf = _timed(lambda: pb.backproject_fourier(qb, out=ib), stream, flush, 2)
        pb.close()
        return {"direct_ms": msd, "direct_Gupdates_s": N * N * nt / msd / 1e6, "fourier_ms": msf,
                "fourier_equiv_Gupdates_s": N * N * nt / msf / 1e6}
    guard("slice8192_bins8192_ang6000", big)
    return out


# ----------------------------------------------------------------------------------------------- GPU arm
def run_gpu(args, world, rank, local):
    import torch

    import __graft_entry__
    from paper_1608_03589_gb300 import bp, synth

    if rank == 0 or world == 1:
        __graft_entry__.build()
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist = dist_mod
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        if rank != 0:
            __graft_entry__.build()
        dist.barrier()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)

    wl = synth.LARGE
    g_host = wl.sinogram(slice_id=replica_slice(rank)).astype(np.float32)
    plan = bp.Plan(wl.N, wl.n_det, wl.theta, wl.det_spacing)
    g = torch.from_numpy(g_host).to(dev)
    q = torch.empty_like(g)
    img = torch.empty((wl.N, wl.N), dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        plan.filter(g, "shepp-logan", out=q)
        plan.backproject(q, out=img)

    # launch shape of the direct R* picked by the library's autotuner (untimed setup), or fixed
    if args.shape:
        plan.set_shape(tuple(int(v) for v in args.shape.split(",")), "direct", torch.float32, 1)
        shape, picked = plan.get_shape("direct", torch.float32, 1), "--shape"
    elif args.no_tune:
        shape, picked = plan.get_shape("direct", torch.float32, 1), "default rule"
    else:
        shape, _ = plan.autotune("direct", torch.float32, 1)
        picked = "bp_autotune"

    for _ in range(max(3, args.warmup)):
        step()
        flush.zero_()
    torch.cuda.synchronize()
    if args.only:
        only = tuple(x for x in args.only.split(",") if x)
        res = other_paths(plan, q, img, flush, stream, dev, only)
        if rank == 0:
            print(json.dumps({"only": list(only), "paths": res}), flush=True)
        plan.close()
        return

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(_gpu_id_for_smi(local))
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.zero_()  # L2 flush outside the timed interval
        e0, e1, e2 = ev[i]
        e0.record(stream)
        plan.filter(g, "shepp-logan", out=q)
        e1.record(stream)
        plan.backproject(q, out=img)
        e2.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(c) for a, b, c in ev]
    bp_ms = [b.elapsed_time(c) for a, b, c in ev]
    filt_ms = [a.elapsed_time(b) for a, b, c in ev]
    total_ms = sum(step_ms)
    total_ms = max_over_ranks(total_ms, dist, dev)

    if args.no_extras:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        if rank == 0:
            print(json.dumps({"value": throughput(wl.updates, world, args.steps, total_ms),
                              "unit": "Gupdates/s", "kernel_ms": statistics.mean(bp_ms), "partial": True}))
        return
    # end to end through the host-buffer C-ABI call: n_e2e steps as one call over n_e2e pinned
    # host sinograms (each step's copy in and copy out inside the timed region; the call
    # overlaps the copies of neighbouring slices with the kernels of the current one)
    n_e2e = max(3, min(args.steps, 20))
    g_pin = torch.from_numpy(np.broadcast_to(g_host, (n_e2e, *g_host.shape)).copy()).pin_memory()
    img_pin = torch.empty((n_e2e, wl.N, wl.N), dtype=torch.float32).pin_memory()
    plan.fbp_host(g_pin, "shepp-logan", out=img_pin)
    if dist:
        dist.barrier()
    e2e_t, e2e_reps = 0.0, 2
    for _ in range(e2e_reps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.fbp_host(g_pin, "shepp-logan", out=img_pin)
        e2e_t += time.perf_counter() - t0
    e2e_t = max_over_ranks(e2e_t, dist, dev)
    n_e2e *= e2e_reps

    # other operators and workloads of the path (reported under "paths", not part of the step)
    extra = {} if args.no_paths else other_paths(plan, q, img, flush, stream, dev,
                                                 tuple(x for x in args.only.split(",") if x))
    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    props = torch.cuda.get_device_properties(dev)
    peaks = _peaks()
    sm_max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak_tflops = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12
    bp_avg_s = statistics.mean(bp_ms) / 1e3
    achieved = wl.updates * FLOPS_PER_UPDATE / bp_avg_s / 1e12
    traffic = _traffic_record(shape)
    # the library takes the 2 x 2-block kernel when every pixel step |c|, |s| = |cos|, |sin| dx/dt <= 1
    ratio = (2.0 / wl.N) / wl.det_spacing
    steps = np.abs(np.stack([np.cos(wl.theta), np.sin(wl.theta)])) * ratio
    kernel = "bp_direct_quad_sync_kernel" if float(np.max(steps.astype(np.float32))) <= 1.0 else "bp_direct_tma_kernel"
    smem_cap = SMEM_UPDATES_PER_CLK[kernel] * props.multi_processor_count * sm_max_mhz * 1e6
    line = {
        "metric": "backprojection G pixel·angle updates/s at 2048²×1800; % of roofline",
        "value": throughput(wl.updates, world, args.steps, total_ms),
        "unit": "Gupdates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl.name, "N": wl.N, "n_det": wl.n_det, "n_theta": wl.n_theta,
                   "phantom": "50 seeded random ellipses + 1% Gaussian noise", "filter": "shepp-logan",
                   "step": "bp_filter + bp_backproject_direct", "l2": "flushed (256 MiB write) between steps",
                   "launch_shape": {"stage": shape[0], "angle_groups": shape[1],
                                    "picked_by": picked},
                   "parallelism": f"independent slice per GPU x{world}"},
        "roofline": {"bound": "alu", "kernel": kernel, "achieved": achieved,
                     "peak": peak_tflops, "unit": "TFLOP/s", "frac": achieved / peak_tflops,
                     "flops_per_update": FLOPS_PER_UPDATE,
                     "peak_basis": f"{props.multi_processor_count} SM x {FP32_LANES_PER_SM} FP32 lanes x 2 x "
                                   f"{sm_max_mhz:.0f} MHz (max SM clock)",
                     "traffic": (traffic["dram_bytes_per_launch"] if traffic else None),
                     "algorithmic_bytes": wl.n_theta * wl.n_det * 4 + wl.N * wl.N * 4,
                     "kernel_ms": bp_avg_s * 1e3, "filter_ms": statistics.mean(filt_ms),
                     "smem_limit": {
                         "resource": "shared-memory wavefronts, 1/clk/SM (" + (
                             "one 16-byte table entry per 2 x 2 pixel block" if kernel == "bp_direct_quad_sync_kernel"
                             else "one 8-byte table pair per update") + ")",
                         "cap_Gupdates_s": smem_cap / 1e9,
                         "frac": wl.updates / bp_avg_s / smem_cap},
                     "issue_limit": ({
                         "resource": "instruction issue, 1 warp instruction/clk per SM sub-partition",
                         "warp_inst_per_update_ncu": traffic["warp_inst_per_update"],
                         "cap_Gupdates_s": 4 * 32 / traffic["warp_inst_per_update"] * props.multi_processor_count *
                                           sm_max_mhz / 1e3,
                         "frac": wl.updates / bp_avg_s / (4 * 32 / traffic["warp_inst_per_update"] *
                                                          props.multi_processor_count * sm_max_mhz * 1e6)}
                                     if traffic and "warp_inst_per_update" in traffic else None)},
        "e2e": {"value": wl.updates * world * n_e2e / e2e_t / 1e9, "unit": "Gupdates/s",
                "h2d_bytes_per_step": g_host.nbytes, "d2h_bytes_per_step": wl.N * wl.N * 4,
                "call": "bp_fbp_host over %d pinned host slices per call (copies of neighbouring slices "
                        "overlap the kernels)" % (n_e2e // e2e_reps)},
        "gpu_launches": 2 * args.steps,
        "clocks": clocks,
        "paths": extra,
    }
    if not args.no_cpu_baseline:
        try:
            line["cpu_baseline"] = cpu_baseline()
        except Exception as exc:  # pragma: no cover
            line["cpu_baseline"] = {"unavailable": str(exc)[:120]}
    print(json.dumps(line), flush=True)
    plan.close()
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the e2e and other-operator timings")
    ap.add_argument("--no-paths", action="store_true", help="skip the other workloads under 'paths'")
    ap.add_argument("--only", default="", help="comma-separated path names: run only these (profiling)")
    ap.add_argument("--no-tune", action="store_true", help="time the direct R* with its default launch shape")
    ap.add_argument("--shape", default="", help="fixed direct R* launch shape 'stage,angle_groups' (no tuning)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    world, rank, local = _dist_init()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_gpu(args, world, rank, local)


if __name__ == "__main__":
    main()
