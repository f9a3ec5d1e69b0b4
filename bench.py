"""Benchmark: filtered backprojection of one 2048^2 slice (2048 bins, 1800 angles) on GB300.

One step = the hot path over one synthetic slice through the C ABI: bp_fbp_direct, the
Shepp-Logan row filter (its filtered rows written straight into the row tables of the
four-image direct R*) followed by the direct pixel-driven R*.
Metric: backprojection pixel-angle updates per second (N^2 * n_theta per step), in G/s.

Prints ONE JSON line on rank 0.  `e2e` is the same metric through bp_fbp_host from pinned
host memory: the e2e steps run as one call over that many slices, each slice copied in and
its image copied out inside the timed region (the call overlaps the copies of neighbouring
slices with the kernels; the median of three timed calls).  `--impl reference` times the FP64
CPU oracle instead.
Multi-GPU (torchrun): each rank backprojects its own independent slice (no data-path
collective); the barrier and max-over-ranks timing are the only cross-rank traffic.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
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
# sources whose content the committed DRAM-traffic record of a kernel is tied to
_FOURIER_SOURCES = ("fourier.cu", "fft.cuh", "fft_pt.cuh", "tma.cuh", "geometry.cuh")
_LP_SOURCES = ("logpolar.cu", "lp_rows.cuh", "fft.cuh", "fft_pt.cuh", "tma.cuh")
KERNEL_SOURCES = {
    "bp_direct_klein_kernel": ("direct_klein.cu", "direct_tile.cuh", "tma.cuh", "f32x2.cuh", "geometry.cuh"),
    "bp_direct_quad_sync_kernel": ("direct.cu", "direct_tile.cuh", "tma.cuh", "geometry.cuh", "f32x2.cuh"),
    "filter_pt_kernel": ("filter.cu", "filter_pt.cuh", "fft.cuh", "fft_pt.cuh"),
    "klein_filter_tables_kernel": ("direct_klein.cu", "filter_pt.cuh", "fft.cuh", "fft_pt.cuh"),
    "fourier_spectra_pt_kernel": _FOURIER_SOURCES,
    "gridding": _FOURIER_SOURCES,
    "ifft_pt_kernel (y pass)": _FOURIER_SOURCES,
    "ifft_pt_kernel (x pass)": _FOURIER_SOURCES,
    "lp_rows_fwd_kernel": _LP_SOURCES,
    "lp_cols_kernel": _LP_SOURCES,
    "lp_rows_inv_kernel": _LP_SOURCES,
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def kernel_hash(kernel: str) -> str:
    h = hashlib.sha256()
    for fn in KERNEL_SOURCES.get(kernel, ()):
        with open(os.path.join(ROOT, "paper_1608_03589_gb300", "csrc", fn), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def traffic_path(kernel: str) -> str:
    slug = "".join(ch if ch.isalnum() else "_" for ch in kernel).strip("_")
    while "__" in slug:
        slug = slug.replace("__", "_")
    return os.path.join(ROOT, "profiles", f"{slug}_traffic.json")


def _traffic_record(kernel, shape=None, workload=None):
    """The committed ncu DRAM-traffic record of `kernel` (per call of its operator), if the
    kernel's sources are unchanged since that capture and it ran the same launch shape (direct
    kernels) on the same workload; else None."""
    try:
        with open(traffic_path(kernel)) as f:
            rec = json.load(f)
        if rec.get("kernel_hash") != kernel_hash(kernel):
            return None
        if shape is not None and list(rec.get("launch_shape", [])) != list(shape):
            return None
        if workload is not None and rec.get("workload") != workload:
            return None
        return rec
    except Exception:
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


def cpu_baseline(img_gpu=None):
    """The oracle as it stands on this host's cores: the whole filtered backprojection of the
    2048^2 x 1800 workload (oracle Shepp-Logan filter on all rows, oracle R* on all pixels); and
    the step's GPU image against that FP64 result (the same float32 input)."""
    import oracle
    from paper_1608_03589_gb300 import synth

    wl = synth.LARGE
    g = wl.sinogram().astype(np.float32).astype(np.float64)  # the float32 values the device reads
    t0 = time.perf_counter()
    q = oracle.filter_rows(g, wl.det_spacing, oracle.SHEPP_LOGAN)
    t1 = time.perf_counter()
    b = oracle.bp_linear(q, wl.N, wl.theta, wl.det_spacing)
    t2 = time.perf_counter()
    base = {"value": wl.updates / (t2 - t0) / 1e9, "unit": "Gupdates/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"the full workload once: FP64 oracle Shepp-Logan filter on all {wl.n_theta} rows "
                      f"({t1 - t0:.1f} s) + oracle R* on all {wl.N}x{wl.N} pixels ({t2 - t1:.1f} s)"}
    err = None
    if img_gpu is not None:
        err = {"rel_l2": oracle.rel_l2(img_gpu, b),
               "against": "FP64 oracle filter + R* of the same float32 sinogram, whole image (the step's output: "
                          "FP32 filter and R* together)"}
    return base, err


# ----------------------------------------------------------------------------------------------- kernel rooflines
# FP32 peak of the ALU roofline, TFLOP/s at 2070 MHz: the derived 152 SM x 128 lanes x 2 x f_clk
# figure.  An FFMA-throughput probe on a GB300 of this machine reached FP32_PROBE_TFLOPS (recorded in
# the design notes); the roofline uses the smaller of the two.
FP32_PROBE_TFLOPS = 79.48  # paired-FMA (f32x2) issue probe, 152 SMs, clocks at 2070 MHz (scalar FFMA: 76.7)


def fp32_peak_tflops(sm_count: int, sm_max_mhz: float):
    derived = sm_count * FP32_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12
    if FP32_PROBE_TFLOPS and FP32_PROBE_TFLOPS < derived:
        return FP32_PROBE_TFLOPS, f"measured by an FFMA-throughput probe ({FP32_PROBE_TFLOPS:.1f} TFLOP/s, below " \
                                  f"the derived {derived:.1f})"
    return derived, f"{sm_count} SM x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_max_mhz:.0f} MHz (max SM clock)"


def klein_table_entries(N: int, n_det: int, theta, dt: float) -> int:
    """Entries per row of the four-image form's row tables (the bins its blocks reach plus 4 on
    each side), restated for the byte count of klein_tables_kernel."""
    r = (2.0 / N) / dt
    nr = (N // 2 + 31) // 32
    E = 32 * nr - 1
    c, s = np.cos(theta) * r, np.sin(theta) * r
    u00 = (c + s) * (0.5 - 0.5 * N) + 0.5 * (n_det - 1)
    lo = u00 + np.minimum(0, c * E) + np.minimum(0, s * E)
    hi = u00 + np.maximum(0, c * E) + np.maximum(0, s * E)
    return int(np.floor(hi.max()) + 4 - (np.floor(lo.min()) - 4) + 1)


def _pow2_at_least(n: int) -> int:
    p = 1
    while p < n:
        p <<= 1
    return p


def lp_meshes(N: int, n_det: int, n_theta: int, dt: float) -> dict:
    """Mesh sizes of the adaptive-rho_0 log-polar R* (Section 5.1-5.2; the library builds the
    same from these formulas): rho nodes, output nodes, angle nodes and the rho transform length."""
    dx = 2.0 / N
    s_max = 0.5 * (n_det - 1) * dt + dt
    rho0, top = math.log(0.5 * dx), math.log(s_max)
    step = -math.log(1.0 - dt / s_max)
    n_rho = math.ceil((top - rho0) / step) + 1
    drho = (top - rho0) / (n_rho - 1)
    r_far = math.sqrt(2.0) * (1.0 - 0.5 * dx)
    n_out = math.ceil((math.log(max(r_far, 0.5 * dx)) - rho0) / drho) + 2
    return {"lp_nphi": _pow2_at_least(2 * n_theta), "lp_L": _pow2_at_least(n_rho + n_out), "lp_nout": n_out}


def lpp_meshes(N: int, n_det: int, n_theta: int, dt: float, Q: int, a_r: float) -> dict:
    """Mesh sizes of the partial (sector) log-polar R* with Q sectors and shift ratio a_r."""
    dx, R = 2.0 / N, math.sqrt(2.0)
    n_half = _pow2_at_least(max(n_theta, 1))
    K = n_half // Q
    dphi, d = math.pi / n_half, R * (1.0 - a_r) / a_r
    beta, alpha = 0.5 * (K - 1) * dphi, math.asin(R / d)
    gamma = alpha + beta + 3.0 * dphi
    step = -math.log(1.0 - dt / (d + R))
    rho0, top = math.log((d - R) * math.cos(gamma)) - 2.0 * step, math.log(d + R)
    n_rho = math.ceil((top - rho0) / step) + 1
    drho = (top - rho0) / (n_rho - 1)
    c_lo = math.floor((math.log(d - R) - rho0) / drho)
    n_out = n_rho - c_lo
    A = alpha / dphi
    a_lo, a_hi = math.floor(0.5 * (K - 1) - A) - 1, math.ceil(0.5 * (K - 1) + A) + 1
    n_aout = a_hi - a_lo + 1
    b_lo, b_hi = a_lo - (K - 1), a_hi
    kmax = math.floor(-math.log(math.cos(max(-b_lo, b_hi) * dphi)) / drho) + 1
    return {"lpp_Q": Q, "lpp_K": K, "lpp_nout": n_out, "lpp_naout": n_aout,
            "lpp_Lr": _pow2_at_least(n_rho + kmax + 1), "lpp_Lp": _pow2_at_least(max(b_hi - b_lo + 1, n_aout, K))}


def kernel_work(name: str, c: dict):
    """Algorithmic (bytes, flops) of one launch of kernel `name` on workload c (N, n_det, n_theta,
    esz, P, M, W, and the BST / log-polar mesh sizes; an FFT of n points counts 5 n log2 n flops,
    an FMA 2): the per-unit figures of the measurement plan times the units one slice (one call)
    processes.  None when no model is kept."""
    N, nd, nt, esz = c["N"], c["n_det"], c["n_theta"], c.get("esz", 4)
    P, M, W = c.get("P", 0), c.get("M", 0), c.get("W", 6)
    upd = N * N * nt
    lg = lambda n: math.log2(n) if n else 0.0
    if name.startswith("bp_direct") or name in ("radon_quad_kernel", "radon_direct_kernel"):
        return nt * nd * esz + 4 * N * N, 7 * upd
    if name == "klein_tables_kernel":
        L = klein_table_entries(N, nd, c["theta"], c["dt"])
        return nt * nd * esz + 2 * 16 * nt * L, 8 * nt * L
    if name == "klein_filter_tables_kernel":  # the row filter with the tables as its output
        L = klein_table_entries(N, nd, c["theta"], c["dt"])
        return nt * nd * esz + 2 * 16 * nt * L, nt * (5 * P * lg(P) + P) + 8 * nt * L
    if name.startswith("memset"):
        return c.get("memset_bytes", 4 * N * N), 0
    if name in ("filter_pt_kernel", "filter_kernel"):
        return nt * nd * (esz + 4), nt * (5 * P * lg(P) + P)
    if name in ("fourier_spectra_pt_kernel", "fourier_spectra_kernel"):
        return nt * nd * esz + nt * (P // 2) * 8, nt * (2.5 * P * lg(P) + 6 * P)
    if name == "gridding":
        return nt * (P // 2) * 8 + 8 * M * M, 8 * W * W * nt * (P // 2)
    if name in ("ifft_pt_kernel (y pass)", "ifft_pass_y_kernel"):
        return 8 * M * M + 8 * N * M, M * 5 * M * lg(M)
    if name in ("ifft_pt_kernel (x pass)", "ifft_pass_x_kernel"):
        return 8 * N * M + 4 * N * N, N * 5 * M * lg(M)
    if name == "fft_pt_fwd_kernel (x pass)":
        return 4 * N * N + 8 * N * M, N * 5 * M * lg(M)
    if name in ("fft_pt_fwd_cols_kernel", "fft_pt_fwd_kernel (y pass)"):
        return 8 * N * M + 8 * M * M, M * 5 * M * lg(M)
    if name == "adj_interp_tiled_kernel":
        return 8 * M * M + nt * (P // 2) * 8, 8 * W * W * nt * (P // 2)
    if name == "adj_rows_pt_kernel":
        return nt * (P // 2) * 8 + 4 * nt * nd, nt * (2.5 * P * lg(P) + 6 * P)
    # the paper's BST (Pb-point polar transforms of projection pairs, bilinear polar -> Cartesian
    # interpolation of complex values) and its windowed semi-polar rows
    Pb = c.get("Pb", 0)
    if name == "bst_window_rows_kernel":
        npr = 2 * (nd // 2 + 1) - 1
        return nt * nd * esz + 4 * nt * npr, 2 * nt * npr
    if name == "bst_polar_kernel" and Pb:
        return nt * nd * c.get("bst_in_esz", esz) + nt * (Pb // 2) * 8, (nt / 2) * 5 * Pb * lg(Pb)
    if name == "bst_interp_kernel" and Pb:
        return nt * (Pb // 2) * 8 + 8 * M * M, 16 * M * M
    # log-polar: rho transforms of n_phi rows of length L (two real rows per complex transform),
    # phi transforms of the L columns (forward, kernel product, inverse), Cartesian interpolation
    nphi, Llp, nout = c.get("lp_nphi", 0), c.get("lp_L", 0), c.get("lp_nout", 0)
    if nphi:
        if name == "lp_rows_fwd_kernel":
            return nt * nd * esz + 8 * nphi * Llp, (nphi / 2) * 5 * Llp * lg(Llp)
        if name == "lp_cols_kernel":
            return 3 * 8 * nphi * Llp, Llp * (10 * nphi * lg(nphi) + 6 * nphi)
        if name == "lp_rows_inv_kernel":
            return 8 * nphi * Llp + 4 * nphi * nout, (nphi / 2) * 5 * Llp * lg(Llp)
        if name == "lp_cart_kernel":
            return 20 * N * N + 4 * nphi * nout, 10 * N * N
    Q = c.get("lpp_Q", 0)
    if Q:
        K, Lr, Lp, na, no = c["lpp_K"], c["lpp_Lr"], c["lpp_Lp"], c["lpp_naout"], c["lpp_nout"]
        if name == "lpp_rows_fwd_kernel":
            return nt * nd * esz + Q * 8 * K * Lr, Q * (K / 2) * 5 * Lr * lg(Lr)
        if name == "lpp_cols_kernel":
            return Q * 8 * Lr * (K + Lp + na), Q * Lr * (10 * Lp * lg(Lp) + 6 * Lp)
        if name == "lpp_rows_inv_kernel":
            return Q * (8 * na * Lr + 4 * na * no), Q * (na / 2) * 5 * Lr * lg(Lr)
        if name == "lpp_cart_kernel":
            return Q * 24 * N * N, Q * 10 * N * N
    return None


def kernel_rooflines(times: dict, ctx: dict, hbm_gbs: float, fp32_tflops: float) -> dict:
    """Per kernel of one call: its time (CUDA events on the launching stream, averaged over the
    profiled calls), launches, algorithmic bytes and flops, and the fraction of the slower of the
    HBM and FP32 bounds it reaches.  The two gridding kernels are reported together."""
    times = dict(times)
    gp = [k for k in ("grid_gather_pair_kernel", "grid_gather_core_kernel") if k in times]
    if gp:
        times["gridding"] = {"ms": sum(times[k]["ms"] for k in gp),
                             "launches_per_call": sum(times[k]["launches_per_call"] for k in gp),
                             "kernels": gp}
        for k in gp:
            times.pop(k)
    out = {}
    for name, t in times.items():
        row = dict(t)
        w = kernel_work(name, ctx)
        if w is not None and t["ms"] > 0:
            b, f = w
            if not name.startswith("memset"):  # per-slice models; memset_bytes covers the whole call
                b, f = b * ctx.get("batch", 1), f * ctx.get("batch", 1)
            t_hbm = b / (hbm_gbs * 1e9)
            t_alu = f / (fp32_tflops * 1e12)
            sec = t["ms"] / 1e3
            bound = "hbm" if t_hbm >= t_alu else "alu"
            row.update({"bytes": b, "flops": f, "bound": bound,
                        "achieved": (b / sec / 1e9) if bound == "hbm" else (f / sec / 1e12),
                        "peak": hbm_gbs if bound == "hbm" else fp32_tflops,
                        "unit": "GB/s" if bound == "hbm" else "TFLOP/s",
                        "frac": max(t_hbm, t_alu) / sec})
            rec = None if name.startswith("bp_direct") or ctx.get("batch", 1) != 1 else \
                _traffic_record(name, None, ctx.get("workload"))
            if rec and all(ctx.get(k) == v for k, v in rec.get("match", {}).items()):  # ncu dram__bytes_read.sum + dram__bytes_write.sum of the same kernel(s), per call
                row["traffic"] = rec["dram_bytes_per_call"]
                row["traffic_over_algorithmic"] = rec["dram_bytes_per_call"] / b
        out[name] = row
    return out


def kernel_profile(plan, fn, flush, reps=3):
    """Per-kernel CUDA-event times of `fn` (calls on `plan`) from the library's stage timer: the
    average per call over `reps` calls, the L2 flushed before each."""
    import torch
    plan.stage_timing(True)
    plan.stage_times()
    for _ in range(reps):
        flush.zero_()
        fn()
    torch.cuda.synchronize()
    t = plan.stage_times()
    plan.stage_timing(False)
    return {k: {"ms": ms / reps, "launches_per_call": n / reps} for k, (ms, n) in t.items()}


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


def other_paths(plan, q, img, flush, stream, dev, only=(), peaks=(6778.3, 80.5), checks=None):
    """Every other row of the path on its own workload, each timed with CUDA events; per kernel its
    own event time and roofline fraction; for each, a check against the FP64 oracle is queued in
    `checks` (name -> callable returning (rel_l2, what)), run later in the CPU-baseline leg."""
    import numpy as np
    import torch

    from paper_1608_03589_gb300 import autograd as ag
    from paper_1608_03589_gb300 import bp, synth

    wl = synth.LARGE
    hbm, fp32 = peaks
    out = {}
    checks = {} if checks is None else checks
    ctx = {"N": wl.N, "n_det": wl.n_det, "n_theta": wl.n_theta, "esz": 4, "P": 4096, "M": 4096, "W": 6,
           "theta": wl.theta, "dt": wl.det_spacing, "workload": wl.name}
    qh = q.double().cpu().numpy()  # the exact float32 values the kernels read, as FP64
    rng = np.random.default_rng(11)
    pix2048 = rng.choice(wl.N * wl.N, 120, replace=False)

    def pick(t, idx):
        return t.reshape(-1)[torch.from_numpy(np.asarray(idx)).to(t.device)].double().cpu().numpy()

    def rel(a, b):
        a, b = np.asarray(a, np.float64).ravel(), np.asarray(b, np.float64).ravel()
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

    def guard(name, fn):
        if only and name not in only:
            return
        try:
            out[name] = fn()
        except Exception as exc:  # reported, never hidden
            out[name] = {"unavailable": f"{type(exc).__name__}: {str(exc)[:160]}"}
        torch.cuda.empty_cache()

    def prof(p, fn, c=ctx, reps=3):
        return kernel_rooflines(kernel_profile(p, fn, flush, reps), c, hbm, fp32)

    # 2048^2 x 1800 slice: Fourier R*, R (direct and Fourier adjoint), BF16 storage
    def fourier():
        ms = _timed(lambda: plan.backproject_fourier(q, out=img), stream, flush, 10)
        kern = prof(plan, lambda: plan.backproject_fourier(q, out=img))
        got6 = pick(img, pix2048)
        plan.set_fourier_width(4)
        ms4 = _timed(lambda: plan.backproject_fourier(q, out=img), stream, flush, 10)
        kern4 = prof(plan, lambda: plan.backproject_fourier(q, out=img), dict(ctx, W=4))
        got4 = pick(img, pix2048)
        plan.set_fourier_width(6)

        def chk():
            import oracle
            ref = oracle.bp_trig_points(qh, wl.N, wl.theta, wl.det_spacing, pix2048)
            return ({"width6": rel(got6, ref), "width4": rel(got4, ref)},
                    f"band-limited oracle (bp_trig_points) at {len(pix2048)} random pixels")
        checks["fourier_backprojection_2048"] = chk
        return {"ms": ms, "equiv_Gupdates_s": wl.updates / ms / 1e6, "kernel_width": 6, "kernels": kern,
                "width4_ms": ms4, "width4_equiv_Gupdates_s": wl.updates / ms4 / 1e6, "width4_kernels": kern4}
    guard("fourier_backprojection_2048", fourier)

    def fbp_fourier():
        tmp = torch.empty_like(q)
        fused = _timed(lambda: plan.fbp_fourier(q, "shepp-logan", out=img), stream, flush, 10)
        kern = prof(plan, lambda: plan.fbp_fourier(q, "shepp-logan", out=img))
        got = pick(img, pix2048)
        two = _timed(lambda: (plan.filter(q, "shepp-logan", out=tmp), plan.backproject_fourier(tmp, out=img)),
                     stream, flush, 10)

        def chk():
            import oracle
            qf = oracle.filter_rows(qh, wl.det_spacing, oracle.SHEPP_LOGAN)
            return rel(got, oracle.bp_trig_points(qf, wl.N, wl.theta, wl.det_spacing, pix2048)), \
                "oracle Shepp-Logan filter + band-limited R* at %d random pixels" % len(pix2048)
        checks["fbp_fourier_fused_2048"] = chk
        return {"fused_ms": fused, "filter_then_fourier_ms": two, "equiv_Gupdates_s": wl.updates / fused / 1e6,
                "kernels": kern}
    guard("fbp_fourier_fused_2048", fbp_fourier)

    def bst():
        res, imgs = {}, {}
        for os_ in (1, 4):
            ms = _timed(lambda: plan.backproject_bst(q, os_, out=img), stream, flush, 10)
            kern = prof(plan, lambda: plan.backproject_bst(q, os_, out=img), dict(ctx, Pb=4096 * os_))
            imgs[os_] = img.double().cpu().numpy()
            res[f"oversampling_{os_}"] = {"ms": ms, "equiv_Gupdates_s": wl.updates / ms / 1e6, "kernels": kern}

        def chk():
            import oracle
            return ({f"oversampling_{o}": rel(imgs[o], oracle.bp_bst_interp(qh, wl.N, wl.theta, wl.det_spacing,
                                                                             P=oracle.fourier_pad(wl.n_det) * o))
                     for o in (1, 4)}, "the oracle of the paper's BST algorithm (bp_bst_interp), whole image")
        checks["bst_interpolation_2048"] = chk
        return res
    guard("bst_interpolation_2048", bst)

    def bst_windowed():
        res, imgs = {}, {}
        for os_ in (1, 4):
            ms = _timed(lambda: plan.backproject_bst_windowed(q, 6.0, os_, out=img), stream, flush, 10)
            kern = prof(plan, lambda: plan.backproject_bst_windowed(q, 6.0, os_, out=img),
                        dict(ctx, Pb=4096 * os_, bst_in_esz=4))
            imgs[os_] = img.double().cpu().numpy()
            res[f"oversampling_{os_}"] = {"ms": ms, "equiv_Gupdates_s": wl.updates / ms / 1e6, "beta": 6.0,
                                          "kernels": kern}

        def chk():
            import oracle
            return ({f"oversampling_{o}": rel(imgs[o], oracle.bp_bst_semipolar(qh, wl.N, wl.theta, wl.det_spacing,
                                                                                6.0, P=oracle.fourier_pad(wl.n_det) * o))
                     for o in (1, 4)}, "the oracle of the windowed semi-polar BST (bp_bst_semipolar), whole image")
        checks["bst_windowed_2048"] = chk
        return res
    guard("bst_windowed_2048", bst_windowed)

    def logpolar():
        ms = _timed(lambda: plan.backproject_logpolar(q, out=img), stream, flush, 5)
        kern = prof(plan, lambda: plan.backproject_logpolar(q, out=img),
                    dict(ctx, **lp_meshes(wl.N, wl.n_det, wl.n_theta, wl.det_spacing)))
        got = img.double().cpu().numpy()

        def chk():
            import oracle
            return rel(got, oracle.bp_logpolar(qh, wl.N, wl.theta, wl.det_spacing)), \
                "the oracle of Andersson's log-polar method (bp_logpolar), whole image"
        checks["logpolar_2048"] = chk
        return {"ms": ms, "equiv_Gupdates_s": wl.updates / ms / 1e6, "kernels": kern}
    guard("logpolar_2048", logpolar)

    def logpolar_partial():
        plan.backproject_logpolar_partial(q, 8, 0.25, out=img)  # workspace and pixel tables (untimed)
        ms = _timed(lambda: plan.backproject_logpolar_partial(q, 8, 0.25, out=img), stream, flush, 5)
        kern = prof(plan, lambda: plan.backproject_logpolar_partial(q, 8, 0.25, out=img),
                    dict(ctx, **lpp_meshes(wl.N, wl.n_det, wl.n_theta, wl.det_spacing, 8, 0.25)))
        got = img.double().cpu().numpy()

        def chk():
            import oracle
            return rel(got, oracle.bp_logpolar_partial(qh, wl.N, wl.theta, wl.det_spacing, Q=8, a_r=0.25)), \
                "the oracle of the partial (sector) log-polar method, whole image"
        checks["logpolar_partial_2048"] = chk
        return {"ms": ms, "equiv_Gupdates_s": wl.updates / ms / 1e6, "sectors": 8, "a_r": 0.25, "kernels": kern}
    guard("logpolar_partial_2048", logpolar_partial)

    # the image R and R_F act on: the direct R* of the workload (as a realistic input)
    plan.backproject(q, out=img)
    f_img = img.clone()
    fh = f_img.double().cpu().numpy()
    sino = torch.empty_like(q)

    def radon():
        shape, _ = plan.autotune("radon", batch=1)
        ms = _timed(lambda: plan.radon(f_img, out=sino), stream, flush, 5)
        kern = prof(plan, lambda: plan.radon(f_img, out=sino))
        ks = np.sort(rng.choice(wl.n_theta, 6, replace=False))
        got = sino[torch.from_numpy(ks).to(dev)].double().cpu().numpy()

        def chk():
            import oracle
            return rel(got, oracle.radon(fh, wl.n_det, wl.theta[ks], wl.det_spacing)), \
                f"oracle R on {len(ks)} random angles (all bins)"
        checks["radon_direct_2048"] = chk
        return {"ms": ms, "Gupdates_s": wl.updates / ms / 1e6, "launch_shape": {"angles_per_cta": shape[0],
                                                                               "bands": shape[1]}, "kernels": kern}
    guard("radon_direct_2048", radon)

    def radon_f():
        ms = _timed(lambda: plan.radon(f_img, out=sino, fourier=True), stream, flush, 10)
        kern = prof(plan, lambda: plan.radon(f_img, out=sino, fourier=True))
        kj = np.array([k * wl.n_det + j for k in rng.choice(wl.n_theta, 4, replace=False)
                       for j in rng.integers(wl.n_det // 4, 3 * wl.n_det // 4, 4)])
        got = pick(sino, kj)

        def chk():
            import oracle
            return rel(got, oracle.radon_trig_points(fh, wl.n_det, wl.theta, wl.det_spacing, kj)), \
                f"oracle of the Fourier-path transpose at {len(kj)} sinogram entries"
        checks["radon_fourier_2048"] = chk
        return {"ms": ms, "equiv_Gupdates_s": wl.updates / ms / 1e6, "kernels": kern}
    guard("radon_fourier_2048", radon_f)

    def bf16():
        q16 = q.to(torch.bfloat16)
        shape, _ = plan.autotune("direct", torch.bfloat16, 1)
        ms = _timed(lambda: plan.backproject(q16, out=img), stream, flush, 10)
        kern = prof(plan, lambda: plan.backproject(q16, out=img), dict(ctx, esz=2, workload=None))
        got = pick(img, pix2048)
        q16h = q16.double().cpu().numpy()

        def chk():
            import oracle
            return rel(got, oracle.bp_linear_points(q16h, wl.N, wl.theta, wl.det_spacing, pix2048)), \
                f"oracle R* on the BF16-rounded sinogram at {len(pix2048)} random pixels"
        checks["direct_bf16_storage_2048"] = chk
        return {"ms": ms, "Gupdates_s": wl.updates / ms / 1e6, "launch_shape": {"stage": shape[0],
                                                                               "angle_groups": shape[1]},
                "kernels": kern}
    guard("direct_bf16_storage_2048", bf16)

    # 256^2 slice, 256 bins, 180 angles: default launch shape vs autotuned
    def small():
        S = synth.SMALL
        ps = bp.Plan(S.N, S.n_det, S.theta, S.det_spacing)
        gs = torch.from_numpy(S.sinogram().astype(np.float32)).to(dev)
        qs = ps.filter(gs, "ramlak")
        ims = torch.empty((S.N, S.N), dtype=torch.float32, device=dev)
        res = {}
        used = ps.get_shape("direct", torch.float32, 1)
        ms = _timed(lambda: ps.backproject(qs, out=ims), stream, flush, 20)
        res["default"] = {"ms": ms, "Gupdates_s": S.updates / ms / 1e6, "launch_shape": list(used)}
        shape, _ = ps.autotune("direct", torch.float32, 1)
        ms = _timed(lambda: ps.backproject(qs, out=ims), stream, flush, 20)
        sctx = {"N": S.N, "n_det": S.n_det, "n_theta": S.n_theta, "theta": S.theta, "dt": S.det_spacing}
        res["autotuned"] = {"ms": ms, "Gupdates_s": S.updates / ms / 1e6, "launch_shape": list(shape),
                            "kernels": prof(ps, lambda: ps.backproject(qs, out=ims), sctx)}
        got = ims.double().cpu().numpy()
        qsh = qs.double().cpu().numpy()
        ps.close()

        def chk():
            import oracle
            return rel(got, oracle.bp_linear(qsh, S.N, S.theta, S.det_spacing)), "oracle R*, whole image"
        checks["slice256_bins256_ang180_shapes"] = chk
        return res
    guard("slice256_bins256_ang180_shapes", small)

    # volume: 256 slices of 2048^2 from BF16 sinograms; the fused filtered backprojection (one
    # launch filters all slices into their row tables, one persistent launch backprojects them)
    # captured in a CUDA graph, the R* launch shape tuned at batch 256
    def volume():
        V = synth.VOLUME
        n = synth.VOLUME_SLICES
        raw = torch.empty((n, V.n_theta, V.n_det), dtype=torch.bfloat16, device=dev)
        for i in range(n):
            e = synth.random_ellipses(V.n_ellipses, V.seed + i)
            raw[i] = synth.ellipse_sinogram_torch(e, V.theta, V.n_det, V.det_spacing, dev).to(torch.bfloat16)
        pv = bp.Plan(V.N, V.n_det, V.theta, V.det_spacing)
        filt = torch.empty((n, V.n_theta, V.n_det), dtype=torch.float32, device=dev)
        imgs = torch.empty((n, V.N, V.N), dtype=torch.float32, device=dev)
        shape, _ = pv.autotune("direct", torch.float32, n)

        def step():
            pv.fbp_direct(raw, "shepp-logan", out=imgs)
        step()
        kern = kernel_rooflines(kernel_profile(pv, step, flush, 1), dict(ctx, esz=2, memset_bytes=4 * n * V.N * V.N,
                                                                           batch=n), hbm, fp32)
        s2 = torch.cuda.Stream(dev)
        s2.wait_stream(torch.cuda.current_stream(dev))
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s2):
            step()
        ms = _timed(graph.replay, stream, flush, 3)
        sl = [0, n - 1]
        got = {i: pick(imgs[i], pix2048) for i in sl}
        pv.filter(raw, "shepp-logan", out=filt)  # the fused call's filtered values (n_theta even), for the check
        fh = {i: filt[i].double().cpu().numpy() for i in sl}
        rawh = {i: raw[i].double().cpu().numpy() for i in sl}
        launches = sum(v["launches_per_call"] for v in kern.values())
        pv.close()
        del raw, filt, imgs

        def chk():
            import oracle
            e_bp = max(rel(got[i], oracle.bp_linear_points(fh[i], V.N, V.theta, V.det_spacing, pix2048)) for i in sl)
            e_f = max(rel(fh[i], oracle.filter_rows(rawh[i], V.det_spacing, oracle.SHEPP_LOGAN)) for i in sl)
            return {"direct": e_bp, "filter": e_f}, (f"slices {sl}: oracle R* at {len(pix2048)} random pixels on the "
                                                     "filtered sinogram the device made; oracle filter on the BF16 "
                                                     "input, all rows")
        checks["volume256_bf16_graph"] = chk
        return {"slices": n, "ms": ms, "Gupdates_s": n * V.updates / ms / 1e6, "storage": "bf16",
                "step": "bp_fbp_direct in one CUDA graph: one launch filters all slices into the four-image "
                        "form's row tables (and clears the images), one persistent launch backprojects all slices",
                "launch_shape": {"stage": shape[0], "angle_groups": shape[1], "tuned_at_batch": n},
                "launches_per_replay": launches, "kernels": kern}
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
                "Gupdates_s": 2 * 50 * B * N * N * nt / ms / 1e6,
                "err_vs_fp64": {"not_measured": "iterative; its operators are checked against the oracle by the tests"}}
    guard("tv_reconstruction_8x1024", tv)

    # uneven batch: 64 slices, widths in {512..4096}, 360-3000 angles, FP16: one launch writes every
    # slice's row tables, one persistent four-image launch backprojects all slices
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
        kern = kernel_profile(plans[0], lambda: bp.backproject_batched(plans, sinos, imgs2), flush, 1)
        for name, t in kern.items():  # the whole batch's algorithmic work (7 flops per update)
            if name.startswith("bp_direct") and t["ms"] > 0:
                t.update({"flops": 7 * upd, "bound": "alu", "achieved": 7 * upd / (t["ms"] / 1e3) / 1e12,
                          "peak": fp32, "unit": "TFLOP/s", "frac": 7 * upd / (fp32 * 1e12) / (t["ms"] / 1e3)})
        sel = [0, int(np.argmax([g[0] for g in geo]))]
        chk_data = []
        for i in sel:
            N, nd, nt = geo[i]
            px = rng.choice(N * N, 100, replace=False)
            chk_data.append((N, nd, synth.uniform_theta(nt), sinos[i].double().cpu().numpy(), px, pick(imgs2[i], px)))
        for pi in plans:
            pi.close()

        def chk():
            import oracle
            return max(rel(got, oracle.bp_linear_points(sh, N, th, 2.0 / nd, px)) for N, nd, th, sh, px, got in chk_data), \
                f"slices {sel}: oracle R* on the FP16-rounded sinograms at 100 random pixels each"
        checks["mixed64_fp16_persistent"] = chk
        return {"slices": len(geo), "updates": upd, "ms": ms, "Gupdates_s": upd / ms / 1e6, "storage": "fp16",
                "launch": "bp_backproject_batched: one launch writes every slice's four-image row tables (and clears "
                          "the images), one persistent launch backprojects all slices", "kernels": kern}
    guard("mixed64_fp16_persistent", mixed)

    # single 8192^2 slice, 8192 bins, 6000 angles: direct and Fourier
    def big():
        H = synth.HIRES
        pb = bp.Plan(H.N, H.n_det, H.theta, H.det_spacing)
        g = synth.ellipse_sinogram_torch(synth.random_ellipses(H.n_ellipses, H.seed), H.theta, H.n_det, H.det_spacing,
                                         dev).float()
        qb = pb.filter(g, "shepp-logan")
        del g
        ib = torch.empty((H.N, H.N), dtype=torch.float32, device=dev)
        pb.autotune("direct", torch.float32, 1)
        hctx = {"N": H.N, "n_det": H.n_det, "n_theta": H.n_theta, "esz": 4, "P": 16384, "M": 16384, "W": 6,
                "theta": H.theta, "dt": H.det_spacing}
        msd = _timed(lambda: pb.backproject(qb, out=ib), stream, flush, 2)
        kd = kernel_rooflines(kernel_profile(pb, lambda: pb.backproject(qb, out=ib), flush, 1), hctx, hbm, fp32)
        pxd = rng.choice(H.N * H.N, 150, replace=False)
        gotd = pick(ib, pxd)
        msf = _timed(lambda: pb.backproject_fourier(qb, out=ib), stream, flush, 2)
        kf = kernel_rooflines(kernel_profile(pb, lambda: pb.backproject_fourier(qb, out=ib), flush, 1), hctx, hbm, fp32)
        pxf = rng.choice(H.N * H.N, 24, replace=False)
        gotf = pick(ib, pxf)
        qbh = qb.double().cpu().numpy()
        pb.close()

        def chk():
            import oracle
            return ({"direct": rel(gotd, oracle.bp_linear_points(qbh, H.N, H.theta, H.det_spacing, pxd)),
                     "fourier": rel(gotf, oracle.bp_trig_points(qbh, H.N, H.theta, H.det_spacing, pxf))},
                    f"oracle R* at {len(pxd)} and band-limited oracle at {len(pxf)} random pixels")
        checks["slice8192_bins8192_ang6000"] = chk
        return {"direct_ms": msd, "direct_Gupdates_s": H.updates / msd / 1e6, "direct_kernels": kd,
                "fourier_ms": msf, "fourier_equiv_Gupdates_s": H.updates / msf / 1e6, "fourier_kernels": kf}
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
        plan.fbp_direct(g, "shepp-logan", out=img)

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
    plan.filter(g, "shepp-logan", out=q)  # the filtered sinogram, input of the other paths (untimed)
    torch.cuda.synchronize()
    if args.only:
        only = tuple(x for x in args.only.split(",") if x)
        res = other_paths(plan, q, img, flush, stream, dev, only)
        if rank == 0:
            print(json.dumps({"only": list(only), "paths": res}), flush=True)
        plan.close()
        return

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    sampler = ClockSampler(_gpu_id_for_smi(local))
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.zero_()  # L2 flush outside the timed interval
        e0, e1 = ev[i]
        e0.record(stream)
        plan.fbp_direct(g, "shepp-logan", out=img)
        e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    img_step = img.double().cpu().numpy()  # the last timed step's image (checked against the oracle below)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    total_ms = max_over_ranks(total_ms, dist, dev)

    if args.no_extras:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        if rank == 0:
            print(json.dumps({"value": throughput(wl.updates, world, args.steps, total_ms),
                              "unit": "Gupdates/s", "step_ms": statistics.mean(step_ms), "partial": True}))
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
    # three timed calls; the median call is reported (all three are in the line)
    e2e_calls = []
    for _ in range(3):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plan.fbp_host(g_pin, "shepp-logan", out=img_pin)
        e2e_calls.append(time.perf_counter() - t0)
    e2e_t = max_over_ranks(statistics.median(e2e_calls), dist, dev)

    props = torch.cuda.get_device_properties(dev)
    peaks = _peaks()
    sm_max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    hbm_gbs = float(peaks.get("hbm_gbs", 6778.3))
    peak_tflops, peak_basis = fp32_peak_tflops(props.multi_processor_count, sm_max_mhz)
    # per-kernel event times of the step (a separate pass after the timed region, from the library's
    # stage timer on the launching stream)
    ctx = {"N": wl.N, "n_det": wl.n_det, "n_theta": wl.n_theta, "esz": 4, "P": 4096, "M": 4096, "W": 6,
           "theta": wl.theta, "dt": wl.det_spacing, "workload": wl.name}
    step_kernels = kernel_rooflines(kernel_profile(plan, step, flush, max(3, min(args.steps, 10))), ctx, hbm_gbs,
                                    peak_tflops)
    launches_per_step = int(round(sum(v["launches_per_call"] for v in step_kernels.values())))
    # other operators and workloads of the path (reported under "paths", not part of the step)
    checks = {}
    extra = {} if args.no_paths else other_paths(plan, q, img, flush, stream, dev,
                                                 tuple(x for x in args.only.split(",") if x),
                                                 (hbm_gbs, peak_tflops), checks)
    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return

    # the dominant kernel of the step: its own event time and algorithmic flops
    dom = max(step_kernels, key=lambda k: step_kernels[k]["ms"])
    dk = step_kernels[dom]
    traffic = _traffic_record(dom, shape)
    line = {
        "metric": "backprojection G pixel·angle updates/s at 2048²×1800; % of roofline",
        "value": throughput(wl.updates, world, args.steps, total_ms),
        "unit": "Gupdates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": wl.name, "N": wl.N, "n_det": wl.n_det, "n_theta": wl.n_theta,
                   "phantom": "50 seeded random ellipses + 1% Gaussian noise", "filter": "shepp-logan",
                   "step": "bp_fbp_direct: one launch filters the rows into the four-image form's row tables "
                           "and clears the image, one launch runs the direct R* kernel",
                   "l2": "flushed (256 MiB write) between steps",
                   "launch_shape": {"stage": shape[0], "angle_groups": shape[1],
                                    "picked_by": picked},
                   "parallelism": f"independent slice per GPU x{world}"},
        "roofline": {"bound": dk.get("bound", "alu"), "kernel": dom, "achieved": dk.get("achieved"),
                     "peak": dk.get("peak"), "unit": dk.get("unit"), "frac": dk.get("frac"),
                     "flops_per_update": FLOPS_PER_UPDATE, "peak_basis": peak_basis, "hbm_peak_gbs": hbm_gbs,
                     "traffic": (traffic["dram_bytes_per_launch"] if traffic else None),
                     "algorithmic_bytes": dk.get("bytes"), "kernel_ms": dk["ms"],
                     "kernel_ms_basis": "CUDA events around the kernel on its stream (library stage timer), "
                                        "average over a pass after the timed region",
                     "step_ms_mean": statistics.mean(step_ms),
                     "step_kernels": step_kernels},
        "e2e": {"value": wl.updates * world * n_e2e / e2e_t / 1e9, "unit": "Gupdates/s",
                "h2d_bytes_per_step": g_host.nbytes, "d2h_bytes_per_step": wl.N * wl.N * 4,
                "call": "bp_fbp_host over %d pinned host slices per call (copies of neighbouring slices "
                        "overlap the kernels); the median of three timed calls" % n_e2e,
                "calls_ms": [round(x * 1e3, 3) for x in e2e_calls]},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "paths": extra,
    }
    if not args.no_cpu_baseline:
        try:
            line["cpu_baseline"], line["err_vs_fp64"] = cpu_baseline(img_step)
        except Exception as exc:  # pragma: no cover
            line["cpu_baseline"] = {"unavailable": str(exc)[:120]}
        # every other path against the FP64 oracle, outside every timed region
        for name, chk in checks.items():
            try:
                t0 = time.perf_counter()
                err, what = chk()
                extra[name]["err_vs_fp64"] = {"rel_l2": err, "against": what,
                                              "oracle_s": round(time.perf_counter() - t0, 1)}
            except Exception as exc:  # pragma: no cover
                extra[name]["err_vs_fp64"] = {"unavailable": f"{type(exc).__name__}: {str(exc)[:120]}"}
    else:
        line["err_vs_fp64"] = {"not_measured": "--no-cpu-baseline (the oracle runs only in that leg)"}
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
