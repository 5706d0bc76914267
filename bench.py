#!/usr/bin/env python
"""Benchmark: even-odd staggered CG on one GB300 (one JSON line on rank 0).

A step is one pass of the whole path on the 32^4 workload (links
exp(i 0.3 H), m = 0.01, one Gaussian even-site source): pack the canonical
FP64 links into the internal layout, round the FP32 copy, pack the source,
solve (m^2 - D_eo D_oe) x = b by mixed-precision CG (FP32 inner iteration on
two-row 16-bit fixed-point links, FP64 reliable updates) to a true relative
residual of 1e-10, and unpack the
solution.  ``value`` is solves per second over all ranks with inputs resident
in HBM; ``e2e`` is the same through ``qex_cg_host`` from page-locked host
buffers (copies inside the timed region).  Ranks are independent replicas
(the lattice is not split across GPUs).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Dslash GB/s & GFLOP/s vs HBM roofline; CG time to 1e-10 residual, mixed vs FP64"
WORKLOAD = "cfg32"
TOL = 1e-10
DELTA = 0.01           # reliable-update threshold (sweep on this workload: same iterations, fewest updates)
INNER = "f32r12h"      # inner CG precision: FP32 fields, two-row 16-bit fixed-point SU(3) links
FLOP_NN = 570          # flops per output site of the one-hop Dslash (8 mat-vecs x 66 + 7 x 6 adds)
# 8 links + 8 input vectors counted once + 1 output vector, per output site
BYTES_NN = {"f64": 1248, "f32": 624, "f32r12": 432, "f32r12h": 240, "f32s16": 368}
L2_BYTES = 135528448   # sm_103a L2 (cudaDevAttrL2CacheSize on GB300)
# FP64 FMA units per SM and clock on GB300: the nominal 1.25 TFLOP/s FP64 at 2070 MHz over 152 SMs
# (1.25e12 / (2 x 152 x 2.07e9) = 1.99)
FP64_FMA_PER_SM_CLK = 2
# kernels of one mixed-precision iteration (16-bit two-row links), in launch order, with their
# algorithmic bytes per even site: links 8 x 24 B; FP32 vectors 24 B each
ITER_KERNELS = (
    ("dslash_kernel<float, 16-bit two-row, one-hop, EPI_PUPD>: p = r + beta p_old, D_oe p, pending x += alpha p_old",
     "dslash_f32r12h_pupd_32^4", 336),   # links 192 + r, p_old, x in 72 + out, p_new, x out 72
    ("dslash_kernel<float, 16-bit two-row, one-hop, EPI_NORMAL>: A p = m^2 p - D_eo tmp, <p, A p>",
     "dslash_f32r12h_normal_32^4", 264),  # links 192 + tmp, p in 48 + A p out 24
    ("update_xr_kernel<float, no x>: r -= alpha A p, ||r||^2", "update_r_f32_32^4", 72),  # r, A p in + r out
)
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-step-seconds", type=float, default=3.0,
                    help="reference arm: oracle CPU time of one step (a bounded sample of the solve)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--sweep", action="store_true",
                    help="Dslash bandwidth sweep over L^3 x T volumes (and 48^4, 64^4), with and without the Naik "
                         "term, in every precision: one JSON line per case")
    ap.add_argument("--sweep-cg", action="store_true",
                    help="with --sweep: also the mixed-precision CG of the 64^4 Naik workload")
    ap.add_argument("--mrhs", action="store_true",
                    help="multi-RHS case: 24^4 Haar links, 16 Gaussian sources, batched Dslash and CG against "
                         "single-RHS calls")
    ap.add_argument("--batch", action="store_true",
                    help="multi-lattice case: 8 lattices 8^4 .. 32^4, Haar links, masses 0.005 * 20^(k/7), one "
                         "batched solve against sequential single-lattice solves")
    ap.add_argument("--profile-iteration", action="store_true",
                    help="profiling case: one mixed-precision solve of the workload, driven from the host (the "
                         "graph solve's kernels launched one by one), inside cudaProfilerStart/Stop")
    ap.add_argument("--dslash-only", action="store_true",
                    help="profiling case: two launches each of the 16-bit two-row, two-row FP32, FP32 and FP64 "
                         "one-hop Dslash on the workload, no timing")
    return ap.parse_args()


def workload_desc(wl):
    lx, ly, lz, lt = wl["dims"]
    return (f"{lx}x{ly}x{lz}x{lt} staggered, links exp(i {wl['a']} H) SU(3), m={wl['mass']}, "
            f"1 Gaussian even-site source, mixed-precision CG to true residual {TOL:g}")


# ------------------------------------------------------------------ distributed

class Dist:
    def __init__(self, want_gpu: bool):
        import torch

        self.rank = int(os.environ.get("RANK", 0))
        self.world = int(os.environ.get("WORLD_SIZE", 1))
        self.local = int(os.environ.get("LOCAL_RANK", 0))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist

            backend = "nccl" if (want_gpu and torch.cuda.is_available()) else "gloo"
            if backend == "nccl":
                torch.cuda.set_device(self.local)
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, v: float) -> float:
        if not self.pg:
            return v
        import torch

        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ----------------------------------------------------------------------- clocks

class Clocks:
    """nvidia-smi samples every 100 ms while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            if self.file is not None:
                self.file.close()
                os.unlink(self.file.name)
            return
        # the sampler's start-up (driver and NVML initialisation) must not overlap the timed region: a
        # host-path solve that ran alongside it took 72-118 ms instead of 23; wait for its first sample
        t0 = time.time()
        while time.time() - t0 < 3.0 and self.proc.poll() is None:
            if os.path.getsize(self.file.name) > 0:
                break
            time.sleep(0.02)

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) == 7:
                    rows.append(parts)
        os.unlink(self.file.name)
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        reasons = sorted({self.NAMES[k] for r in rows for k in range(4) if r[3 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# -------------------------------------------------------------------- helpers

def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash() -> str:
    """Hash of the Dslash kernel's device code: the shared headers and the
    kernel section of dslash.cu (host-side launch code excluded)."""
    h = hashlib.sha256()
    for rel in ("paper_1612_02750_gb300/csrc/qex_common.cuh", "paper_1612_02750_gb300/csrc/qex_dslash_site.cuh"):
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    with open(os.path.join(ROOT, "paper_1612_02750_gb300/csrc/dslash.cu"), "rb") as f:
        src = f.read()
    a, b = src.find(b"struct DsParams"), src.find(b"// Shape of a Dslash launch")
    h.update(src[a:b] if 0 <= a < b else src)
    return h.hexdigest()[:16]


def files_hash(rels) -> str:
    """Hash of whole source files (kernels outside dslash.cu)."""
    h = hashlib.sha256()
    for rel in rels:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel_key: str):
    """DRAM bytes per launch from the committed ncu summary, or None when the
    kernel source changed since the capture (the Dslash device code, or the
    files a record names in "hash_files")."""
    path = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)[kernel_key]
    except (OSError, KeyError, ValueError):
        return None
    want = files_hash(rec["hash_files"]) if "hash_files" in rec else kernel_source_hash()
    if rec.get("source_hash") != want:
        return None
    return rec.get("dram_bytes_per_launch")


def oracle_baseline(wl, u, b):
    """The oracle as it stands on the host cores: one full FP64 CG solve of the
    workload to the true residual tol (all cores), one normal-operator
    application on one thread (the cost of an iteration), and the 4^4 solve
    (Haar links, m = 0.1) in CPU-seconds on one thread."""
    import resource

    import fieldgen as fg
    import oracle

    oracle.build()
    cores = oracle.threads()
    dims, mass = wl["dims"], wl["mass"]
    t0 = time.perf_counter()
    _, ok, iters, tr = oracle.cg(dims, u, b, mass, tol=TOL, maxiter=50000)
    full_s = time.perf_counter() - t0
    def best3(fn):
        ts = []
        for _ in range(3):
            t0 = time.perf_counter()
            fn()
            ts.append(time.perf_counter() - t0)
        return min(ts)

    dslash_all_s = best3(lambda: oracle.dslash_parity(dims, u, b, 1))
    oracle.set_threads(1)
    try:
        dslash_one_s = best3(lambda: oracle.dslash_parity(dims, u, b, 1))
        t0 = time.perf_counter()
        oracle.normal_op(dims, u, b, mass)
        one_thread_op_s = time.perf_counter() - t0
        w0 = fg.workload("cfg4x4")
        u0, _, b0 = fg.make_inputs(w0["dims"], w0["fat"], False, w0["seed"])
        r0 = resource.getrusage(resource.RUSAGE_SELF)
        _, ok0, it0, tr0 = oracle.cg(w0["dims"], u0, b0, w0["mass"], tol=TOL, maxiter=10000)
        r1 = resource.getrusage(resource.RUSAGE_SELF)
    finally:
        oracle.set_threads(cores)
    cpu0 = (r1.ru_utime - r0.ru_utime) + (r1.ru_stime - r0.ru_stime)
    lat = "x".join(map(str, dims))
    return {"value": round(1.0 / full_s, 6), "unit": "solves/s", "cores": cores, "kind": "oracle",
            "sample": f"one full oracle FP64 CG solve of the {lat} workload to true residual {TOL:g} on {cores} "
                      f"threads ({iters} iterations, {full_s:.1f} s, converged={ok}, true residual {tr:.2e})",
            "seconds_per_solve": round(full_s, 2), "iters": iters, "true_rel_resid": tr,
            "seconds_per_iteration": round(full_s / (iters + 2), 4),
            "one_thread": {"normal_op_s": round(one_thread_op_s, 3),
                           "note": "one application of m^2 - D_eo D_oe on the full lattice, 1 thread"},
            "dslash_d_oe": {"all_cores_s": round(dslash_all_s, 4), "one_thread_s": round(dslash_one_s, 4),
                            "note": "oracle D_oe (full-lattice operator, output on odd sites), best of 3"},
            "cfg4x4": {"cpu_seconds": round(cpu0, 4), "iters": it0, "converged": ok0, "true_rel_resid": tr0,
                       "note": "4^4 Haar links, m = 0.1, FP64 CG to 1e-10 on 1 thread, getrusage user+system"}}


def oracle_check(wl, u, b, x_mixed, x_fp64):
    """The oracle's true residual of the benchmarked solutions and their
    difference."""
    import fieldgen as fg
    import oracle

    dims, mass = wl["dims"], wl["mass"]
    ev = fg.even_mask(dims)
    d = x_mixed[ev] - x_fp64[ev]
    return {"mixed_true_rel_resid": oracle.true_residual(dims, u, b, x_mixed, mass),
            "fp64_true_rel_resid": oracle.true_residual(dims, u, b, x_fp64, mass),
            "mixed_vs_fp64_rel_diff": float(np.linalg.norm(d) / np.linalg.norm(x_fp64[ev])),
            "mixed_vs_fp64_max_elem_diff": float(np.abs(d).max() / np.abs(x_fp64[ev]).max())}


def make_inputs(wl):
    import fieldgen as fg

    u, _, b = fg.make_inputs(wl["dims"], wl["fat"], False, wl["seed"], wl["a"])
    return u, b


# --------------------------------------------------------------------- native

def run_native(args):
    import torch

    import fieldgen as fg
    import paper_1612_02750_gb300 as q
    from paper_1612_02750_gb300 import build as qbuild

    dist = Dist(want_gpu=True)
    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA device (no CPU fallback)")
    torch.cuda.set_device(dist.local)
    qbuild.build()
    q.load()
    # the headline solve keeps every reliable update in FP64 (the scheme's true-residual recomputation);
    # the float-float updates are measured apart below
    os.environ.pop("QEX_RU_FF", None)
    wl = fg.workload(WORKLOAD)
    dims, mass = wl["dims"], wl["mass"]
    u, b = make_inputs(wl)
    lat = q.Lattice(dims, antiperiodic=True)
    vh = lat.half_volume

    U_h = torch.from_numpy(u).pin_memory()
    B_h = torch.from_numpy(b).pin_memory()
    X_h = torch.empty_like(B_h).pin_memory()
    U_d = U_h.cuda()
    B_d = B_h.cuda()
    X_d = torch.zeros_like(B_d)
    fat64 = q.empty_links(lat, "f64")
    fat32 = q.empty_links(lat, INNER)
    bh = q.empty_field(lat, "f64")
    x = q.empty_field(lat, "f64")
    stream = torch.cuda.current_stream()

    def step(inner=INNER):
        q.qex_pack_links_pair(lat, U_d, INNER, fat64, fat32)  # FP64 and 16-bit two-row sets, one pass
        q.qex_pack_field(lat, "f64", 0, B_d, bh)
        x.zero_()
        _, stats = q.qex_cg(lat, inner, fat64, None, fat32, None, 0.0, mass, bh, x, tol=TOL, maxiter=200000,
                            delta=DELTA)
        q.qex_unpack_field(lat, "f64", 0, x, X_d)
        return stats

    for _ in range(args.warmup):
        stats = step()
    clocks = Clocks(torch.cuda.current_device())
    dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    n0 = q.qex_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    all_stats = [step() for _ in range(args.steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    launches = q.qex_launch_count() - n0
    clk = clocks.stop()
    dist.barrier()
    ms = e0.elapsed_time(e1) / args.steps
    ms_max = dist.max(ms)
    value = dist.world * 1000.0 / ms_max
    mixed = all_stats[-1]
    x_mixed = X_d.cpu().numpy() if dist.rank == 0 else None

    # end to end from page-locked host buffers through qex_cg_host, right after the device-timed region
    # (same clocks; the FP64 and single-kernel timings below run afterwards)
    e2e = None
    if not args.no_e2e:
        # W untimed calls as for the device-timed steps (the first calls on the host path build its work
        # area and solve graph and load kernels: one of them took 87 ms instead of 24)
        for _ in range(max(1, args.warmup)):
            q.qex_cg_host(lat, INNER, U_h, None, 0.0, mass, B_h, X_h, tol=TOL, maxiter=200000, delta=DELTA)
        dist.barrier()
        torch.cuda.synchronize()
        clocks_e2e = Clocks(torch.cuda.current_device())
        clocks_e2e.start()
        solve_ms, call_ms = [], []
        t0 = time.perf_counter()
        for _ in range(args.steps):
            c0 = time.perf_counter()
            _, _, st_h = q.qex_cg_host(lat, INNER, U_h, None, 0.0, mass, B_h, X_h, tol=TOL, maxiter=200000,
                                       delta=DELTA)
            call_ms.append((time.perf_counter() - c0) * 1e3)
            solve_ms.append(st_h["time_ms"])
        torch.cuda.synchronize()
        e2e_s = dist.max((time.perf_counter() - t0) / args.steps)
        clk_e2e = clocks_e2e.stop()
        # the host link alone: the same bytes as one plain copy each, best of three
        link = []
        for _ in range(3):
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            U_d.copy_(U_h, non_blocking=True)
            B_d.copy_(B_h, non_blocking=True)
            c1.record(stream)
            torch.cuda.synchronize()
            link.append(c0.elapsed_time(c1))
        h2d_bytes = U_h.numel() * 16 + B_h.numel() * 16
        e2e = {"value": round(dist.world / e2e_s, 4), "unit": "solves/s",
               "h2d_bytes_per_step": h2d_bytes, "d2h_bytes_per_step": X_h.numel() * 16,
               "ms_per_step": round(e2e_s * 1e3, 3),
               "h2d_plain_copy_ms": round(min(link), 3),
               "h2d_plain_copy_gbs": round(h2d_bytes / (min(link) * 1e-3) / 1e9, 1),
               "solve_ms_median": round(statistics.median(solve_ms), 3),
               "call_ms_median": round(statistics.median(call_ms), 3), "call_ms_max": round(max(call_ms), 3),
               "clocks_sm_mhz": clk_e2e.get("sm_mhz"), "clock_reasons": clk_e2e.get("reasons")}

    # the same step with the optional float-float intermediate reliable updates (QEX_RU_FF=1), reported
    # apart from the headline: convergence is still judged on an FP64 true residual
    ff_rec = None
    if dist.rank == 0:
        os.environ["QEX_RU_FF"] = "1"
        try:
            step()
            torch.cuda.synchronize()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            ff_stats = [step() for _ in range(5)]
            f1.record(stream)
            torch.cuda.synchronize()
        finally:
            os.environ.pop("QEX_RU_FF", None)
        s_ff = ff_stats[-1]
        ff_rec = {"env": "QEX_RU_FF=1", "step_ms": round(f0.elapsed_time(f1) / 5, 3),
                  "solve_ms_median": round(statistics.median(s["time_ms"] for s in ff_stats), 3),
                  "iters": s_ff["iters"], "reliable_updates": s_ff["reliable_updates"],
                  "ff_updates": s_ff["ff_updates"], "true_rel_resid": s_ff["true_rel_resid"]}

    # FP64 CG on the same inputs (the "mixed vs FP64" half of the metric)
    torch.cuda.synchronize()
    f0 = time.perf_counter()
    st64 = step("f64")
    torch.cuda.synchronize()
    fp64_ms = (time.perf_counter() - f0) * 1e3
    x_fp64 = X_d.cpu().numpy() if dist.rank == 0 else None

    # the kernels of the mixed iteration, timed inside a solve (same order, shapes, buffers and L2 state
    # as the timed solve; events on the solve's stream between the kernels)
    x_prof = torch.zeros_like(bh)
    prof_ms = q.qex_cg_profile(lat, INNER, fat64, None, fat32, None, 0.0, mass, bh, x_prof, iters=100)
    peak, peak_kind = measured_peak()
    in_solve = []
    for (name, key, nbytes), ms_k in zip(ITER_KERNELS, prof_ms):
        ach = nbytes * vh / (ms_k * 1e-3) / 1e9
        in_solve.append({"kernel": name, "traffic_key": key, "bytes_per_site": nbytes, "avg_launch_ms": round(ms_k, 5),
                         "GB/s": round(ach, 1), "frac": round(ach / peak, 4)})
    dom = max(in_solve, key=lambda k: k["avg_launch_ms"])
    roofline = {"bound": "hbm", "kernel": dom["kernel"], "achieved": dom["GB/s"], "peak": peak, "unit": "GB/s",
                "frac": dom["frac"], "frac_of_nominal_8TBps": round(dom["GB/s"] / 8000.0, 4),
                "traffic": ncu_traffic(dom["traffic_key"]),
                "peak_source": f"{peak_kind} HBM copy bandwidth", "bytes_per_site": dom["bytes_per_site"],
                "sites_per_launch": vh, "avg_launch_ms": dom["avg_launch_ms"],
                "timing": "qex_cg_profile: 100 iterations of the solve's own kernels (first two dropped), CUDA "
                          "events between the kernels on the solve's stream",
                "iteration": in_solve,
                "iteration_ms": round(sum(prof_ms), 5),
                "iteration_frac": round(sum(k["bytes_per_site"] for k in in_solve) * vh / (sum(prof_ms) * 1e-3) / 1e9
                                        / peak, 4)}

    # the plain one-hop Dslash in every format, each launch timed alone after a read of twice the L2 size
    # (a read leaves no dirty lines for the kernel to write back)
    flush = torch.zeros(2 * L2_BYTES // 4, dtype=torch.float32, device="cuda")

    def time_dslash(prec, fat, reps=40):
        inp = q.empty_field(lat, prec).normal_()
        out = q.empty_field(lat, prec)
        for _ in range(5):
            q.qex_dslash(lat, prec, fat, None, 0.0, 1, inp, out)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
        for ea, ez in evs:
            torch.sum(flush)
            ea.record(stream)
            q.qex_dslash(lat, prec, fat, None, 0.0, 1, inp, out)
            ez.record(stream)
        torch.cuda.synchronize()
        return sum(ea.elapsed_time(ez) for ea, ez in evs) / reps

    full32 = q.qex_convert_links(lat, "f64", fat64, "f32")
    r12 = q.qex_convert_links(lat, "f64", fat64, "f32r12")
    times = {"f32r12h": time_dslash("f32r12h", fat32), "f32r12": time_dslash("f32r12", r12),
             "f32": time_dslash("f32", full32), "f64": time_dslash("f64", fat64)}
    del full32, r12, flush

    def gbs(prec):
        return BYTES_NN[prec] * vh / (times[prec] * 1e-3) / 1e9

    dslash = {p: {"ms": round(t, 5), "GB/s": round(gbs(p), 1), "frac": round(gbs(p) / peak, 4),
                  "GFLOP/s": round(FLOP_NN * vh / (t * 1e-3) / 1e9, 1)} for p, t in times.items()}
    rates = q.qex_fma_rates()
    f64_flops = 2 * 288 * vh / (times["f64"] * 1e-3) / 1e9  # 288 FP64 FMAs issued per site
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    mhz = clk.get("sm_mhz") or 2070.0
    f64_peak = sms * FP64_FMA_PER_SM_CLK * 2 * mhz * 1e6 / 1e9
    dslash["f64"]["bound"] = "alu"
    dslash["f64"]["alu"] = {"achieved_gflops": round(f64_flops, 1), "peak_gflops": round(f64_peak, 1),
                            "frac": round(f64_flops / f64_peak, 4), "unit": "GFLOP/s",
                            "peak_source": f"derived: {sms} SMs x {FP64_FMA_PER_SM_CLK} FP64 FMA per clock x 2 flops x "
                                           f"{mhz:.0f} MHz (median SM clock of the timed region)",
                            "fma_per_site": 288,
                            "probe_gflops": round(rates["fp64_gflops"], 1),
                            "probe": "qex_fma_rates: dependent FP64 FMA chains, best of five bursts; they plateau "
                                     "below what the Dslash sustains, so the derived peak is the ceiling"}
    dslash["fp32_fma_gflops"] = round(rates["fp32_gflops"], 1)
    dslash["timing"] = "D_oe alone, cold L2 (read of 2x L2 before each launch), 40 launches, CUDA events"
    dslash["traffic_f32r12h"] = ncu_traffic("dslash_f32r12h_nn_32^4")

    # CPU-baseline leg (rank 0 at N = 1): the oracle timed on the host cores, and the oracle's judgement
    # of the two benchmarked solutions
    cpu = checks = None
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        checks = oracle_check(wl, u, b, x_mixed, x_fp64)
        cpu = oracle_baseline(wl, u, b)

    if dist.rank == 0:
        mixed_rec = {"iters": mixed["iters"], "reliable_updates": mixed["reliable_updates"],
                     "ff_updates": mixed["ff_updates"], "true_rel_resid": mixed["true_rel_resid"],
                     "solve_ms": round(mixed["time_ms"], 3)}
        if ff_rec:
            mixed_rec["with_float_float_updates"] = ff_rec
        fp64_rec = {"iters": st64["iters"], "true_rel_resid": st64["true_rel_resid"],
                    "solve_ms": round(st64["time_ms"], 3), "step_ms": round(fp64_ms, 3)}
        if checks:
            mixed_rec["oracle_true_rel_resid"] = checks["mixed_true_rel_resid"]
            mixed_rec["rel_diff_vs_fp64_solution"] = checks["mixed_vs_fp64_rel_diff"]
            mixed_rec["max_elem_diff_vs_fp64_solution"] = checks["mixed_vs_fp64_max_elem_diff"]
            fp64_rec["oracle_true_rel_resid"] = checks["fp64_true_rel_resid"]
        line = {
            "metric": METRIC, "value": round(value, 4), "unit": "solves/s", "n_gpus": dist.world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": workload_desc(wl), "lattice": list(dims), "mass": mass, "tol": TOL,
                       "delta": DELTA, "parallelism": f"replicas{dist.world}",
                       "l2": f"inputs larger than L2: {fat32.numel() * 4 / 1e6:.0f} MB FP32 and "
                             f"{fat64.numel() * 8 / 1e6:.0f} MB FP64 links per step vs {L2_BYTES / 1e6:.0f} MB L2"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches), "clocks": clk,
            "mixed": mixed_rec, "fp64": fp64_rec, "dslash": dslash,
            "launch_shapes": {INNER: q.qex_tune_info(lat, INNER), "f64": q.qex_tune_info(lat, "f64")},
        }
        print(json.dumps(line), flush=True)
    lat.close()
    dist.close()


# ------------------------------------------------------------------ reference

def run_reference(args):
    """The oracle on the host cores (rank 0 only; the other ranks exit at
    once).  Each of the W + K steps is a bounded sample of the workload: a
    fixed number of oracle CG iterations on the full lattice (about
    --ref-step-seconds each), timed for ms_per_step; then one full solve to
    the true residual tol is timed, and value is one over its seconds."""
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if rank != 0:
        return
    import fieldgen as fg
    import oracle

    oracle.build()
    wl = fg.workload(WORKLOAD)
    dims, mass = wl["dims"], wl["mass"]
    u, b = make_inputs(wl)
    t0 = time.perf_counter()
    oracle.normal_op(dims, u, b, mass)
    t_op = time.perf_counter() - t0
    n = max(1, int(args.ref_step_seconds / max(t_op, 1e-6)) - 2)
    times = []
    for k in range(args.warmup + args.steps):
        s0 = time.perf_counter()
        oracle.cg(dims, u, b, mass, tol=TOL, maxiter=n)
        if k >= args.warmup:
            times.append(time.perf_counter() - s0)
    step_s = sum(times) / len(times)
    t0 = time.perf_counter()
    _, ok, iters, tr = oracle.cg(dims, u, b, mass, tol=TOL, maxiter=50000)
    full_s = time.perf_counter() - t0
    value = 1.0 / full_s
    lat = "x".join(map(str, dims))
    sample = (f"each step: {n} oracle FP64 CG iterations on the full {lat} lattice ({step_s:.2f} s); value: one full "
              f"oracle solve to true residual {TOL:g} timed after the steps ({iters} iterations, {full_s:.1f} s, "
              f"converged={ok}, true residual {tr:.2e})")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(step_s * 1e3, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(wl).replace("mixed-precision", "FP64"), "lattice": list(dims),
                   "mass": mass, "tol": TOL, "parallelism": "host cores"},
        "cpu_baseline": {"kind": "oracle", "cores": oracle.threads(), "sample": sample, "value": round(value, 6),
                         "unit": "solves/s", "seconds_per_solve": round(full_s, 2),
                         "seconds_per_iteration": round(step_s / (n + 2), 4)},
        "e2e": {"value": round(value, 6), "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_profile_iteration():
    """One warm solve (tuning, graph), then one host-driven solve of the same
    kernels between cudaProfilerStart and cudaProfilerStop, for
    ``ncu --profile-from-start off``."""
    import torch

    import fieldgen as fg
    import paper_1612_02750_gb300 as q
    from paper_1612_02750_gb300 import build as qbuild

    qbuild.build()
    wl = fg.workload(WORKLOAD)
    u, b = make_inputs(wl)
    lat = q.Lattice(wl["dims"], antiperiodic=True)
    fat64 = q.qex_pack_links(lat, "f64", torch.from_numpy(u).cuda())
    fat16 = q.qex_convert_links(lat, "f64", fat64, INNER)
    bh = q.qex_pack_field(lat, "f64", 0, torch.from_numpy(b).cuda())
    x = torch.zeros_like(bh)
    q.qex_cg(lat, INNER, fat64, None, fat16, None, 0.0, wl["mass"], bh, x, tol=TOL, maxiter=200000, delta=DELTA)
    os.environ["QEX_CG_MODE"] = "host"
    x.zero_()
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStart()
    _, st = q.qex_cg(lat, INNER, fat64, None, fat16, None, 0.0, wl["mass"], bh, x, tol=TOL, maxiter=200000,
                     delta=DELTA)
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStop()
    print("profile-iteration done", json.dumps(st))


def run_dslash_only():
    import torch

    import fieldgen as fg
    import paper_1612_02750_gb300 as q
    from paper_1612_02750_gb300 import build as qbuild

    qbuild.build()
    wl = fg.workload(WORKLOAD)
    u, b = make_inputs(wl)
    lat = q.Lattice(wl["dims"], antiperiodic=True)
    fat64 = q.qex_pack_links(lat, "f64", torch.from_numpy(u).cuda())
    fat32 = q.qex_convert_links(lat, "f64", fat64, "f32")
    fatr12 = q.qex_convert_links(lat, "f64", fat64, "f32r12")
    fatr12h = q.qex_convert_links(lat, "f64", fat64, "f32r12h")
    src = torch.from_numpy(b).cuda()
    for prec, fat in (("f32r12h", fatr12h), ("f32r12", fatr12), ("f32", fat32), ("f64", fat64)):
        inp = q.qex_pack_field(lat, prec, 0, src)
        for _ in range(2):
            out = q.qex_dslash(lat, prec, fat, None, 0.0, 1, inp)
    torch.cuda.synchronize()
    print("dslash-only done", float(out.abs().sum()))


SWEEP_L = (8, 12, 16, 24, 32)
SWEEP_T = (8, 12, 16, 24, 32, 48, 64)
# 8 fat + 8 long links + the input vector once + 1 out; 16-bit formats read 40-byte long links
BYTES_NAIK = {"f64": 2400, "f32": 1200, "f32r12": 1008, "f32r12h": 560, "f32s16": 688}
FLOP_NAIK = 1146


def run_sweep(args):
    """Dslash timing over the paper's L^3 x T volume grid plus 48^4 and 64^4.
    Links and fields are random device tensors (timing only; parity is tested
    elsewhere); each case is 5 warm-up launches, then 3 replays of a CUDA
    graph of 30 launches (device time per launch)."""
    import torch

    import paper_1612_02750_gb300 as q
    from paper_1612_02750_gb300 import build as qbuild

    qbuild.build()
    q.load()
    peak, peak_kind = measured_peak()
    shapes = [(L, L, L, T) for L in SWEEP_L for T in SWEEP_T] + [(48, 48, 48, 48), (64, 64, 64, 64)]
    gen = torch.Generator(device="cuda").manual_seed(7)
    for dims in shapes:
        lat = q.Lattice(dims)
        vh = lat.half_volume
        fat64 = torch.randn(q.qex_links_bytes(lat, "f64") // 8, dtype=torch.float64, device="cuda", generator=gen)
        lng64 = torch.randn_like(fat64)
        sets = {"f64": (fat64, lng64), "f32": (fat64.float(), lng64.float())}
        lng16 = q.qex_convert_links(lat, "f64", lng64, "f32s16")
        sets["f32r12"] = (q.qex_convert_links(lat, "f64", fat64, "f32r12"), sets["f32"][1])
        sets["f32r12h"] = (q.qex_convert_links(lat, "f64", fat64, "f32r12h"), lng16)
        sets["f32s16"] = (q.qex_convert_links(lat, "f64", fat64, "f32s16"), lng16)
        for prec, (fat, lng) in sets.items():
            inp = q.empty_field(lat, prec).normal_(generator=gen)
            out = q.empty_field(lat, prec)
            for naik in (False, True):
                lg = lng if naik else None
                for _ in range(5):  # warm-up (and the launch-shape tuning of this case)
                    q.qex_dslash(lat, prec, fat, lg, -1.0 / 24, 1, inp, out)
                torch.cuda.synchronize()
                # 30 launches captured in one CUDA graph, so that small (L2-resident) volumes are timed
                # by the device, not by the host's launch rate
                graph, side = torch.cuda.CUDAGraph(), torch.cuda.Stream()
                with torch.cuda.stream(side):
                    with torch.cuda.graph(graph, stream=side):
                        for _ in range(30):
                            q.qex_dslash(lat, prec, fat, lg, -1.0 / 24, 1, inp, out, stream=side)
                graph.replay()
                a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                for _ in range(3):
                    graph.replay()
                z.record()
                torch.cuda.synchronize()
                ms = a.elapsed_time(z) / 90
                del graph
                nbytes = (BYTES_NAIK if naik else BYTES_NN)[prec] * vh
                flops = (FLOP_NAIK if naik else FLOP_NN) * vh
                gbs = nbytes / (ms * 1e-3) / 1e9
                print(json.dumps({"sweep": "dslash", "lattice": list(dims), "naik": naik, "prec": prec,
                                  "us": round(ms * 1e3, 2), "GB/s": round(gbs, 1), "frac": round(gbs / peak, 4),
                                  "GFLOP/s": round(flops / (ms * 1e-3) / 1e9, 1),
                                  "l2_resident": nbytes < L2_BYTES, "peak": f"{peak_kind} {peak}"}), flush=True)
        del sets, fat64, lng64, fat, lng, inp, out
        lat.close()
        torch.cuda.empty_cache()
    if args.sweep_cg:
        import fieldgen as fg

        wl = fg.workload("cfg64naik")
        u, w, b = fg.make_inputs_sliced(wl["dims"], wl["fat"], True, wl["seed"])
        lat = q.Lattice(wl["dims"])
        fat64 = q.qex_pack_links(lat, "f64", torch.from_numpy(u).cuda())
        lng64 = q.qex_pack_links(lat, "f64", torch.from_numpy(w).cuda())
        del u, w
        torch.cuda.empty_cache()
        bh = q.qex_pack_field(lat, "f64", 0, torch.from_numpy(b).cuda())
        # inner formats: FP32 two-row fat + FP32 long links, and 16-bit two-row fat + 16-bit scaled long links
        for inner, delta in (("f32r12", DELTA), ("f32r12h", DELTA)):
            fati = q.qex_convert_links(lat, "f64", fat64, inner)
            lngi = q.qex_convert_links(lat, "f64", lng64, q.qex_long_links_prec(inner))
            x = torch.zeros_like(bh)
            st, stats = q.qex_cg(lat, inner, fat64, lng64, fati, lngi, -1.0 / 24, wl["mass"], bh, x, tol=TOL,
                                 maxiter=80000, delta=delta, check=False)
            print(json.dumps({"sweep": "cg", "workload": "64^4 Naik, Haar fat links, Gaussian/sqrt(3) long links, "
                              "c3=-1/24, m=0.005", "inner": inner, "long_links": q.qex_long_links_prec(inner),
                              "delta": delta, "status": st, **stats}), flush=True)
            del fati, lngi, x
            torch.cuda.empty_cache()


MRHS_MASS = 0.05  # the 16-source solve's mass (the workload names masses only for the multi-lattice case)


def run_mrhs(args):
    """24^4, Haar links (seed 4), 16 Gaussian even-site sources: batched
    two-row FP32 Dslash per right-hand side vs the single-RHS kernel, and the
    batched mixed-precision solve vs 16 single-RHS solves of the same
    sources."""
    import torch

    import fieldgen as fg
    import paper_1612_02750_gb300 as q
    from paper_1612_02750_gb300 import build as qbuild

    qbuild.build()
    q.load()
    dims, nrhs, seed = (24, 24, 24, 24), 16, 4
    st = fg.rng_streams(seed)
    u = fg.random_links(dims, "haar", st["links"])
    ev = fg.even_mask(dims)
    srcs = []
    for _ in range(nrhs):
        b = fg.gaussian_field(st["source"], dims)
        b[~ev] = 0
        srcs.append(b)
    lat = q.Lattice(dims)
    vh = lat.half_volume
    fat64 = q.qex_pack_links(lat, "f64", torch.from_numpy(u).cuda())
    fatr = q.qex_convert_links(lat, "f64", fat64, "f32r12")
    n64 = q.qex_field_bytes(lat, "f64") // 8
    B = torch.cat([q.qex_pack_field(lat, "f64", 0, torch.from_numpy(b).cuda()) for b in srcs]).contiguous()
    peak, _ = measured_peak()

    def tev(fn, reps=30):
        for _ in range(3):
            fn()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        z.record()
        torch.cuda.synchronize()
        return a.elapsed_time(z) / reps

    inp = q.empty_fields(lat, "f32r12", nrhs).normal_()
    out = q.empty_fields(lat, "f32r12", nrhs)
    one_in, one_out = inp[: inp.numel() // nrhs].contiguous(), q.empty_field(lat, "f32r12")
    t_m = tev(lambda: q.qex_dslash_mrhs(lat, "f32r12", fatr, None, 0.0, 1, nrhs, inp, out))
    t_1 = tev(lambda: q.qex_dslash(lat, "f32r12", fatr, None, 0.0, 1, one_in, one_out))
    mbytes = (384 + nrhs * 48) * vh
    print(json.dumps({"mrhs": "dslash", "lattice": list(dims), "nrhs": nrhs, "prec": "f32r12",
                      "batched_ms": round(t_m, 4), "single_ms": round(t_1, 4),
                      "per_rhs_speedup": round(t_1 * nrhs / t_m, 2),
                      "batched_GB/s": round(mbytes / (t_m * 1e-3) / 1e9, 1),
                      "batched_frac": round(mbytes / (t_m * 1e-3) / 1e9 / peak, 4),
                      "bytes_per_site": 384 + nrhs * 48}), flush=True)
    X = torch.zeros_like(B)
    q.qex_cg_mrhs(lat, "f32r12", fat64, None, fatr, None, 0.0, MRHS_MASS, nrhs, B, X, tol=TOL, delta=DELTA)
    X.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    _, stm = q.qex_cg_mrhs(lat, "f32r12", fat64, None, fatr, None, 0.0, MRHS_MASS, nrhs, B, X, tol=TOL, delta=DELTA)
    torch.cuda.synchronize()
    t_batched = time.perf_counter() - t0
    t0 = time.perf_counter()
    its = []
    for r in range(nrhs):
        x1 = torch.zeros(n64, dtype=torch.float64, device="cuda")
        _, s1 = q.qex_cg(lat, "f32r12", fat64, None, fatr, None, 0.0, MRHS_MASS, B[r * n64:(r + 1) * n64].contiguous(),
                         x1, tol=TOL, delta=DELTA)
        its.append(s1["iters"])
    torch.cuda.synchronize()
    t_single = time.perf_counter() - t0
    print(json.dumps({"mrhs": "cg", "lattice": list(dims), "nrhs": nrhs, "mass": MRHS_MASS, "links": "Haar",
                      "batched_s": round(t_batched, 4), "sequential_single_s": round(t_single, 4),
                      "speedup": round(t_single / t_batched, 2),
                      "batched_iters": [x["iters"] for x in stm], "single_iters": its,
                      "max_true_rel_resid": max(x["true_rel_resid"] for x in stm),
                      "all_converged": all(x["converged"] for x in stm)}), flush=True)


BATCH_DIMS = [(8, 8, 8, 8), (12, 12, 12, 12), (16, 16, 16, 16), (16, 16, 16, 32), (20, 20, 20, 20),
              (24, 24, 24, 24), (24, 24, 24, 48), (32, 32, 32, 32)]


def run_batch(args):
    """Eight independent lattices (Haar links, seed 4 + 10k, masses
    m_k = 0.005 * 20^(k/7) in the listed order, one Gaussian source each):
    one qex_cg_batch call against eight qex_cg calls, 16-bit inner links."""
    import torch

    import fieldgen as fg
    import paper_1612_02750_gb300 as q
    from paper_1612_02750_gb300 import build as qbuild

    qbuild.build()
    q.load()
    items = []
    for k, dims in enumerate(BATCH_DIMS):
        u, _, b = fg.make_inputs(dims, "haar", False, 4 + 10 * k)
        lat = q.Lattice(dims)
        fat64 = q.qex_pack_links(lat, "f64", torch.from_numpy(u).cuda())
        bh = q.qex_pack_field(lat, "f64", 0, torch.from_numpy(b).cuda())
        items.append({"lat": lat, "fat64": fat64, "fat32": q.qex_convert_links(lat, "f64", fat64, INNER),
                      "mass": 0.005 * 20 ** (k / 7), "b64": bh, "x64": torch.zeros_like(bh)})
    delta = DELTA
    q.qex_cg_batch(items, INNER, tol=TOL, maxiter=400000, delta=delta)  # warm-up (builds scratch)
    for it in items:  # warm-up of the single solves (launch-shape tuning, graph capture)
        x = torch.zeros_like(it["b64"])
        q.qex_cg(it["lat"], INNER, it["fat64"], None, it["fat32"], None, 0.0, it["mass"], it["b64"], x, tol=TOL,
                 maxiter=400000, delta=delta)
        it["x64"].zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, stats = q.qex_cg_batch(items, INNER, tol=TOL, maxiter=400000, delta=delta)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    singles = []
    t0 = time.perf_counter()
    for it in items:
        x = torch.zeros_like(it["b64"])
        _, s1 = q.qex_cg(it["lat"], INNER, it["fat64"], None, it["fat32"], None, 0.0, it["mass"], it["b64"], x,
                         tol=TOL, maxiter=400000, delta=delta)
        singles.append(s1)
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    print(json.dumps({"batch": "cg", "lattices": ["x".join(map(str, d)) for d in BATCH_DIMS],
                      "masses": [round(it["mass"], 5) for it in items], "status": st,
                      "batched_s": round(t_batch, 4), "sequential_s": round(t_seq, 4),
                      "speedup": round(t_seq / t_batch, 3),
                      "batched_iters": [x["iters"] for x in stats], "single_iters": [x["iters"] for x in singles],
                      "max_true_rel_resid": max(x["true_rel_resid"] for x in stats),
                      "all_converged": all(x["converged"] for x in stats)}), flush=True)


def main():
    args = parse()
    if args.batch:
        run_batch(args)
    elif args.mrhs:
        run_mrhs(args)
    elif args.sweep:
        run_sweep(args)
    elif args.dslash_only:
        run_dslash_only()
    elif args.profile_iteration:
        run_profile_iteration()
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
