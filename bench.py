"""Benchmark: time-to-certified-solve of XM on the 10155-camera workload (Q resident in HBM),
with the Q.Y sweep's achieved HBM bandwidth, the FP32-bulk vs FP64 comparison, an
end-to-end number from pinned host arrays through the C ABI, and the FP64 oracle timed on the
host cores.  Prints one JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload c3] [--prec fp32]
    python bench.py --impl reference ...      # the oracle on the host cores, same metric/unit

A "step" is one certified solve (Alg. 1 + RTR-tCG + certificate + rounding) from the
[I, ..., I] start on a Q already built on the device.
"""
from __future__ import annotations

import argparse
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

import scenes  # noqa: E402

METRIC = "time-to-certified-solve (s) at 10k cams; Q·Y GB/s vs HBM peak, FP32 vs FP64"
WORKLOADS = {
    "c3": (scenes.config3, 10155, "10155 cameras, 1.5M landmarks, ~7.5M observations, track "
                                  "2+Geom(1/4), 5% outliers, noise N(0,0.02^2), w~U[0.5,1]; BM rank "
                                  "4 start with staircase"),
    "c2": (scenes.config2, 1934, "1934 cameras, 300k landmarks, ~1.5M observations, 2% outliers"),
    "c4": (scenes.config4, 2000, "2000-frame indoor trajectory, 400k landmarks, multiplicative depth "
                                 "noise; App. D scale regularisation weight 10"),
    "c1": (scenes.config1, 20, "20 cameras on a circle, 200 landmarks x 4 observers"),
}
# objective options per workload: the trajectory's unregularised optimum collapses the scales of
# later frames towards zero (App. D), so it is solved with the scale regulariser
WORKLOAD_OPTS = {"c4": {"scale_reg": 10.0}}
# solver options of the timed certified solve per workload beyond the objective's: none (the
# defaults hand the FP32 bulk phase over at its noise floor and precondition the tCG when it
# keeps stopping at its iteration cap, which the trajectory needs and the other workloads do not)
SOLVE_OPTS = {}
BATCH_DESC = ("256 independent scenes, cameras log-uniform in [10, 400] (floor), 50 landmarks per "
              "camera x 4 observers, keypoint noise N(0, 0.01^2), unit weights; FP32 bulk, one "
              "persistent launch per rank class under a CUDA graph, autotuned block-row tiling")
PRECS = {"fp64": 0, "fp32": 1, "bf16": 2}
DTYPES = {"fp64": "f64", "fp32": "f32", "bf16": "bf16/f32"}
# Sweeps of one certified FP32-bulk solve of each workload as measured on a B300 by the GPU arm
# of this benchmark with the default options (bulk-phase tCG solves of at most 60 iterations;
# 10155 cameras: mean of the 5 timed solves of a default run; 1934 cameras and the trajectory:
# mean of 3 solves); the reference arm multiplies the oracle's time per sweep by it (an
# extrapolation, labelled as such in its line).
REFERENCE_SWEEPS = {"c3": 1720, "c2": 570, "c4": 10190, "c1": 500}
L2_BYTES = 126e6
# DRAM bytes (read + write) over algorithmic bytes of qy_packed_kernel<float,4,8> from one ncu
# capture at the 10155-camera size itself (n = 30465: 1.88 GB read + 0.00412 GB written per
# launch against 1.8573 GB algorithmic, as ncu prints them), on the kernel as it stands (swizzled
# Y_J, paired tile-row order, column partials through the reducer warp).  Applied only at that
# size (other sizes get traffic = null); must be re-measured (or set to None) whenever the
# sweep kernel changes.
SWEEP_TRAFFIC_RATIO = (1.88 + 0.00412) / 1.857268
SWEEP_TRAFFIC_N = 30465
# The same ratio for k_batched<4> on the 256-scene batch with pairs only (one launch per batch):
# DRAM read + write of that launch over the dense sweep bytes of its scenes, from one ncu
# capture (0.90: L2 serves part of the small scenes' re-reads).  With the automatic mixed teams
# the batch is two launches running side by side, which ncu serialises (the first then drains
# both queues alone, with L2 serving most of its reads), so no capture measures that mode's
# traffic: it is reported as null.
BATCH_TRAFFIC_RATIO_PAIRS = (78.787872 + 2.726973) / 90.936067344


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi sampled every 200 ms while the timed region runs."""

    def __init__(self, index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def sweep_bytes(n: int, r: int, bq: int, by: int) -> float:
    """Algorithmic bytes of one sweep: the unique entries of symmetric Q plus Y read and W written."""
    return n * (n + 1) / 2 * bq + 2 * n * r * by


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_sweep_seconds(n: int, r: int, reps: int = 2, seed: int = 0) -> float:
    """Host time of one oracle sweep (dense FP64 Q @ Y plus the oracle's per-camera dual blocks
    and tangent projection) at size n.  Q's values do not change the time of a dense product; a
    seeded random symmetric matrix of the workload's size is used."""
    from oracle import xm_oracle as O
    rng = np.random.default_rng(seed)
    Q = rng.standard_normal((n, n))
    Q += Q.T
    Y = O.initial_point(n // 3, r)
    t0 = time.perf_counter()
    for _ in range(reps):
        G = Q @ Y
        L = O.lambdas(Y, G)
        O.proj_tangent(Y, 2.0 * (G - O.apply_blockdiag(L, Y)))
    return (time.perf_counter() - t0) / reps


def whole_job_seconds(local_total: float, steps: int, world: int, dist=None, device=None) -> float:
    """Replicas only: every rank solves its own copy; the job's time is the slowest rank's timed
    region (max over ranks) and the value is that time over all solves of all ranks."""
    total = float(local_total)
    if dist is not None and world > 1:
        import torch
        t = torch.tensor([total], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total = float(t.item())
    return total / (steps * world)


def run_reference(args):
    """The oracle as it stands on the host cores: each step times one oracle sweep at the
    workload's size; the value is that time per sweep times the sweeps of one certified solve."""
    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    if args.workload == "c5":
        scs = scenes.config5()
        vals = []
        for i in range(args.warmup + args.steps):
            cb = oracle_batch_sample(scs, budget_s=10.0)
            if i >= args.warmup:
                vals.append(cb["value"])
        v = statistics.mean(vals)
        cb["value"] = v
        print(json.dumps({"impl": "reference", "metric": "batched certified solves: scenes/s and "
                          "p50/p99 per-scene latency", "value": v, "unit": "scenes/s",
                          "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak",
                          "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                          "config": {"workload": f"c5: {BATCH_DESC}"}, "cpu_baseline": cb,
                          "e2e": {"value": v, "unit": "scenes/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}), flush=True)
        return 0
    _, N, desc = WORKLOADS[args.workload]
    n = 3 * N
    S = REFERENCE_SWEEPS[args.workload]
    from oracle import xm_oracle as O
    rng = np.random.default_rng(0)
    Q = rng.standard_normal((n, n))
    Q += Q.T
    Y = O.initial_point(N, 4)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        G = Q @ Y
        L = O.lambdas(Y, G)
        O.proj_tangent(Y, 2.0 * (G - O.apply_blockdiag(L, Y)))
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    del Q
    per = statistics.mean(times)
    value = per * S
    full = oracle_full_solve_c2()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: {desc}", "prec": "fp64 (oracle)"},
        "cpu_baseline": {"value": value, "unit": "s", "cores": host_cores(),
                         "kind": "oracle, extrapolated",
                         "sample": f"one oracle sweep (dense FP64 Q@Y on a seeded random symmetric Q "
                                   f"of the workload's size n={n}, r=4, plus dual blocks and "
                                   f"projection; the product's time does not depend on Q's values) "
                                   f"timed per step, times the {S} sweeps of the GPU arm's mean "
                                   f"certified solve"},
        "e2e": {"value": value, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "oracle_end_to_end_c2": full,
    }
    print(json.dumps(line), flush=True)
    return 0


def oracle_full_solve_c2() -> dict:
    """One complete oracle run on the 1934-camera workload, measured end to end on the host cores
    (no extrapolation): Q by the Schur form, then the staircase (Alg. 1 + RTR-tCG), certificate
    and rounding."""
    from oracle import xm_oracle as O
    sc = scenes.config2()
    t0 = time.perf_counter()
    Q = O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w)
    t1 = time.perf_counter()
    res = O.solve(Q, r0=4)
    t2 = time.perf_counter()
    return {"workload": "c2: 1934 cameras, 300k landmarks, ~1.5M observations, 2% outliers",
            "build_s": t1 - t0, "solve_s": t2 - t1, "certified": bool(res.certified),
            "sweeps": int(res.sweeps), "f": res.f, "cores": host_cores(), "kind": "oracle, measured"}


def run_sweep_only(args):
    """Q.Y sweep alone (FP32 storage, r = 4, the solver's dominant launch configuration) on a
    seeded random symmetric Q of the given number of cameras; prints one JSON line."""
    import torch
    from paper_2502_04640_b300 import xm
    N = args.sweep_only
    n = 3 * N
    ctx = xm.Context(0)
    g = torch.Generator(device="cuda").manual_seed(1)
    Q = torch.randn((n, n), dtype=torch.float64, device="cuda", generator=g)
    Q = (Q + Q.T) * 0.5
    q = xm.xm_qmat_from_dense(ctx, Q, xm.XM_STORE_FP32)
    del Q
    torch.cuda.empty_cache()
    ms, ms_min = xm.xm_bench_qy(q, xm.XM_FP32_BULK, 4, max(args.steps, 1))
    alg = sweep_bytes(n, 4, 4, 4)
    peak, kind = peaks()
    line = {"sweep_only": True, "N": N, "n": n, "ms": ms, "ms_min": ms_min,
            "GBps": alg / (ms * 1e-3) / 1e9, "frac": alg / (ms * 1e-3) / 1e9 / peak,
            "peak": peak, "peak_kind": kind}
    q.free()
    if args.sweep_table:
        # every storage precision and padded width on the same Q (mean of 20 after warm-up)
        Q = torch.randn((n, n), dtype=torch.float64, device="cuda",
                        generator=torch.Generator(device="cuda").manual_seed(1))
        Q = (Q + Q.T) * 0.5
        table = {}
        for name, store, pv, bq, by in (("fp32", xm.XM_STORE_FP32, xm.XM_FP32_BULK, 4, 4),
                                        ("bf16", xm.XM_STORE_BF16, xm.XM_BF16Q_BULK, 2, 4),
                                        ("fp64", xm.XM_STORE_FP64, xm.XM_FP64, 8, 8)):
            qq = xm.xm_qmat_from_dense(ctx, Q, store)
            for r in (1, 4, 8):
                m_ms, _ = xm.xm_bench_qy(qq, pv, r, 20)
                gbs = sweep_bytes(n, r, bq, by) / (m_ms * 1e-3) / 1e9
                table[f"{name}_r{r}"] = {"us": m_ms * 1e3, "GBps": gbs, "frac": gbs / peak}
            qq.free()
        del Q
        line["table"] = table
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def update_tensor_flops(N: int) -> float:
    """BF16 tensor FLOPs of the translation elimination on the tensor cores: 36 digit pairs
    (levels 0..7) of (a) the rank-(N-1) product over the n(n+1)/2 entries of the upper
    triangle, (b) the blocked triangular solve: per 1024-row block the product with the diagonal
    block's inverse and the block update of the rows below, and (c) the trailing updates of the
    blocked Cholesky factor (lower triangle), 512-row blocks; n = 3N."""
    n, K = 3 * N, N - 1
    syrk = 36 * 2.0 * K * n * (n + 1) / 2
    trsm = sum(36 * 2.0 * (K - i0) * n * min(1024, K - i0) for i0 in range(0, K, 1024))
    chol = sum(36 * 2.0 * (K - i0 - min(512, K - i0)) ** 2 / 2 * min(512, K - i0) for i0 in range(0, K, 512))
    return syrk + trsm + chol


def update_report(N: int, path: int, t_update: float) -> dict:
    """The build's translation elimination (triangular solve + rank-(N-1) update + packing): its
    path, device time and, for the tensor-core path, its tensor-core roofline (BF16 peak,
    measured burst) and FP64-equivalent rate ((n^2 K + K^2 n + K^3 / 3) / t)."""
    n, K = 3 * N, N - 1
    rep = {"path": {0: "none", 1: "fp64_dpotrf_dtrsm_dsyrk", 2: "split_bf16_tcgen05"}.get(path, str(path)),
           "seconds": t_update,
           "fp64_equivalent_tflops": (n * n * K + K * K * n + K ** 3 / 3) / t_update / 1e12
           if t_update > 0 else None}
    if path == 2 and t_update > 0:
        pk = None
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                pk = json.load(f).get("bf16_tflops")
        except (OSError, ValueError):
            pk = None
        kind = "measured" if pk else "fallback"
        pk = pk or 1800.0
        ach = update_tensor_flops(N) / t_update / 1e12
        rep["roofline"] = {"bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                           "frac": ach / pk, "traffic": None,
                           "kernel": "k_oz_mma<SYRK> + k_oz_mma<GEMM> (triangular solve, Cholesky updates) "
                                     "(+ digit splits, FP64 diagonal inverses, Cholesky diagonal "
                                     "blocks and panels, packing)",
                           "flops": update_tensor_flops(N), "peak_kind": kind + " bf16 burst"}
    return rep


def run_build_only(args):
    """xm_build_Q alone on a seeded random scene of N cameras (30 N landmarks, track 2+Geom(1/4),
    5 % outliers): one warm-up, then --steps builds with the tensor-core update and one with the
    FP64 update; prints one JSON line."""
    import torch
    from paper_2502_04640_b300 import xm
    N = args.build_only
    sc = scenes.random_scene(N, 30 * N, noise=0.02, outlier_frac=0.05, seed=1)
    ctx = xm.Context(0)
    tens = xm.scene_tensors(sc)
    res = {}
    for mode, reps in ((xm.XM_BUILD_SPLIT_BF16, max(args.steps, 1)), (xm.XM_BUILD_FP64, 1)):
        xm.xm_set_build_mode(ctx, mode)
        walls, upds = [], []
        for i in range(reps + (1 if mode == xm.XM_BUILD_SPLIT_BF16 else 0)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            q = xm.xm_build_Q(ctx, sc.N, sc.M, *tens)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            path, tu = xm.xm_qmat_build_info(q)
            q.free()
            if mode == xm.XM_BUILD_SPLIT_BF16 and i == 0:
                continue    # first call: library set-up
            walls.append(wall)
            upds.append(tu)
        res[mode] = (statistics.median(walls), statistics.median(upds), path)
    ws, us, ps = res[xm.XM_BUILD_SPLIT_BF16]
    wf, uf, pf = res[xm.XM_BUILD_FP64]
    cpu = None if args.no_cpu else oracle_build_sample(N)
    print(json.dumps({"build_only": True, "N": N, "n": 3 * N, "E": sc.E,
                      "split": {"build_s": ws, **update_report(N, ps, us)},
                      "fp64": {"build_s": wf, **update_report(N, pf, uf)},
                      "cpu_baseline": cpu}), flush=True)
    ctx.close()
    return 0


def _pct(xs, q):
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q)) if len(xs) else float("nan")


def batched_measure(ctx, scs, warmup: int, steps: int, time_limit: float = 60.0) -> dict:
    """Builds every scene's Q, packs the batch, autotunes its tiling, then W untimed and K timed
    batched solves (CUDA events on the context's stream around the K graph replays, and the
    wall clock; the larger counts); per-scene latency from the device clock of each scene's CTA
    in the last batch: completion after the batch's first scene started (p50/p99) and the
    scene's own solve time."""
    import torch
    from paper_2502_04640_b300 import xm
    S = len(scs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    qs = [xm.xm_build_Q(ctx, sc.N, sc.M, *xm.scene_tensors(sc)) for sc in scs]
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t0
    t0 = time.perf_counter()
    b = xm.xm_batch_create(ctx, qs)
    t_pack = time.perf_counter() - t0
    for q in qs:
        q.free()
    t0 = time.perf_counter()
    tiling = xm.xm_batch_autotune(b, reps=8)
    t_tune = time.perf_counter() - t0
    opts = xm.xm_default_opts(time_limit_s=time_limit)
    tot = sum(sc.N for sc in scs)
    R = torch.zeros((tot, 3, 3), dtype=torch.float64, device="cuda:0")
    s = torch.zeros((tot,), dtype=torch.float64, device="cuda:0")
    for _ in range(warmup):
        xm.xm_solve_batched(b, opts, R=R, s=s)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(ctx.stream)
    wall0 = time.perf_counter()
    infos = []
    for _ in range(steps):
        infos.append(xm.xm_solve_batched(b, opts, R=R, s=s)["info"])
    ev1.record(ctx.stream)
    torch.cuda.synchronize()
    per_step = max(time.perf_counter() - wall0, ev0.elapsed_time(ev1) / 1e3) / steps
    launches, quads = xm.xm_batch_launches(b)
    last = infos[-1]
    t_first = min(i["t_begin_ns"] for i in last)
    done_ms = [(i["t_end_ns"] - t_first) / 1e6 for i in last]
    own_ms = [(i["t_end_ns"] - i["t_begin_ns"]) / 1e6 for i in last]
    # bytes the dense sweeps read: FP32 sweeps n x ldq x 4, FP64 sweeps n x ldq x 8 (Y in shared memory)
    by = 0.0
    for sc, i in zip(scs, last):
        n = 3 * sc.N
        ldq = (n + 3) & ~3
        by += (i["n_sweeps"] - i["n_sweeps_fp64"]) * n * ldq * 4 + i["n_sweeps_fp64"] * n * ldq * 8
    peak, peak_kind = peaks()
    achieved = by / per_step / 1e9
    q_bytes = sum(3 * sc.N * ((3 * sc.N + 3) & ~3) for sc in scs) * 4
    return {
        "b": b, "opts": opts, "R": R, "s": s, "tot": tot,
        "scenes_per_s": S / per_step, "s_per_batch": per_step,
        "latency_ms": {"p50": _pct(done_ms, 50), "p99": _pct(done_ms, 99), "max": max(done_ms),
                       "scene_solve_p50": _pct(own_ms, 50), "scene_solve_p99": _pct(own_ms, 99)},
        "certified": sum(i["certified"] for i in last), "scenes": S, "cameras": tot,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": None,
                     "traffic_note": ("null: the batch's two launches run side by side and ncu "
                                      "serialises them; " if quads else "null: ") +
                                     "with pairs only (one launch, before the shared second queue) ncu "
                                     f"measured DRAM read+write = {BATCH_TRAFFIC_RATIO_PAIRS:.2f} of the "
                                     "dense sweep bytes",
                     "kernel": "k_batched<4>" + (" (4-CTA and 2-CTA launches side by side)" if quads else ""),
                     "bytes_per_launch": by, "launch_ms": per_step * 1e3, "peak_kind": peak_kind,
                     "note": "dense sweep bytes of all scenes / batch time; the FP32 copies total "
                             f"{q_bytes / 1e6:.0f} MB, so part of every sweep is served by L2"},
        "l2": f"per-scene Q re-read every sweep; the batch's FP32 copies total {q_bytes / 1e6:.0f} MB",
        "tiling_rows_chunks": tiling,
        "sweeps": int(sum(i["n_sweeps"] for i in last)),
        "sweeps_fp64": int(sum(i["n_sweeps_fp64"] for i in last)),
        "escapes": int(sum(i["n_escapes"] for i in last)),
        "ranks": {str(r): sum(1 for i in last if i["rank"] == r) for r in sorted({i["rank"] for i in last})},
        "build_q_s": t_build, "pack_s": t_pack, "autotune_s": t_tune,
        "launches_per_batch": launches, "quad_scenes": quads,
    }


def run_batched(args):
    """The serving-style batch: every scene's Q resident, W untimed and K timed batched solves;
    value = scenes per second."""
    import torch
    from paper_2502_04640_b300 import xm
    scs = scenes.config5()
    S = len(scs)
    ctx = xm.Context(0)
    clocks = ClockSampler(0)
    m = batched_measure(ctx, scs, args.warmup, args.steps,
                        args.time_limit if args.time_limit > 0 else 60.0)
    clk = clocks.stop()
    b, opts, R, s, tot = m.pop("b"), m.pop("opts"), m.pop("R"), m.pop("s"), m.pop("tot")
    # end to end from pinned host arrays: copies, Q builds, batch packing, solve, results back
    e2e = None
    if args.e2e_steps > 0:
        def pin(a, dt):
            return torch.from_numpy(np.ascontiguousarray(a)).to(dt).pin_memory()
        host = [(pin(sc.cam, torch.int32), pin(sc.lmk, torch.int32), pin(sc.ukp, torch.float64),
                 pin(sc.w, torch.float64)) for sc in scs]
        Rh = torch.zeros((tot, 3, 3), dtype=torch.float64).pin_memory()
        sh = torch.zeros((tot,), dtype=torch.float64).pin_memory()
        h2d = sum(int(sc.E * (4 + 4 + 24 + 8)) for sc in scs)
        torch.cuda.synchronize()
        te = time.perf_counter()
        for _ in range(args.e2e_steps):
            qs2 = []
            for sc, (hc, hl, hu, hw) in zip(scs, host):
                dt = [x.to("cuda:0", non_blocking=True) for x in (hc, hl, hu, hw)]
                qs2.append(xm.xm_build_Q(ctx, sc.N, sc.M, *dt))
            b2 = xm.xm_batch_create(ctx, qs2)
            for q in qs2:
                q.free()
            o2 = xm.xm_solve_batched(b2, opts, R=R, s=s)
            Rh.copy_(o2["R"], non_blocking=True)
            sh.copy_(o2["s"], non_blocking=True)
            torch.cuda.synchronize()
            b2.free()
        e2e_s = (time.perf_counter() - te) / args.e2e_steps
        e2e = {"value": S / e2e_s, "unit": "scenes/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": int(tot * (72 + 8)), "seconds_per_batch": e2e_s}
    cpu = None
    if not args.no_cpu:
        cpu = oracle_batch_sample(scs, budget_s=20.0)
    line = {
        "metric": "batched certified solves: scenes/s and p50/p99 per-scene latency",
        "value": m["scenes_per_s"], "unit": "scenes/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": m["s_per_batch"] * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64", "data": "synthetic",
        "config": {"workload": f"c5: {BATCH_DESC}", "scenes": S, "cameras": tot, "l2": m.pop("l2")},
        "latency_ms": m["latency_ms"], "certified": m["certified"], "roofline": m["roofline"],
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": m["launches_per_batch"] * args.steps, "clocks": clk,
        **{k: m[k] for k in ("tiling_rows_chunks", "sweeps", "sweeps_fp64", "escapes", "ranks",
                             "build_q_s", "pack_s", "autotune_s")},
    }
    print(json.dumps(line), flush=True)
    b.free()
    ctx.close()
    return 0


def factored_bytes_flops(N: int, M: int, E: int, r: int) -> tuple:
    """Algorithmic bytes and FP64 flops of one factored product (App. A's elimination in product
    form): the landmark-major copy of (u, w, camera) read twice (u once), the camera-major copy
    (u, w, landmark) twice, per landmark its offsets and 1/d_k twice and the two means written and
    read (8 doubles a row), the packed -Sbar^{-1} once, Y read and W written (row offsets and the
    (N-1) x R sweep vectors are negligible).  Flops: a_e three times (2 x 3r each), the means and
    sums (2r each), the output outer products (2 x 3r) and the symmetric sweep (2 (N-1)^2 r)."""
    m = N - 1
    by = (E * (36 + 12 + 36 + 36) + M * (2 * 8 + 2 * 8 + 4 * 8 * 8) + m * (m + 1) / 2 * 8
          + 2 * 3 * N * r * 8)
    fl = E * (3 * 6 * r + 3 * 2 * r + 6 * r) + 2.0 * m * m * r
    return by, fl


def factored_measure(ctx, sc, q, reps: int = 20) -> dict:
    """The factored Q operator next to the dense sweeps on the same scene: set-up time, resident
    bytes, time per product (CUDA events on the context stream, after 3 warm-up products), its
    algorithmic bytes and FP64 flops, and the largest difference from the dense FP64 sweep
    relative to that sweep's largest entry."""
    import torch
    from paper_2502_04640_b300 import xm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    f = xm.xm_qfact_create(ctx, sc.N, sc.M, *xm.scene_tensors(sc))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    Y = torch.as_tensor(np.random.default_rng(3).standard_normal((3 * sc.N, 4)), device="cuda:0")
    W = torch.empty_like(Y)
    for _ in range(3):
        xm.lib().xm_qy_factored(ctx.h, f.h, 4, Y.data_ptr(), W.data_ptr())
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(ctx.stream)
    for _ in range(reps):
        xm.lib().xm_qy_factored(ctx.h, f.h, 4, Y.data_ptr(), W.data_ptr())
    ev1.record(ctx.stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / reps
    res = {"setup_s": setup_s, "resident_GB": f.bytes / 1e9, "ms_per_product_r4": ms}
    by, fl = factored_bytes_flops(sc.N, sc.M, sc.E, 4)
    res.update({"bytes_per_product": by, "fp64_flops_per_product": fl,
                "achieved_GBps": by / (ms * 1e-3) / 1e9, "achieved_fp64_tflops": fl / (ms * 1e-3) / 1e12})
    if q is not None and (q.mask & xm.XM_STORE_FP64):
        Wd = xm.xm_qy(q, Y, xm.XM_FP64)
        res["max_diff_vs_dense_fp64_rel"] = float((W - Wd).abs().max() / Wd.abs().max())
        d_ms, _ = xm.xm_bench_qy(q, xm.XM_FP64, 4, 10)
        res["dense_fp64_sweep_ms"] = d_ms
        res["speedup_vs_dense_fp64"] = d_ms / ms
    if q is not None and (q.mask & xm.XM_STORE_FP32):
        res["dense_fp32_sweep_ms"] = xm.xm_bench_qy(q, xm.XM_FP32_BULK, 4, 10)[0]
    f.free()
    return res


def depth_noise_table(ctx, count: int = 8, N: int = 100, M: int = 2000) -> dict:
    """Robustness to the depth-noise model of the paper's noise analysis (every observation's depth
    scaled by (1 + eps)^x, x ~ U(-1, 1)): per noise level, `count` community-photo-shaped scenes
    of N cameras solved in the FP32-bulk mode; certified count, Eq. 18's eta (median, max), the
    rounded rotations' angular error against the ground truth (median over cameras and scenes,
    worst camera), the median |log| scale error, and the median solve time."""
    from paper_2502_04640_b300 import xm
    table = {}
    for eps in scenes.DEPTH_NOISE_EPS:
        cert, etas, angs, worst, lserr, times = 0, [], [], [], [], []
        for sc in scenes.depth_noise_scenes(eps, count=count, N=N, M=M):
            q = xm.xm_build_Q(ctx, sc.N, sc.M, *xm.scene_tensors(sc))
            o = xm.xm_solve(q, xm.xm_default_opts(prec=xm.XM_FP32_BULK))
            q.free()
            info = o["info"]
            R, s, _, _ = sc.anchored_gt()
            Rg, sg = o["R"].cpu().numpy(), o["s"].cpu().numpy()
            c = np.clip((np.einsum("iab,iab->i", Rg, R) - 1.0) / 2.0, -1.0, 1.0)
            a = np.degrees(np.arccos(c))[1:]
            cert += int(info["certified"])
            etas.append(info["eta"])
            angs.append(a)
            worst.append(a.max())
            lserr.append(np.median(np.abs(np.log(np.maximum(sg[1:], 1e-300) / s[1:]))))
            times.append(info["t_solve_s"])
        table[f"{eps:g}"] = {"certified": cert, "scenes": count, "eta_median": float(np.median(etas)),
                             "eta_max": float(np.max(etas)),
                             "rot_err_deg_median": float(np.median(np.concatenate(angs))),
                             "rot_err_deg_worst": float(np.max(worst)),
                             "log_scale_err_median": float(np.median(lserr)),
                             "solve_s_median": float(np.median(times))}
    return {"model": "depth x (1 + eps)^x, x ~ U(-1, 1) per observation", "N": N, "M": M,
            "scenes_per_level": count, "table": table}


def other_workloads(ctx, steps: int = 3) -> dict:
    """The other workloads of the benchmark, measured in the same run after the main line's timed
    region (rank 0): the 1934-camera plain-vs-mixed comparison, the 2000-frame trajectory's
    certified solve (both hand-over settings) and adjoint, and the 256-scene batch.  Each entry
    records its own error instead of failing the run."""
    out = {}
    for name, fn in (("c2", _c2_compare), ("c4", _c4_solve_and_adjoint), ("c5", _c5_batch),
                     ("depth_noise", lambda c, k: depth_noise_table(c, count=4))):
        t0 = time.perf_counter()
        try:
            out[name] = fn(ctx, steps)
        except Exception as e:      # noqa: BLE001 - reported in the line, the main number stands
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        out[name]["wall_s"] = time.perf_counter() - t0
    return out


def _timed_solves(xm, q, opts, warmup: int, steps: int):
    import torch
    for _ in range(warmup):
        xm.xm_solve(q, opts)
    outs, walls = [], []
    for _ in range(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        o = xm.xm_solve(q, opts)
        walls.append(time.perf_counter() - t0)
        outs.append(o)
    return outs, walls


def _errs(o, ref):
    fi = ref["info"]
    return {"f_rel": abs(o["info"]["f"] - fi["f"]) / (1 + abs(fi["f"])),
            "rho_hat_rel": abs(o["info"]["rho_hat"] - fi["rho_hat"]) / (1 + abs(fi["rho_hat"])),
            "eta_abs": abs(o["info"]["eta"] - fi["eta"]),
            "lambda_min_abs": abs(o["info"]["lambda_min_deflated"] - fi["lambda_min_deflated"]),
            "R_max_abs": float((o["R"] - ref["R"]).abs().max()),
            "s_max_rel": float(((o["s"] - ref["s"]).abs() / ref["s"].abs()).max())}


def _c2_compare(ctx, steps):
    """1934 cameras: certified solve in the FP32-bulk, BF16-storage and plain FP64 forms, with
    per-result errors against the FP64 form."""
    from paper_2502_04640_b300 import xm
    sc = scenes.config2()
    q = xm.xm_build_Q(ctx, sc.N, sc.M, *xm.scene_tensors(sc), xm.XM_STORE_ALL)
    n = q.n
    res = {"N": sc.N, "E": sc.E, "l2": f"L2-resident: packed FP32 Q {n * (n + 1) / 2 * 4 / 1e6:.0f} MB "
                                     f"< 126 MB L2 (no flush between solves)"}
    ref = None
    for name, pv in (("fp64", 0), ("fp32", 1), ("bf16", 2)):
        outs, walls = _timed_solves(xm, q, xm.xm_default_opts(prec=pv), 1, steps)
        res[f"{name}_solve_s"] = statistics.median(walls)
        res[f"{name}_certified"] = all(o["info"]["certified"] for o in outs)
        res[f"{name}_sweeps"] = outs[-1]["info"]["n_sweeps"]
        if pv == 0:
            ref = outs[-1]
        else:
            res[f"{name}_vs_fp64"] = _errs(outs[-1], ref)
    res["eta"] = ref["info"]["eta"]
    res["factored_qy"] = factored_measure(ctx, sc, q)
    for pname, pv, bq, byy in (("fp32", 1, 4, 4), ("bf16", 2, 2, 4), ("fp64", 0, 8, 8)):
        ms, _ = xm.xm_bench_qy(q, pv, 4, 20)
        res[f"qy_{pname}_r4_us"] = ms * 1e3
        res[f"qy_{pname}_r4_GBps"] = sweep_bytes(n, 4, bq, byy) / (ms * 1e-3) / 1e9
    q.free()
    return res


def _c4_solve_and_adjoint(ctx, steps):
    """2000-frame trajectory (App. D weight 10): the certified FP32-bulk solve with the default
    options (automatic hand-over, adaptive tCG preconditioner), once without either (the bulk
    then runs to its iteration cap), and the adjoint (FP32 inner CG in FP64 refinement)."""
    import torch
    from paper_2502_04640_b300 import xm
    sc = scenes.config4()
    wopts = dict(WORKLOAD_OPTS["c4"])
    q = xm.xm_build_Q(ctx, sc.N, sc.M, *xm.scene_tensors(sc), xm.XM_STORE_ALL)
    res = {"N": sc.N, "E": sc.E, "opts": wopts}
    outs, walls = _timed_solves(xm, q, xm.xm_default_opts(prec=1, **wopts), 1, steps)
    res["solve_default_s"] = statistics.median(walls)
    res["solve_default_certified"] = all(o["info"]["certified"] for o in outs)
    out = outs[0]      # the adjoint's forward solve: default options (its stationarity sets the floor)
    plain, walls = _timed_solves(xm, q, xm.xm_default_opts(prec=1, bulk_stall=0, precond=0, **wopts), 0, 1)
    res["solve_no_handover_s"] = walls[0]
    res["solve_no_handover_certified"] = plain[0]["info"]["certified"]
    r = out["info"]["rank"]
    t = xm.scene_tensors(sc)
    D = torch.as_tensor(np.random.default_rng(5).standard_normal((sc.N, 3, 3)), device="cuda:0")
    opts = xm.xm_default_opts(prec=1, **wopts)
    xm.xm_backward(q, out["Y"], r, sc.M, *t, D, opts)
    walls, infos = [], []
    for _ in range(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        infos.append(xm.xm_backward(q, out["Y"], r, sc.M, *t, D, opts)[3])
        walls.append(time.perf_counter() - t0)
    res["adjoint_s"] = statistics.median(walls)
    res["adjoint_grads_per_s"] = sc.E * 4 / res["adjoint_s"]
    res["adjoint"] = {k: infos[-1][k] for k in ("res_rel", "n_cg", "n_refine", "t_lambda_s", "t_resid_s",
                                                 "t_precond_s")}
    res["factored_qy"] = factored_measure(ctx, sc, q)
    q.free()
    return res


def _c5_batch(ctx, steps):
    m = batched_measure(ctx, scenes.config5(), 2, steps)
    m.pop("b").free()
    for k in ("opts", "R", "s", "tot"):
        m.pop(k)
    return m


def oracle_batch_sample(scs, budget_s=20.0):
    """The oracle's own certified solve, scene by scene over every 16th scene of the batch (a
    size-stratified sample), until about budget_s; scenes per second."""
    sys.path.insert(0, ROOT)
    from oracle import xm_oracle as O
    done, t_used = 0, 0.0
    for sc in scs[::16]:
        t0 = time.perf_counter()
        Q = O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w)
        O.solve(Q, r0=4)
        t_used += time.perf_counter() - t0
        done += 1
        if t_used > budget_s:
            break
    return {"value": done / t_used, "unit": "scenes/s", "cores": host_cores(), "kind": "oracle",
            "sample": f"oracle build + staircase solve of {done} scenes (every 16th of the batch, "
                      f"{t_used:.1f} s of host time)"}


def oracle_adjoint_sample(sc, mu: float, n_cams: int = 120) -> dict:
    """The oracle's adjoint on a bounded prefix of the workload (its first n_cams cameras and
    their landmarks): oracle build and solve untimed, one adjoint call timed."""
    from oracle import xm_oracle as O
    sub = scenes.sub_scene(sc, min(n_cams, sc.N))
    Q = O.build_Q_schur(sub.N, sub.M, sub.cam, sub.lmk, sub.ukp, sub.w)
    res = O.solve(Q, r0=4, mu=mu)
    D = np.random.default_rng(5).standard_normal((sub.N, 3, 3))
    t0 = time.perf_counter()
    O.adjoint(sub.N, sub.M, sub.cam, sub.lmk, sub.ukp, sub.w, res.Y, D, Q=Q, mu=mu)
    dt = time.perf_counter() - t0
    return {"value": dt, "unit": "s per backward", "cores": host_cores(), "kind": "oracle",
            "sample": f"oracle adjoint (dense FP64) on the first {sub.N} cameras ({sub.E} observations) "
                      f"of the workload, one call after an untimed oracle build and solve"}


def oracle_build_sample(N: int, n_cap: int = 1500) -> dict:
    """The oracle's Q construction (Schur form, dense FP64) on the same scene generator at
    min(N, n_cap) cameras."""
    from oracle import xm_oracle as O
    Ns = min(N, n_cap)
    sc = scenes.random_scene(Ns, 30 * Ns, noise=0.02, outlier_frac=0.05, seed=1)
    t0 = time.perf_counter()
    O.build_Q_schur(sc.N, sc.M, sc.cam, sc.lmk, sc.ukp, sc.w)
    dt = time.perf_counter() - t0
    return {"value": dt, "unit": "s per build", "cores": host_cores(), "kind": "oracle",
            "sample": f"oracle build_Q_schur on the seeded random scene of {Ns} cameras "
                      f"({sc.E} observations)"}


def run_recover(args):
    """Translations and landmarks of the solution (Eq. 7) with per-observation residual terms,
    and the XM^2 re-run (Sec. 5) on a workload: one certified solve, then W untimed and K timed
    xm_recover_tp calls and one timed xm_solve_xm2; prints one JSON line."""
    import torch
    from paper_2502_04640_b300 import xm
    mk, _, desc = WORKLOADS[args.workload]
    sc = mk()
    ctx = xm.Context(0)
    t = xm.scene_tensors(sc)
    wopts = WORKLOAD_OPTS.get(args.workload, {})
    q = xm.xm_build_Q(ctx, sc.N, sc.M, *t, xm.XM_STORE_ALL)
    out = xm.xm_solve(q, xm.xm_default_opts(prec=1, **wopts))
    q.free()
    for _ in range(args.warmup):
        xm.xm_recover_tp(ctx, sc.N, sc.M, *t, out["R"], out["s"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        tt, pp, res2 = xm.xm_recover_tp(ctx, sc.N, sc.M, *t, out["R"], out["s"])
    torch.cuda.synchronize()
    rec_s = (time.perf_counter() - t0) / args.steps
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    xm2 = {}
    try:
        x2 = xm.xm_solve_xm2(ctx, sc.N, sc.M, *t, xm.xm_default_opts(prec=1, **wopts))
        torch.cuda.synchronize()
        # cameras left in the solved component (an isolated camera comes back with zero scale)
        kept_cams = int((x2["s"] != 0).sum().item())
        xm2 = {"xm2_s": time.perf_counter() - t0, "xm2_first_certified": x2["info_first"]["certified"],
               "xm2_second_certified": x2["info_second"]["certified"],
               "xm2_kept": int(x2["keep"].sum().item()), "xm2_dropped": int((~x2["keep"]).sum().item()),
               "xm2_cameras_solved": kept_cams, "xm2_eta_second": x2["info_second"]["eta"],
               "xm2_solve_first_s": x2["info_first"]["t_solve_s"],
               "xm2_solve_second_s": x2["info_second"]["t_solve_s"],
               "xm2_sweeps_second": x2["info_second"]["n_sweeps"]}
    except xm.XmError as e:
        # dropping the largest residuals can leave a camera or landmark unobserved
        xm2 = {"xm2_status": xm.STATUS_NAMES.get(e.status, str(e.status)), "xm2_message": str(e)}
    cpu = None
    if not args.no_cpu:
        from oracle import xm_oracle as O
        sub = scenes.sub_scene(sc, min(60, sc.N))   # the oracle's sparse solve is slow: keep it bounded
        Q = O.build_Q_schur(sub.N, sub.M, sub.cam, sub.lmk, sub.ukp, sub.w)
        res = O.solve(Q, r0=4, mu=wopts.get("scale_reg", 0.0))
        U3 = np.concatenate([res.s[i] * res.R[i] for i in range(sub.N)], axis=1)
        c0 = time.perf_counter()
        O.recover_tp(sub.N, sub.M, sub.cam, sub.lmk, sub.ukp, sub.w, U3)
        cpu = {"value": time.perf_counter() - c0, "unit": "s per recovery", "cores": host_cores(),
               "kind": "oracle", "sample": f"oracle recover_tp on the first {sub.N} cameras "
                                           f"({sub.E} observations) of the workload"}
    print(json.dumps({"recover": True, "workload": f"{args.workload}: {desc}", "N": sc.N, "M": sc.M,
                      "E": sc.E, "steps": args.steps, "warmup": args.warmup,
                      "recover_tp_s": rec_s, "observations_per_s": sc.E / rec_s, **xm2,
                      "cpu_baseline": cpu}), flush=True)
    ctx.close()
    return 0


def run_adjoint(args):
    """Adjoint of the certified optimum on a workload (default: the 2000-frame trajectory):
    one certified FP32-bulk solve, then W untimed and K timed xm_backward calls per inner
    precision for L = <D, G> with a seeded D; prints one JSON line."""
    import torch
    from paper_2502_04640_b300 import xm
    mk, _, desc = WORKLOADS[args.workload]
    sc = mk()
    ctx = xm.Context(0)
    t = xm.scene_tensors(sc)
    q = xm.xm_build_Q(ctx, sc.N, sc.M, *t, xm.XM_STORE_ALL)
    wopts = WORKLOAD_OPTS.get(args.workload, {})
    out = xm.xm_solve(q, xm.xm_default_opts(prec=1, **wopts))
    r = out["info"]["rank"]
    D = torch.as_tensor(np.random.default_rng(5).standard_normal((sc.N, 3, 3)), device="cuda:0")
    res = {}
    for name, pv in (("fp32_refined", 1), ("fp64", 0)):
        opts = xm.xm_default_opts(prec=pv, **wopts)
        for _ in range(args.warmup):
            xm.xm_backward(q, out["Y"], r, sc.M, *t, D, opts)
        infos = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            infos.append(xm.xm_backward(q, out["Y"], r, sc.M, *t, D, opts)[3])
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / args.steps
        last = infos[-1]
        res[name] = {"s_per_backward": dt, "grads_per_s": sc.E * 4 / dt,
                     **{k: last[k] for k in ("res_rel", "n_refine", "n_cg", "n_sweeps_fp32",
                                             "n_sweeps_fp64", "t_lambda_s", "t_resid_s", "t_precond_s",
                                             "launches")}}
    cpu = None
    if not args.no_cpu:
        cpu = oracle_adjoint_sample(sc, wopts.get("scale_reg", 0.0))
    print(json.dumps({"adjoint": True, "workload": f"{args.workload}: {desc}", "opts": wopts, "N": sc.N, "M": sc.M,
                      "E": sc.E, "rank": r, "forward_solve_s": out["info"]["t_solve_s"],
                      "certified": out["info"]["certified"], "steps": args.steps,
                      "warmup": args.warmup, **res, "cpu_baseline": cpu}), flush=True)
    q.free()
    ctx.close()
    return 0


def run_spd_inverse(args):
    """xm_spd_inverse on A = G G^T / n + 0.05 I (G seeded standard normal, n x n FP32): W untimed
    and K timed calls (CUDA events on the context stream, a fresh copy of A before each), the
    residual A X - I in FP64 on 64 seeded columns; flops n^3 (n^3 / 2 multiply-adds), BF16 tensor
    flops 6 n^3 (six digit products per multiply-add)."""
    import torch
    from paper_2502_04640_b300 import xm
    n = args.spd_inverse
    ctx = xm.Context(0)
    g = torch.Generator(device="cuda").manual_seed(0)
    G = torch.randn(n, n, device="cuda", generator=g, dtype=torch.float32)
    A = torch.addmm(torch.eye(n, device="cuda"), G, G.T, beta=0.05, alpha=1.0 / n)
    A = 0.5 * (A + A.T)
    del G
    X = torch.empty_like(A)
    st = torch.cuda.current_stream()
    times = []
    for i in range(args.warmup + args.steps):
        X.copy_(A)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        xm.xm_spd_inverse(ctx, X)
        e1.record(st)
        torch.cuda.synchronize()
        if i >= args.warmup:
            times.append(e0.elapsed_time(e1) * 1e-3)
    idx = torch.randint(0, n, (64,), device="cuda", generator=torch.Generator(device="cuda").manual_seed(1))
    Rm = A.double() @ X[:, idx].double()
    Rm[idx, torch.arange(64, device="cuda")] -= 1.0
    t = statistics.median(times)
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            bf16, kind = float(json.load(fh)["bf16_tflops"]), "measured"
    except Exception:
        bf16, kind = 1800.0, "fallback"
    print(json.dumps({"spd_inverse": True, "n": n, "steps": args.steps, "warmup": args.warmup,
                      "s_median": t, "s_min": min(times), "launches": xm.xm_last_launch_count(),
                      "fp32_equiv_tflops": n ** 3 / t / 1e12, "bf16_tensor_tflops": 6 * n ** 3 / t / 1e12,
                      "bf16_peak_tflops": bf16, "peak_kind": kind,
                      "frac_of_bf16_peak": (6 * n ** 3 / t / 1e12) / bf16,
                      "residual_max": Rm.abs().max().item()}), flush=True)
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="c3", choices=sorted(WORKLOADS) + ["c5"])
    ap.add_argument("--prec", default="fp32", choices=sorted(PRECS))
    ap.add_argument("--impl", default="xm", choices=["xm", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-compare", action="store_true", help="skip the FP64 / BF16 comparison solves")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--profile-solve", action="store_true",
                    help="build Q and run exactly one solve inside the NVTX range 'timed' (profiler "
                         "launch lists); prints the solve's info")
    ap.add_argument("--bulk-stall", type=int, default=None, metavar="K",
                    help="opts.bulk_stall = K: hand the FP32 bulk phase to the FP64 polish after K "
                         "outer steps of stagnation (0: off)")
    ap.add_argument("--time-limit", type=float, default=0.0,
                    help="wall-clock cap of each solve in seconds (0: none)")
    ap.add_argument("--sweep-only", type=int, default=0, metavar="N",
                    help="time only the Q.Y sweep on a seeded random symmetric Q of N cameras "
                         "(the small case used for profiler captures)")
    ap.add_argument("--sweep-table", action="store_true",
                    help="with --sweep-only: also time every storage precision at r = 1, 4, 8")
    ap.add_argument("--build-only", type=int, default=0, metavar="N",
                    help="time only xm_build_Q (tensor-core and FP64 rank-k update) on a seeded random "
                         "scene of N cameras (also the small case for profiler captures)")
    ap.add_argument("--recover", action="store_true",
                    help="time xm_recover_tp (Eq. 7) and xm_solve_xm2 (Sec. 5) on --workload")
    ap.add_argument("--adjoint", action="store_true",
                    help="time xm_backward (the adjoint of the certified optimum) on --workload")
    ap.add_argument("--noise-sweep", action="store_true",
                    help="depth-noise robustness table (certified rate, eta, rotation and scale errors "
                         "across the noise levels of the paper's noise analysis)")
    ap.add_argument("--spd-inverse", type=int, default=0, metavar="n",
                    help="time only xm_spd_inverse (the adjoint preconditioner's dense inverse) on a "
                         "seeded SPD n x n FP32 matrix (n = 30465 is the 10155-camera size)")
    ap.add_argument("--no-others", action="store_true",
                    help="skip the other workloads (1934 cameras, trajectory + adjoint, batch) that the "
                         "default line measures after its timed region")
    args = ap.parse_args()
    if args.adjoint:
        return run_adjoint(args)
    if args.noise_sweep:
        from paper_2502_04640_b300 import xm
        ctx = xm.Context(0)
        print(json.dumps({"noise_sweep": True, **depth_noise_table(ctx)}), flush=True)
        ctx.close()
        return 0
    if args.recover:
        return run_recover(args)
    if args.spd_inverse:
        return run_spd_inverse(args)

    if args.warmup < 3 and not args.profile_solve:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "c5":
        if int(os.environ.get("WORLD_SIZE", "1")) > 1:
            ap.error("--workload c5 runs on one GPU")
        return run_batched(args)
    if args.sweep_only:
        return run_sweep_only(args)
    if args.build_only:
        return run_build_only(args)

    import torch
    from paper_2502_04640_b300 import xm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"

    mk, _, desc = WORKLOADS[args.workload]
    sc = mk()    # every replica solves the same synthetic scene (replicas only: no exchange)
    ctx = xm.Context(local)
    prec = PRECS[args.prec]
    cam, lmk, ukp, w = xm.scene_tensors(sc, local)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    q = xm.xm_build_Q(ctx, sc.N, sc.M, cam, lmk, ukp, w, xm.XM_STORE_ALL)
    torch.cuda.synchronize()
    t_build = time.perf_counter() - t0
    build_path, t_update = xm.xm_qmat_build_info(q)
    del cam, lmk, ukp, w
    torch.cuda.empty_cache()
    wopts = dict(WORKLOAD_OPTS.get(args.workload, {}))
    wopts.update(SOLVE_OPTS.get(args.workload, {}))
    if args.bulk_stall is not None:
        wopts["bulk_stall"] = args.bulk_stall
    opts = xm.xm_default_opts(prec=prec, time_limit_s=args.time_limit, **wopts)
    stream = ctx.stream

    if args.profile_solve:
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")
        o = xm.xm_solve(q, opts)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        print(json.dumps({"profile_solve": True, "launches": xm.xm_last_launch_count(), **o["info"]}))
        q.free()
        ctx.close()
        return 0
    for _ in range(args.warmup):
        xm.xm_solve(q, opts)
    # ---- timed region: exactly K certified solves
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    ev0.record(stream)
    wall0 = time.perf_counter()
    launches = 0
    timed = []
    out = None
    per_step = []
    for _ in range(args.steps):
        ts = time.perf_counter()
        out = xm.xm_solve(q, opts)     # synchronises before returning
        per_step.append(time.perf_counter() - ts)
        launches += xm.xm_last_launch_count()
        timed.append(out["info"])
    ev1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    clk = clocks.stop()
    dev_s = ev0.elapsed_time(ev1) / 1e3
    value = whole_job_seconds(max(dev_s, wall), args.steps, world, dist, dev)
    info = timed[-1]
    certified = all(i["certified"] for i in timed)

    # ---- roofline of the dominant kernel, from the sweeps timed live inside the solves
    n = q.n
    key = "qy_ms_fp64" if prec == 0 else "qy_ms_fp32"
    live = [i[key] for i in timed if i[key] > 0]
    qy_ms = statistics.mean(live) if live else float("nan")
    bq, by = (8, 8) if prec == 0 else (4, 4)
    alg = sweep_bytes(n, 4, bq, by)
    peak, peak_kind = peaks()
    achieved = alg / (qy_ms * 1e-3) / 1e9
    measured_here = prec == 1 and SWEEP_TRAFFIC_RATIO and n == SWEEP_TRAFFIC_N
    traffic = alg * SWEEP_TRAFFIC_RATIO if measured_here else None
    roofline = {"bound": "hbm" if prec != 0 else "alu", "achieved": achieved, "peak": peak,
                "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                "traffic_note": "ncu DRAM read+write of one launch at n = 30465 (this sweep "
                                "size), as a ratio to the algorithmic bytes" if traffic else
                                "no ncu DRAM capture at this size",
                "kernel": f"qy_packed_kernel<{'double' if prec == 0 else 'float'},4,8>",
                "bytes_per_launch": alg, "launch_ms": qy_ms, "peak_kind": peak_kind}

    extra = {}
    if rank == 0 and not args.no_compare:
        # plain FP64 GPU form and the BF16-Q trial, one solve each, errors against the FP64 run
        ref = xm.xm_solve(q, xm.xm_default_opts(prec=0, **wopts))
        fi = ref["info"]
        extra["fp64_solve_s"] = fi["t_solve_s"]
        extra["fp64_certified"] = fi["certified"]
        extra["fp64_sweeps"] = fi["n_sweeps"]

        def errs(o):
            return {"f_rel": abs(o["info"]["f"] - fi["f"]) / (1 + abs(fi["f"])),
                    "rho_hat_rel": abs(o["info"]["rho_hat"] - fi["rho_hat"]) / (1 + abs(fi["rho_hat"])),
                    "lambda_min_abs": abs(o["info"]["lambda_min_deflated"] - fi["lambda_min_deflated"]),
                    "R_max_abs": float((o["R"] - ref["R"]).abs().max()),
                    "s_max_rel": float(((o["s"] - ref["s"]).abs() / ref["s"].abs()).max())}
        extra["fp32_vs_fp64"] = errs(out)
        # the plain FP64 form on the factored operator alone (Q never formed)
        try:
            qf = xm.xm_build_Q(ctx, sc.N, sc.M, *xm.scene_tensors(sc, local), xm.XM_STORE_FACTORED)
            ff = xm.xm_solve(qf, xm.xm_default_opts(prec=0, **wopts))
            extra["fp64_factored_solve_s"] = ff["info"]["t_solve_s"]
            extra["fp64_factored_certified"] = ff["info"]["certified"]
            extra["fp64_factored_vs_fp64"] = errs(ff)
            qf.free()
        except Exception as e:      # noqa: BLE001 - reported, the main number stands
            extra["fp64_factored_error"] = f"{type(e).__name__}: {e}"
        if prec != 2:
            b = xm.xm_solve(q, xm.xm_default_opts(prec=2, **wopts))
            extra["bf16q_solve_s"] = b["info"]["t_solve_s"]
            extra["bf16q_certified"] = b["info"]["certified"]
            extra["bf16q_vs_fp64"] = errs(b)
        try:
            extra["factored_qy"] = factored_measure(ctx, sc, q)
        except Exception as e:      # noqa: BLE001 - reported, the main number stands
            extra["factored_qy"] = {"error": f"{type(e).__name__}: {e}"}
        for pname, pv in (("fp32", 1), ("bf16", 2), ("fp64", 0)):
            mean_ms, _ = xm.xm_bench_qy(q, pv, 4, 10)
            bqq = {1: 4, 2: 2, 0: 8}[pv]
            byy = 8 if pv == 0 else 4
            extra[f"qy_{pname}_r4_ms"] = mean_ms
            extra[f"qy_{pname}_r4_GBps"] = sweep_bytes(n, 4, bqq, byy) / (mean_ms * 1e-3) / 1e9

    # ---- end to end through the C ABI from pinned host arrays (H2D, build, solve, D2H)
    e2e = None
    q.free()
    if rank == 0 and args.e2e_steps > 0:
        def pin(a, dt):
            return torch.from_numpy(np.ascontiguousarray(a)).to(dt).pin_memory()
        hc, hl = pin(sc.cam, torch.int32), pin(sc.lmk, torch.int32)
        hu, hw = pin(sc.ukp, torch.float64), pin(sc.w, torch.float64)
        Rh = torch.zeros((sc.N, 3, 3), dtype=torch.float64).pin_memory()
        sh = torch.zeros(sc.N, dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        te = time.perf_counter()
        for _ in range(args.e2e_steps):
            xm.xm_pipeline_host_ptrs(ctx, sc.N, sc.M, hc, hl, hu, hw, opts, Rh, sh)
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - te) / args.e2e_steps
        e2e = {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(sc.E * (4 + 4 + 24 + 8)),
               "d2h_bytes_per_step": int(sc.N * (72 + 8))}

    others = None
    if rank == 0 and not args.no_others:
        others = other_workloads(ctx, steps=3)

    cpu = None
    if rank == 0 and not args.no_cpu:
        dt = oracle_sweep_seconds(n, 4, reps=2)
        S = int(info["n_sweeps"])
        cpu = {"value": dt * S, "unit": "s", "cores": host_cores(), "kind": "oracle",
               "sample": f"two oracle sweeps (dense FP64 Q@Y, n={n}, r=4, dual blocks, projection) "
                         f"timed, times the {S} sweeps of this certified solve"}

    qb = n * (n + 1) / 2 * {0: 8, 1: 4, 2: 2}[prec]
    l2_label = (f"inputs larger than L2 (packed Q {qb / 1e9:.2f} GB > 126 MB)" if qb > L2_BYTES else
                f"L2-resident: packed Q {qb / 1e6:.0f} MB < 126 MB L2 (not flushed between solves)")
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": value * 1e3 * world, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[args.prec], "data": "synthetic",
            "config": {"workload": f"{args.workload}: {desc}", "prec": args.prec, "opts": wopts,
                       "replicas": world, "l2": l2_label, "N": sc.N, "M": sc.M, "E": sc.E},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
            "certified": certified,
            "solve": {k: info[k] for k in ("f", "grad_norm", "lambda_min", "lambda_min_deflated",
                                           "lambda_max", "dual", "rho_hat", "eta", "eta_robust", "rank",
                                           "n_sweeps", "n_sweeps_fp64", "n_outer", "n_tcg",
                                           "n_lanczos", "n_escapes", "t_cert_s")},
            "step_s": {"mean": statistics.mean(per_step), "median": statistics.median(per_step),
                       "p90": _pct(per_step, 90), "min": min(per_step), "max": max(per_step)},
            "per_step": [{"s": round(t, 4), "n_tcg": i["n_tcg"], "n_outer": i["n_outer"],
                          "n_sweeps": i["n_sweeps"], "t_cert_s": round(i["t_cert_s"], 4),
                          "certified": i["certified"]} for t, i in zip(per_step, timed)],
            "build_q_s": t_build,
            "build_update": update_report(sc.N, build_path, t_update),
            **extra,
        }
        if others is not None:
            line["other_workloads"] = others
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    ctx.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
