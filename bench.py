#!/usr/bin/env python
"""Benchmark of the fast directional Burton-Miller BEM on GB300.

Workload: rigid unit sphere, icosphere level 7 (327,680 flat triangles,
collocation at centroids), k = 50 (kD = 100), plane wave along +z, octree
leaves <= 64 elements, SVD threshold eps = 1e-4, GMRES tolerance 1e-4.
Synthetic input: the icosphere stands in for the paper's sphere meshes.

A timed step is one FDA matrix-vector product (Steps 2-4 of the paper's
algorithm: near field, S2M, M2M, M2L, L2L, L2T) through the C ABI on inputs
resident in HBM.  `value` is FDA matvec/s of the chosen form (FP32 far field
and FP32 near-field storage); the JSON line also carries the plain FP64
matvec rate, the setup time (tree, lists, quadrature, SVD precompute) and
GMRES solve seconds of both forms at 1e-4, with the FP64 residual.

`--impl reference` times the FP64 CPU oracle (dense on-the-fly matvec) on a
bounded sample of rows of the same workload, on the host cores.
"""
from __future__ import annotations

import argparse
import datetime
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FDA matvec/s & GMRES solve s, kD=100 N=327,680, plain vs chosen form @1e-4"
WORKLOAD = "rigid unit sphere, icosphere level 7 (327,680 triangles), k=50 (kD=100), plane wave +z, eps=1e-4"


def _workload(args, n):
    """The headline workload's name, or the same description for another
    --level / --k / --eps."""
    if (args.level, args.k, args.eps) == (7, 50.0, 1e-4):
        return WORKLOAD
    return "rigid unit sphere, icosphere level %d (%s triangles), k=%g (kD=%g), plane wave +z, eps=%g" % (
        args.level, format(n, ","), args.k, 2 * args.k, args.eps)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class RankGroup:
    """One process per GPU (torchrun): barrier and max over ranks.  NCCL
    between GPUs, gloo on CPU (the same code path the tests run)."""

    def __init__(self, backend=None):
        self.ws, self.rank, self.local = _dist()
        self.dist = None
        self.backend = backend
        if self.ws > 1:
            import torch
            import torch.distributed as dist
            if self.backend is None:
                self.backend = "nccl" if torch.cuda.is_available() else "gloo"
            dist.init_process_group(self.backend)
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max(self, v):
        if self.dist is None:
            return v
        import torch
        dev = "cuda" if self.backend == "nccl" else "cpu"
        t = torch.tensor([float(v)], dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()
            self.dist = None


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.p = None
        self.path = os.path.join("/tmp", "fda_clocks_%d_%d.csv" % (os.getpid(), gpu_index))

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                                       "--format=csv,noheader,nounits", "-lms", "20"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def mark(self, which):
        """Wall-clock start or end of the timed region (samples outside it are dropped)."""
        setattr(self, which, datetime.datetime.now())

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0, t1 = getattr(self, "t_begin", None), getattr(self, "t_end", None)
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f")
                if t0 is not None and t1 is not None and not (t0 <= ts <= t1):
                    continue
                sm.append(float(parts[2]))
                smax.append(float(parts[3]))
            except ValueError:
                continue
            for n, v in zip(names, parts[6:10]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def _cpu_oracle_rate(v, f, k, x, rows_n, seed=7):
    """Oracle matvec rate on sampled rows (matvec/s equivalent); also returns
    the rows and the oracle's values there, for the GPU results' error."""
    import numpy as np
    import oracle
    rows = np.random.default_rng(seed).choice(len(f), rows_n, replace=False)
    t0 = time.perf_counter()
    ref = oracle.matvec(v, f, k, x, rows=rows)
    dt = time.perf_counter() - t0
    return (rows_n / len(f)) / dt, dt, oracle.num_threads(), rows, ref


def _rel(a, b):
    import numpy as np
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    from inputs import icosphere, complex_normal
    v, f = icosphere(args.level)
    n = len(f)
    x = complex_normal(n, seed=1234)
    # rows per step: at most --ref-rows, and about 10,000 rows over the run so
    # that any --steps finishes within a few minutes on the host cores
    rows_n = max(16, min(args.ref_rows, 10000 // max(1, args.steps)))
    rows = np.random.default_rng(7).choice(n, rows_n, replace=False)
    oracle.load()
    for _ in range(args.warmup):
        oracle.matvec(v, f, args.k, x, rows=rows[:max(1, rows_n // 8)])
    t0 = time.perf_counter()
    for s in range(args.steps):
        r = np.random.default_rng(100 + s).choice(n, rows_n, replace=False)
        oracle.matvec(v, f, args.k, x, rows=r)
    dt = time.perf_counter() - t0
    value = args.steps * (rows_n / n) / dt
    cores = oracle.num_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "matvec/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": _workload(args, n), "N": n, "k": args.k},
            "cpu_baseline": {"kind": "oracle", "value": value, "unit": "matvec/s", "cores": cores,
                             "sample": "%d sampled rows of the dense FP64 oracle matvec per step (of %d)" % (rows_n, n)},
            "e2e": {"value": value, "unit": "matvec/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_native(args):
    import numpy as np
    import torch

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    group = RankGroup()
    from paper_1403_4747_gb300 import build as lib_build
    lib_build.build()
    import paper_1403_4747_gb300 as F
    from inputs import icosphere, complex_normal
    barrier, reduce_max = group.barrier, group.max

    v, f = icosphere(args.level)
    n = len(f)
    k = args.k
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    P = F.FDAProblem(v, f, k, stream=stream, precision=F.FDA_CHOSEN_FP32, eps=args.eps,
                     precond=0 if args.no_precond else 1, restart=args.restart, max_rhs=max(1, args.batch))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    st = P.stats()
    nlev = st.n_levels

    x = torch.from_numpy(complex_normal(n, seed=1234)).cuda()
    y = torch.empty_like(x)
    for _ in range(args.warmup):
        P.apply(x, y)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nl0 = F.fda_launch_count()
    gr0 = P.stats().graph_replays
    clocks.mark("t_begin")
    e0.record(stream)
    for _ in range(args.steps):
        P.apply(x, y)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks.mark("t_end")
    launches = F.fda_launch_count() - nl0
    graph_replays = P.stats().graph_replays - gr0
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms = reduce_max(ms)
    value = ws * 1e3 / ms
    y_chosen = y.cpu().numpy()

    # end to end through the C ABI with host buffers (pinned)
    xh = torch.from_numpy(complex_normal(n, seed=99)).pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    F.fda_apply_host(P.h, xh.data_ptr(), yh.data_ptr(), 1, n)
    te = time.perf_counter()
    ne = max(3, args.steps // 2)
    for _ in range(ne):
        F.fda_apply_host(P.h, xh.data_ptr(), yh.data_ptr(), 1, n)
    e2e_ms = reduce_max((time.perf_counter() - te) / ne * 1e3)

    # per-pass device times (CUDA events recorded by the library on its stream)
    def pass_times(reps):
        F.fda_set_timing(P.h, True)
        acc = np.zeros(6)
        for _ in range(reps):
            P.apply(x, y)
            acc += np.array(F.fda_get_pass_times(P.h))
        F.fda_set_timing(P.h, False)
        return acc / reps

    pt32 = pass_times(5)
    # the same passes with the FP32 SIMT M2L, for comparison
    F.fda_set_tensor_cores(P.h, 0)
    pt32_simt = pass_times(3)
    F.fda_set_tensor_cores(P.h, 1)
    F.fda_set_precision(P.h, F.FDA_PLAIN_FP64)
    P.apply(x, y)
    torch.cuda.synchronize()
    tp = time.perf_counter()
    nplain = max(1, args.plain_steps)
    for _ in range(nplain):
        P.apply(x, y)
    torch.cuda.synchronize()
    plain_ms = (time.perf_counter() - tp) / nplain * 1e3
    y_plain = y.cpu().numpy()
    pt64 = pass_times(1)
    F.fda_set_precision(P.h, F.FDA_CHOSEN_FP32)

    # the same workload with every reduced M2L operator applied in full
    # (Sec. 4.2's low-rank step off), for comparison
    lowrank_off = None
    if not args.no_lowrank_off:
        t0 = time.perf_counter()
        Q = F.FDAProblem(v, f, k, stream=stream, precision=F.FDA_CHOSEN_FP32, eps=args.eps, lowrank=0,
                         max_rhs=1)
        torch.cuda.synchronize()
        setup_off = time.perf_counter() - t0
        for _ in range(3):
            Q.apply(x, y)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(20):
            Q.apply(x, y)
        e1.record(stream)
        torch.cuda.synchronize()
        off_ms = e0.elapsed_time(e1) / 20
        F.fda_set_timing(Q.h, True)
        acc = np.zeros(6)
        for _ in range(5):
            Q.apply(x, y)
            acc += np.array(F.fda_get_pass_times(Q.h))
        F.fda_set_timing(Q.h, False)
        F.fda_set_precision(Q.h, F.FDA_PLAIN_FP64)
        Q.apply(x, y)
        torch.cuda.synchronize()
        tq = time.perf_counter()
        for _ in range(max(1, args.plain_steps)):
            Q.apply(x, y)
        torch.cuda.synchronize()
        off_plain_ms = (time.perf_counter() - tq) / max(1, args.plain_steps) * 1e3
        lowrank_off = {"ms_per_matvec": off_ms, "matvec_per_s": 1e3 / off_ms, "setup_s": setup_off,
                       "chosen_pass_ms": dict(zip(["s2m", "m2m", "m2l", "l2l", "l2t", "near"], (acc / 5).tolist())),
                       "m2l_bytes": _m2l_bytes(Q), "m2l_flops": _m2l_flops(Q),
                       "plain_fp64_ms_per_matvec": off_plain_ms}
        Q.close()
        del Q
        torch.cuda.empty_cache()

    # many right-hand sides per pass (incidence directions): every operator
    # read serves all of them
    batched = None
    if args.batch > 1:
        xb = torch.from_numpy(complex_normal(n, seed=77, nrhs=args.batch)).cuda()
        yb = torch.empty_like(xb)
        for _ in range(2):
            P.apply(xb, yb)
        torch.cuda.synchronize()
        nb_steps = max(3, args.steps // 4)
        e0.record(stream)
        for _ in range(nb_steps):
            P.apply(xb, yb)
        e1.record(stream)
        torch.cuda.synchronize()
        bms = reduce_max(e0.elapsed_time(e1) / nb_steps)
        F.fda_set_timing(P.h, True)
        P.apply(xb, yb)
        bpt = np.array(F.fda_get_pass_times(P.h))
        F.fda_set_timing(P.h, False)
        m2l_b = _m2l_flops(P) * args.batch
        batched = {"nrhs": args.batch, "ms_per_pass": bms,
                   "rhs_matvec_per_s": ws * args.batch * 1e3 / bms,
                   "pass_ms": dict(zip(["s2m", "m2m", "m2l", "l2l", "l2t", "near"], bpt.tolist())),
                   "m2l_tflops": m2l_b / (bpt[2] * 1e-3) / 1e12}
        del xb, yb

    # roofline of the dominant kernel: the tensor-core translation kernel in
    # the M2L pass (all levels).  Algorithmic work of one apply: every
    # distinct compressed operator read once (8 bytes per complex entry, FP32
    # or bf16 hi + lo), the source densities read once and the target
    # densities read and written once; 8 real flops per complex
    # multiply-add.  The binding roof is the larger of bytes / HBM peak and
    # flops / bf16 peak.
    peaks, src = _peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    fp32_peak_tflops = nsm * 128 * 2 * sm_mhz * 1e6 / 1e12
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    bf16_peak = float(peaks.get("bf16_tflops", 1900.0))
    m2l_flops = _m2l_flops(P)
    m2l_bytes = _m2l_bytes(P)
    m2l_ms = pt32[2]
    t_hbm, t_tc = m2l_bytes / (hbm_peak * 1e9), m2l_flops / (bf16_peak * 1e12)
    m2l_gbs = m2l_bytes / (m2l_ms * 1e-3) / 1e9
    m2l_tflops = m2l_flops / (m2l_ms * 1e-3) / 1e12
    if t_hbm >= t_tc:
        roofline = {"bound": "hbm", "achieved": m2l_gbs, "peak": hbm_peak, "unit": "GB/s",
                    "frac": m2l_gbs / hbm_peak}
    else:
        roofline = {"bound": "tensor", "achieved": m2l_tflops, "peak": bf16_peak, "unit": "TFLOP/s",
                    "frac": m2l_tflops / bf16_peak}
    roofline.update({
        "traffic": _m2l_traffic(args),
        "kernel": "k_btr_tc (tcgen05 gather-GEMM-scatter), M2L launches of one apply (one per level)",
        "peak_source": "MEASURED_PEAKS.json (%s): hbm_gbs %.0f, bf16_tflops %.1f (burst)" % (src, hbm_peak, bf16_peak),
        "ms_per_apply": m2l_ms,
        "algorithmic_bytes_per_apply": m2l_bytes,
        "algorithmic_flops_per_apply": m2l_flops,
        "tensor": {"achieved_tflops": m2l_tflops, "frac_of_bf16": m2l_tflops / bf16_peak,
                   "executed_tflops": 3 * m2l_flops / (m2l_ms * 1e-3) / 1e12,
                   "note": "split bf16 executes 3 products per multiply-add"},
        "simt_fp32_m2l": {"ms": pt32_simt[2], "achieved_tflops": m2l_flops / (pt32_simt[2] * 1e-3) / 1e12,
                          "peak": fp32_peak_tflops,
                          "frac": m2l_flops / (pt32_simt[2] * 1e-3) / 1e12 / fp32_peak_tflops,
                          "peak_source": "FP32 FMA rate: %d SMs x 128 lanes x 2 flops x %.0f MHz" % (nsm, sm_mhz)}})
    near_bytes = 8 * st.nnz_near + 24 * n  # FP32 entries read once; x read and y written once
    near_gbs = near_bytes / (pt32[5] * 1e-3) / 1e9
    near_roof = {"kernel": "k_near_apply", "bound": "hbm", "achieved": near_gbs, "peak": hbm_peak, "unit": "GB/s",
                 "frac": near_gbs / hbm_peak, "ms_per_apply": pt32[5], "algorithmic_bytes_per_apply": near_bytes}

    solve = {}
    u_chosen = b_host = None
    if not args.no_solve:
        b = P.rhs_plane_wave(np.array([0.0, 0.0, 1.0]))
        b_host = b.cpu().numpy()
        runs = [("chosen", F.FDA_CHOSEN_FP32, 0)]
        if not args.no_plain_unpreconditioned:
            runs.append(("plain", F.FDA_PLAIN_FP64, 0))
        for name, prec, pc in runs:
            F.fda_set_precision(P.h, prec)
            F.fda_set_precond(P.h, pc)
            torch.cuda.synchronize()
            ts = time.perf_counter()
            xs, info = P.solve(b, args.tol, raise_on_not_converged=False)
            torch.cuda.synchronize()
            if name == "chosen":
                u_chosen = xs.cpu().numpy()
            solve[name] = {"solve_s": time.perf_counter() - ts, "iters": info.iters,
                           "refinements": info.refinements, "rel_resid_fp64": info.rel_resid_fp64,
                           "matvec_s": info.matvec_s, "precond": ["none", "blockdiag"][pc]}
        F.fda_set_precision(P.h, F.FDA_CHOSEN_FP32)
        F.fda_set_precond(P.h, 0)
        if not args.no_precond:
            solve["preconditioners"] = _precond_block(F, P, b, args)
        if "plain" in solve and solve["chosen"]["solve_s"] > 0:
            solve["speedup_chosen_over_plain"] = solve["plain"]["solve_s"] / solve["chosen"]["solve_s"]
        solve["setup_s"] = setup_s
        solve["restart"] = args.restart
        solve["coupling"] = "alpha = -i/k with the normal into the body (library default; the paper's operator)"
        if not args.no_alt_coupling:
            # the coupling as printed, alpha = +i/k: same scattering problem,
            # sphere eigenvalues around 0, many more iterations
            P.close()
            t0 = time.perf_counter()
            Q = F.FDAProblem(v, f, k, stream=stream, precision=F.FDA_CHOSEN_FP32, eps=args.eps, alpha_sign=1.0,
                             restart=args.restart)
            torch.cuda.synchronize()
            setup_q = time.perf_counter() - t0
            bq = Q.rhs_plane_wave(np.array([0.0, 0.0, 1.0]))
            alt = {}
            forms = [("chosen", F.FDA_CHOSEN_FP32)] + ([("plain", F.FDA_PLAIN_FP64)] if args.alt_plain else [])
            for name, prec in forms:
                F.fda_set_precision(Q.h, prec)
                torch.cuda.synchronize()
                ts = time.perf_counter()
                xq, info = Q.solve(bq, args.tol, raise_on_not_converged=False)
                torch.cuda.synchronize()
                alt[name] = {"solve_s": time.perf_counter() - ts, "iters": info.iters,
                             "refinements": info.refinements, "rel_resid_fp64": info.rel_resid_fp64}
            alt["setup_s"] = setup_q
            if "plain" in alt:
                alt["speedup_chosen_over_plain"] = alt["plain"]["solve_s"] / max(alt["chosen"]["solve_s"], 1e-9)
            solve["printed_coupling_plus_i_over_k"] = alt
            Q.close()
            P = None

    cpu = None
    err = None
    if rank == 0 and not args.no_cpu:
        import oracle
        xc = complex_normal(n, seed=1234)
        rate, dt, cores, rows, ref = _cpu_oracle_rate(v, f, k, xc, args.cpu_rows)
        cpu = {"value": rate, "unit": "matvec/s", "cores": cores, "kind": "oracle",
               "sample": "%d random rows of the dense FP64 oracle matvec (of %d), %.1f s" % (args.cpu_rows, n, dt)}
        # the timed GPU products against the same oracle rows (same x)
        err = {"rows": int(args.cpu_rows), "row_seed": 7, "metric": "relative L2 over the sampled rows",
               "chosen_matvec": _rel(y_chosen[rows], ref), "plain_matvec": _rel(y_plain[rows], ref)}
        if u_chosen is not None:
            # the chosen solve's solution: residual b - A u with the oracle's A on
            # the first 256 sampled rows, and its distance to the Mie series
            r2 = rows[:256]
            err["solution_oracle_residual"] = _rel(oracle.matvec(v, f, k, u_chosen, rows=r2), b_host[r2])
            c = np.mean(v[f], axis=1)
            err["solution_vs_mie"] = _rel(u_chosen, oracle.mie_surface_field(k, c[:, 2] / np.linalg.norm(c, axis=1)))

    if cpu is not None and solve and "plain" in solve:
        # the oracle's matrix-free GMRES at this size, from its matvec rate and
        # the FP64 solve's iteration count (too long to run: days)
        cpu["solve_s_extrapolated"] = solve["plain"]["iters"] / cpu["value"]
    line = {"metric": METRIC, "value": value, "unit": "matvec/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": _workload(args, n), "N": n, "k": k, "eps": args.eps, "leaf_max": 64,
                       "form": "chosen (FP32 far field and near storage, FP64 setup)",
                       "l2": "inputs larger than L2 (near-field matrix %.2f GB FP32)" % (st.bytes_near / 2 / 1e9),
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "e2e": {"value": ws * 1e3 / e2e_ms, "unit": "matvec/s", "h2d_bytes_per_step": 16 * n,
                    "d2h_bytes_per_step": 16 * n},
            "gpu_launches": launches,
            "cuda_graph_replays": graph_replays,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "clocks": clk,
            "plain_fp64": {"matvec_per_s": 1e3 / plain_ms, "ms_per_matvec": plain_ms,
                           "pass_ms": dict(zip(["s2m", "m2m", "m2l", "l2l", "l2t", "near"], pt64.tolist()))},
            "chosen_pass_ms": dict(zip(["s2m", "m2m", "m2l", "l2l", "l2t", "near"], pt32.tolist())),
            "chosen_simt_m2l_pass_ms": dict(zip(["s2m", "m2m", "m2l", "l2l", "l2t", "near"], pt32_simt.tolist())),
            "err_vs_oracle": err,
            "near_field_roofline": near_roof,
            "batched_rhs": batched,
            "lowrank_off": lowrank_off,
            "solve": solve,
            "tree": {"levels": nlev, "boxes": st.n_boxes, "leaves": st.n_leaves, "nnz_near": st.nnz_near,
                     "m2l_pairs": st.n_m2l, "m2l_ops": st.n_m2l_ops,
                     "rank_per_level": [st.level_rank[l] for l in range(nlev)],
                     "regime_per_level": [st.level_regime[l] for l in range(nlev)],
                     "cones_per_level": [st.level_cones[l] for l in range(nlev)],
                     "m2l_pairs_per_level": [st.level_m2l_pairs[l] for l in range(nlev)],
                     "m2l_ops_per_level": [st.level_m2l_ops[l] for l in range(nlev)],
                     "lowrank_ops_per_level": [st.level_lr_ops[l] for l in range(nlev)],
                     "lowrank_pairs_per_level": [st.level_lr_pairs[l] for l in range(nlev)],
                     "lowrank_rank_mean_per_level": [round(st.level_lr_rank_mean[l], 1) for l in range(nlev)],
                     "lowrank_rank_max_per_level": [st.level_lr_rank_max[l] for l in range(nlev)],
                     "lowrank_tc_form_per_level": [st.level_lr_tc[l] for l in range(nlev)],
                     "tc_shape_m2m_m2l_l2l_per_level": [list(st.level_tc_shape[l]) for l in range(nlev)],
                     "device_gb": st.device_bytes / 1e9}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if P is not None:
        P.close()
    group.close()
    return 0


def _precond_block(F, P, b, args):
    """GMRES in the chosen form (the headline's coupling and tolerance) with
    no preconditioner, the leaf block-diagonal inverse, and the learned
    network on the near-field pattern trained on this mesh's own near-field
    matrix (Adam, 64 leaves per step, weights seed 1); times include neither
    training nor setting M, which are reported beside them."""
    import torch
    w = F.fda_sai_init_weights(1)
    cfg = F.fda_sai_default_config(epochs=args.sai_epochs, pattern=1, sample_leaves=64)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rep = F.fda_sai_train([P.h], cfg, w)
    train_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    F.fda_sai_set_pattern(P.h, w, 1, want_loss=False)
    torch.cuda.synchronize()
    set_s = time.perf_counter() - t0
    out = {}
    x_ref = None
    for name, pc in (("none", 0), ("blockdiag", 1), ("learned_near", 2)):
        F.fda_set_precond(P.h, pc)
        torch.cuda.synchronize()
        ts = time.perf_counter()
        x, info = P.solve(b, args.tol, raise_on_not_converged=False)
        torch.cuda.synchronize()
        if x_ref is None:
            x_ref = x.clone()
        out[name] = {"iters": info.iters, "solve_s": time.perf_counter() - ts, "rel_resid_fp64": info.rel_resid_fp64,
                     "diff_vs_none": float((x - x_ref).norm() / x_ref.norm())}
    F.fda_set_precond(P.h, 0)
    out["learned_near_setup"] = {"epochs": args.sai_epochs, "sample_leaves": 64, "loss_init": rep.loss_init,
                                 "loss_final": rep.loss_final, "train_s": train_s, "set_s": set_s,
                                 "note": "loss on one fixed draw of 64 leaves, before and after training"}
    return out


def _m2l_traffic(args):
    """DRAM bytes of the M2L pass per matvec from the committed ncu summary
    (sphere level 7, k = 50, eps 1e-4), or None for another workload or if the
    kernel's source (the k_btr_tc template and the tcgen05 helpers) changed
    since the counters were taken."""
    import hashlib
    if (args.level, args.k, args.eps) != (7, 50.0, 1e-4):
        return None
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "k_btr_tc_traffic_sphere_l7_k50.json")))
        csrc = os.path.join(ROOT, "paper_1403_4747_gb300", "csrc")
        lines = open(os.path.join(csrc, "translate_tc.cu")).read().split("\n")
        i = [j for j, s in enumerate(lines) if "k_btr_tc(const tc_tile" in s][0] - 1
        e = next(j for j in range(i, len(lines)) if lines[j] == "}")
        src = "\n".join(lines[i:e + 1]) + "\n" + open(os.path.join(csrc, "tc_util.cuh")).read()
        if hashlib.sha256(src.encode()).hexdigest()[:16] != rec["source_sha256_16"]:
            return None
        return rec["m2l_dram_bytes_per_matvec"]
    except Exception:
        return None


def _m2l_bytes(P):
    """Algorithmic bytes of the M2L pass per apply, as the library counts
    them from its batches: every operator applied read once (8 bytes per
    complex entry: T^2 in full form, 2 r T in the low-rank form of Sec. 4.2
    with the operator's own rank r), source densities read once, target
    densities read and written once, each low-rank pair's intermediate
    written and read once."""
    st = P.stats()
    return int(sum(st.level_m2l_bytes[l] for l in range(st.n_levels)))


def _m2l_flops(P):
    """Real flops of the M2L pass per apply that the method performs: 8 T^2
    per pair in full form, 8 (2 r T) per pair in low-rank form."""
    st = P.stats()
    return int(sum(st.level_m2l_flops[l] for l in range(st.n_levels)))


def run_many_meshes(args):
    """Eight meshes (sphere and ellipsoid icospheres, levels 5-7, kD 20-100)
    times 64 plane-wave directions behind one batch apply per step: one CUDA
    graph per step, one branch per mesh.  Reports (mesh x right-hand side)
    matvecs per second.  Not the headline workload; run with
    --workload many_meshes."""
    import numpy as np
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    group = RankGroup()
    from paper_1403_4747_gb300 import build as lib_build
    lib_build.build()
    import paper_1403_4747_gb300 as F
    from inputs import multi_mesh_set, complex_normal
    mm = multi_mesh_set()
    nrhs = args.batch
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    B = F.FDABatch([(v, f) for v, f, _ in mm], [k for _, _, k in mm], stream=stream,
                   precision=F.FDA_CHOSEN_FP32, eps=args.eps, max_rhs=nrhs)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    xs = [torch.from_numpy(complex_normal(len(f), seed=500 + i, nrhs=nrhs)).cuda() for i, (v, f, _) in enumerate(mm)]
    ys = [torch.empty_like(x) for x in xs]
    for _ in range(max(3, args.warmup)):
        B.apply(xs, ys)
    torch.cuda.synchronize()
    steps = max(3, args.steps // 20)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    group.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nl0 = F.fda_launch_count()
    gr0 = B.stats().graph_replays
    clocks.mark("t_begin")
    e0.record(stream)
    for _ in range(steps):
        B.apply(xs, ys)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks.mark("t_end")
    launches = F.fda_launch_count() - nl0
    st = B.stats()
    group.barrier()
    clk = clocks.stop()
    ms = group.max(e0.elapsed_time(e1) / steps)
    # each mesh alone through its own handle, for comparison with the batch
    alone_ms = []
    for i in range(len(mm)):
        h = B.mesh(i)
        n = len(mm[i][1])
        F.fda_apply(h, xs[i].data_ptr(), ys[i].data_ptr(), nrhs, n)
        F.fda_apply(h, xs[i].data_ptr(), ys[i].data_ptr(), nrhs, n)
        torch.cuda.synchronize()
        e0.record(stream)
        F.fda_apply(h, xs[i].data_ptr(), ys[i].data_ptr(), nrhs, n)
        e1.record(stream)
        torch.cuda.synchronize()
        alone_ms.append(e0.elapsed_time(e1))
    # one right-hand side per mesh: the batch's graph branches against the
    # meshes' own graph replays one after another
    x1 = [x[:1].contiguous() for x in xs]
    y1 = [torch.empty_like(x) for x in x1]
    for _ in range(3):
        B.apply(x1, y1)
        for i in range(len(mm)):
            F.fda_apply(B.mesh(i), x1[i].data_ptr(), y1[i].data_ptr(), 1, len(mm[i][1]))
    torch.cuda.synchronize()
    reps = 20
    e0.record(stream)
    for _ in range(reps):
        B.apply(x1, y1)
    e1.record(stream)
    torch.cuda.synchronize()
    one_batch_ms = e0.elapsed_time(e1) / reps
    e0.record(stream)
    for _ in range(reps):
        for i in range(len(mm)):
            F.fda_apply(B.mesh(i), x1[i].data_ptr(), y1[i].data_ptr(), 1, len(mm[i][1]))
    e1.record(stream)
    torch.cuda.synchronize()
    one_seq_ms = e0.elapsed_time(e1) / reps
    line = {"metric": "many-mesh batched FDA matvec (mesh x right-hand side)/s", "value": ws * len(mm) * nrhs * 1e3 / ms,
            "unit": "matvec/s", "n_gpus": ws, "steps": steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16x3/f64",
            "data": "synthetic",
            "config": {"workload": "8 meshes (sphere/ellipsoid icospheres L5-L7, 20,480-327,680 triangles, kD 20-100) "
                                   "x %d right-hand sides, chosen form, eps %g" % (nrhs, args.eps),
                       "meshes": [{"n": len(f), "k": k} for _, f, k in mm], "n_total": int(st.n_total),
                       "l2": "inputs larger than L2 (%.1f GB of right-hand sides per step)"
                             % (st.n_total * nrhs * 16 * 2 / 1e9)},
            "setup_s": setup_s, "device_gb": st.device_bytes / 1e9, "gpu_launches": launches,
            "cuda_graph_replays": st.graph_replays - gr0, "graph_fallback": st.graph_fallback,
            "sequential_handles_ms": sum(alone_ms), "per_mesh_ms": alone_ms,
            "one_rhs": {"batch_ms": one_batch_ms, "sequential_handles_ms": one_seq_ms,
                        "batch_matvec_per_s": len(mm) * 1e3 / one_batch_ms},
            "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)
    B.close()
    group.close()
    return 0


def run_pulsating(args):
    """The pulsating unit sphere of Sec. 5.1 over the paper's sphere family
    N = 512 * 4^m, k = pi 2^m (octahedral spheres, m = 0..6): right-hand side
    of the Burton-Miller equation for du/dn = 1 by the fast directional
    algorithm, GMRES to tol = eps, error against 1/(1 - ik); eps = 1e-3 and
    1e-4, chosen form.  The shape of Table tab_usphpls; not the headline
    workload (--workload pulsating)."""
    import math
    import numpy as np
    import torch
    from paper_1403_4747_gb300 import build as lib_build
    lib_build.build()
    import paper_1403_4747_gb300 as F
    from inputs import octasphere
    rows = []
    max_level = min(9, args.pulsating_max_level)
    for eps in (1e-3, 1e-4):
        for level in range(3, max_level + 1):
            m = level - 3
            k = math.pi * 2 ** m
            v, f = octasphere(level)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            P = F.FDAProblem(v, f, k, precision=F.FDA_CHOSEN_FP32, eps=eps, alpha_sign=args.alpha_sign)
            q = torch.ones(len(f), dtype=torch.complex128, device="cuda")
            b = P.rhs_neumann(q)
            torch.cuda.synchronize()
            setup_s = time.perf_counter() - t0
            u, info = P.solve(b, eps, raise_on_not_converged=False)
            ue = 1.0 / (1.0 - 1j * k)
            un = u.cpu().numpy()
            err = float(np.linalg.norm(un - ue) / (abs(ue) * math.sqrt(len(f))))
            st = P.stats()
            rows.append({"N": len(f), "k_over_pi": 2 ** m, "eps": eps, "alpha_sign": args.alpha_sign,
                         "setup_s": round(setup_s, 3),
                         "solve_s": round(info.solve_s, 4), "iters": info.iters,
                         "matvec_ms": round(info.matvec_s * 1e3, 3), "rel_resid": info.rel_resid_fp64,
                         "l2_error": err, "device_gb": round(st.device_bytes / 1e9, 2)})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
            P.close()
            del P, q, b, u
            torch.cuda.empty_cache()
    line = {"metric": "pulsating unit sphere: solve time and L2 error vs N (Table tab_usphpls shape)",
            "value": rows[-1]["solve_s"] if rows else None, "unit": "s", "higher_is_better": False,
            "n_gpus": 1, "dtype": "f32+bf16x3/f64", "data": "synthetic",
            "config": {"workload": "octahedral unit spheres N = 512 4^m, k = pi 2^m, du/dn = 1, chosen form"},
            "rows": rows}
    print(json.dumps(line), flush=True)
    return 0


def run_point_source(args):
    """Rigid unit sphere, point source at (-2, 0, 0) (the comparison of Sec.
    5.2): k = 5 and 50 on spheres of about the paper's size (N = 131,072)
    and the headline sphere (N = 327,680); GMRES to eps = 1e-3 as there,
    error against the closed form.  Not the headline workload
    (--workload point_source)."""
    import numpy as np
    import torch
    from paper_1403_4747_gb300 import build as lib_build
    lib_build.build()
    import paper_1403_4747_gb300 as F
    from inputs import octasphere, icosphere
    from scipy import special
    src = np.array([-2.0, 0.0, 0.0])

    def exact(k, cg):
        # -(1/(4 pi k)) sum (2n+1) h_n(2k) P_n(cos g) / h_n'(k)
        u = np.zeros(cg.shape, dtype=np.complex128)
        for n in range(int(k + 10 * k ** (1 / 3) + 40)):
            h = special.spherical_jn(n, 2 * k) + 1j * special.spherical_yn(n, 2 * k)
            hd = special.spherical_jn(n, k, True) + 1j * special.spherical_yn(n, k, True)
            u += -(2 * n + 1) / (4 * np.pi * k) * h / hd * special.eval_legendre(n, cg)
        return u

    rows = []
    for name, mesh in (("octasphere L7", lambda: octasphere(7)), ("icosphere L7", lambda: icosphere(7))):
        v, f = mesh()
        for k in (5.0, 50.0):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            P = F.FDAProblem(v, f, k, precision=F.FDA_CHOSEN_FP32, eps=1e-3, alpha_sign=args.alpha_sign)
            torch.cuda.synchronize()
            setup_s = time.perf_counter() - t0
            b = P.rhs_point_source(src)
            u, info = P.solve(b, 1e-3, raise_on_not_converged=False)
            c = np.mean(v[f], axis=1)
            cg = (c / np.linalg.norm(c, axis=1, keepdims=True)) @ (src / 2.0)
            ue = exact(k, cg)
            err = float(np.linalg.norm(u.cpu().numpy() - ue) / np.linalg.norm(ue))
            rows.append({"mesh": name, "N": len(f), "k": k, "alpha_sign": args.alpha_sign,
                         "setup_s": round(setup_s, 3), "solve_s": round(info.solve_s, 4), "iters": info.iters,
                         "T_it_ms": round(info.solve_s / max(1, info.iters) * 1e3, 3),
                         "rel_resid": info.rel_resid_fp64, "l2_error": err})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
            P.close()
            del P, b, u
            torch.cuda.empty_cache()
    line = {"metric": "point-source sphere scattering: time per GMRES iteration and error (Sec. 5.2)",
            "value": rows[1]["T_it_ms"], "unit": "ms", "higher_is_better": False, "n_gpus": 1,
            "dtype": "f32+bf16x3/f64", "data": "synthetic",
            "config": {"workload": "rigid unit sphere, point source (-2, 0, 0), k = 5 and 50, eps = tol = 1e-3"},
            "rows": rows}
    print(json.dumps(line), flush=True)
    return 0


def run_p0_sweep(args):
    """The p0 study of Table tab_varp0: points per direction p = ceil(ln(1/eps))
    + p0 for the low-frequency cubes (and two more for the high-frequency cone
    grids), p0 = 0..3, on the pulsating sphere with eps = 1e-3 (N = 524,288,
    k = 32 pi here; the paper uses N = 2,097,152).  Not the headline workload
    (--workload p0_sweep)."""
    import math
    import numpy as np
    import torch
    from paper_1403_4747_gb300 import build as lib_build
    lib_build.build()
    import paper_1403_4747_gb300 as F
    from inputs import octasphere
    level = args.p0_level
    v, f = octasphere(level)
    k = math.pi * 2 ** (level - 3)
    eps = 1e-3
    rows = []
    for p0 in range(4):
        p_lf = int(math.ceil(math.log(1.0 / eps))) + p0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        try:
            P = F.FDAProblem(v, f, k, precision=F.FDA_CHOSEN_FP32, eps=eps, p_lf=p_lf, p_hf=p_lf + 2,
                             alpha_sign=args.alpha_sign)
        except F.FDAError as e:
            rows.append({"p0": p0, "p_lf": p_lf, "p_hf": p_lf + 2, "error": str(e)})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
            continue
        b = P.rhs_neumann(torch.ones(len(f), dtype=torch.complex128, device="cuda"))
        torch.cuda.synchronize()
        setup_s = time.perf_counter() - t0
        u, info = P.solve(b, eps, raise_on_not_converged=False)
        ue = 1.0 / (1.0 - 1j * k)
        err = float(np.linalg.norm(u.cpu().numpy() - ue) / (abs(ue) * math.sqrt(len(f))))
        x = torch.ones(len(f), dtype=torch.complex128, device="cuda")
        y = torch.empty_like(x)
        for _ in range(3):
            P.apply(x, y)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            P.apply(x, y)
        e1.record()
        torch.cuda.synchronize()
        st = P.stats()
        rows.append({"p0": p0, "p_lf": p_lf, "p_hf": p_lf + 2, "setup_s": round(setup_s, 3),
                     "solve_s": round(info.solve_s, 4), "iters": info.iters,
                     "matvec_ms": round(e0.elapsed_time(e1) / 10, 3), "l2_error": err,
                     "device_gb": round(st.device_bytes / 1e9, 2),
                     "ranks": [int(st.level_rank[l]) for l in range(st.n_levels)]})
        print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
        P.close()
        del P, b, u, x, y
        torch.cuda.empty_cache()
    line = {"metric": "p0 study (Table tab_varp0 shape): error, time and memory vs points per direction",
            "value": rows[1]["matvec_ms"], "unit": "ms", "higher_is_better": False, "n_gpus": 1,
            "dtype": "f32+bf16x3/f64", "data": "synthetic",
            "config": {"workload": "pulsating octahedral sphere N = %d, k = %g pi, eps = 1e-3" % (len(f), k / math.pi)},
            "rows": rows}
    print(json.dumps(line), flush=True)
    return 0


def run_precond_study(args):
    """Preconditioners at the large size (icosphere level 9, N = 5,242,880,
    k = 200): the learned network trained on the leaf blocks of level 6-8
    spheres and ellipsoids with kD in {50, 100, 200, 300} (weights seed 0),
    and the network on the near-field pattern trained on the target mesh's
    own near-field matrix; GMRES to 1e-4 with none, the leaf block-diagonal
    inverse and both learned preconditioners (chosen form).  Not the
    headline workload (--workload precond)."""
    import numpy as np
    import torch
    from paper_1403_4747_gb300 import build as lib_build
    lib_build.build()
    import paper_1403_4747_gb300 as F
    from inputs import icosphere, ellipsoid_from_icosphere
    train = [("sphere L6", icosphere(6), 25.0), ("ellipsoid L7", ellipsoid_from_icosphere(7), 50.0),
             ("sphere L8", icosphere(8), 100.0), ("ellipsoid L8", ellipsoid_from_icosphere(8), 150.0)]
    hs = []
    t0 = time.perf_counter()
    for name, (v, f), k in train:
        hs.append(F.FDAProblem(v, f, k, precision=F.FDA_CHOSEN_FP32, alpha_sign=args.alpha_sign))
    w = F.fda_sai_init_weights(0)
    rep = F.fda_sai_train([P.h for P in hs], F.fda_sai_default_config(epochs=400, seed=0), w)
    train_setup_s = time.perf_counter() - t0
    for P in hs:
        P.close()
    del hs
    torch.cuda.empty_cache()
    v, f = icosphere(args.precond_level)
    k = args.precond_k
    t0 = time.perf_counter()
    P = F.FDAProblem(v, f, k, precision=F.FDA_CHOSEN_FP32, precond=1, alpha_sign=args.alpha_sign, maxit=600)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    set_loss = F.fda_sai_set(P.h, w)
    b = P.rhs_plane_wave([0.0, 0.0, 1.0])
    res = {}
    x_ref = None

    def run(name, pc):
        nonlocal x_ref
        F.fda_set_precond(P.h, pc)
        x, info = P.solve(b, 1e-4, raise_on_not_converged=False)
        if x_ref is None:
            x_ref = x.clone()
        res[name] = {"iters": info.iters, "solve_s": round(info.solve_s, 3), "rel_resid": info.rel_resid_fp64,
                     "diff_vs_none": float((x - x_ref).norm() / x_ref.norm())}
        print(json.dumps({name: res[name]}), file=sys.stderr, flush=True)

    for name, pc in (("none", 0), ("blockdiag", 1), ("learned", 2)):
        run(name, pc)
    # the network on the near-field pattern, trained on this mesh's own
    # near-field matrix (64 leaves per Adam step), then M on the whole pattern
    wn = F.fda_sai_init_weights(1)
    t0 = time.perf_counter()
    rep_near = F.fda_sai_train([P.h], F.fda_sai_default_config(epochs=args.sai_epochs, pattern=1,
                                                                sample_leaves=64), wn)
    near_train_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    F.fda_sai_set_pattern(P.h, wn, 1, want_loss=False)
    torch.cuda.synchronize()
    near_set_s = time.perf_counter() - t0
    run("learned_near", 2)
    st = P.stats()
    P.close()
    line = {"metric": "GMRES iterations and solve time at 1e-4: none vs block-diagonal vs learned (leaf blocks, "
                      "near field)",
            "value": res["learned"]["solve_s"], "unit": "s", "higher_is_better": False, "n_gpus": 1,
            "dtype": "f32+bf16x3/f64", "data": "synthetic",
            "config": {"workload": "icosphere level %d (N = %d), k = %g, plane wave +z, chosen form"
                                   % (args.precond_level, len(f), k), "alpha_sign": args.alpha_sign,
                       "training": [{"mesh": n, "N": len(m[1]), "k": kk} for n, m, kk in train]},
            "train": {"loss_init": rep.loss_init, "loss_final": rep.loss_final, "train_s": rep.train_s,
                      "setup_and_train_s": train_setup_s},
            "train_near": {"pattern": "near field, trained on the target mesh", "epochs": args.sai_epochs,
                           "sample_leaves": 64, "loss_init": rep_near.loss_init, "loss_final": rep_near.loss_final,
                           "train_s": near_train_s, "set_s": near_set_s},
            "target_loss": set_loss, "setup_s": setup_s, "device_gb": st.device_bytes / 1e9, "solves": res}
    print(json.dumps(line), flush=True)
    return 0


def run_far_field(args):
    """Far-field pattern of the headline sphere (level 7, N = 327,680,
    k = 50, plane wave along +z, chosen form, tol 1e-4) on 720 directions in
    the xz-plane against the Mie series, the scattered field on a grid of
    the xz-plane directly and through the fast algorithm, and reciprocity on
    the ellipsoid of the same level.  Not the headline workload
    (--workload far_field)."""
    import numpy as np
    import torch
    from scipy import special
    from paper_1403_4747_gb300 import build as lib_build
    lib_build.build()
    import paper_1403_4747_gb300 as F
    from inputs import icosphere, ellipsoid_from_icosphere
    k = 50.0
    th = np.arange(720) * (2 * np.pi / 720)
    dirs = np.stack([np.sin(th), np.zeros_like(th), np.cos(th)], axis=1)
    nmax = int(np.ceil(k + 10 * k ** (1 / 3) + 10))
    mie = np.zeros(len(th), dtype=np.complex128)
    for n in range(nmax + 1):
        jd = special.spherical_jn(n, k, True)
        hd = jd + 1j * special.spherical_yn(n, k, True)
        mie += (2 * n + 1) * jd / hd * special.eval_legendre(n, np.cos(th))
    mie *= 1j / k
    v, f = icosphere(7)
    P = F.FDAProblem(v, f, k, precision=F.FDA_CHOSEN_FP32, alpha_sign=args.alpha_sign)
    u, info = P.solve(P.rhs_plane_wave([0.0, 0.0, 1.0]), 1e-4)
    P.far_field(u, dirs[:8])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Fp = P.far_field(u, dirs)
    torch.cuda.synchronize()
    t_pat = time.perf_counter() - t0
    Fp = Fp.cpu().numpy()
    err = float(np.linalg.norm(Fp - mie) / np.linalg.norm(mie))
    # the same pattern through the fast algorithm's upward pass
    P.far_field(u, dirs[:8], fast=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Ff = P.far_field(u, dirs, fast=True)
    torch.cuda.synchronize()
    t_fast = time.perf_counter() - t0
    Ff = Ff.cpu().numpy()
    fast = {"ms": t_fast * 1e3, "rel_l2_vs_direct": float(np.linalg.norm(Ff - Fp) / np.linalg.norm(Fp)),
            "rel_l2_error_vs_mie": float(np.linalg.norm(Ff - mie) / np.linalg.norm(mie))}
    # the scattered field on a 40 x 40 grid of the xz-plane over [-2.5, 2.5]^2
    # (points with r >= 1.05), directly and through the fast algorithm
    g = np.linspace(-2.5, 2.5, 40)
    X, Z = np.meshgrid(g, g)
    pts = np.stack([X.ravel(), np.zeros(X.size), Z.ravel()], axis=1)
    pts = pts[np.linalg.norm(pts, axis=1) >= 1.05]
    times = {}
    vals = {}
    for name, fl in (("direct", False), ("fast", True)):
        P.scattered_field(u, pts[:8], fast=fl)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        vals[name] = P.scattered_field(u, pts, fast=fl)
        torch.cuda.synchronize()
        times[name] = (time.perf_counter() - t0) * 1e3
        vals[name] = vals[name].cpu().numpy()
    field = {"points": int(len(pts)), "direct_ms": times["direct"], "fast_ms": times["fast"],
             "fast_rel_l2_vs_direct": float(np.linalg.norm(vals["fast"] - vals["direct"])
                                           / np.linalg.norm(vals["direct"]))}
    P.close()
    ve, fe = ellipsoid_from_icosphere(7)
    Q = F.FDAProblem(ve, fe, k, precision=F.FDA_CHOSEN_FP32, alpha_sign=args.alpha_sign)
    d = np.array([0.0, 0.0, 1.0])
    a = np.array([0.6, 0.0, 0.8])
    u1, _ = Q.solve(Q.rhs_plane_wave(d), 1e-5)
    u2, _ = Q.solve(Q.rhs_plane_wave(-a), 1e-5)
    f1 = complex(Q.far_field(u1, [a]).cpu().numpy()[0])
    f2 = complex(Q.far_field(u2, [-d]).cpu().numpy()[0])
    Q.close()
    line = {"metric": "far-field pattern: 720 directions, error vs Mie, evaluation time", "value": t_pat * 1e3,
            "unit": "ms", "higher_is_better": False, "n_gpus": 1, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "icosphere level 7 (N = 327,680), k = 50, plane wave +z; ellipsoid level 7 "
                                   "reciprocity", "alpha_sign": args.alpha_sign},
            "pattern_rel_l2_error_vs_mie": err, "fast_pattern": fast, "scattered_field": field,
            "solve_iters": info.iters,
            "solve_s": info.solve_s,
            "reciprocity": {"F(a;d)": [f1.real, f1.imag], "F(-d;-a)": [f2.real, f2.imag],
                            "rel_gap": abs(f1 - f2) / abs(f1)}}
    print(json.dumps(line), flush=True)
    return 0


def run_profile_apply(args):
    """Profiling harness (--workload profile_apply): setup of the icosphere of
    --level at --k (chosen form, eager launches), one warm apply of --batch
    right-hand sides, then one more apply between cudaProfilerStart and
    cudaProfilerStop, so that `ncu --profile-from-start off` captures exactly
    the launches of one apply.  Prints one JSON line with the workload."""
    import numpy as np
    import torch
    from paper_1403_4747_gb300 import build as lib_build
    lib_build.build()
    import paper_1403_4747_gb300 as F
    from inputs import icosphere, complex_normal
    v, f = icosphere(args.level)
    n = len(f)
    nrhs = max(1, args.batch)
    P = F.FDAProblem(v, f, args.k, precision=F.FDA_CHOSEN_FP32, eps=args.eps, max_rhs=nrhs, graphs=0,
                     lowrank=0 if args.no_lowrank else 1)
    if args.tc_tiles:
        F.fda_set_tc_tiles(P.h, *[int(c) for c in args.tc_tiles.split(",")])
    x = torch.from_numpy(complex_normal(n, seed=77, nrhs=nrhs if nrhs > 1 else None)).cuda()
    y = torch.empty_like(x)
    P.apply(x, y)
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStart()
    P.apply(x, y)
    torch.cuda.synchronize()
    torch.cuda.cudart().cudaProfilerStop()
    # per-pass device times of five more applies (events on the library stream)
    F.fda_set_timing(P.h, True)
    acc = np.zeros(6)
    for _ in range(5):
        P.apply(x, y)
        acc += np.array(F.fda_get_pass_times(P.h))
    F.fda_set_timing(P.h, False)
    st = P.stats()
    print(json.dumps({"workload": "profile_apply", "level": args.level, "N": n, "k": args.k, "nrhs": nrhs,
                      "lowrank": not args.no_lowrank, "tc_tiles": args.tc_tiles or "tuned",
                      "pass_ms": dict(zip(["s2m", "m2m", "m2l", "l2l", "l2t", "near"], (acc / 5).round(4).tolist())),
                      "lowrank_tc_levels": [st.level_lr_tc[l] for l in range(st.n_levels)],
                      "tc_shape_m2m_m2l_l2l": [list(st.level_tc_shape[l]) for l in range(st.n_levels)],
                      "m2l_pairs_per_level": [st.level_m2l_pairs[l] for l in range(st.n_levels)],
                      "m2l_bytes_per_level": [st.level_m2l_bytes[l] for l in range(st.n_levels)],
                      "rank_per_level": [st.level_rank[l] for l in range(st.n_levels)]}), flush=True)
    P.close()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--level", type=int, default=7)
    ap.add_argument("--k", type=float, default=50.0)
    ap.add_argument("--eps", type=float, default=1e-4)
    ap.add_argument("--tol", type=float, default=1e-4)
    ap.add_argument("--plain-steps", type=int, default=3)
    ap.add_argument("--cpu-rows", type=int, default=1024)
    ap.add_argument("--ref-rows", type=int, default=384)
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-plain-unpreconditioned", action="store_true")
    ap.add_argument("--no-alt-coupling", action="store_true")
    ap.add_argument("--no-lowrank", action="store_true", help="profile_apply: Sec. 4.2's low-rank step off")
    ap.add_argument("--tc-tiles", default="", help="profile_apply: force one tensor-core tile shape "
                    "'columns,row_tiles,stages' (fda_set_tc_tiles) in place of the tuned ones")
    ap.add_argument("--no-lowrank-off", action="store_true",
                    help="skip the comparison run with the low-rank M2L step (Sec. 4.2) off")
    ap.add_argument("--alt-plain", action="store_true",
                    help="also solve the alpha = +i/k problem with the plain FP64 form (about a minute)")
    ap.add_argument("--no-precond", action="store_true",
                    help="skip the preconditioner comparison (block-diagonal, learned near-field) of the solve")
    ap.add_argument("--sai-epochs", type=int, default=150, help="Adam steps of the learned near-field preconditioner")
    ap.add_argument("--restart", type=int, default=100)
    ap.add_argument("--batch", type=int, default=64, help="right-hand sides per pass for the batched measurement")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--workload", default="sphere_l7_k50", choices=["sphere_l7_k50", "many_meshes", "pulsating", "point_source", "far_field",
                             "p0_sweep", "precond", "profile_apply"],
                    help="many_meshes: the eight-mesh batch; pulsating: the pulsating-sphere study")
    ap.add_argument("--pulsating-max-level", type=int, default=9)
    ap.add_argument("--p0-level", type=int, default=8, help="octahedral sphere level of the p0 study")
    ap.add_argument("--precond-level", type=int, default=9, help="icosphere level of the preconditioner study")
    ap.add_argument("--precond-k", type=float, default=200.0)
    ap.add_argument("--alpha-sign", type=float, default=-1.0, choices=[-1.0, 1.0],
                    help="coupling alpha = sign * i/k of the pulsating and point-source studies "
                         "(-1: the paper's time convention)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "many_meshes":
        return run_many_meshes(args)
    if args.workload == "pulsating":
        return run_pulsating(args)
    if args.workload == "point_source":
        return run_point_source(args)
    if args.workload == "far_field":
        return run_far_field(args)
    if args.workload == "p0_sweep":
        return run_p0_sweep(args)
    if args.workload == "precond":
        return run_precond_study(args)
    if args.workload == "profile_apply":
        return run_profile_apply(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
