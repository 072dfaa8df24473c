"""Benchmark: HOD-BF apply of the VIE system matrix on one GB300 (or N replicas).

Workload: homogeneous lossy sphere, radius 2 lambda0, eps_r = 4 - 0.1j, voxel
pitch lambda0/10 with 6 Kuhn tetrahedra per voxel (N = 410,208 SWG unknowns),
HOD-BF with leaf 64 and chi_con = 1e-4, factors stored in complex FP32, one
right-hand side.  A step is one application of the compressed operator
Y = Z X (cluster-tree gather, every stage of the butterfly program, scatter).

Metric: algorithmic bytes moved per apply / time, in GB/s, where the
algorithmic bytes are 8 E + 16 N nrhs (E = complex entries of all stored
factor blocks, c64; X read once, Y written once).  The factor data (tens of
GB) is far larger than L2, so no flush is needed between steps.

Usage: python bench.py [--gpus N --steps K --warmup W] [--impl reference] [--radius R]
Under torchrun each rank builds its own replica (weak scaling, no collective on
the data path) and rank 0 prints one JSON line.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "HOD-BF apply GB/s (algorithmic bytes / apply time), single RHS"
UNIT = "GB/s"
# DRAM traffic / algorithmic bytes of the single-RHS stage kernel, from an ncu capture of all
# 11 stages of one apply of the r = 1.0 sphere (N = 52,584, 5.04 GB of factors, larger than
# L2) with the current kernel; the traffic is the factor stream, so it scales with the
# algorithmic bytes to the benchmark operator.
TRAFFIC_RATIO = 1.019
TRAFFIC_NOTE = ("ncu dram bytes of stage1_kernel<4>, all 11 stages of one apply at r=1.0 (N=52,584) = "
                "1.019 x algorithmic, scaled by the algorithmic bytes")
# the same ratio for the shared-memory bulk-staged kernel (autotuner candidates 9-11): not captured
# since the kernel last changed
BULK_TRAFFIC_RATIO = None
BULK_TRAFFIC_NOTE = "no ncu capture of stage1_bulk_kernel since it last changed; traffic not measured"


def single_rhs_kernels(tune):
    """Kernel names and DRAM-traffic ratio of the single-RHS stages for an autotuner choice list
    (candidates 0-8 stage1_kernel<4>, 9-11 stage1_bulk_kernel, 12-20 stage1_kernel<8>)."""
    kinds = {"stage1_kernel<4>" if c < 9 else "stage1_bulk_kernel" if c < 12 else "stage1_kernel<8>"
             for c in ([0] if tune is None else [int(c) for c in tune])}
    names = " + ".join(sorted(kinds))
    if kinds == {"stage1_kernel<4>"}:
        return names, TRAFFIC_RATIO, TRAFFIC_NOTE
    if kinds == {"stage1_bulk_kernel"}:
        return names, BULK_TRAFFIC_RATIO, BULK_TRAFFIC_NOTE
    return names, None, "no ncu capture of this kernel mix; traffic ratio not measured"


def _bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured bf16 dense (burst)"
    except Exception:
        return 1900.0, "fallback bf16 dense"


BF16_PEAK = _bf16_peak()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def workload(radius: float, kind: str = "sphere"):
    """The body of an apply benchmark.

    sphere: homogeneous sphere of the given radius, eps_r = 4 - 0.1j, pitch lambda0/10
            (radius 2: N = 410,208, the benchmark workload);
    shell:  Drude plasma shell 1.5/1.2 lambda0, vacuum core, pitch lambda0/20 (N = 690,768);
    cube:   5 lambda0 cube, eps_r = 1 + 49 Phi(GRF), pitch lambda0/10 (N = 1,515,000)."""
    if kind == "shell":
        return W.plasma_shell(), ("plasma shell 1.5/1.2 lambda0, Drude eps_r=-2.2319-0.1616j, vacuum core, "
                                  "pitch lambda0/20, N={n}")
    if kind == "cube":
        return W.cube_grf(5.0, 0.1), ("cube 5 lambda0, eps_r=1+49*Phi(GRF, corr 0.5, seed 20211101), "
                                      "pitch lambda0/10, N={n}")
    body = W.sphere(radius, 4.0 - 0.1j, 1.0 / 10, name=f"sphere_r{radius:g}_eps4-0.1j")
    desc = f"sphere r={radius:g} lambda0, eps_r=4-0.1j, pitch lambda0/10, 6 Kuhn tets/voxel, N={{n}}"
    return body, desc


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
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
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_operator():
    """The FP64 oracle's HOD-BF of a bounded sample of the workload: a sphere of the same
    permittivity at radius 0.25 and pitch 1/16 (N = 3,672), built with full-row IDs."""
    from oracle.entries import Elements, zblock
    from oracle.hodbf import HODBF, cluster_tree, face_centroids
    from oracle.mesh import build_mesh

    body = W.sphere(0.25, 4.0 - 0.1j, 1.0 / 16, name="sample")
    mesh = build_mesh(body)
    n = len(mesh["faces"])
    Z = zblock(Elements(mesh, W.K0), np.arange(n), np.arange(n))
    perm, LH, bounds = cluster_tree(face_centroids(mesh), 64)
    Zt = Z[np.ix_(perm, perm)]
    H = HODBF(lambda r, c: Zt[np.ix_(r, c)], bounds, LH, 1e-4)
    return H, n


def oracle_sample_desc(H, n, reps, dt):
    return (f"oracle FP64 HOD-BF apply of a sphere r=0.25 eps_r=4-0.1j pitch 1/16 (N={n}, chi_con=1e-4, "
            f"{H.entries()} complex128 entries), {reps} applies of {dt * 1e3:.2f} ms; one Python thread "
            f"driving NumPy, whose BLAS may use up to `cores` threads per block product")


def oracle_apply_sample(seconds_budget: float = 15.0):
    """Time the FP64 oracle's HOD-BF apply on host cores (bounded sample of the workload)."""
    H, n = oracle_operator()
    x = W.random_block(n, 1, seed=1)
    nbytes = 16 * H.entries() + 32 * n  # complex128 factors, x read and y written
    reps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds_budget or reps < 3:
        H.apply(x)
        reps += 1
    dt = (time.perf_counter() - t0) / reps
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return dict(value=nbytes / dt / 1e9, unit=UNIT, cores=cores, kind="oracle",
                sample=oracle_sample_desc(H, n, reps, dt), ms_per_apply=dt * 1e3, n=n)


def run_reference(args):
    """The oracle arm: the plain FP64 CPU HOD-BF apply, timed on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    H, n = oracle_operator()
    x = W.random_block(n, 1, seed=1)
    nbytes = 16 * H.entries() + 32 * n
    for _ in range(args.warmup):
        H.apply(x)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        H.apply(x)
        times.append(time.perf_counter() - t0)
    dt = statistics.median(times)
    v = nbytes / dt / 1e9
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    _, desc = workload(args.radius)
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic",
            "config": {"workload": desc.format(n="410208") + " (oracle on a bounded sample, see cpu_baseline)"},
            "cpu_baseline": {"value": round(v, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": oracle_sample_desc(H, n, args.steps, dt)},
            "e2e": {"value": round(v, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def serving_operators():
    """Resident scatterers of the serving workload: the kinds of the eight-operator mix (spheres
    of eps_r 2, 4, 10 and 40, a negative-permittivity shell, a lossy sphere) at reduced sizes
    (N = 7.1k-27.7k; the full mix holds 1.18 M unknowns), pitch lambda_d/10, capped at
    lambda0/20 for eps_r = 40 as in the mix."""
    r2 = 1.0 / (10 * 2 ** 0.5)
    r10 = 1.0 / (10 * 10 ** 0.5)
    return [W.sphere(0.5, 2.0, r2, name="S1 sphere r=0.5 eps=2"),
            W.sphere(0.3, 4.0, 1.0 / 20, name="sphere r=0.3 eps=4"),
            W.shell(0.5, 0.4, -4.0 - 0.3j, 1.0 / 20, name="P2' shell 0.5/0.4 eps=-4-0.3j"),
            W.sphere(0.4, 4.0 - 0.1j, 1.0 / 20, name="sphere r=0.4 eps=4-0.1j"),
            W.sphere(0.25, 10.0, r10, name="S2' sphere r=0.25 eps=10"),
            W.sphere(0.25, 40.0, 1.0 / 20, name="S3' sphere r=0.25 eps=40")]


def serving_tol_fact(bodies):
    """chi_fact = 1e-3 for negative permittivity (Sec. IV-A), 1e-2 for 10 <= |eps_r| < 40 and
    1e-3 from 40 on (high-contrast operators need a tighter inverse for GMRES to reach 1e-3 in
    tens of iterations), 1e-1 otherwise (Sec. IV-A, IV-B)."""
    out = []
    for b in bodies:
        e = np.asarray(b.eps)
        out.append(1e-3 if np.real(e).min() < 0 or np.abs(e).max() >= 40 else
                   (1e-2 if np.abs(e).max() >= 10 else 1e-1))
    return out


def run_serving(args):
    """Continuous-batching solves (C32 factors, tensor-core multi-column applies, FP64 refinement)
    against the plain FP64 one-request-at-a-time GPU solver on the same requests."""
    print(json.dumps(serving_line(args)), flush=True)
    return 0


def serving_line(args):
    import torch

    import paper_2111_01730_gb300 as pkg

    torch.cuda.set_device(0)
    bodies = serving_operators()[:max(1, getattr(args, "serve_ops", 6))]
    t0 = time.perf_counter()
    mixed = [pkg.Operator(b, W.K0, tol_con=1e-3, tol_fact=fact, leaf=64, factor_dtype="c64")
             for b, fact in zip(bodies, serving_tol_fact(bodies))]
    build_mixed = time.perf_counter() - t0
    # where each operator's multi-column applies switch to the tensor cores (timed per operator)
    crossover = [[m.autotune_rhs(pkg.VIE_OP_Z), m.autotune_rhs(pkg.VIE_OP_ZINV)] for m in mixed]
    rng = np.random.default_rng(7)
    nreq = args.requests
    reqs = []
    for i in range(nreq):
        op = int(rng.integers(len(mixed)))
        nr = int(rng.integers(1, 33))
        k, p = W.planewave_random(nr, seed=1000 + i)
        reqs.append((op, k, p))
    rhs = [mixed[op].rhs_planewave(k, p).cpu().numpy() for op, k, p in reqs]
    arrivals = np.cumsum(rng.exponential(1.0 / args.rate, size=nreq))
    total_rhs = sum(r.shape[1] for r in rhs)

    def serve(sat: bool):
        srv = pkg.Server(mixed, restart=30, max_iter=300, mem_budget=48 << 30)
        ids, lat, rels, its = {}, [], [], []
        torch.cuda.synchronize()
        start = time.perf_counter()
        nxt = 0
        while len(lat) < nreq:
            now = time.perf_counter() - start
            while nxt < nreq and (sat or arrivals[nxt] <= now):
                ids[srv.submit(reqs[nxt][0], rhs[nxt], rtol=1e-3)] = nxt
                nxt += 1
            srv.step()
            for rid in list(ids):
                i = ids[rid]
                r = srv.result(rid, mixed[reqs[i][0]].n, rhs[i].shape[1])
                if r is not None:
                    lat.append(r[3])
                    rels.append(r[2].max())
                    its.append(int(r[1].max()))
                    del ids[rid]
        wall = time.perf_counter() - start
        srv.close()
        return wall, np.array(lat), np.array(rels), np.array(its)

    serve(True)  # warm-up: tensor-core tiles, workspaces
    wall_s, lat_s, rel_s, it_s = serve(True)
    wall_p, lat_p, rel_p, it_p = serve(False)
    try:
        grouped = grouped_timing(mixed, pkg, torch)
    except Exception as exc:  # reported, the serving numbers stand on their own
        grouped = {"error": f"{type(exc).__name__}: {exc}"[:300]}
    # plain FP64 GPU solver, one request and one right-hand side at a time, on a bounded sample
    for m in mixed:
        m.close()
    fp64 = [pkg.Operator(b, W.K0, tol_con=1e-3, tol_fact=fact, leaf=64, factor_dtype="c128")
            for b, fact in zip(bodies, serving_tol_fact(bodies))]
    ns = min(nreq, args.baseline_requests)
    done_rhs, t_busy, rel_b = 0, 0.0, []
    for i in range(ns):
        op, k, p = reqs[i]
        V = fp64[op].rhs_planewave(k, p)
        for j in range(V.shape[1]):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            I, it, rel, st = fp64[op].solve(V[:, j:j + 1].contiguous(), rtol=1e-3, restart=30, max_iter=300)
            torch.cuda.synchronize()
            t_busy += time.perf_counter() - t1
            rel_b.append(float(rel.max()))
            done_rhs += 1
    base = done_rhs / t_busy
    line = {"metric": "solves/s (right-hand sides solved per second), continuous batching, rtol 1e-3",
            "value": round(total_rhs / wall_s, 2), "unit": "solves/s", "higher_is_better": True,
            "config": {"workload": "; ".join(f"{b.name} (N={m.n})" for b, m in zip(bodies, fp64)),
                       "requests": nreq, "rhs_total": int(total_rhs), "rhs_per_request": "uniform 1-32",
                       "chi_con": 1e-3, "chi_fact": "1e-1 (eps > 0), 1e-2 (10 <= |eps| < 40), 1e-3 (eps < 0 or |eps| >= 40)", "restart": 30, "build_seconds": round(build_mixed, 1),
                       "tensor_core_from_columns": {"Z": [c[0] for c in crossover], "Zinv": [c[1] for c in crossover]}},
            "saturated": {"solves_per_s": round(total_rhs / wall_s, 2), "p50_s": round(float(np.median(lat_s)), 4),
                          "p99_s": round(float(np.percentile(lat_s, 99)), 4), "max_relres": float(rel_s.max()),
                          "max_iters": int(it_s.max())},
            "poisson": {"rate_req_per_s": args.rate, "solves_per_s": round(total_rhs / wall_p, 2),
                        "p50_s": round(float(np.median(lat_p)), 4), "p99_s": round(float(np.percentile(lat_p, 99)), 4),
                        "max_relres": float(rel_p.max())},
            "plain_fp64_one_at_a_time": {"solves_per_s": round(base, 2), "sample_rhs": done_rhs,
                                         "max_relres": max(rel_b)},
            "speedup_vs_plain_fp64": round(total_rhs / wall_s / base, 2),
            "grouped_apply": grouped}
    return line


def grouped_timing(ops, pkg, torch, reps: int = 20):
    """Z (Zinv x) of every resident operator at 1 and 8 columns: one apply per operator (each
    replayed from its CUDA graph) against one grouped launch sequence for all of them
    (vie_apply_group, one launch per stage depth); CUDA events, median of the repetitions,
    and whether the grouped results equal the separate ones bit for bit."""
    out = {}
    stream = torch.cuda.current_stream()
    for nrhs in (1, 8):
        X = [torch.from_numpy(W.random_block(o.n, nrhs, seed=21 + i).astype(np.complex64)).cuda().t().contiguous().t()
             for i, o in enumerate(ops)]
        jobs = [(o, x, pkg.VIE_OP_ZINV) for o, x in zip(ops, X)]

        def separate():
            return [o.apply(x, op=k) for o, x, k in jobs]

        def grouped():
            return pkg.apply_group(jobs)

        same = all(torch.equal(a, b) for a, b in zip(separate(), grouped()))
        times = {}
        for name, fn in (("separate", separate), ("grouped", grouped)):
            for _ in range(3):
                fn()
            ms = []
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                fn()
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            times[name] = round(float(np.median(ms)), 4)
        out[f"nrhs_{nrhs}"] = {"separate_ms": times["separate"], "grouped_ms": times["grouped"],
                               "speedup": round(times["separate"] / times["grouped"], 3), "bit_identical": same}
    out["operators"] = len(ops)
    out["op"] = "Zinv"
    return out


def serving_summary(args):
    """A short serving run for the default line: 40 requests of 1-32 plane waves on the four
    resident operators (continuous batching, grouped launches, rtol 1e-3), saturated and at
    Poisson arrivals of 100 req/s, against the plain FP64 solver on a 2-request sample."""
    import argparse

    sub = argparse.Namespace(requests=40, rate=100.0, baseline_requests=2, serve_ops=6)
    full = serving_line(sub)
    keep = ("metric", "value", "unit", "saturated", "poisson", "plain_fp64_one_at_a_time", "speedup_vs_plain_fp64",
            "grouped_apply")
    out = {k: full[k] for k in keep}
    out["config"] = {k: full["config"][k] for k in ("workload", "requests", "rhs_total", "rhs_per_request", "chi_con",
                                                    "chi_fact", "restart")}
    return out


def zinv_timing(op, pkg, x, y, steps, torch):
    """Zinv apply (Algorithm 1 levels present in the operator) and one preconditioned MVP (Z + Zinv)."""
    st = op.get_stats()
    ez = int(op.program_info(pkg.VIE_OP_ZINV)[0].sum())
    t = torch.empty_like(y)
    for _ in range(3):
        op.apply(x, y, op=pkg.VIE_OP_ZINV)
    stream = torch.cuda.current_stream()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    torch.cuda.synchronize()
    e[0].record(stream)
    for _ in range(steps):
        op.apply(x, y, op=pkg.VIE_OP_ZINV)
    e[1].record(stream)
    for _ in range(steps):
        op.apply(x, t, op=pkg.VIE_OP_ZINV)
        op.apply(t, y)
    e[2].record(stream)
    torch.cuda.synchronize()
    ms = e[0].elapsed_time(e[1]) / steps
    return {"ms_per_apply": round(ms, 4), "gbs": round((8 * ez + 16 * op.n * x.numel() // op.n) / (ms * 1e-3) / 1e9, 1),
            "factor_entries": ez, "stages": int(st.apply_stages_zinv), "top_level": int(st.zinv_top_level),
            "invert_seconds": round(st.invert_seconds, 2),
            "mvp_with_precond_ms": round(e[1].elapsed_time(e[2]) / steps, 4)}


def multi_rhs_timing(op, pkg, torch, nrhs: int = 128, steps: int = 5):
    """The same operator applied to a block of right-hand sides on the tensor cores (tcgen05,
    BF16x3 split products): useful complex flops 8 E nrhs over the apply time."""
    n = op.n
    E = int(op.program_info(pkg.VIE_OP_Z)[0].sum())
    X = torch.from_numpy(W.random_block(n, nrhs, seed=11).astype(np.complex64)).cuda().t().contiguous().t()
    Y = torch.empty_like(X)
    for _ in range(2):  # the first packs the tensor-core tiles
        op.apply(X, Y)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        op.apply(X, Y)
    e1.record(stream)
    torch.cuda.synchronize()
    op.check()
    ms = e0.elapsed_time(e1) / steps
    tf = 8.0 * E * nrhs / (ms * 1e-3) / 1e12
    out = {"nrhs": nrhs, "ms_per_apply": round(ms, 3), "useful_tflops": round(tf, 2),
           "frac_of_bf16_peak": round(tf / BF16_PEAK[0], 4), "peak_note": BF16_PEAK[1],
           "factor_gbs": round(8.0 * E / (ms * 1e-3) / 1e9, 1),
           "kernel": "tc_stage_kernel<BF16x3> (+ stage_kernel for blocks under 16 x 32)"}
    # the TF32 variant on the same operator and block (tiles repacked), then back to BF16x3
    op.set_prec(pkg.VIE_P_TC_TF32)
    Yb = Y.clone()
    for _ in range(2):
        op.apply(X, Y)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        op.apply(X, Y)
    e1.record(stream)
    torch.cuda.synchronize()
    op.check()
    ms32 = e0.elapsed_time(e1) / steps
    tf32 = 8.0 * E * nrhs / (ms32 * 1e-3) / 1e12
    out["tf32"] = {"ms_per_apply": round(ms32, 3), "useful_tflops": round(tf32, 2),
                   "rel_diff_vs_bf16x3": float(torch.linalg.norm(Y - Yb) / torch.linalg.norm(Yb)),
                   "kernel": "tc_stage_kernel<TF32>"}
    op.set_prec(pkg.VIE_P_TC_BF16X3)
    return out


def precond_section(pkg, torch, steps: int = 20):
    """Zinv from products (Algorithms 1-2, BF_random_matvec) and one preconditioned solve, on a
    sphere of the benchmark's permittivity and pitch at radius 1 (N = 52,584): the four top
    levels of the inverse are built from products only (nodes above 4,096 unknowns), the rest
    from their dense blocks.  The solve (x-polarized plane wave along +z, left-preconditioned
    TFQMR to 1e-3) is compared with the plain FP64 path (complex FP64 factors, unpreconditioned
    GMRES to 1e-6)."""
    body = W.sphere(1.0, 4.0 - 0.1j, 1.0 / 10, name="sphere_r1_eps4-0.1j")
    t0 = time.perf_counter()
    op = pkg.Operator(body, W.K0, tol_con=1e-4, tol_fact=1e-2, leaf=64, factor_dtype="c64", seed=1,
                      inv_dense_max=4096)
    build = time.perf_counter() - t0
    st = op.get_stats()
    n = op.n
    ez = int(op.program_info(pkg.VIE_OP_ZINV)[0].sum())
    x = torch.from_numpy(W.random_block(n, 1, seed=5)[:, 0].astype(np.complex64)).cuda()
    y = torch.empty_like(x)
    for _ in range(3):
        op.apply(x, y, op=pkg.VIE_OP_ZINV)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        op.apply(x, y, op=pkg.VIE_OP_ZINV)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    ident = op.apply(op.apply(x), op=pkg.VIE_OP_ZINV)
    k, p = W.planewave_x_along_z()
    V = op.rhs_planewave(k, p)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    I, it, rel, stt = op.solve_tfqmr(V, rtol=1e-3, max_iter=300)
    torch.cuda.synchronize()
    t_solve = time.perf_counter() - t1
    op.close()
    ref = pkg.Operator(body, W.K0, tol_con=1e-4, leaf=64, factor_dtype="c128", seed=1)
    I64, it64, rel64, st64 = ref.solve(ref.rhs_planewave(k, p), rtol=1e-6, restart=200, max_iter=2000)
    err = (torch.linalg.norm(I - I64) / torch.linalg.norm(I64)).item()
    ref.close()
    return {"workload": f"sphere r=1 lambda0, eps_r=4-0.1j, pitch lambda0/10, N={n}", "chi_fact": 1e-2,
            "invert_seconds": round(st.invert_seconds, 1), "build_seconds": round(build, 1),
            "product_levels": int(st.zinv_product_levels), "products": int(st.inverse_products),
            "zinv_top_level": int(st.zinv_top_level),
            "zinv_apply_ms": round(ms, 4), "zinv_apply_gbs": round((8 * ez + 16 * n) / (ms * 1e-3) / 1e9, 1),
            "zinv_z_identity_error": round((torch.linalg.norm(ident - x) / torch.linalg.norm(x)).item(), 5),
            "tfqmr_iterations": int(it[0]), "tfqmr_relres": float(rel[0]), "solve_seconds": round(t_solve, 3),
            "status": int(stt),
            "fp64_reference": {"gmres_iterations": int(it64[0]), "relres": float(rel64[0])},
            "solution_error_vs_fp64_path": round(err, 6)}


def nrhs_for_tune(args):
    """The stage-tiling autotuner serves the single-RHS kernel."""
    return args.nrhs == 1 and not args.no_autotune


def job_value(alg_bytes_per_rank: float, total_ms: float, steps: int, world: int, dist=None, device=None):
    """Whole-job throughput: the units all ranks processed / the slowest rank's time.

    Each rank times its own replica; the max over ranks (all_reduce MAX) is the job's time.
    Returns (GB/s of the job, ms per step of the slowest rank)."""
    if dist is not None and world > 1:
        import torch

        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_step = total_ms / steps
    return world * alg_bytes_per_rank / (ms_step * 1e-3) / 1e9, ms_step


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--radius", type=float, default=2.0,
                    help="sphere radius in wavelengths (2.0 = the benchmark workload; smaller for checks/profiles)")
    ap.add_argument("--workload", default="sphere", choices=["sphere", "shell", "cube"],
                    help="sphere (default, the benchmark workload), shell (plasma shell) or cube (GRF cube)")
    ap.add_argument("--chi-con", type=float, default=1e-4, help="compression tolerance of Z")
    ap.add_argument("--nrhs", type=int, default=1,
                    help="right-hand sides per apply (>= 16 runs the tensor-core path)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default stage tiling")
    ap.add_argument("--tiling", type=int, default=None,
                    help="use one autotuner candidate on every stage (0-8 streaming kernel, 9-11 shared-memory "
                         "bulk kernel, 12-20 streaming kernel with 8 loads in flight)")
    ap.add_argument("--zinv", action="store_true", help="also build Zinv (chi_fact 1e-1) and time its apply")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the 128-RHS apply and the preconditioned-solve keys of the default line")
    ap.add_argument("--serve", action="store_true", help="serving benchmark (solves/s, p50/p99 latency)")
    ap.add_argument("--requests", type=int, default=120)
    ap.add_argument("--rate", type=float, default=100.0, help="Poisson arrival rate (requests/s) for --serve")
    ap.add_argument("--baseline-requests", type=int, default=6)
    ap.add_argument("--serve-ops", type=int, default=6, help="serve the first N resident operators of the mix")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.serve:
        return run_serving(args)

    import torch

    import paper_2111_01730_gb300 as pkg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    hbm, peak_kind = peaks()
    body, desc = workload(args.radius, args.workload)
    t0 = time.perf_counter()
    op = pkg.Operator(body, W.K0, tol_con=args.chi_con, tol_fact=(1e-1 if args.zinv else 0.0), leaf=64,
                      factor_dtype="c64", seed=1)
    build_s = time.perf_counter() - t0
    if args.tiling is not None:  # one fixed kernel/tiling candidate on every stage (profiling)
        tune = np.full(op.get_stats().apply_stages_z, args.tiling, dtype=np.int32)
        op.set_tiling(tune)
    else:
        tune = op.autotune(pkg.VIE_OP_Z) if nrhs_for_tune(args) else None
    st = op.get_stats()
    n = op.n
    entries, sbytes, tiles = op.program_info(pkg.VIE_OP_Z)
    E = int(entries.sum())
    nrhs = args.nrhs
    alg_bytes = 8 * E + 16 * n * nrhs  # per apply
    if nrhs == 1:
        x = torch.from_numpy(W.random_block(n, 1, seed=7)[:, 0].astype(np.complex64)).cuda()
    else:
        x = torch.from_numpy(W.random_block(n, nrhs, seed=7).astype(np.complex64)).cuda().t().contiguous().t()
    y = torch.empty_like(x)
    stream = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        op.apply(x, y)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    torch.cuda.synchronize()
    evs[0].record(stream)
    for i in range(args.steps):
        op.apply(x, y)
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    per = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    total_ms = evs[0].elapsed_time(evs[-1])
    # per-stage timing of the dominant kernel (stage kernels), CUDA events on the launch stream
    prof = []
    for _ in range(5):
        ms, launches = op.apply_profile(x, y)
        prof.append(ms)
    clk = clocks.stop()
    prof = np.median(np.array(prof), axis=0)
    stage_ms = prof[1:-1]
    launches_per_apply = int(launches)
    value, ms_step = job_value(alg_bytes, total_ms, args.steps, world, dist, "cuda")
    # end to end through the public API: pinned host X -> device, apply, device -> host Y
    xh = x.cpu().pin_memory()
    yh = torch.empty_like(xh).pin_memory()
    xd = torch.empty_like(x)
    for _ in range(3):
        xd.copy_(xh, non_blocking=True)
        op.apply(xd, y)
        yh.copy_(y, non_blocking=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        xd.copy_(xh, non_blocking=True)
        op.apply(xd, y)
        yh.copy_(y, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / args.steps
    # roofline of the dominant kernel: the stage kernel, all its launches of one apply
    stage_alg = 8 * E
    achieved = stage_alg / (stage_ms.sum() * 1e-3) / 1e9
    useful_tflops = 8.0 * E * nrhs / (stage_ms.sum() * 1e-3) / 1e12
    if rank == 0:
        k_names, k_ratio, k_note = single_rhs_kernels(tune)
        line = {
            "metric": METRIC if nrhs == 1 else METRIC.replace("single RHS", f"{nrhs} RHS"), "value": round(value, 2), "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(ms_step, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64", "data": "synthetic",
            "config": {"workload": desc.format(n=n), "n": n, "levels": st.levels, "chi_con": args.chi_con, "leaf": 64, "nrhs": nrhs,
                       "factor_entries": E, "factor_bytes_stored": int(sbytes.sum()), "max_rank": st.max_rank,
                       "build_seconds": round(build_s, 2),
                       "autotuned_tiling": None if tune is None else [int(c) for c in tune],
                       "build_split_s": {"entries": round(st.build_entries_seconds, 1), "ids": round(st.build_id_seconds, 1),
                                         "host_sampling": round(st.build_host_seconds, 1)},
                       "l2": "inputs (factor data) larger than L2, no flush",
                       "parallelism": f"replicas x{world}"},
            "apply_latency_ms": {"p50": round(float(np.percentile(per, 50)), 4),
                                 "p99": round(float(np.percentile(per, 99)), 4)},
            "roofline": ({"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
                          "frac": round(achieved / hbm, 4), "traffic": k_ratio and round(k_ratio * stage_alg),
                          "traffic_note": k_note,
                          "kernel": k_names + " (single-RHS stages, autotuned per stage; all launches of one apply)"}
                         if nrhs < 16 else
                         {"bound": "tensor", "achieved": round(useful_tflops, 2), "peak": BF16_PEAK[0], "unit": "TFLOP/s",
                          "frac": round(useful_tflops / BF16_PEAK[0], 4), "traffic": None,
                          "peak_note": BF16_PEAK[1] + "; useful complex flops 8*E*nrhs (the BF16x3 split issues 3x)",
                          "hbm_gbs": round(achieved, 1),
                          "kernel": "tc_stage_kernel + stage_kernel remainder (all stages of one apply)"}),
            "e2e": {"value": round(alg_bytes / (e2e_ms * 1e-3) / 1e9, 2), "unit": UNIT,
                    "h2d_bytes_per_step": 8 * n * nrhs, "d2h_bytes_per_step": 8 * n * nrhs,
                    "ms_per_step": round(e2e_ms, 4)},
            "gpu_launches": launches_per_apply * args.steps,
            "clocks": clk,
        }
        if args.zinv:
            try:
                line["zinv"] = zinv_timing(op, pkg, x, y, args.steps, torch)
            except Exception as exc:  # an extra key: the headline line must still print
                line["zinv"] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
        if nrhs == 1 and not args.no_extras:
            try:
                line["multi_rhs"] = multi_rhs_timing(op, pkg, torch)
            except Exception as exc:  # an extra key: the headline line must still print
                line["multi_rhs"] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
        line["roofline"].update({"peak_kind": peak_kind, "stage_ms": [round(float(v), 4) for v in stage_ms],
                                 "stage_gbs": [round(8 * float(e) / (float(t) * 1e6), 1)
                                               for e, t in zip(entries, stage_ms)]})
        if nrhs == 1 and not args.no_extras and world == 1:
            op.close()
            torch.cuda.empty_cache()
            try:
                line["preconditioned_solve"] = precond_section(pkg, torch)
            except Exception as exc:  # an extra key: the headline line must still print
                line["preconditioned_solve"] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
            torch.cuda.empty_cache()
            try:
                line["serving"] = serving_summary(args)
            except Exception as exc:  # the headline line must still print
                line["serving"] = {"error": f"{type(exc).__name__}: {exc}"[:300]}
        if not args.no_cpu_baseline and world == 1:
            cb = oracle_apply_sample(15.0)
            line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
