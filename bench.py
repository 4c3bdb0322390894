#!/usr/bin/env python3
"""Throughput of batched FP32 finite-element assembly of CDR transport equations.

One step = one fea_assemble call over the whole workload: gather, Gauss-point
geometry, per-equation coefficients, element matrices and RHS, scatter into the
CSR values and RHS of every equation.  On the default workload (Hex8 256^3, 32
equations) a step is a time step: the assembly, then the seeded update of the
field, K of them recorded in one CUDA graph.  Inputs are resident in HBM; the
inputs plus outputs of every workload are larger than the 129 MB L2, so no L2
flush is needed between steps.  The default run then measures the other
paper-shaped workloads the same way ("workloads" in the output).

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
instead (a bounded sample of the same workload on the host cores).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2107_11541_gb300 import meshgen as G  # noqa: E402

WORKLOADS = {"tet4_100_perm_1eq": 1, "hex8_128_21eq": 2, "hex27_48_11eq": 3, "hex8_256_32eq": 4}
# meshes of several element types (not among the paper-shaped configurations): cells per axis, equations
MIXED_WORKLOADS = {"mixed_96_4eq": (96, 4)}
NG = {G.TET4: 4, G.HEX8: 8, G.HEX27: 27, G.PEN6: 6, G.PYR5: 12}
# the largest paper-shaped configuration that fits one GPU: Hex8 256^3, 32 equations, 10 time steps
# in one CUDA graph; the default run also measures the other paper-shaped workloads (SIDE_WORKLOADS)
DEFAULT_WORKLOAD = "hex8_256_32eq"
SIDE_WORKLOADS = ("hex8_128_21eq", "hex27_48_11eq", "tet4_100_perm_1eq")
METRIC = "elements x equations assembled per second (FP32 batched)"
UNIT = "elem*eq/s"
HBM_PEAK_FALLBACK = 6800.0
FP32_LANES_PER_SM = 128
SM_MAX_MHZ_FALLBACK = 2070.0
NEN = {G.TET4: 4, G.HEX8: 8, G.HEX27: 27}


def closed_form_nnz(workload: str, n=None) -> int:
    """nnz of a paper-shaped workload's pattern by counting (pinned against the oracle's pattern by
    the CPU tests): Kuhn tetrahedra of n^3 cubes have N + 2 x (edges) entries, edges = 3n(n+1)^2
    axis edges + 3n^2(n+1) face diagonals + n^3 body diagonals; a tensor grid of Hex8 (Hex27)
    elements has (3n+1)^3 ((8n+1)^3) entries, the cube of its 1-D row lengths."""
    cfg = G.CONFIGS[WORKLOADS[workload]]
    n, t = cfg["n"] if n is None else n, cfg["elem_type"]
    if t == G.TET4:
        return (n + 1) ** 3 + 2 * (3 * n * (n + 1) ** 2 + 3 * n * n * (n + 1) + n ** 3)
    return (3 * n + 1) ** 3 if t == G.HEX8 else (8 * n + 1) ** 3


def device_alu_peak():
    """FP32 FMA peak of the current device in TFLOP/s: its SM count x 128 lanes x 2 flop x the
    maximum SM clock (the measured one from MEASURED_PEAKS.json where present)."""
    import torch
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    peaks = measured_peaks()
    mhz = float(peaks.get("sm_max_mhz", SM_MAX_MHZ_FALLBACK)) if peaks else SM_MAX_MHZ_FALLBACK
    return sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12, f"{sms} SMs x 128 FP32 lanes x 2 flop x {mhz:.0f} MHz"


def rooflines(abytes: float, aflops: float, kernel_ms: float, traffic):
    """(binding, other) roofline objects of a kernel time: HBM against the measured copy
    bandwidth, FP32 ALU against the device's FMA peak; the binding one has the longer ideal time."""
    peaks = measured_peaks()
    hbm_peak = peaks["hbm_gbs"] if peaks else HBM_PEAK_FALLBACK
    alu_peak, alu_src = device_alu_peak()
    hbm_ach = abytes / (kernel_ms * 1e-3) / 1e9
    alu_ach = aflops / (kernel_ms * 1e-3) / 1e12
    hbm_obj = {"bound": "hbm", "achieved": hbm_ach, "peak": hbm_peak, "unit": "GB/s", "frac": hbm_ach / hbm_peak,
               "traffic": traffic, "algorithmic_bytes": abytes, "peak_source": "measured" if peaks else "fallback"}
    alu_obj = {"bound": "alu", "achieved": alu_ach, "peak": alu_peak, "unit": "TFLOP/s", "frac": alu_ach / alu_peak,
               "traffic": traffic, "algorithmic_flops": aflops, "peak_source": alu_src}
    t_hbm, t_alu = abytes / (hbm_peak * 1e9), aflops / (alu_peak * 1e12)
    return (alu_obj, hbm_obj) if t_alu > t_hbm else (hbm_obj, alu_obj)


def algorithmic_bytes(E, N, nnz, nen, q, s=4):
    """conn + coordinates and velocity + per-equation k, s, phi + values and RHS written once."""
    return 4 * E * nen + 6 * N * s + 3 * q * N * s + q * (nnz + N) * s


def algorithmic_flops_per_elem_eq(nen, ng=None):
    """Multiply-adds of the operator in its direct form, per element and equation: the rank-NG
    Galerkin/SUPG product (NG NEN^2), the symmetric diffusion sum (NG NEN(NEN+1)/2) and the
    interpolation/test-function/RHS vectors (6 NG NEN); NG = NEN except for the pyramid (12)."""
    ng = nen if ng is None else ng
    return 2 * (ng * nen * nen + ng * nen * (nen + 1) // 2 + 6 * ng * nen)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return None


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.dev = device_index

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.dev)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def kernel_source_digest():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2107_11541_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        if fn.endswith((".cu", ".cuh")):
            with open(os.path.join(csrc, fn), "rb") as f:
                h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current kernels."""
    path = os.path.join(ROOT, "profiles", f"dram_traffic_{workload}.txt")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_digest") != kernel_source_digest():
        return None
    try:
        return float(vals["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def make(workload: str, n=None):
    """The named workload with FP32 fields (the values the FP32 path consumes; the oracle widens
    them); ``n`` shrinks it to n cells per axis (profiling captures only)."""
    return G.make_workload(WORKLOADS[workload], n=n, dtype=np.float32)


def cpu_oracle_sample(w, budget_s: float):
    """Oracle throughput on the first elements of the workload (all equations), single thread."""
    import oracle as O
    m = w.mesh
    q = w.fields.n_eq
    n0 = 64 if m.elem_type == G.HEX27 else 512
    c0, k0, a0 = _oracle_submesh(m, w.fields, 0, n0)
    rp0, ci0, _ = O.pattern(m.elem_type, k0, c0.shape[0], with_pos=False)
    t0 = time.perf_counter()
    O.assemble(m.elem_type, c0, k0, rp0, ci0, G.Fields(*a0, w.fields.dt))
    rate = n0 / max(time.perf_counter() - t0, 1e-9)
    ne = int(min(m.n_elem, max(n0, rate * budget_s)))
    c, k, a = _oracle_submesh(m, w.fields, 0, ne)
    rp, ci, _ = O.pattern(m.elem_type, k, c.shape[0], with_pos=False)
    f = G.Fields(*a, w.fields.dt)
    t0 = time.perf_counter()
    O.assemble(m.elem_type, c, k, rp, ci, f)
    dt = time.perf_counter() - t0
    return ne, q, dt, (rp, ci)


def _oracle_submesh(m, f, e0, e1):
    """Elements [e0, e1) as a compact mesh: their nodes renumbered in ascending order."""
    conn = m.conn[e0:e1]
    nodes, inv = np.unique(conn, return_inverse=True)
    arrays = tuple(np.ascontiguousarray(a[:, nodes].astype(np.float32).astype(np.float64))
                   for a in (f.velocity, f.diffusivity, f.reaction, f.phi_old))
    return np.ascontiguousarray(m.coords[nodes]), inv.reshape(conn.shape).astype(np.int32), arrays


def _oracle_worker(elem_type, coords, conn, arrays, dt, reps, barrier, out):
    """One host core of the all-cores oracle timing: the unmodified oracle assembles this
    process's elements ``reps`` times; every repetition starts at the barrier."""
    try:
        import oracle as O
        f = G.Fields(*arrays, dt)
        rp, ci, _ = O.pattern(elem_type, conn, coords.shape[0], with_pos=False)
        times = []
        for _ in range(reps):
            barrier.wait(timeout=600)
            t0 = time.perf_counter()
            O.assemble(elem_type, coords, conn, rp, ci, f)
            times.append(time.perf_counter() - t0)
        out.put((int(conn.shape[0]), times))
    except Exception as exc:  # reported to the parent, which raises
        barrier.abort()
        out.put((-1, repr(exc)))


def oracle_all_cores(w, per_worker_s: float, reps: int):
    """The FP64 oracle on all host cores: one spawned process per core, each assembling its own
    contiguous element chunk into its own outputs (no shared writes, the oracle unchanged).
    Returns (elements x equations per second per timed repetition, processes, elements timed);
    a repetition's rate is all processes' units over the slowest process's time."""
    import multiprocessing as mp
    import oracle as O
    m = w.mesh
    f = w.fields  # each chunk's columns are rounded to FP32 (the arrays the GPU path consumes)
    q = f.n_eq
    procs = max(1, len(os.sched_getaffinity(0)))
    n0 = 64 if m.elem_type == G.HEX27 else 512
    c0, k0, a0 = _oracle_submesh(m, f, 0, n0)
    rp0, ci0, _ = O.pattern(m.elem_type, k0, c0.shape[0], with_pos=False)
    f0 = G.Fields(*a0, f.dt)
    t0 = time.perf_counter()
    O.assemble(m.elem_type, c0, k0, rp0, ci0, f0)
    rate = n0 / max(time.perf_counter() - t0, 1e-9)  # elements per second on one core
    chunk = int(min(m.n_elem // procs, max(n0, rate * per_worker_s)))
    ctx = mp.get_context("spawn")
    barrier, out = ctx.Barrier(procs), ctx.Queue()
    workers = []
    for i in range(procs):
        c, k, arr = _oracle_submesh(m, f, i * chunk, (i + 1) * chunk)
        workers.append(ctx.Process(target=_oracle_worker, args=(m.elem_type, c, k, arr, f.dt, reps, barrier, out)))
    for pr in workers:
        pr.start()
    try:
        res = [out.get(timeout=900) for _ in workers]
    finally:
        for pr in workers:
            pr.join(timeout=60)
    bad = [r[1] for r in res if r[0] < 0]
    if bad:
        raise RuntimeError(f"oracle worker failed: {bad[0]}")
    units = sum(r[0] for r in res) * q
    rates = [units / max(r[1][k] for r in res) for k in range(reps)]
    return rates, procs, procs * chunk


def run_reference(args, w, rank):
    if rank != 0:
        return
    m = w.mesh
    q = w.fields.n_eq
    reps = args.warmup + args.steps
    rates, procs, ne = oracle_all_cores(w, max(2.0, 120.0 / max(1, reps)), reps)
    value = len(rates[args.warmup:]) / sum(1.0 / r for r in rates[args.warmup:])  # units over the summed times
    t = ne * q / value
    sample = (f"elements [0, {ne}) of {m.n_elem} in {procs} contiguous chunks, one process per host core, "
              f"all {q} equations, per step")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": dict(config_dict(args.workload, w, closed_form_nnz(args.workload, m.n_cells)),
                          sampled=f"each step times elements [0, {ne}) of {m.n_elem}"),
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def field_update_parity(mesh, phi0, phi_gpu, prm, seq):
    """Max |phi_gpu - oracle| on 4096 sampled nodes after the bench's field updates, applied
    with the parameter rows ``seq`` in order (warm-up steps, the update timed outside the
    graph, then the graph's steps)."""
    import oracle as O
    rng = np.random.default_rng(7)
    idx = np.sort(rng.choice(mesh.n_node, size=min(4096, mesh.n_node), replace=False))
    phi = phi0[:, idx].astype(np.float64)
    for s in seq:
        phi = O.update_fields(mesh.coords[idx], phi, prm[s].astype(np.float64))
    err = float(np.abs(phi_gpu[:, idx] - phi).max())
    return {"nodes": int(idx.size), "updates": len(seq), "max_abs_err": err, "tol": 1e-5, "pass": err <= 1e-5}


def aggregate_over_ranks(ms, kernel_ms, units_per_rank, world, dist, device):
    """Replica runs: the slowest rank's step time (max over ranks) and the whole job's rate,
    every rank's units divided by that time.  dist is torch.distributed or None (one rank)."""
    if dist is not None:
        import torch
        t = torch.tensor([ms, kernel_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms, kernel_ms = float(t[0]), float(t[1])
    return ms, kernel_ms, units_per_rank * world / (ms * 1e-3)


def tuned_dict(tc: dict) -> dict:
    """The autotuned configuration (fea_tuned_config) in words."""
    return {"scatter": {1: "atomic", 2: "rowowned", 3: "gather"}.get(tc["scatter"], str(tc["scatter"])),
            "eq_groups": tc["eq_groups"],
            "mapping": {1: "type kernel", 2: "warp per element"}.get(tc["mapping"], str(tc["mapping"])),
            "elems_per_cta": tc["elems_per_cta"] or "rule",
            "contraction": {1: "cuda cores", 2: "tensor cores bf16x3", 3: "tensor cores 3xtf32"}.get(
                tc["contraction"], str(tc["contraction"])),
            "tuning_from_cache": bool(tc["from_cache"])}


def config_dict(workload, w, nnz):
    m = w.mesh
    return {"workload": workload, "elem_type": G.NAMES[m.elem_type], "elements": m.n_elem, "nodes": m.n_node,
            "nnz": nnz, "n_eq": w.fields.n_eq, "precision": "f32_fused",
            "l2": "no flush: inputs + outputs per step exceed the 129 MB L2"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS) + sorted(MIXED_WORKLOADS))
    ap.add_argument("--scatter", type=int, default=0, help="0 auto, 1 atomic, 2 row-owned, 3 gather")
    ap.add_argument("--mapping", type=int, default=0,
                    help="Gauss-point mapping: 0 auto, 1 type kernel, 2 warp per element, 3 two threads per item "
                         "(row-owned Hex8)")
    ap.add_argument("--eq-groups", type=int, default=0, help="row-owned equation groups (0: tuned or 1)")
    ap.add_argument("--host-parts", type=int, default=0, help="parts of the end-to-end call (0: automatic)")
    ap.add_argument("--contraction", type=int, default=0,
                    help="Hex27 element matrices: 0 auto, 1 CUDA cores, 2 tensor cores bf16x3, 3 tensor cores bf16x6")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-f64", action="store_true")
    ap.add_argument("--no-parity", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--cells", type=int, default=None, help="shrink to this many cells per axis (profiling)")
    ap.add_argument("--residual", action="store_true",
                    help="also time the matrix-free residual r = b - A phi (fea_residual) on the same workload")
    ap.add_argument("--spmv", action="store_true",
                    help="also time the batched SpMV y_q = A_q x_q (fea_spmv) on the assembled matrices")
    ap.add_argument("--pcg", action="store_true",
                    help="also time the batched Jacobi-preconditioned CG (fea_pcg) on the MASS + DIFF matrices")
    ap.add_argument("--explicit", action="store_true",
                    help="also time explicit SSP-RK3 steps (fea_explicit_step: three matrix-free operator "
                         "applications with the lumped mass) on the same workload")
    ap.add_argument("--laplacian", action="store_true",
                    help="also time the Laplacian of the same mesh (the DIFF term alone, k = 1, one equation)")
    ap.add_argument("--graph", type=int, default=None,
                    help="1: time the K steps as one CUDA graph of K (assemble, field update) time steps "
                         "(default on for hex8_256_32eq)")
    ap.add_argument("--side", default=None,
                    help="comma-separated further workloads measured after the headline one (their results go "
                         "into 'workloads'); default: the other paper-shaped workloads when the headline is the "
                         "default workload on one GPU, 'none' to skip")
    args = ap.parse_args()
    if args.graph is None:
        args.graph = 1 if args.workload == "hex8_256_32eq" else 0
    if args.side is None:
        args.side = list(SIDE_WORKLOADS) if (args.workload == DEFAULT_WORKLOAD and args.cells is None) else []
    elif args.side == "none":
        args.side = []
    else:
        args.side = [x for x in args.side.split(",") if x]
        bad = [x for x in args.side if x not in WORKLOADS]
        if bad:
            ap.error(f"unknown side workloads: {bad}")
    rank, world, local = dist_env()
    if args.workload in MIXED_WORKLOADS:
        run_mixed(args, rank, world, local)
        return
    w = make(args.workload, args.cells)
    if args.impl == "reference":
        run_reference(args, w, rank)
        return
    w0 = w  # the workload as drawn (the graph mode replaces w with the stepped field for its parity check)

    import torch
    from paper_2107_11541_gb300 import fea

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    m, fld = w.mesh, w.fields
    q = fld.n_eq
    stream = torch.cuda.Stream()
    h = fea.fea_mesh_create(m.coords, m.conn, m.elem_type, stream)
    p = fea.fea_pattern_build(h)
    nnz = fea.fea_pattern_get(p)[3]
    f32 = fld if fld.diffusivity.dtype == np.float32 else fld.astype(np.float32)
    with torch.cuda.stream(stream):
        dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda(non_blocking=False)
               for a in (f32.velocity, f32.diffusivity, f32.reaction, f32.phi_old)]
        values = torch.empty((q, nnz), dtype=torch.float32, device="cuda")
        rhs = torch.empty((q, m.n_node), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    opts = fea.fea_default_opts(scatter=args.scatter, contraction=args.contraction, mapping=args.mapping,
                                eq_groups=args.eq_groups)

    def step(ev=None):
        if ev is not None:
            opts.event_begin, opts.event_end = ev[0].cuda_event, ev[1].cuda_event
        else:
            opts.event_begin = opts.event_end = None
        fea.fea_assemble(h, p, *dev, fld.dt, q, opts, values, rhs)

    graph = None
    if args.graph:
        # time steps: assemble, then the seeded field perturbation, K of them in one CUDA graph
        prm = torch.from_numpy(G.step_params(max(args.steps, args.warmup), q)).cuda()
        for s in range(args.warmup):
            step()
            fea.fea_update_fields(h, dev[3], q, prm[s])
    else:
        for _ in range(args.warmup):
            step()
    fea.fea_sync(h)
    n_kev = 1 if args.graph else args.steps
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_kev)]
    for a, b in kev:  # torch creates the CUDA events lazily, on first record
        a.record(stream)
        b.record(stream)
    update_ms = None
    if args.graph:
        # kernel times outside the graph: one assembly and one field update, each between events
        step(kev[0])
        ua, ub = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ua.record(stream)
        fea.fea_update_fields(h, dev[3], q, prm[0])
        ub.record(stream)
        torch.cuda.synchronize()
        update_ms = ua.elapsed_time(ub)
        opts.event_begin = opts.event_end = None
        graph = fea.fea_graph_capture_steps(h, p, *dev, fld.dt, q, opts, values, rhs, prm, args.steps)
    t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = fea.fea_kernel_launches()
    clocks.start()
    time.sleep(0.3)
    t0e.record(stream)
    if graph is not None:
        fea.fea_graph_launch(graph)
    else:
        for s in range(args.steps):
            step(kev[s])
    t1e.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = fea.fea_kernel_launches() - launches0
    fea.fea_sync(h)
    if graph is not None:
        fea.fea_graph_destroy(graph)
    ms = t0e.elapsed_time(t1e) / args.steps
    kernel_ms = sum(a.elapsed_time(b) for a, b in kev) / len(kev)
    ms, kernel_ms, value = aggregate_over_ranks(ms, kernel_ms, m.n_elem * q, world, dist, "cuda")

    # roofline of the dominant kernel
    peaks = measured_peaks()
    hbm_peak = peaks["hbm_gbs"] if peaks else HBM_PEAK_FALLBACK
    nen = NEN[m.elem_type]
    abytes = algorithmic_bytes(m.n_elem, m.n_node, nnz, nen, q)
    aflops = algorithmic_flops_per_elem_eq(nen) * m.n_elem * q
    roof, other = rooflines(abytes, aflops, kernel_ms, profiled_traffic(args.workload))

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config_dict(args.workload, w, nnz),
           "clocks": clk, "gpu_launches": int(launches), "kernel_ms": kernel_ms, "roofline": roof,
           "roofline_other": other}
    try:
        tc = fea.fea_tuned_config(p, q)
        out["config"].update(tuned_dict(tc))
    except fea.FeaError:
        out["config"]["scatter"] = {0: "auto", 1: "atomic", 2: "rowowned", 3: "gather"}[args.scatter]
    if args.graph:
        out["graph"] = {"time_steps": args.steps, "launches": 1, "step": "assemble, then field update",
                        "update_ms": update_ms, "assemble_ms": kernel_ms}
        if rank == 0 and not args.no_parity:
            # the graph's last assembly used the field before the last update; check an eager assembly of
            # the current field instead (same code), and the updated field on sampled nodes
            fea.fea_assemble(h, p, *dev, fld.dt, q, opts, values, rhs)
            fea.fea_sync(h)
            fld = G.Fields(fld.velocity, fld.diffusivity, fld.reaction,
                           dev[3].cpu().numpy().astype(np.float64), fld.dt)
            w = G.Workload(w.name, w.mesh, fld, w.precision)
            seq = list(range(args.warmup)) + [0] + list(range(args.steps))
            out["field_update_parity"] = field_update_parity(w.mesh, f32.phi_old, fld.phi_old,
                                                             G.step_params(max(args.steps, args.warmup), q), seq)

    if rank == 0 and not args.no_parity:
        out["parity"] = sampled_parity(w, values, rhs, p, nnz)
    if args.spmv:
        xs = torch.ones((q, m.n_node), dtype=torch.float32, device="cuda")
        ys = torch.empty_like(xs)
        fea.fea_spmv(p, values, xs, ys, q, 0, stream)
        sa, sb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        sa.record(stream)
        for _ in range(5):
            fea.fea_spmv(p, values, xs, ys, q, 0, stream)
        sb.record(stream)
        torch.cuda.synchronize()
        sms = sa.elapsed_time(sb) / 5
        sbytes = 4 * q * nnz + 4 * nnz + 8 * (m.n_node + 1) + 2 * 4 * q * m.n_node  # values, colind, rowptr, x, y
        out["spmv"] = {"ms": sms, "algorithmic_bytes": sbytes, "achieved_gbs": sbytes / (sms * 1e-3) / 1e9,
                       "frac_of_hbm": sbytes / (sms * 1e-3) / 1e9 / hbm_peak}
        del xs, ys
    if args.pcg:
        # symmetric positive definite systems of the same mesh: mass + diffusion; 10 iterations with rtol 0 keep
        # every equation iterating (many more drive the mass-dominated FP32 residual to exactly 0, which stops it)
        po = fea.fea_default_opts(terms=fea.FEA_TERM_MASS | fea.FEA_TERM_DIFF, scatter=args.scatter)
        fea.fea_assemble(h, p, *dev, fld.dt, q, po, values, rhs)
        fea.fea_sync(h)
        xs = torch.zeros((q, m.n_node), dtype=torch.float32, device="cuda")
        fea.fea_pcg(p, values, rhs, xs, q, 3, 0.0, stream)  # workspace and diagonal positions
        n_it = 10
        xs.zero_()
        pa, pb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        pa.record(stream)
        iters, rel = fea.fea_pcg(p, values, rhs, xs, q, n_it, 0.0, stream)
        pb.record(stream)
        torch.cuda.synchronize()
        pms = pa.elapsed_time(pb) / max(1, int(iters.max()))
        # per iteration: the SpMV (values, colind, rowptr, p, Ap) and 13 vector passes of 4 q N bytes
        pbytes = 4 * q * nnz + 4 * nnz + 8 * (m.n_node + 1) + 2 * 4 * q * m.n_node + 13 * 4 * q * m.n_node
        out["pcg"] = {"ms_per_iteration": pms, "iterations": int(iters.max()), "rel_resid_max": float(rel.max()),
                      "algorithmic_bytes_per_iteration": pbytes, "achieved_gbs": pbytes / (pms * 1e-3) / 1e9,
                      "frac_of_hbm": pbytes / (pms * 1e-3) / 1e9 / hbm_peak,
                      "system": "MASS + DIFF terms (symmetric positive definite), b = the assembled RHS"}
        del xs
    if args.laplacian:
        # the Laplacian of the same mesh: the diffusion term alone with k = 1, one equation (Algorithm 1
        # assembles it once per run); the first call also tunes the scatter for one equation
        lf = G.Fields(np.zeros((3, m.n_node)), np.ones((1, m.n_node)), np.zeros((1, m.n_node)),
                      np.zeros((1, m.n_node)), 1.0)
        ld = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
              for a in (lf.velocity, lf.diffusivity, lf.reaction, lf.phi_old)]
        lv = torch.empty((1, nnz), dtype=torch.float32, device="cuda")
        lr = torch.empty((1, m.n_node), dtype=torch.float32, device="cuda")
        lo = fea.fea_default_opts(terms=fea.FEA_TERM_DIFF, scatter=args.scatter)
        fea.fea_assemble(h, p, *ld, lf.dt, 1, lo, lv, lr)
        fea.fea_sync(h)
        la, lb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        la.record(stream)
        for _ in range(5):
            fea.fea_assemble(h, p, *ld, lf.dt, 1, lo, lv, lr)
        lb.record(stream)
        torch.cuda.synchronize()
        lms = la.elapsed_time(lb) / 5
        out["laplacian"] = {"ms": lms, "value": m.n_elem / (lms * 1e-3), "unit": "elements/s",
                            "what": "K = sum_e int grad N_a . grad N_b (DIFF term, k = 1), FP32, one equation"}
        try:
            out["laplacian"].update(tuned_dict(fea.fea_tuned_config(p, 1, fea.FEA_TERM_DIFF)))
        except fea.FeaError:
            pass
        if rank == 0 and not args.no_parity:
            out["laplacian"]["parity"] = sampled_parity(G.Workload(w.name, m, lf, w.precision), lv, lr, p, nnz,
                                                        terms=fea.FEA_TERM_DIFF)
        del ld, lv, lr
    if args.explicit:
        phx = dev[3].clone()
        xo = fea.fea_default_opts()
        fea.fea_explicit_step(h, p, *dev[:3], phx, 1e-4, q, 3, xo)  # lumped mass and workspace
        xa, xb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        xa.record(stream)
        for _ in range(3):
            fea.fea_explicit_step(h, p, *dev[:3], phx, 1e-4, q, 3, xo)
        xb.record(stream)
        torch.cuda.synchronize()
        xms = xa.elapsed_time(xb) / 3
        out["explicit_rk3"] = {"ms_per_step": xms, "value": m.n_elem * q / (xms * 1e-3), "unit": UNIT,
                               "what": "one SSP-RK3 step of M_L dphi/dt = -(C + K + R) phi, FP32: three "
                                       "matrix-free operator applications and stage updates"}
        del phx
    if args.residual:
        r = torch.empty((q, m.n_node), dtype=torch.float32, device="cuda")
        ro = fea.fea_default_opts()
        fea.fea_residual(h, p, *dev, dev[3], fld.dt, q, ro, r)
        ra, rb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ra.record(stream)
        for _ in range(3):
            fea.fea_residual(h, p, *dev, dev[3], fld.dt, q, ro, r)
        rb.record(stream)
        torch.cuda.synchronize()
        rms = ra.elapsed_time(rb) / 3
        out["residual"] = {"ms_per_step": rms, "value": m.n_elem * q / (rms * 1e-3), "unit": UNIT,
                           "what": "matrix-free r = b - A phi_old, FP32"}
        del r

    if not args.no_f64 and rank == 0:
        q64 = q if m.n_elem * q <= 60_000_000 else 4
        d64 = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
               for a in (fld.velocity, fld.diffusivity[:q64], fld.reaction[:q64], fld.phi_old[:q64])]
        del values
        v64 = torch.empty((q64, nnz), dtype=torch.float64, device="cuda")
        r64 = torch.empty((q64, m.n_node), dtype=torch.float64, device="cuda")
        o64 = fea.fea_default_opts(precision=fea.FEA_F64_PLAIN)
        fea.fea_assemble(h, p, *d64, fld.dt, q64, o64, v64, r64)
        fea.fea_sync(h)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fea.fea_assemble(h, p, *d64, fld.dt, q64, o64, v64, r64)
        b.record(stream)
        torch.cuda.synchronize()
        t64 = a.elapsed_time(b)
        v_f64 = m.n_elem * q64 / (t64 * 1e-3)
        out["fp64_plain"] = {"value": v_f64, "unit": UNIT, "ms_per_step": t64, "equations_timed": q64,
                             "speedup_f32_fused": value / world / v_f64}
        del v64, r64, d64
        values = torch.empty((q, nnz), dtype=torch.float32, device="cuda")

    if not args.no_e2e:
        out["e2e"] = end_to_end(h, p, f32, m, nnz, q, stream, min(args.steps, 5), world, dist, values_dev=values,
                                parity_of=(w0, None) if rank == 0 and not args.no_parity else None,
                                host_parts=args.host_parts)

    if rank == 0 and world == 1 and not args.no_cpu:
        w = w0
        ne, qq, dt, _ = cpu_oracle_sample(w, args.cpu_budget)
        single = {"value": ne * qq / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                  "sample": f"elements [0, {ne}) of {m.n_elem}, all {qq} equations, FP64 C oracle, single thread"}
        rates, procs, ne_all = oracle_all_cores(w, args.cpu_budget / 3.0, 2)
        out["cpu_baseline"] = {"value": rates[-1], "unit": UNIT, "cores": procs, "kind": "oracle",
                               "sample": f"elements [0, {ne_all}) of {m.n_elem} in {procs} contiguous chunks, one "
                                         f"process per host core, all {qq} equations, FP64 C oracle"}
        out["cpu_baseline_single"] = single
    fea.fea_pattern_destroy(p)
    fea.fea_mesh_destroy(h)
    if world == 1 and args.side:
        del values, rhs, dev
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        out["workloads"] = {nm: side_workload(nm, max(3, min(args.steps, 10)), args.warmup, not args.no_parity)
                            for nm in args.side}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def side_workload(name: str, steps: int, warmup: int, parity: bool):
    """One more paper-shaped workload measured like the headline one (device-resident inputs, the
    autotuned FP32 fused path, CUDA events around every assembly), with its rooflines, clocks,
    sampled parity against the oracle and the plain FP64 path on the same GPU."""
    import torch
    from paper_2107_11541_gb300 import fea
    w = make(name)
    m, fld = w.mesh, w.fields
    q = fld.n_eq
    stream = torch.cuda.Stream()
    h = fea.fea_mesh_create(m.coords, m.conn, m.elem_type, stream)
    p = fea.fea_pattern_build(h)
    nnz = fea.fea_pattern_get(p)[3]
    f32 = fld if fld.diffusivity.dtype == np.float32 else fld.astype(np.float32)
    with torch.cuda.stream(stream):
        dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (f32.velocity, f32.diffusivity,
                                                                          f32.reaction, f32.phi_old)]
        values = torch.empty((q, nnz), dtype=torch.float32, device="cuda")
        rhs = torch.empty((q, m.n_node), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    opts = fea.fea_default_opts()
    for _ in range(warmup):
        fea.fea_assemble(h, p, *dev, fld.dt, q, opts, values, rhs)
    fea.fea_sync(h)
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in kev:
        a.record(stream)
        b.record(stream)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    for a, b in kev:
        opts.event_begin, opts.event_end = a.cuda_event, b.cuda_event
        fea.fea_assemble(h, p, *dev, fld.dt, q, opts, values, rhs)
    torch.cuda.synchronize()
    clk = clocks.stop()
    opts.event_begin = opts.event_end = None
    fea.fea_sync(h)
    kernel_ms = sum(a.elapsed_time(b) for a, b in kev) / len(kev)
    nen = NEN[m.elem_type]
    roof, other = rooflines(algorithmic_bytes(m.n_elem, m.n_node, nnz, nen, q),
                            algorithmic_flops_per_elem_eq(nen) * m.n_elem * q, kernel_ms, profiled_traffic(name))
    res = {"config": config_dict(name, w, nnz), "steps": steps, "warmup": warmup, "kernel_ms": kernel_ms,
           "value": m.n_elem * q / (kernel_ms * 1e-3), "unit": UNIT, "roofline": roof, "roofline_other": other,
           "clocks": clk}
    try:
        res["config"].update(tuned_dict(fea.fea_tuned_config(p, q)))
    except fea.FeaError:
        pass
    if parity:
        res["parity"] = sampled_parity(w, values, rhs, p, nnz)
    del values
    q64 = q if m.n_elem * q <= 60_000_000 else 4
    d64 = [torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
           for a in (fld.velocity, fld.diffusivity[:q64], fld.reaction[:q64], fld.phi_old[:q64])]
    v64 = torch.empty((q64, nnz), dtype=torch.float64, device="cuda")
    r64 = torch.empty((q64, m.n_node), dtype=torch.float64, device="cuda")
    o64 = fea.fea_default_opts(precision=fea.FEA_F64_PLAIN)
    fea.fea_assemble(h, p, *d64, fld.dt, q64, o64, v64, r64)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    fea.fea_assemble(h, p, *d64, fld.dt, q64, o64, v64, r64)
    b.record(stream)
    torch.cuda.synchronize()
    t64 = a.elapsed_time(b)
    v_f64 = m.n_elem * q64 / (t64 * 1e-3)
    res["fp64_plain"] = {"value": v_f64, "unit": UNIT, "ms_per_step": t64, "equations_timed": q64,
                         "speedup_f32_fused": res["value"] / v_f64}
    del v64, r64, d64, dev, rhs
    fea.fea_pattern_destroy(p)
    fea.fea_mesh_destroy(h)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return res


def make_mixed(workload: str, n=None):
    """The Hex8 / Pyr5 / Pen6 layered unit cube (interior nodes moved by up to 0.1 h) and its
    fields, seeded like the other workloads."""
    cells, q = MIXED_WORKLOADS[workload]
    mm = G.mixed_mesh(n or cells)
    rng = np.random.default_rng(G.SEED_BASE + 100)
    G.perturb_interior(mm, rng, 0.1)
    return mm, G.draw_fields(rng, mm.coords, q, 50.0)


def mixed_parity(mm, fields, values, rhs, rowptr, colind, n_rows=48, seed=5):
    """Sampled rows of a mesh of several element types against the oracle: the elements incident
    to the sampled nodes, of every block, assembled by the oracle give those rows complete."""
    import oracle as O
    rng = np.random.default_rng(seed)
    rows = np.unique(np.concatenate([[0, mm.n_node - 1], rng.integers(0, mm.n_node, n_rows)]))
    sub = [(t, c[np.isin(c, rows).any(axis=1)]) for t, c in mm.blocks]
    sub = [(t, c) for t, c in sub if c.shape[0] > 0]
    srp, sci, _ = O.pattern_mixed(sub, mm.n_node, with_pos=False)
    wide = fields.astype(np.float32).astype(np.float64)
    ref, refb, _, absb = O.assemble_mixed(mm.coords, sub, srp, sci, wide, with_abs=True)
    worst_a = worst_b = 0.0
    for r in rows:
        k0, k1, s0, s1 = rowptr[r], rowptr[r + 1], srp[r], srp[r + 1]
        assert np.array_equal(colind[k0:k1], sci[s0:s1])
        got = values[:, k0:k1].astype(np.float64)
        want = ref[:, s0:s1]
        den = np.sqrt((want ** 2).sum(axis=1))
        worst_a = max(worst_a, float((np.sqrt(((got - want) ** 2).sum(axis=1)) / np.where(den > 0, den, 1)).max()))
        eb = np.abs(rhs[:, r].astype(np.float64) - refb[:, r]) / np.where(absb[:, r] > 0, absb[:, r], 1.0)
        worst_b = max(worst_b, float(eb.max()))
    return {"rows": int(rows.size), "max_row_err_A": worst_a, "max_err_b": worst_b, "tol": 1e-5,
            "pass": worst_a <= 1e-5 and worst_b <= 1e-5}


def run_mixed(args, rank, world, local):
    """A mesh of Hex8, Pyr5 and Pen6 blocks: the same measurement as the single-type workloads
    (device-resident step, end to end, FP64 plain, sampled parity, oracle on the host)."""
    mm, fld = make_mixed(args.workload, args.cells)
    q = fld.n_eq
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the reference arm times the paper-shaped "
                              "configurations; this workload has no oracle-on-all-cores line"}), flush=True)
        return
    import torch
    from paper_2107_11541_gb300 import fea
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.Stream()
    h = fea.fea_mesh_create_mixed(mm.coords, mm.blocks, stream)
    p = fea.fea_pattern_build(h)
    r_, c_, _, nnz = fea.fea_pattern_get(p)
    f32 = fld if fld.diffusivity.dtype == np.float32 else fld.astype(np.float32)
    with torch.cuda.stream(stream):
        dev = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (f32.velocity, f32.diffusivity,
                                                                          f32.reaction, f32.phi_old)]
        values = torch.empty((q, nnz), dtype=torch.float32, device="cuda")
        rhs = torch.empty((q, mm.n_node), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    opts = fea.fea_default_opts()
    for _ in range(args.warmup):
        fea.fea_assemble(h, p, *dev, fld.dt, q, opts, values, rhs)
    fea.fea_sync(h)
    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for a, b in kev:
        a.record(stream)
        b.record(stream)
    t0e, t1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = fea.fea_kernel_launches()
    clocks.start()
    time.sleep(0.3)
    t0e.record(stream)
    for a, b in kev:
        opts.event_begin, opts.event_end = a.cuda_event, b.cuda_event
        fea.fea_assemble(h, p, *dev, fld.dt, q, opts, values, rhs)
    t1e.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = fea.fea_kernel_launches() - launches0
    fea.fea_sync(h)
    opts.event_begin = opts.event_end = None
    ms = t0e.elapsed_time(t1e) / args.steps
    kernel_ms = sum(a.elapsed_time(b) for a, b in kev) / len(kev)
    ms, kernel_ms, value = aggregate_over_ranks(ms, kernel_ms, mm.n_elem * q, world, dist, "cuda")
    abytes = sum(4 * c.size for _, c in mm.blocks) + 6 * mm.n_node * 4 + 3 * q * mm.n_node * 4 + \
        q * (nnz + mm.n_node) * 4
    aflops = sum(algorithmic_flops_per_elem_eq(G.NEN[t], NG[t]) * c.shape[0] for t, c in mm.blocks) * q
    roof, other = rooflines(abytes, aflops, kernel_ms, None)
    config = {"workload": args.workload, "elem_types": {G.NAMES[t]: int(c.shape[0]) for t, c in mm.blocks},
              "elements": mm.n_elem, "nodes": mm.n_node, "nnz": int(nnz), "n_eq": q, "precision": "f32_fused",
              "l2": "no flush: inputs + outputs per step exceed the 129 MB L2", "scatter": "atomic"}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config, "clocks": clk,
           "gpu_launches": int(launches), "kernel_ms": kernel_ms, "roofline": roof, "roofline_other": other}
    if rank == 0 and not args.no_parity:
        rowptr = torch.as_tensor(fea._DevView(r_, (mm.n_node + 1,), "<i8"), device="cuda").cpu().numpy()
        colind = torch.as_tensor(fea._DevView(c_, (nnz,), "<i4"), device="cuda").cpu().numpy()
        out["parity"] = mixed_parity(mm, fld, values.cpu().numpy(), rhs.cpu().numpy(), rowptr, colind)
    if not args.no_f64:
        d64 = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (fld.velocity, fld.diffusivity,
                                                                          fld.reaction, fld.phi_old)]
        v64 = torch.empty((q, nnz), dtype=torch.float64, device="cuda")
        r64 = torch.empty((q, mm.n_node), dtype=torch.float64, device="cuda")
        o64 = fea.fea_default_opts(precision=fea.FEA_F64_PLAIN)
        fea.fea_assemble(h, p, *d64, fld.dt, q, o64, v64, r64)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fea.fea_assemble(h, p, *d64, fld.dt, q, o64, v64, r64)
        b.record(stream)
        torch.cuda.synchronize()
        t64 = a.elapsed_time(b)
        v_f64 = mm.n_elem * q / (t64 * 1e-3)
        out["fp64_plain"] = {"value": v_f64, "unit": UNIT, "ms_per_step": t64, "equations_timed": q,
                             "speedup_f32_fused": value / world / v_f64}
        del d64, v64, r64
    if not args.no_e2e:
        out["e2e"] = end_to_end(h, p, f32, mm, nnz, q, stream, min(args.steps, 5), world, dist)
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle as O
        sub = [(t, c[: max(1, c.shape[0] // 64)]) for t, c in mm.blocks]
        srp, sci, _ = O.pattern_mixed(sub, mm.n_node, with_pos=False)
        wide = fld.astype(np.float32).astype(np.float64)
        t0 = time.perf_counter()
        O.assemble_mixed(mm.coords, sub, srp, sci, wide)
        dt_cpu = time.perf_counter() - t0
        ne = sum(c.shape[0] for _, c in sub)
        out["cpu_baseline"] = {"value": ne * q / dt_cpu, "unit": UNIT, "cores": 1, "kind": "oracle",
                               "sample": f"the first 1/64 of every block ({ne} of {mm.n_elem} elements), all {q} "
                                         f"equations, FP64 C oracle, single thread"}
    fea.fea_pattern_destroy(p)
    fea.fea_mesh_destroy(h)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def sampled_parity(w, values, rhs, p, nnz, n_rows=48, seed=5, terms=None, wide=None):
    """Sampled full-size rows against the oracle (computed row by row from incident elements).
    values/rhs may be device or host tensors; ``wide`` is the FP32 fields widened to FP64 (made
    here when not given)."""
    import oracle as O
    from paper_2107_11541_gb300 import fea
    m = w.mesh
    rp_t, ci_t, _ = fea.pattern_tensors(p, m.n_node, 0, NEN[m.elem_type])
    rp = rp_t.cpu().numpy()
    if wide is None:
        wide = w.fields.astype(np.float32).astype(np.float64)
    rs = O.RowSampler(m.elem_type, m.coords, m.conn, wide, O.ALL_TERMS if terms is None else terms)
    rng = np.random.default_rng(seed)
    rows = np.unique(np.concatenate([[0, m.n_node - 1], rng.integers(0, m.n_node, n_rows)]))
    worst_a = worst_b = 0.0
    plain = (0.0, 0.0)
    for r in rows:
        cols, ref, _, refb, absb = rs.row(r)
        k0, k1 = rp[r], rp[r + 1]
        assert np.array_equal(ci_t[k0:k1].cpu().numpy(), cols)
        got = values[:, k0:k1].double().cpu().numpy()
        ea = np.sqrt(((got - ref) ** 2).sum(axis=1) / (ref ** 2).sum(axis=1)).max()
        gb = rhs[:, r].double().cpu().numpy()
        eb = (np.abs(gb - refb) / np.where(absb > 0, absb, 1.0)).max()
        nz = np.abs(refb) > 0
        if nz.any():
            pl = np.abs(gb - refb)[nz] / np.abs(refb)[nz]
            i = int(np.argmax(pl))
            if pl[i] > plain[0]:
                plain = (float(pl[i]), float(absb[nz][i] / np.abs(refb)[nz][i]))
        worst_a, worst_b = max(worst_a, ea), max(worst_b, eb)
    return {"rows": int(len(rows)), "max_row_err_A": worst_a, "max_err_b": worst_b, "tol": 1e-5,
            "pass": bool(worst_a <= 1e-5 and worst_b <= 1e-5),
            "max_err_b_plain": plain[0], "cancellation_ratio_of_that_row": plain[1],
            "err_b_definitions": "max_err_b = |b - b*| / (sum of the magnitudes of b*'s Gauss-point summands); "
                                 "max_err_b_plain = |b - b*| / |b*|"}


def host_memory_available() -> int:
    """Bytes this process can still take on the host: MemAvailable, capped by the cgroup limit."""
    avail = None
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                avail = int(line.split()[1]) * 1024
    except OSError:
        pass
    try:
        lim = open("/sys/fs/cgroup/memory.max").read().strip()
        cur = int(open("/sys/fs/cgroup/memory.current").read().strip())
        if lim != "max":
            left = int(lim) - cur
            avail = left if avail is None else min(avail, left)
    except (OSError, ValueError):
        pass
    return avail if avail is not None else 0


def end_to_end(h, p, f32, m, nnz, q, stream, steps, world, dist, values_dev=None, parity_of=None, host_parts=0):
    """Same metric through fea_assemble_host: pinned host inputs copied in, values and RHS read back.
    Also the copy floor of this box: one cudaMemcpyAsync per direction of the step's bytes between
    pinned host memory and the device (values_dev, the device-resident values of the same size, is
    the device end of the output copy), and, when ``parity_of`` = (workload, wide fields) is given,
    sampled rows of the last step's host outputs against the oracle."""
    import torch
    from paper_2107_11541_gb300 import fea
    need = 4 * (f32.velocity.size + f32.diffusivity.size + f32.reaction.size + f32.phi_old.size + q * (nnz + m.n_node))
    local = int(os.environ.get("LOCAL_WORLD_SIZE", world))  # ranks on this host, each pinning its own buffers
    avail = host_memory_available()
    if need * local > 0.6 * avail:  # pinned host buffers this large would crowd the host
        return {"skipped": f"the pinned host buffers ({need / 1e9:.1f} GB per rank, {local} ranks on this host) "
                           f"exceed 60% of the host memory available ({avail / 1e9:.1f} GB)"}
    pin = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
           for a in (f32.velocity, f32.diffusivity, f32.reaction, f32.phi_old)]
    hv = torch.empty((q, nnz), dtype=torch.float32).pin_memory()
    hr = torch.empty((q, m.n_node), dtype=torch.float32).pin_memory()
    opts = fea.fea_default_opts(host_parts=host_parts)
    fea.fea_assemble_host(h, p, *pin, f32.dt, q, opts, hv, hr)
    times = []
    for _ in range(steps):
        if dist is not None:
            dist.barrier()
        t0 = time.perf_counter()
        fea.fea_assemble_host(h, p, *pin, f32.dt, q, opts, hv, hr)
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    if dist is not None:
        tt = torch.tensor([t], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt[0])
    h2d = sum(x.numel() * 4 for x in pin)
    d2h = (hv.numel() + hr.numel()) * 4
    out = {"value": m.n_elem * q * world / t, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "ms_per_step": t * 1e3, "api": "fea_assemble_host"}
    if values_dev is not None:
        # the copy floor: the largest input and the values, one copy each way, CUDA events on the stream
        big = max(pin, key=lambda x: x.numel())
        dbig = torch.empty(big.shape, dtype=big.dtype, device="cuda")
        ea, eb, ec = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        with torch.cuda.stream(stream):
            dbig.copy_(big, non_blocking=True)
            ea.record(stream)
            dbig.copy_(big, non_blocking=True)
            eb.record(stream)
            hv.copy_(values_dev, non_blocking=True)
            ec.record(stream)
        torch.cuda.synchronize()
        h2d_gbs = big.numel() * 4 / (ea.elapsed_time(eb) * 1e-3) / 1e9
        d2h_gbs = hv.numel() * 4 / (eb.elapsed_time(ec) * 1e-3) / 1e9
        floor_ms = (h2d / h2d_gbs + d2h / d2h_gbs) / 1e9 * 1e3
        out["copy_floor"] = {"h2d_gbs": h2d_gbs, "d2h_gbs": d2h_gbs, "ms": floor_ms,
                             "what": "one cudaMemcpyAsync per direction between pinned host memory and the "
                                     "device (largest input array, then the values), CUDA events; ms = the "
                                     "step's bytes at those rates, copies not overlapped"}
        del dbig
        # the timed steps ended with values on the host: redo one so the parity check sees them
        fea.fea_assemble_host(h, p, *pin, f32.dt, q, opts, hv, hr)
    if parity_of is not None:
        wl, wide = parity_of
        out["parity"] = sampled_parity(wl, hv, hr, p, nnz, wide=wide)
    del pin, hv, hr
    return out


if __name__ == "__main__":
    main()
