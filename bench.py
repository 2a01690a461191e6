"""Benchmark: HB butterfly apply throughput (N_v * RHS / s) on one GB300.

Workload: 2D constant-gradient velocity c = 1 + 0.5 z on the unit square,
256 x 256 cells (N_v = 65536), omega = 2 pi * 32, n_I = 16 Chebyshev tables,
HODBF / butterfly compression at eps = 1e-6, 16 seeded complex Gaussian
right-hand sides, mixed precision (factors and vectors as split-BF16 pairs,
three BF16 tensor-core products per complex multiply-add, FP32
accumulation).  One step = one hb_apply: gather + scale into
tree order, every butterfly level of every HODBF block, dense leaves,
scatter back - the whole hot path of the apply.  The factors (hundreds of MB)
exceed the 129 MB L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  ``--impl reference`` times the FP64 CPU oracle (the
only reference this method has) on a bounded row sample of the same
workload.  Under torchrun (N > 1) every rank runs an independent replica of
the workload (the operator does not shard across GPUs here) and rank 0
reports the aggregate.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2210_02698_gb300 import workloads as W  # noqa: E402

WORKLOAD = "grad256"
METRIC = "HB butterfly apply N_v·RHS/s at rel-L2≤1e-4, % roofline, vs plain FP64 GPU"
UNIT = "N_v*RHS/s"


def describe(w):
    """The workload as a config string: medium, grid, frequency, tables, tolerance, sources."""
    med = {"grad": "c=1+0.5z", "homog": "n=1"}.get(w.medium.key.split("_")[0], w.medium.key)
    return (f"{w.name}: {med}, {w.N}x{w.N} cells (N_v={w.grid.Nv}), omega=2pi*{w.omega / (2 * math.pi):g}, "
            f"n_I={w.n_I}, eps={w.eps:g}, chi={w.chi:g}, leaf {w.leaf}, {w.nrhs} RHS ({w.rhs_kind})")


def table_path(w):
    return os.path.join(ROOT, "tests", "golden", "tables", f"{w.medium.key}_nI{w.n_I}.npz")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


PROFILE = os.path.join(ROOT, "profiles", "bf_step_kernel_grad256.md")
PROFILE_WORKLOAD = "grad256"      # the workload the ncu summary was captured on
KERNEL_SOURCES = ["paper_2210_02698_gb300/csrc/bf_mma.cu", "paper_2210_02698_gb300/csrc/build.cu"]


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload, mode):
    """DRAM bytes (read + write) of the step kernels of one apply in launch
    shape `mode` (hb_launch_shape's) from the committed ncu summary, if it
    was taken on the current kernel sources, on this workload and in that
    shape (None otherwise)."""
    if workload != PROFILE_WORKLOAD:
        return None
    try:
        with open(PROFILE) as f:
            txt = f.read()
    except OSError:
        return None
    vals = {}
    for line in txt.splitlines():
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel sources sha256 prefix") != kernel_source_hash():
        return None
    try:
        return float(vals[f"step-kernel DRAM bytes per apply (mode {mode})"])
    except (KeyError, ValueError):
        return None


def cpu_oracle_sample(w, tables, rows_n, seed=1234):
    """Time the oracle's dense sum on a bounded sample of output rows."""
    import oracle.dense as odense
    import oracle.kernel as okernel
    op = okernel.Operator(w.N, tables, w.omega, w.n_cells())
    s = W.workload_sources(w)
    rows = W.sample_rows(w.grid.Nv, rows_n, seed)
    t0 = time.perf_counter()
    U = odense.apply(op, s, rows=rows, chunk=8192)
    dt = time.perf_counter() - t0
    return rows, U, dt


def one_core_rate(w, rows_n, seed=4321):
    """The oracle's dense-sum rate (output rows x RHS per second) with its
    numeric libraries held to one thread: the same sample in a child
    process whose BLAS / OpenMP thread counts are set to 1 before numpy
    loads.  Returns (rate, seconds)."""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--one-core-sample", w.name, str(rows_n),
                        str(seed)], env=env, capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        raise RuntimeError(r.stderr.strip().splitlines()[-1] if r.stderr.strip() else f"exit {r.returncode}")
    dt = float(r.stdout.strip().splitlines()[-1])
    return rows_n * w.nrhs / dt, dt


def one_core_entry(w, rows_n):
    """The one-thread oracle rate as a JSON object (never raises)."""
    try:
        rate, dt = one_core_rate(w, rows_n)
        return {"value": rate, "unit": UNIT, "threads": 1,
                "sample": f"dense HB sum on {rows_n} seeded rows x all sources x {w.nrhs} RHS, "
                          f"BLAS/OpenMP held to one thread ({dt:.1f} s)"}
    except Exception as ex:
        return {"value": None, "unit": UNIT, "threads": 1, "sample": f"failed: {ex}"}


def rank_summary(op):
    """Ranks of the built HODBF (hb_rank_profile): the largest rank at each
    HODBF level l = 1..L_v, and the largest and mean rank at each butterfly
    level k of the top-level (l = 1) butterflies.  Never raises."""
    try:
        mx, mean = op.rank_profile()
        Lv = mx.shape[0] - 1
        return {"max_by_hodbf_level": [int(mx[l].max()) for l in range(1, Lv + 1)],
                "top_level_max_by_butterfly_level": [int(v) for v in mx[1, :Lv]],
                "top_level_mean_by_butterfly_level": [round(float(v), 2) for v in mean[1, :Lv]]}
    except Exception as ex:
        return {"failed": str(ex)}


def cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def load_tables(w):
    z = np.load(table_path(w))
    return {"nodes": z["nodes"], "tau2": z["tau2"], "v0": z["v0"], "v1": z["v1"], "n_I": w.n_I}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = W.WORKLOADS[args.workload]
    tab = load_tables(w)
    rows_per_step = 4
    times = []
    for it in range(args.warmup + args.steps):
        _, _, dt = cpu_oracle_sample(w, tab, rows_per_step, seed=100 + it)
        if it >= args.warmup:
            times.append(dt)
    t = sum(times) / len(times)
    value = rows_per_step * w.nrhs / t
    nc = cores()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": describe(w), "sample": f"{rows_per_step} seeded output rows x all "
                                   f"{w.grid.Nv} sources x {w.nrhs} RHS per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nc, "kind": "oracle",
                             "sample": f"dense HB sum (numpy/scipy FP64) on {rows_per_step} rows per step",
                             "one_core": one_core_entry(w, rows_per_step)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2210_02698_gb300 import binding, build
    build.build()
    w = W.WORKLOADS[args.workload]
    tab = load_tables(w)
    tune = {"tuned": 1, "depth": 0, "dataflow": 2, "tc_leaf": 3, "cones": 4, "pairs": 5, "grid": 6}[args.shape]
    op = binding.Operator(w.N, tab["nodes"], tab["tau2"], tab["v0"], tab["v1"], w.n_cells(), w.omega,
                          eps=w.eps, leaf=w.leaf, chi=w.chi, precision=binding.HB_MIXED_BF16X3, autotune=tune)
    t0 = time.perf_counter()
    op.build()
    build_s = time.perf_counter() - t0
    info = op.info()
    R = w.nrhs
    Nv = w.grid.Nv
    s_host = W.workload_sources(w)
    s_dev = torch.from_numpy(np.ascontiguousarray(s_host.T)).to(dev)
    u_dev = torch.empty_like(s_dev)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        if world > 1:
            t = torch.tensor([ms], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms = float(t.item())
        return ms

    # ---- headline: mixed precision, inputs resident in HBM
    op.set_precision(binding.HB_MIXED_BF16X3)
    apply_mixed = lambda: op.apply(s_dev, u_dev, R, stream)  # noqa: E731
    clocks = Clocks(local)
    for _ in range(args.warmup):
        apply_mixed()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    ms_eager = timed(apply_mixed, args.steps, 0)
    # the timed region: CUDA-graph replays of one hb_apply (scratch and launch
    # plans were set up by the eager calls above); eager timing if capture fails
    ms_graph, graph_note = None, None
    try:
        graph = torch.cuda.CUDAGraph()
        cap = torch.cuda.Stream(dev)
        cap.wait_stream(stream)
        with torch.cuda.graph(graph, stream=cap):
            op.apply(s_dev, u_dev, R, cap)
        torch.cuda.synchronize()
        ms_graph = timed(graph.replay, args.steps, args.warmup)
    except Exception as ex:
        graph_note = f"graph capture failed: {ex}"
    ms = ms_graph if ms_graph is not None else ms_eager
    clk = clocks.stop()
    # large problems keep no full extra copies of the vectors on the device:
    # the rel-L2 checks use the oracle's row sample there
    large = Nv * R > (1 << 24)
    rows_n = 384 if Nv <= (1 << 18) else max(8, 384 * 65536 // Nv)   # ~10-15 s of the oracle
    rows = W.sample_rows(Nv, rows_n, 1234)
    rows_t = torch.from_numpy(rows).to(dev)
    mixed_rows = u_dev[:, rows_t].cpu().numpy().T
    u_mixed = None if large else u_dev.clone()
    # per-kernel-group device time of one apply (events on the launch stream)
    op.set_kernel_timing(True)
    ktimes = {}
    nk = max(3, min(args.steps, 10))
    for _ in range(nk):
        apply_mixed()
    ktimes = op.kernel_times()
    op.set_kernel_timing(False)

    # ---- measured FP64 peaks (the FP64 rooflines): the library's FMA-loop
    # probe and a cuBLAS DGEMM (4096^3, best of three)
    fp64_fma = binding.fp64_fma_peak(stream)
    try:
        A64 = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
        B64 = torch.randn(4096, 4096, dtype=torch.float64, device=dev)
        torch.matmul(A64, B64)
        best = 1e30
        for _ in range(3):
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            g0.record(stream)
            torch.matmul(A64, B64)
            g1.record(stream)
            torch.cuda.synchronize()
            best = min(best, g0.elapsed_time(g1))
        fp64_dgemm = 2 * 4096 ** 3 / (best * 1e-3) / 1e12
        del A64, B64
    except Exception:
        fp64_dgemm = None

    # ---- plain FP64 GPU butterfly apply (same factors, complex128)
    op.set_precision(binding.HB_FP64)
    apply64 = lambda: op.apply(s_dev, u_dev, R, stream)  # noqa: E731
    ms64 = timed(apply64, max(3, args.steps // 4), 2)
    fp64_rows = u_dev[:, rows_t].cpu().numpy().T
    if large:
        rel_mixed_fp64 = float(np.linalg.norm(mixed_rows - fp64_rows) / np.linalg.norm(fp64_rows))
    else:
        rel_mixed_fp64 = float(torch.linalg.norm(u_mixed - u_dev) / torch.linalg.norm(u_dev))
    u64_host = None if large else u_dev.cpu().numpy().T

    # ---- plain FP64 GPU matrix-free dense sum (every entry evaluated on the fly)
    dense_line = {"value": None, "unit": UNIT, "note": "skipped at this size (seconds per entry batch)"}
    if not large:
        apply_dense = lambda: op.apply_dense(s_dev, u_dev, R, stream)  # noqa: E731
        ms_dense = timed(apply_dense, 1, 1)
        # counted FP64 flops per entry: tau^2, v0, v1 by 16-term contractions
        # (48 FMA), the per-source-cell contraction shared by 64 outputs (12
        # FMA per entry), the complex multiply-add per right-hand side (4 FMA);
        # the Hankel evaluation is not counted, so the fraction is a lower bound
        dflops = 2.0 * (48 + 12 + 4 * R) * float(Nv) * Nv
        dense_line = {"value": Nv * R * world / (ms_dense * 1e-3), "unit": UNIT, "ms_per_step": ms_dense,
                      "rel_l2_mixed_vs_dense": float(torch.linalg.norm(u_mixed - u_dev) / torch.linalg.norm(u_dev)),
                      "roofline": {"bound": "alu", "achieved": dflops / (ms_dense * 1e-3) / 1e12,
                                   "peak": fp64_fma, "unit": "TFLOP/s",
                                   "frac": dflops / (ms_dense * 1e-3) / 1e12 / fp64_fma,
                                   "flops_per_entry": 2 * (48 + 12 + 4 * R),
                                   "peak_kind": "measured FP64 FMA loop (Hankel flops not counted)"}}
    op.set_precision(binding.HB_MIXED_BF16X3)
    u_mixed = None

    # ---- end to end through the public API with host buffers: every step
    # copies its input from pinned host memory, applies, and reads its result
    # back into pinned host memory.  Steps are pipelined as a serving loop
    # would run them: copy-in, apply and copy-out on three streams, two device
    # buffer pairs, each step's copy-in waiting for the apply that last used
    # its buffer and each apply for the copy-out that last read its output.
    # (one buffer pair when the device has no room for a second one)
    s_pin = torch.from_numpy(np.ascontiguousarray(s_host.T)).pin_memory()
    free_b, _ = torch.cuda.mem_get_info(dev)
    nbuf = 2 if free_b > 2 * s_dev.numel() * s_dev.element_size() + (1 << 30) else 1
    u_pin = [torch.empty_like(s_pin).pin_memory() for _ in range(nbuf)]
    s_buf = [s_dev] + [torch.empty_like(s_dev) for _ in range(nbuf - 1)]
    u_buf = [u_dev] + [torch.empty_like(u_dev) for _ in range(nbuf - 1)]
    st_in, st_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def e2e_run(steps):
        ev_c, ev_o = [], []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st_in)
        for i in range(steps):
            b = i % nbuf
            if i >= nbuf:
                st_in.wait_event(ev_c[i - nbuf])
            with torch.cuda.stream(st_in):
                s_buf[b].copy_(s_pin, non_blocking=True)
            ev_i = torch.cuda.Event()
            ev_i.record(st_in)
            stream.wait_event(ev_i)
            if i >= nbuf:
                stream.wait_event(ev_o[i - nbuf])
            op.apply(s_buf[b], u_buf[b], R, stream)
            ev_c.append(torch.cuda.Event())
            ev_c[i].record(stream)
            st_out.wait_event(ev_c[i])
            with torch.cuda.stream(st_out):
                u_pin[b].copy_(u_buf[b], non_blocking=True)
            ev_o.append(torch.cuda.Event())
            ev_o[i].record(st_out)
        e1.record(st_out)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    e2e_run(2)
    ms_e2e = e2e_run(args.steps)
    if world > 1:
        t = torch.tensor([ms_e2e], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_e2e = float(t.item())
    # the last step's result as read back to the host equals the device-timed
    # apply's output on the sampled rows (same input, deterministic kernels)
    e2e_same = bool(np.array_equal(u_pin[(args.steps - 1) % nbuf].numpy()[:, rows].T, mixed_rows))

    # ---- the source-inversion step of the 512^2 workload: loss
    # ||P u(s) - d||^2 over 256 seeded receivers and its gradient through the
    # adjoint apply (forward + backward, mixed precision)
    autograd_line = None
    if w.nrhs == 1 and w.medium.kind == "gradient":
        from paper_2210_02698_gb300.autograd import hb_apply
        rng = np.random.default_rng(512)
        P = torch.from_numpy(np.sort(rng.choice(Nv, 256, replace=False))).to(dev)
        d_obs = torch.zeros(256, dtype=torch.complex128, device=dev)
        s_var = s_dev[:1].clone().requires_grad_(True)

        def fwd_bwd():
            s_var.grad = None
            loss = (hb_apply(s_var, op)[:, P] - d_obs).abs().pow(2).sum()
            loss.backward()

        ms_ag = timed(fwd_bwd, args.steps, args.warmup)
        autograd_line = {"ms_per_step": ms_ag, "what": "loss ||P u(s) - d||^2 over 256 receivers and its "
                         "gradient (hb_apply forward, hb_apply_adjoint backward), mixed precision"}

    result = {}
    if rank == 0:
        hbm, peak_kind = peaks()
        step_ms = sum(v[0] for k, v in ktimes.items() if k.startswith("bf_")) / nk
        gather_ms = sum(v[0] for k, v in ktimes.items() if k in ("gather", "scatter")) / nk
        E = info["factor_entries"]
        fac_bytes = E * 8
        mt = min(2, (R + 15) // 16)
        shape = op.launch_shape(False, mt)
        passes = (R + 31) // 32
        # algorithmic bytes of the timed kernels of one apply: every factor
        # entry once (8-byte split-BF16 pair), the output written once (FP64
        # complex), every skeleton vector written once and read once (8-byte
        # pairs), and the input: read once as FP64 complex by the dataflow
        # launch, which gathers it itself, or read once as the 8-byte pairs the
        # separate gather wrote, when the step kernels run one launch per depth
        # (the tensor-core leaf shape's gather also writes x in the operand
        # layout the leaf kernel reads: not algorithmic, not counted)
        in_bytes = 16 if shape["mode"] == 1 else 8
        alg_bytes = fac_bytes + Nv * R * (in_bytes + 16) + 2 * info["skeleton_rows"] * R * 8
        kernel_what = {1: "one persistent dataflow launch per pass of 32 right-hand sides (gather and every "
                          "butterfly level)",
                       0: "butterfly step kernels of one apply (one launch per dependency depth)",
                       2: "butterfly step kernels of one apply (one launch per dependency depth; the leaf "
                          "outputs on the tcgen05 tensor-core kernel)",
                       3: "butterfly step kernels of one apply (the first four butterfly levels as cones in "
                          "one launch, then one launch per dependency depth)",
                       4: "butterfly step kernels of one apply (cone launch, one launch per remaining depth, "
                          "the leaf outputs on the tcgen05 tensor-core kernel)",
                       5: "butterfly step kernels of one apply (the transfer depths fused in pairs, one launch "
                          "per pair, then the leaf outputs)",
                       6: "butterfly step kernels of one apply (the transfer depths fused in pairs; the leaf "
                          "outputs on the tcgen05 tensor-core kernel)",
                       7: "butterfly step kernel of one apply (every dependency depth in one cooperative "
                          "launch, grid barriers between depths)"}[shape["mode"]]
        ndepth = info["levels"] + 1
        launches = passes * {1: 1, 0: 1 + ndepth, 2: 1 + ndepth,
                             3: 2 + max(0, ndepth - 4), 4: 2 + max(0, ndepth - 4),
                             5: 2 + (ndepth - 1 + 1) // 2, 6: 2 + (ndepth - 1 + 1) // 2, 7: 2}[shape["mode"]]
        achieved = alg_bytes / (step_ms * 1e-3) / 1e9
        value = Nv * R * world / (ms * 1e-3)
        nc = cores()
        # cpu baseline: oracle dense sum on a bounded row sample, plus the
        # rel-L2 of our mixed output on those rows
        cpu = {}
        try:
            if args.skip_cpu:
                raise RuntimeError("skipped (--skip-cpu)")
            rows2, U_ref, dt = cpu_oracle_sample(w, tab, rows_n)
            assert np.array_equal(rows2, rows)
            got, got64 = mixed_rows, fp64_rows
            cpu = {"value": rows_n * R / dt, "unit": UNIT, "cores": nc, "kind": "oracle",
                   "sample": f"dense FP64 HB sum, {rows_n} seeded rows x {Nv} sources x {R} RHS "
                             f"({dt:.1f} s; numpy's BLAS threads over all {nc} cores)",
                   "one_core": one_core_entry(w, max(4, rows_n // 8)),
                   "rel_l2_mixed_vs_oracle": float(np.linalg.norm(got - U_ref) / np.linalg.norm(U_ref)),
                   "rel_l2_fp64_vs_oracle": float(np.linalg.norm(got64 - U_ref) / np.linalg.norm(U_ref))}
            if w.rhs_kind == "mixed64":
                # the four source kinds (quarters of the columns) on their own:
                # smooth bumps and wavepackets radiate little at this frequency
                q = R // 4
                kinds = ("point", "line", "gaussian_bump", "wavepacket")
                cpu["rel_l2_mixed_by_source_kind"] = {
                    kinds[k]: float(np.linalg.norm(got[:, k * q:(k + 1) * q] - U_ref[:, k * q:(k + 1) * q]) /
                                    np.linalg.norm(U_ref[:, k * q:(k + 1) * q])) for k in range(4)}
                cpu["output_norm_by_source_kind"] = {
                    kinds[k]: float(np.linalg.norm(U_ref[:, k * q:(k + 1) * q])) for k in range(4)}
        except Exception as ex:  # the baseline must never break the bench line
            cpu = {"value": None, "unit": UNIT, "cores": nc, "kind": "oracle", "sample": f"failed: {ex}"}
        # the oracle's CPU butterfly apply over the saved factors (all rows, all RHS)
        cpu_bf = {}
        try:
            if args.skip_cpu:
                raise RuntimeError("skipped (--skip-cpu)")
            if large:
                raise RuntimeError("skipped at this size (the factor file would be too large)")
            from oracle.factor_file import FactorFile
            with tempfile.TemporaryDirectory() as td:
                path = os.path.join(td, "op.hbf")
                op.save(path)
                F = FactorFile(path)
            t0 = time.perf_counter()
            u_cpu = F.apply(s_host)
            dt = time.perf_counter() - t0
            cpu_bf = {"value": Nv * R / dt, "unit": UNIT, "cores": nc, "kind": "oracle",
                      "sample": f"full FP64 butterfly apply of the saved factors, {Nv} rows x {R} RHS "
                                f"({dt:.1f} s, numpy)",
                      "rel_l2_fp64_gpu_vs_cpu_butterfly":
                          float(np.linalg.norm(u64_host - u_cpu) / np.linalg.norm(u_cpu))}
        except Exception as ex:
            cpu_bf = {"value": None, "unit": UNIT, "cores": nc, "kind": "oracle", "sample": f"failed: {ex}"}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": describe(w),
                       "l2": f"factors {fac_bytes / 2**20:.0f} MiB > 129 MB L2, no flush",
                       "precision": "factors and vectors as split-BF16 pairs (hi + lo), three BF16 "
                                    "tensor-core products per complex MAC, FP32 accumulate, FP64 output",
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": profiled_traffic(args.workload, shape["mode"]),
                         "kernel": kernel_what,
                         "alg_bytes": alg_bytes, "kernel_ms": step_ms,
                         "peak_kind": f"{peak_kind} copy bandwidth"},
            "e2e": {"value": Nv * R * world / (ms_e2e * 1e-3), "unit": UNIT,
                    "h2d_bytes_per_step": Nv * R * 16, "d2h_bytes_per_step": Nv * R * 16,
                    "ms_per_step": ms_e2e,
                    "pipeline": f"copy-in, hb_apply, copy-out on three streams, {nbuf} device buffer pair(s)",
                    "result_equals_device_run": e2e_same},
            "gpu_launches": launches * args.steps,
            "launch_shape": {**shape, "requested": args.shape},
            "timed": "CUDA-graph replay of hb_apply" if ms_graph is not None else graph_note,
            "eager_ms_per_step": ms_eager,
            "clocks": clk,
            "cpu_baseline": cpu,
            "cpu_butterfly": cpu_bf,
            "fp64_gpu": {"value": Nv * R * world / (ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64,
                         "roofline": {"bound": "alu", "achieved": 8.0 * E * R / (ms64 * 1e-3) / 1e12,
                                      "peak": fp64_fma, "unit": "TFLOP/s",
                                      "frac": 8.0 * E * R / (ms64 * 1e-3) / 1e12 / fp64_fma,
                                      "flops": "8 per stored complex factor entry and right-hand side",
                                      "peak_kind": "measured FP64 FMA loop"}},
            "fp64_peaks": {"fma_loop_tflops": fp64_fma, "dgemm_tflops": fp64_dgemm,
                           "note": "measured in this run: the library's FMA-loop probe; cuBLAS DGEMM 4096^3"},
            "fp64_gpu_dense": dense_line,
            "speedup_vs_fp64_gpu": ms64 / ms,
            "rel_l2_mixed_vs_fp64_butterfly": rel_mixed_fp64,
            "rel_l2_scope": f"oracle row sample ({rows_n} rows)" if large else "all rows",
            "build_s": build_s,
            "factor_entries": E,
            "factor_bytes": {"fp64": info["factor_bytes_fp64"], "mixed_per_direction": info["factor_bytes_mixed"],
                             "total_device": info["factor_bytes_fp64"] + 2 * info["factor_bytes_mixed"]},
            "max_rank": info["max_rank"],
            "ranks": rank_summary(op),
            "kernel_ms_per_apply": {k: v[0] / nk for k, v in ktimes.items()},
            **({"autograd": autograd_line} if autograd_line else {}),
            "gather_scatter_ms": gather_ms,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def run_inclusion(args):
    """The inclusion apply (Sec. 3.2, Eq. m_v2v_inclu) on the workload's
    grid with a circle of args.inclusion segments (centre (0.5, 0.5), radius
    0.3): K^{v2v} compressed (split-BF16), the surface part in FP64 - first
    with the dense K^{v2s} / K^{s2v}, then with their butterflies
    (hb_curve_compress).  One JSON line; the roofline is the FP64 arithmetic
    of the two surface butterflies (8 flops per stored complex entry and
    right-hand side) against the measured FP64 FMA rate."""
    import torch
    from paper_2210_02698_gb300 import binding, build
    build.build()
    torch.cuda.set_device(0)
    w = W.WORKLOADS[args.workload]
    tab = load_tables(w)
    op = binding.Operator(w.N, tab["nodes"], tab["tau2"], tab["v0"], tab["v1"], w.n_cells(), w.omega,
                          eps=w.eps, leaf=w.leaf, chi=w.chi, precision=binding.HB_MIXED_BF16X3, autotune=1)
    op.build()
    ns = int(args.inclusion)
    cen, lw = W.circle_segments((0.5, 0.5), 0.3, ns)
    t0 = time.perf_counter()
    op.set_curve(cen, lw, w.medium.n(cen[:, 0], cen[:, 1]))
    set_s = time.perf_counter() - t0
    R, Nv = w.nrhs, w.grid.Nv
    s_dev = torch.from_numpy(np.ascontiguousarray(W.workload_sources(w).T)).to("cuda")
    stream = torch.cuda.current_stream()

    def timed():
        u = torch.empty_like(s_dev)
        for _ in range(args.warmup):
            op.apply_inclusion(s_dev, u, R, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            op.apply_inclusion(s_dev, u, R, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps, u

    ms_dense, u_dense = timed()
    t0 = time.perf_counter()
    op.curve_compress(16)
    compress_s = time.perf_counter() - t0
    ms_bf, u_bf = timed()
    info = [op.curve_info(q) for q in (0, 1)]
    entries = sum(e for _, _, e in info)
    # the surface butterflies alone: the difference to the volume apply
    u = torch.empty_like(s_dev)
    for _ in range(args.warmup):
        op.apply(s_dev, u, R, stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        op.apply(s_dev, u, R, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_v2v = e0.elapsed_time(e1) / args.steps
    peak = binding.fp64_fma_peak(stream)
    surface_ms = max(ms_bf - ms_v2v, 1e-9)
    achieved = 8.0 * entries * R / (surface_ms * 1e-3) / 1e12
    rel = float(torch.linalg.norm(u_bf - u_dense) / torch.linalg.norm(u_dense))
    print(json.dumps({
        "metric": "inclusion apply N_v*RHS/s (K^{v2v} compressed, surface part FP64)", "unit": UNIT,
        "value": Nv * R / (ms_bf * 1e-3), "ms_per_step": ms_bf, "higher_is_better": True,
        "steps": args.steps, "warmup": args.warmup, "data": "synthetic",
        "config": {"workload": describe(w), "segments": ns, "curve": "circle centre (0.5, 0.5) radius 0.3"},
        "dense_surface": {"value": Nv * R / (ms_dense * 1e-3), "ms_per_step": ms_dense,
                          "bytes": 2 * ns * Nv * 16},
        "volume_only_ms": ms_v2v,
        "butterflies": {"v2s": {"levels": info[0][0], "max_rank": info[0][1], "entries": info[0][2]},
                        "s2v": {"levels": info[1][0], "max_rank": info[1][1], "entries": info[1][2]},
                        "compress_s": compress_s, "curve_set_s": set_s},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "kernel": "surface butterflies (inclusion apply minus the volume apply)",
                     "peak_kind": "measured FP64 FMA loop"},
        "rel_l2_compressed_vs_dense_surface": rel}), flush=True)
    op.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(W.WORKLOADS))
    ap.add_argument("--skip-cpu", action="store_true", help="omit the CPU oracle leg (profiling runs)")
    ap.add_argument("--shape", default="tuned",
                    choices=["tuned", "dataflow", "depth", "tc_leaf", "cones", "pairs", "grid"],
                    help="launch shape of the mixed apply: autotuned (default), the persistent dataflow "
                         "launch, one launch per dependency depth, that with the leaf outputs on the "
                         "tcgen05 tensor-core kernel, the cone launch, fused level pairs, or every depth "
                         "in one cooperative launch with grid barriers")
    ap.add_argument("--inclusion", type=int, default=0, metavar="NS",
                    help="time the inclusion apply with a circle of NS segments instead (dense and compressed "
                         "surface operators)")
    ap.add_argument("--one-core-sample", nargs=3, metavar=("WORKLOAD", "ROWS", "SEED"), help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.one_core_sample:
        # child of one_core_rate: print the seconds of one oracle sample
        name, rows_n, seed = args.one_core_sample
        w = W.WORKLOADS[name]
        _, _, dt = cpu_oracle_sample(w, load_tables(w), int(rows_n), seed=int(seed))
        print(dt, flush=True)
    elif args.inclusion:
        run_inclusion(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
