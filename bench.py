#!/usr/bin/env python
"""Benchmark of the GB300 coarse<->fine AMR transfer.

Workload (the uniform batch): 2,048 hanging faces, coarse patches of 9^3
volumes, overlap k = 3, U = 59 unknowns per volume (FP64, AoS), faces cycled
over the six orientations, seeded smooth fields (4 Gaussians + 4 sinusoids per
unknown, 1e-8 relative noise).  One step = Taylor-3 interpolation of all fine
ghost volumes + Taylor-3 restriction of all coarse halo volumes.  The metric
is ghost volume-unknowns per second (interpolated + restricted), with the
interpolation kernel's achieved HBM bandwidth, the d-linear tensor-product
path and Taylor-2 on the same GPU, and the error against the FP64 oracle.

Rank 0 prints one JSON line.  Inputs (4.7 GB) are larger than L2 (129 MB),
so no flush is needed between steps.  ``--impl reference`` times the CPU
oracle instead (a bounded sample of the same workload, on the host cores).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

P, K, U, N_FACES = 9, 3, 59, 2048
METRIC = "ghost volume-unknowns/s (Taylor-3 interpolation + restriction)"
UNIT = "volume-unknowns/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fixed", "split", "fp64"], default="fixed")
    ap.add_argument("--faces", type=int, default=N_FACES)
    ap.add_argument("--no-extra", action="store_true", help="skip the d-linear / Taylor-2 / e2e / oracle legs")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="time only the adjoint (P^T, R^T) of --faces hanging faces and print its JSON object")
    ap.add_argument("--tuning", default=None,
                    help="launch shape threads,smem_budget,restrict_threads,addback,lanes instead of autotuning")
    ap.add_argument("--order", type=int, default=3, choices=[1, 2, 3], help="operator order of the timed step")
    return ap.parse_args()


def dist_setup(n):
    import torch
    import torch.distributed as dist
    if n > 1 or int(os.environ.get("WORLD_SIZE", "1")) > 1:
        rank = int(os.environ["RANK"])
        local = int(os.environ.get("LOCAL_RANK", rank))
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        return dist, rank, dist.get_world_size(), local
    return None, 0, 1, 0


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        self.file.flush()
        self.file.seek(0)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file.read().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        os.unlink(self.file.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# CUDA sources each profiled kernel is compiled from (its own file and the
# headers it includes)
KERNEL_SOURCES = {
    "interp_fixed_kernel": ["fixed_kernels.cuh", "transfer_kernels.cuh", "amr_common.cuh", "split_arith.cuh"],
    "restrict_kernel_fixed": ["restrict_kernels.cuh", "transfer_kernels.cuh", "amr_common.cuh", "split_arith.cuh"],
    "restrict_kernel_fp64": ["restrict_kernels.cuh", "transfer_kernels.cuh", "amr_common.cuh", "split_arith.cuh"],
    "restrict_kernel_split": ["restrict_kernels.cuh", "transfer_kernels.cuh", "amr_common.cuh", "split_arith.cuh"],
}


def kernel_source_hash(kernel=None):
    """sha256 of the CUDA sources a kernel is compiled from (sorted by name;
    every CUDA/C++ source of the library for a kernel not listed)."""
    import hashlib
    d = os.path.join(ROOT, "paper_2504_15814_gb300", "csrc")
    names = KERNEL_SOURCES.get(kernel) or [n for n in os.listdir(d) if n.endswith((".cu", ".cuh", ".cpp", ".hpp"))]
    h = hashlib.sha256()
    for name in sorted(names):
        with open(os.path.join(d, name), "rb") as fh:
            h.update(name.encode() + b"\0" + fh.read())
    return h.hexdigest()


def profiled_traffic(kernel, faces):
    """DRAM bytes per launch of a kernel from a committed ncu summary
    (profiles/<kernel>_uniform_batch.md), scaled to `faces` hanging faces,
    when the summary was taken on these exact sources (else None)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_uniform_batch.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    fields = {}
    for line in text.splitlines():
        if line.startswith("- ") and ": " in line:
            key, val = line[2:].split(": ", 1)
            fields[key.strip()] = val.strip().strip("`")
    if fields.get("source_sha256") != kernel_source_hash(kernel):
        return None
    try:
        return float(fields["dram_bytes_per_face"]) * faces
    except (KeyError, ValueError):
        return None


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0}, "fallback"


def time_kernel(launch, n, stream):
    """Average device time of one launch, CUDA events on the launching stream."""
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    for a, b in evs:
        a.record(stream)
        launch()
        b.record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs) / n


def oracle_sample(items, coarse, fine, n_faces, U):
    """A compact copy of the first n_faces items and their arrays on the host."""
    import numpy as np
    from paper_2504_15814_gb300 import workloads as wl
    sub = items[:n_faces].copy()
    arr = 2 * K * P * P * U
    c = np.empty(n_faces * arr)
    f = np.empty(n_faces * 9 * arr)
    for i in range(n_faces):
        co, fo = int(sub[i]["coarse_offset"]), int(sub[i]["fine_offset"])
        c[i * arr:(i + 1) * arr] = coarse[co:co + arr].cpu().numpy()
        f[i * 9 * arr:(i + 1) * 9 * arr] = fine[fo:fo + 9 * arr].cpu().numpy()
        sub[i]["coarse_offset"] = i * arr
        sub[i]["fine_offset"] = i * 9 * arr
    return sub, c, f


def _oracle_worker(conn, U):
    """Pool process: receives its share of the sampled faces once, builds the
    operators (construction happens once per plan on the GPU side too), then
    runs one interpolate + restrict per "go" message."""
    import numpy as np
    from oracle import transfer as tr
    sub, c, f = conn.recv()
    if len(sub):
        tr.restrict(sub, U, tr.interpolate(sub, U, c, f), c)
    conn.send("ready")
    while conn.recv() == "go":
        f2 = tr.interpolate(sub, U, c, f)
        tr.restrict(sub, U, f2, c)
        conn.send(len(sub))


def oracle_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class OraclePool:
    """The CPU oracle over all host cores: one process per core (spawn
    context, safe after CUDA initialisation), each holding a contiguous share
    of the sampled faces; a step runs every share once in parallel."""

    def __init__(self, U, sub, c, f):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.cores = oracle_cores()
        n = len(sub)
        arr = 2 * K * P * P * U
        self.procs, self.conns = [], []
        for r in range(self.cores):
            lo, hi = r * n // self.cores, (r + 1) * n // self.cores
            s2 = sub[lo:hi].copy()
            s2["coarse_offset"] -= lo * arr
            s2["fine_offset"] -= lo * 9 * arr
            a, b = ctx.Pipe()
            pr = ctx.Process(target=_oracle_worker, args=(b, U), daemon=True)
            pr.start()
            a.send((s2, c[lo * arr:hi * arr].copy(), f[lo * 9 * arr:hi * 9 * arr].copy()))
            self.procs.append(pr)
            self.conns.append(a)
        for a in self.conns:
            a.recv()

    def step(self):
        for a in self.conns:
            a.send("go")
        return sum(a.recv() for a in self.conns)

    def close(self):
        for a in self.conns:
            a.send("stop")
        for pr in self.procs:
            pr.join()


def time_oracle(sub, c, f, U, budget_s=15.0):
    """Oracle interpolate + restrict of the sampled faces on all host cores;
    operators are built before timing.  Returns (volume-unknowns/s, seconds
    per pass, cores)."""
    pool = OraclePool(U, sub, c, f)
    try:
        pool.step()  # warm-up
        reps, t0 = 0, time.perf_counter()
        while True:
            pool.step()
            reps += 1
            el = time.perf_counter() - t0
            if el > budget_s or reps >= 3:
                break
    finally:
        pool.close()
    per = el / reps
    outs = len(sub) * (9 * K * P * P + K * P * P) * U
    return outs / per, per, pool.cores


def run_reference(args):
    """Reference arm: the CPU oracle, as it stands, on a bounded sample of the
    workload, on this machine's host cores."""
    import numpy as np
    import torch
    from paper_2504_15814_gb300 import workloads as wl
    if int(os.environ.get("RANK", "0")) != 0:
        return
    cores = oracle_cores()
    n_sample = 4 * cores  # four hanging faces per host core
    items, coarse, fine = wl.uniform_batch(n_faces=n_sample, p=P, k=K, U=U, order=3, config_index=1)
    c, f = coarse.numpy(), fine.numpy()
    pool = OraclePool(U, items, c, f)  # operators built in the workers before timing
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        pool.step()
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    pool.close()
    per = sum(times) / len(times)
    outs = n_sample * (9 * K * P * P + K * P * P) * U
    value = outs / per
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"uniform batch sample: {n_sample} hanging faces of the 2048-face batch, "
                                   f"p={P}, k={K}, U={U}, Taylor-3 interpolate+restrict",
                       "faces": n_sample, "p": P, "k": K, "U": U},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.cores, "kind": "oracle",
                             "sample": f"{n_sample} hanging faces of the batch per step, Taylor-3 interpolate + "
                                       f"restrict, scipy CSR apply, one process per host core"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import numpy as np
    import torch
    from paper_2504_15814_gb300 import binding as B
    from paper_2504_15814_gb300 import workloads as wl

    dist, rank, world, local = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if args.adjoint_only:
        if rank == 0:
            print(json.dumps(adjoint_leg(B, wl, torch.cuda.current_stream(dev), args.faces, max(args.steps, 1))),
                  flush=True)
        if dist:
            dist.destroy_process_group()
        return
    prec = {"fixed": B.PREC_FIXED, "split": B.PREC_SPLIT, "fp64": B.PREC_FP64}[args.precision]
    # weak scaling: a global batch of faces-per-GPU x N faces, each rank
    # keeping its cost-balanced shard (items are independent: no collective)
    items, coarse, fine = wl.uniform_batch(n_faces=args.faces * world, p=P, k=K, U=U, order=args.order,
                                           config_index=1, device=dev, shard=(rank, world) if world > 1 else None)
    coarse_out = coarse.clone()
    plan = B.Plan(items, U, coarse.numel(), fine.numel(), prec)
    stream = torch.cuda.current_stream(dev)
    if args.tuning:
        plan.set_tuning(*[int(v) for v in args.tuning.split(",")])
        tuning = plan.tuning
    else:
        tuning = plan.autotune(coarse, fine, coarse_out)  # launch shapes for this GPU, before timing
    info = plan.info

    def step():
        plan.interpolate(coarse, fine)
        plan.restrict(fine, coarse_out)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        # per-kernel durations for the roofline (same stream, same launches)
        t_interp = time_kernel(lambda: plan.interpolate(coarse, fine), max(args.steps, 5), stream)
        t_restrict = time_kernel(lambda: plan.restrict(fine, coarse_out), max(args.steps, 5), stream)
    clocks = clk.summary()
    ms = e0.elapsed_time(e1) / args.steps
    if dist:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    outs = (info["interp_outputs"] + info["restrict_outputs"]) * U
    total_outs = outs
    if dist:
        t = torch.tensor([float(outs)], device=dev, dtype=torch.float64)
        dist.all_reduce(t)
        total_outs = float(t.item())
    value = total_outs / (ms * 1e-3)

    peaks, peak_src = measured_peaks()
    hbm_peak = float(peaks["hbm_gbs"])
    interp_gbs = info["interp_bytes"] / (t_interp * 1e-3) / 1e9
    restrict_gbs = info["restrict_bytes"] / (t_restrict * 1e-3) / 1e9
    ikern = {B.PREC_FIXED: "interp_fixed_kernel", B.PREC_SPLIT: "interp_kernel_split",
             B.PREC_FP64: "interp_kernel_fp64"}[prec]
    rkern = {B.PREC_FIXED: "restrict_kernel_fixed", B.PREC_SPLIT: "restrict_kernel_split",
             B.PREC_FP64: "restrict_kernel_fp64"}[prec]
    roofline = {"bound": "hbm", "kernel": ikern, "achieved": interp_gbs, "peak": hbm_peak,
                "unit": "GB/s", "frac": interp_gbs / hbm_peak,
                "traffic": profiled_traffic(ikern, args.faces),
                "algorithmic_bytes_per_launch": info["interp_bytes"], "launch_ms": t_interp,
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else "fallback",
                "restrict_kernel": {"achieved": restrict_gbs, "frac": restrict_gbs / hbm_peak,
                                    "launch_ms": t_restrict, "algorithmic_bytes_per_launch": info["restrict_bytes"],
                                    "kernel": rkern, "traffic": profiled_traffic(rkern, args.faces)}}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": {B.PREC_FIXED: "int64 interpolation, f64 + int64 restriction", B.PREC_SPLIT: "f64 base / f32 increment",
                      B.PREC_FP64: "f64"}[prec],
            "data": "synthetic",
            "config": {"workload": f"uniform batch: {args.faces} hanging faces per GPU, p={P}, k={K}, U={U}, "
                                   f"FP64 AoS, {['d-linear', 'Taylor-2', 'Taylor-3'][args.order - 1]} "
                                   "interpolate+restrict",
                       "faces_per_gpu": args.faces, "p": P, "k": K, "U": U, "order": args.order,
                       "precision": args.precision, "parallelism": f"dp{world}" if world > 1 else "single GPU",
                       "tuning": tuning,
                       "l2": f"inputs ({(coarse.numel() + fine.numel()) * 8 / 1e9:.1f} GB) larger than L2, "
                             "no flush"},
            "roofline": roofline, "clocks": clocks,
            "gpu_launches": args.steps * (info["interp_launches"] + info["restrict_launches"])}

    if rank == 0 and not args.no_extra:
        line["compare"] = compare_paths(B, wl, items, coarse, fine, coarse_out, U, args, stream, plan)
        staged = e2e_leg(plan, coarse, fine, coarse_out, outs, args, stream, items=items)
        line["e2e"] = e2e_zero_copy(plan, items, coarse, fine, coarse_out, outs, stream)
        line["e2e"]["staged_copies"] = staged
        line["err_vs_fp64"] = error_vs_oracle(items, coarse, fine, plan, U)
        n_cpu = 4 * oracle_cores()
        sub, c_h, f_h = oracle_sample(items, coarse, fine, n_cpu, U)
        v, per, cores = time_oracle(sub, c_h, f_h, U)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{n_cpu} hanging faces of the batch (4 per host core), Taylor-3 "
                                          "interpolate + restrict, operators prebuilt, scipy CSR apply, one "
                                          "process per host core"}
        line["workloads"] = other_workloads(B, wl, stream)
    plan.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def _time_steps(step, n, stream):
    import torch
    for _ in range(3):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(n):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / n


def other_workloads(B, wl, stream):
    """The other synthetic workloads of the benchmark family, measured on the
    same GPU: single face (launch latency, direct vs captured graph), uneven
    batch (default vs autotuned launch shapes), split precision on puncture
    fields (error against the FP64 oracle per field class), adjoint."""
    import numpy as np
    import torch
    from oracle import transfer as tr
    out = {}
    # single face: p = 6, k = 3, U = 1, Taylor-2, random quadratic on the unit cube
    items, cl, fl = wl.make_items([0], [-1], [6], [3], [2], 1)
    rng = np.random.Generator(np.random.PCG64(wl.SEED_BASE + 0))
    coef = torch.as_tensor(rng.uniform(-1, 1, 10))
    H = 1.0 / 6

    def quad(x):
        x = x * H
        t = torch.stack([torch.ones_like(x[:, 0]), x[:, 0], x[:, 1], x[:, 2], x[:, 0] ** 2, x[:, 1] ** 2,
                         x[:, 2] ** 2, x[:, 0] * x[:, 1], x[:, 0] * x[:, 2], x[:, 1] * x[:, 2]], 1)
        return (t @ coef.to(x.device))[:, None]

    c, f = wl.polynomial_buffers(items, 1, cl, fl, quad, origins=np.array([[1.0 / H, 0.0, 0.0]]), device="cuda")
    co = c.clone()
    exact_f, exact_c = f.clone(), c.clone()
    plan = B.Plan(items, 1, cl, fl, B.PREC_FP64)
    direct = _time_steps(lambda: (plan.interpolate(c, f), plan.restrict(f, co)), 200, stream)
    plan.capture_step(c, f, co)
    graph = _time_steps(lambda: plan.launch_step(), 200, stream)
    torch.cuda.synchronize()
    err = max(float((f - exact_f).abs().max() / exact_f.abs().max()), float((co - exact_c).abs().max() / exact_c.abs().max()))
    outs = (plan.info["interp_outputs"] + plan.info["restrict_outputs"])
    out["single_face"] = {"workload": "1 hanging face, p=6, k=3, U=1, Taylor-2, quadratic field",
                          "us_per_step_direct": direct * 1e3, "us_per_step_graph": graph * 1e3,
                          "volume_unknowns_per_step": outs, "max_rel_err_vs_exact_quadratic": err,
                          "launches_per_step": 2}
    plan.close()
    # float32 storage of the increments on the uniform batch (2,048 faces)
    items, coarse, fine = wl.uniform_batch(n_faces=2048, U=59, order=3, config_index=1, device="cuda")
    plan = B.Plan(items, 59, coarse.numel(), fine.numel(), B.PREC_SPLIT)
    plan.autotune(coarse, fine, coarse.clone())
    info = plan.info
    incr = torch.empty(info["increment_elems"], dtype=torch.float32, device="cuda")
    t_incr = _time_steps(lambda: plan.interpolate_increments(coarse, incr), 20, stream)
    t_apply = _time_steps(lambda: plan.apply_increments(coarse, incr, fine), 20, stream)
    read_b = info["interp_bytes"] - info["interp_outputs"] * 59 * 8
    incr_b = read_b + info["increment_elems"] * 4
    out["split_f32_increments"] = {
        "workload": "2,048 hanging faces, p=9, k=3, U=59, Taylor-3: float32 increments instead of float64 ghosts",
        "interpolate_increments_ms": t_incr, "algorithmic_bytes": incr_b,
        "achieved_gbs": incr_b / (t_incr * 1e-3) / 1e9, "apply_increments_ms": t_apply,
        "value": info["increment_elems"] / (t_incr * 1e-3), "unit": "interpolated volume-unknowns/s"}
    plan.close()
    del items, coarse, fine, incr
    torch.cuda.empty_cache()
    # least-squares scheme and the sparse-row (CSR, the paper's storage) path
    # on the uniform batch, Taylor-3
    items, coarse, fine = wl.uniform_batch(n_faces=2048, U=59, order=3, config_index=1, device="cuda")
    co = coarse.clone()
    rows = {}
    for name, scheme, flags in (("least_squares", 1, 0), ("least_squares_csr", 1, B.FLAG_CSR),
                                ("csr_finite_difference", 0, B.FLAG_CSR)):
        it = items.copy()
        it["scheme"] = scheme
        for prec_name, prec in (("split", B.PREC_SPLIT), ("fp64", B.PREC_FP64)):
            plan = B.Plan(it, 59, coarse.numel(), fine.numel(), prec, flags)
            if not flags:
                plan.autotune(coarse, fine, co)
            info = plan.info
            t = _time_steps(lambda: (plan.interpolate(coarse, fine), plan.restrict(fine, co)), 5, stream)
            rows[f"{name}_{prec_name}"] = {"ms_per_step": t,
                                           "value": (info["interp_outputs"] + info["restrict_outputs"]) * 59 / (t * 1e-3)}
            plan.close()
    out["taylor3_variants"] = {"workload": "2,048 hanging faces, p=9, k=3, U=59, Taylor-3", **rows}
    del items, coarse, fine, co
    torch.cuda.empty_cache()
    # patch-size sweep (the paper's run time against p at halo 3, Sec. 5.3,
    # where multiples of 3 align coarse and fine cells better): about
    # 2,048 * 81 / p^2 faces per p, so every point moves ~the same data
    sweep = {}
    for pp in (6, 8, 9, 10, 12, 15, 16, 18, 24):
        nf = max(64, int(round(2048 * 81 / (pp * pp))))
        it9, c9, f9 = wl.uniform_batch(n_faces=nf, p=pp, k=3, U=59, order=3, config_index=1, device="cuda")
        co9 = c9.clone()
        row = {"faces": nf}
        for name, order in (("taylor3", 3), ("taylor2", 2), ("dlinear", 1)):
            it = it9.copy()
            it["order"] = order
            plan = B.Plan(it, 59, c9.numel(), f9.numel(), B.PREC_SPLIT)
            tuned = plan.autotune(c9, f9, co9)
            info = plan.info
            t = _time_steps(lambda: (plan.interpolate(c9, f9), plan.restrict(f9, co9)), 10, stream)
            row[name] = {"ms_per_step": t,
                         "value": (info["interp_outputs"] + info["restrict_outputs"]) * 59 / (t * 1e-3),
                         "lanes": tuned["interp_lanes"], "threads": tuned["interp_threads"]}
            plan.close()
        sweep[f"p{pp}"] = row
        del it9, c9, f9, co9
    torch.cuda.empty_cache()
    out["patch_size_sweep"] = {"workload": "k=3, U=59, split precision, autotuned, ~2,048*81/p^2 hanging faces per p",
                               **sweep}
    # uneven batch: 20,000 subface items, p in {6,9,12}, k in {2,3}, orders 1/2/3
    items, coarse, fine = wl.uneven_batch(device="cuda")
    U = 59
    co = coarse.clone()
    for prec_name, prec in (("fixed", B.PREC_FIXED), ("split", B.PREC_SPLIT), ("fp64", B.PREC_FP64)):
        plan = B.Plan(items, U, coarse.numel(), fine.numel(), prec)
        info = plan.info
        outs = (info["interp_outputs"] + info["restrict_outputs"]) * U
        t_default = _time_steps(lambda: (plan.interpolate(coarse, fine), plan.restrict(fine, co)), 10, stream)
        chosen = plan.autotune(coarse, fine, co)
        t_tuned = _time_steps(lambda: (plan.interpolate(coarse, fine), plan.restrict(fine, co)), 10, stream)
        plan.capture_step(coarse, fine, co)
        t_graph = _time_steps(lambda: plan.launch_step(), 10, stream)
        out[f"uneven_batch_{prec_name}"] = {
            "workload": "20,000 subface items, p 6/9/12 (40/40/20 %), k 2/3, orders 1/2/3, U=59",
            "ms_per_step_default": t_default, "ms_per_step_autotuned": t_tuned, "ms_per_step_graph": t_graph,
            "autotuned": chosen, "value": outs / (min(t_tuned, t_graph) * 1e-3), "unit": UNIT,
            "step_gbs": (info["interp_bytes"] + info["restrict_bytes"]) / (min(t_tuned, t_graph) * 1e-3) / 1e9}
        plan.close()
    del items, coarse, fine, co
    torch.cuda.empty_cache()
    # split precision on puncture-like fields: 8,192 faces, Taylor-3
    items, coarse, fine = wl.puncture_batch(device="cuda")
    co = coarse.clone()
    res = {"workload": "8,192 hanging faces, p=9, k=3, U=59, Taylor-3, puncture-like fields"}
    for prec_name, prec in (("fixed", B.PREC_FIXED), ("split", B.PREC_SPLIT), ("fp64", B.PREC_FP64)):
        plan = B.Plan(items, U, coarse.numel(), fine.numel(), prec)
        info = plan.info
        fo = fine.clone()
        t = _time_steps(lambda: (plan.interpolate(coarse, fo), plan.restrict(fine, co)), 5, stream)
        res[f"{prec_name}_ms_per_step"] = t
        res[f"{prec_name}_value"] = (info["interp_outputs"] + info["restrict_outputs"]) * U / (t * 1e-3)
        # error against the FP64 oracle per field class (u mod 3) on 8 sampled faces
        arr = 2 * K * P * P * U
        errs = {0: [], 1: [], 2: []}
        rng = np.random.default_rng(8)
        for i in rng.choice(len(items), 8, replace=False):
            it = items[int(i)].copy()
            c0, f0 = int(it["coarse_offset"]), int(it["fine_offset"])
            one = np.array([it])
            one["coarse_offset"], one["fine_offset"] = 0, 0
            ch, fh = coarse[c0:c0 + arr].cpu().numpy(), fine[f0:f0 + 9 * arr].cpu().numpy()
            for got, ref in ((fo[f0:f0 + 9 * arr].cpu().numpy(), tr.interpolate(one, U, ch, fh)),
                             (co[c0:c0 + arr].cpu().numpy(), tr.restrict(one, U, fh, ch))):
                g2, r2 = got.reshape(-1, U), ref.reshape(-1, U)
                e = np.abs(g2 - r2).max(axis=0) / np.maximum(np.abs(r2).max(axis=0), 1e-300)
                for u in range(U):
                    errs[u % 3].append(e[u])
        names = {0: "psi", 1: "lapse", 2: "shift"}
        res[f"{prec_name}_err_vs_fp64"] = {names[q]: {"max": float(np.max(v)), "rms": float(np.sqrt(np.mean(np.square(v))))}
                                           for q, v in errs.items()}
        plan.close()
        del fo
    out["puncture_split"] = res
    del items, coarse, fine, co
    torch.cuda.empty_cache()
    out["adjoint"] = adjoint_leg(B, wl, stream, 4096)
    # diagonal (edge and vertex) ghost volumes of 256 hanging faces: every
    # fine face array's ghost half widened by k on each tangential side
    items, coarse, fine = wl.uniform_batch(n_faces=256, U=U, order=3, config_index=5, device="cuda")
    plan = B.Plan(items, U, coarse.numel(), fine.numel(), B.PREC_FIXED)
    diag = torch.empty(plan.diagonal_elems, dtype=torch.float64, device="cuda")
    plan.interpolate_diagonal(coarse, diag)  # builds the tile table
    t = time_kernel(lambda: plan.interpolate_diagonal(coarse, diag), 5, stream)
    vols = plan.diagonal_elems // U
    out["diagonal_halos"] = {"workload": "256 hanging faces, p=9, k=3, U=59, Taylor-3: widened ghost boxes "
                                         "(p + 2k)^2 x k per fine face array, float64",
                             "ms_per_call": t, "value": vols * U / (t * 1e-3), "unit": "volume-unknowns/s",
                             "bytes_written": plan.diagonal_elems * 8}
    plan.close()
    del items, coarse, fine, diag
    torch.cuda.empty_cache()
    return out


def compare_paths(B, wl, items, coarse, fine, coarse_out, U, args, stream, plan_main):
    """d-linear and Taylor-2 on the same workload and GPU, in every precision
    mode, with the error of each against the FP64 oracle."""
    out = {}
    for name, order in (("dlinear", 1), ("taylor2", 2), ("taylor3", 3)):
        for prec_name, prec in (("fixed", B.PREC_FIXED), ("fp64", B.PREC_FP64), ("split", B.PREC_SPLIT)):
            it = items.copy()
            it["order"] = order
            plan = B.Plan(it, U, coarse.numel(), fine.numel(), prec)
            plan.autotune(coarse, fine, coarse_out)
            info = plan.info
            step = lambda: (plan.interpolate(coarse, fine), plan.restrict(fine, coarse_out))
            for _ in range(3):
                step()
            import torch
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            n = max(5, args.steps // 2)
            e0.record(stream)
            for _ in range(n):
                step()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / n
            ti = time_kernel(lambda: plan.interpolate(coarse, fine), n, stream)
            tr_ = time_kernel(lambda: plan.restrict(fine, coarse_out), n, stream)
            outs = (info["interp_outputs"] + info["restrict_outputs"]) * U
            out[f"{name}_{prec_name}"] = {
                "value": outs / (ms * 1e-3), "ms_per_step": ms, "interp_ms": ti, "restrict_ms": tr_,
                "interp_gbs": info["interp_bytes"] / (ti * 1e-3) / 1e9,
                "restrict_gbs": info["restrict_bytes"] / (tr_ * 1e-3) / 1e9,
                "step_gbs": (info["interp_bytes"] + info["restrict_bytes"]) / (ms * 1e-3) / 1e9,
                "err_vs_fp64": error_vs_oracle(it, coarse, fine, plan, U, n_faces=4)}
            plan.close()
    return out


def adjoint_leg(B, wl, stream, nf, steps=5):
    """P^T and R^T of a fixed-point Taylor-3 plan over nf hanging faces (p=9,
    k=3, U=59).  Algorithmic bytes: P^T reads the ghost gradients and writes
    the whole coarse arrays, R^T reads the restricted halo gradients and
    writes the whole fine arrays (the API overwrites every gradient entry)."""
    import torch
    U = 59
    items, coarse, fine = wl.uniform_batch(n_faces=nf, U=U, order=3, config_index=4, device="cuda")
    plan = B.Plan(items, U, coarse.numel(), fine.numel(), B.PREC_FIXED)
    gc, gf = torch.empty_like(coarse), torch.empty_like(fine)
    plan.interpolate_adjoint(fine, gc)  # builds the transposed tables
    t = _time_steps(lambda: (plan.interpolate_adjoint(fine, gc), plan.restrict_adjoint(coarse, gf)), steps, stream)
    t_pt = time_kernel(lambda: plan.interpolate_adjoint(fine, gc), steps, stream)
    t_rt = time_kernel(lambda: plan.restrict_adjoint(coarse, gf), steps, stream)
    b_pt = nf * (9 * K * P * P + 2 * K * P * P) * U * 8
    b_rt = nf * (K * P * P + 18 * K * P * P) * U * 8
    hbm = float(measured_peaks()[0]["hbm_gbs"])
    res = {"workload": f"{nf:,} hanging faces, p=9, k=3, U=59, Taylor-3, P^T + R^T",
           "ms_per_step": t, "value": (coarse.numel() + fine.numel()) / (t * 1e-3),
           "unit": "gradient entries/s",
           "interp_adjoint_ms": t_pt, "restrict_adjoint_ms": t_rt,
           "algorithmic_bytes": b_pt + b_rt, "achieved_gbs": (b_pt + b_rt) / (t * 1e-3) / 1e9,
           "frac": (b_pt + b_rt) / (t * 1e-3) / 1e9 / hbm,
           "interp_adjoint_gbs": b_pt / (t_pt * 1e-3) / 1e9,
           "interp_adjoint_frac": b_pt / (t_pt * 1e-3) / 1e9 / hbm,
           "restrict_adjoint_gbs": b_rt / (t_rt * 1e-3) / 1e9}
    plan.close()
    del items, coarse, fine, gc, gf
    torch.cuda.empty_cache()
    return res


def e2e_leg(plan, coarse, fine, coarse_out, outs, args, stream, items=None, n_chunks=8):
    """The same step through the C ABI with the data in pinned host memory:
    every step uploads both buffers, runs interpolate + restrict and downloads
    both results.  The faces are independent, so the batch is cut into
    n_chunks plans over contiguous chunks whose uploads, kernels and
    downloads overlap on three streams (H2D, compute, D2H) ordered by
    events."""
    import torch
    from paper_2504_15814_gb300 import binding as B
    from paper_2504_15814_gb300.sharding import local_items, shard_bounds
    ch = torch.empty_like(coarse, device="cpu").pin_memory()
    fh = torch.empty_like(fine, device="cpu").pin_memory()
    ch.copy_(coarse)
    fh.copy_(fine)
    cho = torch.empty_like(ch).pin_memory()
    fho = torch.empty_like(fh).pin_memory()
    cd, fd, cod = torch.empty_like(coarse), torch.empty_like(fine), torch.empty_like(coarse)
    chunks = []
    for lo, hi in shard_bounds(items, n_chunks):
        if hi <= lo:
            continue
        sub, cl, fl, csrc, fsrc = local_items(items, U, lo, hi)
        c0, f0 = csrc[0][0], fsrc[0][0]
        # the chunk's arrays are contiguous in the global buffers
        cn = csrc[-1][0] + csrc[-1][2] - c0
        fn = fsrc[-1][0] + fsrc[-1][2] - f0
        cplan = B.Plan(sub, U, cn, fn, plan.precision)
        cplan.set_tuning(**plan.tuning)
        chunks.append((cplan, c0, cn, f0, fn))
    s_h2d, s_cmp, s_d2h = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
    drained = [None] * len(chunks)  # per chunk: its last download, before the device buffers are reused

    def step():
        for q, (cplan, c0, cn, f0, fn) in enumerate(chunks):
            up, done = torch.cuda.Event(), torch.cuda.Event()
            if drained[q] is not None:
                s_h2d.wait_event(drained[q])
            with torch.cuda.stream(s_h2d):
                cd[c0:c0 + cn].copy_(ch[c0:c0 + cn], non_blocking=True)
                fd[f0:f0 + fn].copy_(fh[f0:f0 + fn], non_blocking=True)
                up.record(s_h2d)
            s_cmp.wait_event(up)
            with torch.cuda.stream(s_cmp):
                cod[c0:c0 + cn].copy_(cd[c0:c0 + cn], non_blocking=True)
                cplan.interpolate(cd[c0:c0 + cn], fd[f0:f0 + fn], stream=s_cmp)
                cplan.restrict(fd[f0:f0 + fn], cod[c0:c0 + cn], stream=s_cmp)
                done.record(s_cmp)
            s_d2h.wait_event(done)
            with torch.cuda.stream(s_d2h):
                fho[f0:f0 + fn].copy_(fd[f0:f0 + fn], non_blocking=True)
                cho[c0:c0 + cn].copy_(cod[c0:c0 + cn], non_blocking=True)
                drained[q] = torch.cuda.Event()
                drained[q].record(s_d2h)

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    n = 3
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s_h2d)
    for _ in range(n):
        step()
    s_h2d.wait_stream(s_d2h)
    e1.record(s_h2d)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / n
    for cplan, *_ in chunks:
        cplan.close()
    nbytes = (coarse.numel() + fine.numel()) * 8
    return {"value": outs / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": nbytes, "chunks": len(chunks),
            "how": "pinned host buffers; per step H2D of both buffers, interpolate + restrict, D2H of both "
                   "results; chunks of faces overlap on H2D / compute / D2H streams"}


def e2e_zero_copy(plan, items, coarse, fine, coarse_out, outs, stream, chunk_counts=(1, 2, 4, 8)):
    """The same step through the C ABI on buffers that live in pinned host
    memory: the kernels read their inputs and write their results there in
    place, over the host link (no staging copies).  Interpolation writes more
    than it reads and restriction the reverse, so with n chunks of faces (one
    plan each) the restriction of chunk q (stream 2) overlaps the
    interpolation of chunk q + 1 (stream 1); a step starts once the previous
    step's restrictions are done.  Returns the fastest chunk count and all."""
    import torch
    from paper_2504_15814_gb300 import binding as B
    from paper_2504_15814_gb300.sharding import shard_bounds
    c_h = coarse.cpu().pin_memory()
    f_h = fine.cpu().pin_memory()
    co_h = coarse_out.cpu().pin_memory()
    info = plan.info
    w_i, w_r = info["interp_outputs"] * U * 8, info["restrict_outputs"] * U * 8
    h2d = (info["interp_bytes"] - w_i) + (info["restrict_bytes"] - w_r)
    s_i, s_r = torch.cuda.Stream(), torch.cuda.Stream()
    per = {}
    for n_chunks in chunk_counts:
        plans = []
        for lo, hi in shard_bounds(items, n_chunks):
            if hi > lo:
                cp = B.Plan(items[lo:hi], U, c_h.numel(), f_h.numel(), plan.precision)
                cp.set_tuning(**plan.tuning)
                plans.append(cp)

        def step():
            s_i.wait_stream(s_r)
            for cp in plans:
                cp.interpolate(c_h, f_h, stream=s_i)
                ev = torch.cuda.Event()
                ev.record(s_i)
                s_r.wait_event(ev)
                cp.restrict(f_h, co_h, stream=s_r)

        for _ in range(2):
            step()
        torch.cuda.synchronize()
        n = 5
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s_i)
        s_r.wait_stream(s_i)
        for _ in range(n):
            step()
        s_i.wait_stream(s_r)
        e1.record(s_i)
        torch.cuda.synchronize()
        per[n_chunks] = e0.elapsed_time(e1) / n
        for cp in plans:
            cp.close()
    best = min(per, key=per.get)
    ms = per[best]
    return {"value": outs / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": w_i + w_r, "chunks": best,
            "ms_per_step_by_chunks": {str(k): v for k, v in per.items()},
            "link_gbs": (h2d + w_i + w_r) / (ms * 1e-3) / 1e9,
            "how": "buffers in pinned host memory; interpolate + restrict through the C ABI read the inputs and "
                   "write the results in place over the host link (bytes = the kernels' algorithmic reads and "
                   "writes); chunks of faces overlap restriction with the next chunk's interpolation"}


def error_vs_oracle(items, coarse, fine, plan, U, n_faces=8):
    """Max and RMS normwise error of sampled outputs against the FP64 oracle."""
    import numpy as np
    import torch
    from oracle import transfer as tr
    f_out = fine.clone()
    c_out = coarse.clone()
    plan.interpolate(coarse, f_out)
    plan.restrict(fine, c_out)
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    arr = 2 * K * P * P * U
    errs = []
    chosen = rng.choice(len(items), n_faces, replace=False)
    for i in chosen:
        it = items[int(i)]
        co, fo = int(it["coarse_offset"]), int(it["fine_offset"])
        c_h = np.zeros(arr)
        c_h[:] = coarse[co:co + arr].cpu().numpy()
        f_h = fine[fo:fo + 9 * arr].cpu().numpy()
        one = it.copy()
        one["coarse_offset"], one["fine_offset"] = 0, 0
        f_ref = tr.interpolate([one], U, c_h, f_h)
        c_ref = tr.restrict([one], U, f_h, c_h)
        fg = f_out[fo:fo + 9 * arr].cpu().numpy()
        cg = c_out[co:co + arr].cpu().numpy()
        for got, ref in ((fg, f_ref), (cg, c_ref)):
            g = got.reshape(-1, U)
            r = ref.reshape(-1, U)
            errs.append((np.abs(g - r).max(axis=0) / np.maximum(np.abs(r).max(axis=0), 1e-300)))
    e = np.concatenate(errs)
    return {"max": float(e.max()), "rms": float(np.sqrt(np.mean(e ** 2))),
            "sample": f"{n_faces} random hanging faces, all outputs, normwise per (face, unknown)"}


if __name__ == "__main__":
    main()
