#!/usr/bin/env python
"""Benchmark of the matrix-free Q1 operator apply y = A x on the GPU (one JSON line on stdout).

Workload (one "step" = one pass of the hot path over one batch of synthetic input): the matrix-free
FP64 apply of the scalar Laplace operator on a 256^3-cell Cartesian box (16,908,544 free DoF) and
of isotropic elasticity on a 160^3-cell box (12,442,080 free DoF), both with 8 z-layers of
heterogeneous coefficients times per-cell lognormal noise and u = 0 on z = 0.  ``value`` is free
DoF processed per second over both applies (GDoF/s).  The same line carries, measured after the
timed region: the in-library CSR SpMV on the same matrices, CG time-to-1e-8 (matrix-free vs CSR),
the end-to-end throughput through the C ABI with host buffers, the roofline of the dominant
kernel, and the CPU oracle timed on a bounded sample on the host cores.

Launch: ``python bench.py [--gpus N --steps K --warmup W]``; for N > 1 under torchrun every rank
runs an independent replica (the operator needs no exchange between independent problems) and
rank 0 prints the line with value = all ranks' DoF / max-over-ranks time.
``--impl reference`` times the CPU oracle (the deliberately slow reference implementation) on the
host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import shutil
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GDoF/s of matrix-free A.x (Q1 Laplace 256^3 + elasticity 160^3, FP64)"
UNIT = "GDoF/s"
# DRAM bytes (read + write) per launch of the face-marching FP64 kernels at the benchmarked sizes:
# one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) on the 192^3 Laplace and 128^3
# elasticity meshes, scaled by the node count (the traffic is proportional to it).  Part of y is
# still dirty in L2 when a launch ends, so the write share is below the bytes written.
TRAFFIC = {"laplace": round(153548544 * 16974593 / 7189057), "elasticity": round(101496576 * 4173281 / 2146689)}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-laplace", type=int, default=256)
    ap.add_argument("--n-elasticity", type=int, default=160)
    ap.add_argument("--no-cg", action="store_true", help="skip the CG time-to-solution measurements")
    ap.add_argument("--no-csr", action="store_true", help="skip the CSR SpMV measurements")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-solver measurement")
    ap.add_argument("--no-multi", action="store_true", help="skip the multi-RHS measurement")
    ap.add_argument("--no-vector", action="store_true", help="skip the vector Laplace measurement")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision measurement")
    ap.add_argument("--no-tet", action="store_true", help="skip the P1 tetrahedra and Q2 hexahedra measurements")
    ap.add_argument("--n-tet", type=int, default=96, help="boxes per side of the tetrahedral meshes (6 tets each)")
    ap.add_argument("--n-q2", type=int, default=48, help="Q2 hexahedra per side")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-preconditioner measurement")
    ap.add_argument("--n-learned", type=int, default=128)
    ap.add_argument("--pairs", type=int, default=2000)
    ap.add_argument("--train-steps", type=int, default=4000)
    ap.add_argument("--lr", type=float, default=2e-4)
    ap.add_argument("--cg-timeout", type=float, default=90.0)
    ap.add_argument("--variant", type=int, default=0, help="0 = auto (fastest FP64-accurate), 1 = reference")
    ap.add_argument("--no-tune", action="store_true", help="keep the library's default z-segment length")
    ap.add_argument("--tile-segments", default="",
                    help="z-segment lengths 'laplace,elasticity' to use instead of tuning (e.g. the ones a "
                         "tuned run reported), so that a profiled run launches the same grids")
    return ap.parse_args()


# ------------------------------------------------------------------------------------ clocks ----

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 100):
        self.proc = None
        self.path = None
        exe = shutil.which("nvidia-smi")
        if exe is None:
            return
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        self.f = open(self.path, "w")
        self.proc = subprocess.Popen([exe, "-i", str(gpu_index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                      "-lms", str(period_ms)], stdout=self.f, stderr=subprocess.DEVNULL)
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        with open(self.path) as f:
            text = f.read()
        os.unlink(self.path)
        return summarise_clocks(text)


def summarise_clocks(text: str):
    """Median SM clock, maximum SM clock and the throttle reasons seen in `nvidia-smi --query-gpu=
    ClockSampler.FIELDS --format=csv,noheader,nounits` output; rows that are short or hold no number
    (a partial last line, "[N/A]") are skipped.  None when no row parses."""
    sm, smax, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in text.strip().splitlines():
        r = [c.strip() for c in line.split(",")]
        if len(r) < 9:
            continue
        try:
            sm.append(float(r[1]))
            smax.append(float(r[2]))
        except ValueError:
            continue
        for nm, v in zip(names, r[5:9]):
            if v.lower() == "active":
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
            "samples": len(sm)}


# ----------------------------------------------------------------------- multi-rank timing ----

def aggregate(units_per_rank: float, seconds: float, world: int, dist=None, device=None):
    """Whole-job throughput of `world` independent replicas: every rank processed `units_per_rank`
    units; the job took the slowest rank's time (max over ranks, via all_reduce when distributed)."""
    t = seconds
    if dist is not None and world > 1:
        import torch
        v = torch.tensor([seconds], dtype=torch.float64, device=device)
        dist.all_reduce(v, op=dist.ReduceOp.MAX)
        t = float(v.item())
    return world * units_per_rank / t, t


# ------------------------------------------------------------------------------- CPU oracle ----

def slab(p, nz_slab):
    """The bottom ``nz_slab`` cell layers of a box problem (same coordinates and coefficients)."""
    from paper_2308_09839_gb300 import inputs
    nn = (p.nx + 1) * (p.ny + 1) * (nz_slab + 1)
    ne = p.nx * p.ny * nz_slab
    return inputs.Problem(p.name + f"_slab{nz_slab}", p.physics, p.nx, p.ny, nz_slab, p.coords[:nn], p.mat[:ne],
                          p.dirichlet[:nn], p.seed)


def bind_to_gpu_numa(device: int):
    """Bind this process to the CPUs of the NUMA node of `device` (read from sysfs through the GPU's
    PCI address); returns the node, or None when the topology cannot be read (then nothing changes)."""
    try:
        import torch
        pr = torch.cuda.get_device_properties(device)
        addr = f"{pr.pci_domain_id:04x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0"
        node = int(open(f"/sys/bus/pci/devices/{addr}/numa_node").read().strip())
        if node < 0:
            return None
        cpus = set()
        for part in open(f"/sys/devices/system/node/node{node}/cpulist").read().strip().split(","):
            lo, _, hi = part.partition("-")
            cpus.update(range(int(lo), int(hi or lo) + 1))
        if cpus:
            os.sched_setaffinity(0, cpus)
        return node
    except (AttributeError, OSError, ValueError):
        return None


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def _oracle_slab_task(args):
    """One worker's share of the all-core oracle timing: the oracle apply on an n x n x nz_slab box of
    the workload's physics and cell-constant recipe (the cost per cell does not depend on the values),
    counted as cells x the full problem's free DoF per cell (module-level so that a spawned process
    can run it)."""
    kind, n, nz_slab, seed, dof_per_cell = args
    from oracle import fem
    from paper_2308_09839_gb300 import inputs
    make = inputs.laplace_box if kind == "laplace" else inputs.elasticity_box
    s = make(n, nz=nz_slab, sigma=0.5, layered=True, seed=seed)
    x = s.x(seed)
    cells = s.cell_array()
    t0 = time.perf_counter()
    fem.apply(s.physics, s.coords, cells, s.mat, s.dirichlet, x)
    return time.perf_counter() - t0, cells.shape[0] * dof_per_cell


def oracle_all_core_rate(problems, nz_slabs, workers):
    """The oracle on every host core: `workers` spawned processes (spawn: nothing inherited from a CUDA
    context) each apply the oracle to their own slab of each problem at once; returns (free DoF per
    second over the wall time of the parallel phase, wall seconds, description)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    tasks = []
    for p, nzs in zip(problems, nz_slabs):
        tasks += [(p.physics, p.nx, nzs, 100 + w, p.n_free / p.n_cells) for w in range(workers)]
    with ctx.Pool(workers) as pool:
        pool.map(_oracle_slab_task, [(p.physics, 8, 1, 0, 1.0) for p in problems] * workers)  # warm the imports
        t0 = time.perf_counter()
        res = pool.map(_oracle_slab_task, tasks, chunksize=1)
        wall = time.perf_counter() - t0
    dofs = sum(r[1] for r in res)
    desc = "; ".join(f"{workers} x {p.physics} {p.nx}x{p.ny}x{nzs} cells" for p, nzs in zip(problems, nz_slabs))
    return dofs / wall, wall, desc


def oracle_sample_rate(problems, nz_slabs, repeats=1):
    """Time the oracle's apply on slabs of each problem; returns (free DoF per second scaled from
    the full problems' DoF per cell, seconds, description)."""
    from oracle import fem
    dof_equiv, secs, desc = 0.0, 0.0, []
    for p, nzs in zip(problems, nz_slabs):
        s = slab(p, nzs)
        cells = s.cell_array()
        x = s.x()
        t0 = time.perf_counter()
        for _ in range(repeats):
            fem.apply(s.physics, s.coords, cells, s.mat, s.dirichlet, x)
        dt = time.perf_counter() - t0
        dof_equiv += repeats * cells.shape[0] * (p.n_free / p.n_cells)
        secs += dt
        desc.append(f"{p.physics} {p.nx}x{p.ny}x{nzs} cells x{repeats}")
    return dof_equiv / secs, secs, "; ".join(desc)


def workload_name(pL, pE):
    """The benchmarked workload, named the same way by both arms."""
    return (f"Q1 matrix-free apply, Laplace {pL.nx}^3 Cartesian (F={pL.n_free}) + elasticity "
            f"{pE.nx}^3 Cartesian (F={pE.n_free}), 8 z-layers x lognormal(0,0.5)")


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2308_09839_gb300 import inputs
    pL = inputs.cartesian_laplace_256(n=args.n_laplace)
    pE = inputs.cartesian_elasticity_160(n=args.n_elasticity)
    workers = os.cpu_count() or 1
    for _ in range(max(1, args.warmup)):  # untimed warm-up steps (each step creates its own pool)
        oracle_all_core_rate([pL, pE], [1, 1], workers)
    rates, tot = [], 0.0
    for _ in range(args.steps):
        r, s, desc = oracle_all_core_rate([pL, pE], [1, 1], workers)
        rates.append(r)
        tot += s
    value = float(np.mean(rates)) / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(pL, pE), "n_dof_total": [pL.n_dof, pE.n_dof],
                   "parallelism": "host cores", "l2": "not applicable: the oracle runs on the host cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle", "cpu_model": cpu_model(),
                         "sample": "per step: " + desc + " (one-cell-thick slabs of both workloads, one per "
                                   "process, all at once)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------------- GPU arm ----

def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    from paper_2308_09839_gb300 import bytes_model as bm
    from paper_2308_09839_gb300 import inputs, mf

    CG_OK = (mf.MF_OK, mf.MF_NOT_CONVERGED, mf.MF_ERR_TIMEOUT)
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    hbm_src = "of measured" if "hbm_gbs" in peaks else "of fallback"

    pL = inputs.cartesian_laplace_256(n=args.n_laplace)
    pE = inputs.cartesian_elasticity_160(n=args.n_elasticity)
    meshes, segs = [], []
    fixed = [int(s) for s in args.tile_segments.split(",")] if args.tile_segments else None
    for j, p in enumerate((pL, pE)):
        m = mf.Mesh.from_problem(p, device=f"cuda:{local}")
        m.set_variant(args.variant)
        if fixed is not None:
            mf.mf_set_tile_segment(m, fixed[j])
            segs.append(fixed[j])
        elif args.variant == 0 and not args.no_tune:
            from paper_2308_09839_gb300 import autotune
            segs.append(autotune.tune_apply(m, use_cache=False))  # setup, not timed
        x = torch.from_numpy(p.x()).cuda()
        meshes.append((p, m, x, torch.empty_like(x)))
    F = [p.n_free for p in (pL, pE)]
    torch.cuda.synchronize()

    def step():
        for (p, m, x, y) in meshes:
            m.apply(x, y)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    K = args.steps
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    l0 = mf.mf_kernel_launches()
    e0.record()
    for k in range(K):
        step()
    e1.record()
    torch.cuda.synchronize()
    barrier()
    launches = mf.mf_kernel_launches() - l0
    clk = clocks.stop()
    t_local = e0.elapsed_time(e1) / 1e3
    # per-operator kernel time: K back-to-back applies of one operator between two events (the
    # per-step events above include host launch gaps when a kernel is shorter than the launch path)
    t_app = []
    for (p, m, x, y) in meshes:
        m.apply(x, y)
        e0.record()
        for _ in range(K):
            m.apply(x, y)
        e1.record()
        torch.cuda.synchronize()
        t_app.append(e0.elapsed_time(e1) / 1e3 / K)
    value, t_total = aggregate(K * sum(F), t_local, world, dist if world > 1 else None, "cuda")
    value /= 1e9

    # ---- parity spot check of the timed launch configuration (sampled rows vs the oracle)
    extras = {"gdofs_apply": {"laplace": F[0] / t_app[0] / 1e9, "elasticity": F[1] / t_app[1] / 1e9},
              "ms_apply": {"laplace": 1e3 * t_app[0], "elasticity": 1e3 * t_app[1]}}

    # ---- end to end through the C ABI with host buffers (H2D of x, apply, D2H of y every step).
    # The host buffers are allocated (first touch) by a thread bound to the CPUs of the NUMA node
    # the GPU is attached to, so the copies do not cross the link between the host's sockets.
    numa_node = bind_to_gpu_numa(local)
    # Each mesh alternates between two device buffer sets, each on its own stream, so the copies
    # of one step overlap the applies of the other mesh and of the neighbouring step (the copy
    # engines and the SMs work at the same time); every step still moves its full input and output.
    hx = [x.cpu().pin_memory() for (_, _, x, _) in meshes]
    hy = [[torch.empty_like(h).pin_memory() for _ in range(2)] for h in hx]
    dx = [[x, x.clone()] for (_, _, x, _) in meshes]
    dy = [[y, torch.empty_like(y)] for (_, _, _, y) in meshes]
    streams = [[torch.cuda.Stream() for _ in range(2)] for _ in meshes]

    def e2e_step(k):
        b = k & 1
        for j, (p, m, _, _) in enumerate(meshes):
            st = streams[j][b]
            with torch.cuda.stream(st):
                dx[j][b].copy_(hx[j], non_blocking=True)
                m.apply(dx[j][b], dy[j][b], stream=st)
                hy[j][b].copy_(dy[j][b], non_blocking=True)

    for k in range(4):
        e2e_step(k)
    torch.cuda.synchronize()
    Ke = max(6, K // 2) // 2 * 2
    barrier()
    torch.cuda.synchronize()
    main = torch.cuda.current_stream()
    e0.record(main)
    for sl in streams:
        for st in sl:
            st.wait_event(e0)
    for k in range(Ke):
        e2e_step(k)
    for sl in streams:
        for st in sl:
            ev = torch.cuda.Event()
            ev.record(st)
            main.wait_event(ev)
    e1.record(main)
    torch.cuda.synchronize()
    e2e_value, _ = aggregate(Ke * sum(F), e0.elapsed_time(e1) / 1e3, world, dist if world > 1 else None, "cuda")
    io_bytes = sum(h.numel() * 8 for h in hx)
    e2e = {"value": e2e_value / 1e9, "unit": UNIT, "h2d_bytes_per_step": io_bytes, "d2h_bytes_per_step": io_bytes,
           "overlap": "2 streams per mesh, copies overlap applies", "host_numa_node": numa_node}
    del dx, dy

    # ---- roofline of the dominant kernel (the matrix-free apply taking the most time).  The FP64-
    # accurate apply runs in double-word FP32 arithmetic and is bound by the FP32 pipe: achieved =
    # algorithmic FP32-pipe operations per launch / kernel time against SMs x lanes x max clock.
    # The HBM view is reported beside it: the paper's read-once bytes of a matrix-free apply on a
    # general hex mesh (node map, coordinates, cell constants, x, y) and the bytes this kernel must
    # move on a tensor-product grid (cell constants, mask, x, y).
    j = int(np.argmax(t_app))
    p = (pL, pE)[j]
    tp = meshes[j][1].info["tensor_product"] and args.variant == 0
    paper_bytes = bm.kernel_apply_bytes(p.physics, p.n_cells, p.n_nodes, structured=False) - p.n_nodes
    kern_bytes = bm.kernel_apply_bytes(p.physics, p.n_cells, p.n_nodes, structured=True, tensor_product=tp)
    hbm = {"peak": hbm_peak, "unit": "GB/s", "peak_source": hbm_src,
           "paper_model_bytes": paper_bytes, "paper_model_achieved": paper_bytes / t_app[j] / 1e9,
           "paper_model_frac": paper_bytes / t_app[j] / 1e9 / hbm_peak,
           "kernel_bytes": kern_bytes, "kernel_bytes_achieved": kern_bytes / t_app[j] / 1e9,
           "kernel_bytes_frac": kern_bytes / t_app[j] / 1e9 / hbm_peak}
    if tp:
        # headline: the paper's read-once bytes of a matrix-free apply (node map, coordinates, cell
        # constants, x, y) per launch over the kernel time, against the measured copy bandwidth; the
        # FP32-pipe view (what binds this kernel on GB300) beside it
        ops = bm.kernel_apply_ops(p.physics)["total"] * p.n_cells
        peak = bm.fp32_lane_peak() / 1e12
        alu = {"achieved": ops / t_app[j] / 1e12, "peak": peak, "unit": "Tops/s", "frac": ops / t_app[j] / 1e12 / peak,
               "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz",
               "algorithmic_ops": ops, "ops_per_element": bm.kernel_apply_ops(p.physics)["total"]}
        roof = {"kernel": f"matrix-free {p.physics} apply ({p.nx}^3, face-marching DW)", "bound": "hbm",
                "achieved": paper_bytes / t_app[j] / 1e9, "peak": hbm_peak, "unit": "GB/s",
                "frac": paper_bytes / t_app[j] / 1e9 / hbm_peak, "peak_source": hbm_src,
                "algorithmic_bytes": paper_bytes, "bytes_model": "paper read-once model (node map 32 B/cell, "
                "coordinates 24 B/node, cell constants, x and y once)", "traffic": TRAFFIC.get(p.physics),
                "kernel_bytes": kern_bytes, "kernel_bytes_frac": kern_bytes / t_app[j] / 1e9 / hbm_peak, "alu": alu}
    else:
        achieved = kern_bytes / t_app[j] / 1e9
        roof = {"kernel": f"matrix-free {p.physics} apply ({p.nx}^3)", "bound": "hbm", "achieved": achieved,
                "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak, "peak_source": hbm_src,
                "algorithmic_bytes": kern_bytes, "traffic": None}

    # ---- CSR SpMV on the same matrices (in-library matrix-based baseline)
    if not args.no_csr:
        csr = {}
        for (p, m, x, y) in meshes:
            A = m.assemble_csr()
            for _ in range(3):
                A.spmv(x, y)
            torch.cuda.synchronize()
            Ks = max(5, K // 2)
            e0.record()
            for _ in range(Ks):
                A.spmv(x, y)
            e1.record()
            torch.cuda.synchronize()
            ts = e0.elapsed_time(e1) / 1e3 / Ks
            sb = bm.kernel_spmv_bytes(A.info["n_rows"], A.info["nnz"])
            csr[p.physics] = {"gdofs": p.n_free / ts / 1e9, "ms": 1e3 * ts, "nnz": A.info["nnz"],
                              "hbm_frac": sb / ts / 1e9 / hbm_peak}
            if not args.no_cg:
                xs, info = m.cg(torch.from_numpy(p.b()).cuda(), csr=A, timeout_s=args.cg_timeout, ok=CG_OK)
                csr[p.physics]["cg"] = {"seconds": info.seconds, "iters": info.iters, "status": info.status,
                                        "rel_res_true": info.rel_res_true}
            A.close()
            del A
            torch.cuda.empty_cache()
        extras["csr_spmv"] = csr
        extras["mf_over_csr"] = {ph: extras["gdofs_apply"][ph] / csr[ph]["gdofs"] for ph in csr}

    # ---- the 16^3 jittered Laplace problem (lognormal(0, 1) kappa): one apply as the median of 1000
    # launches (device time between events of consecutive launches, and host round trip with a
    # synchronize), L2-resident and latency-bound, plus CG to 1e-8
    p1 = inputs.small_laplace_16(seed=0)
    m1 = mf.Mesh.from_problem(p1, device=f"cuda:{local}")
    x1 = torch.from_numpy(p1.x()).cuda()
    y1 = torch.empty_like(x1)
    for _ in range(20):
        m1.apply(x1, y1)
    torch.cuda.synchronize()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(1001)]
    evs[0].record()
    for k in range(1000):
        m1.apply(x1, y1)
        evs[k + 1].record()
    torch.cuda.synchronize()
    dev_us = sorted(1e3 * evs[k].elapsed_time(evs[k + 1]) for k in range(1000))
    host_us = []
    for _ in range(1000):
        t0 = time.perf_counter()
        m1.apply(x1, y1)
        torch.cuda.synchronize()
        host_us.append(1e6 * (time.perf_counter() - t0))
    host_us.sort()
    c1 = {"mesh": "Laplace 16^3, jitter 0.2h, lognormal(0, 1) kappa", "free_dof": p1.n_free,
          "variant": "partial assembly (double-word)" if m1.info["partial_assembly"] else "general (double-word)",
          "apply_us_median": dev_us[500], "apply_us_p10_p90": [dev_us[100], dev_us[900]],
          "apply_gdofs": p1.n_free / (dev_us[500] * 1e-6) / 1e9, "host_round_trip_us_median": host_us[500]}
    if not args.no_cg:
        b1 = torch.from_numpy(p1.b()).cuda()
        m1.cg(b1, timeout_s=args.cg_timeout, ok=CG_OK)  # graph capture and workspace, not timed
        _, i1 = m1.cg(b1, timeout_s=args.cg_timeout, ok=CG_OK)
        c1["cg"] = {"seconds": i1.seconds, "iters": i1.iters, "status": i1.status, "rel_res_true": i1.rel_res_true,
                    "us_per_iter": 1e6 * i1.seconds / max(i1.iters, 1)}
    extras["laplace16_jittered"] = c1
    m1.close()
    del x1, y1

    # ---- CG time-to-1e-8 with the matrix-free operator
    if not args.no_cg:
        cg = {}
        for (p, m, x, y) in meshes:
            b = torch.from_numpy(p.b()).cuda()
            xs, info = m.cg(b, timeout_s=args.cg_timeout, ok=CG_OK)
            xs = xs.clone()
            cg[p.physics] = {"seconds": info.seconds, "iters": info.iters, "status": info.status,
                             "rel_res_true": info.rel_res_true,
                             "cg_gdofs": p.n_free * info.iters / info.seconds / 1e9,
                             "ms_per_iter": 1e3 * info.seconds / max(info.iters, 1)}
            # the same recurrence with separate vector kernels: same iterates, bitwise
            xsp, isp = m.cg(b, timeout_s=args.cg_timeout, ok=CG_OK, recurrence=mf.MF_CG_CLASSIC_SPLIT)
            cg[p.physics]["split_kernels"] = {"seconds": isp.seconds, "iters": isp.iters,
                                              "ms_per_iter": 1e3 * isp.seconds / max(isp.iters, 1),
                                              "bitwise_equal_solution": bool(torch.equal(xs, xsp))}
            del xsp
            # single-synchronisation recurrence (Chronopoulos-Gear): one kernel fewer per iteration
            _, ip = m.cg(b, timeout_s=args.cg_timeout, ok=CG_OK, recurrence=mf.MF_CG_PIPELINED)
            cg[p.physics]["pipelined"] = {"seconds": ip.seconds, "iters": ip.iters, "status": ip.status,
                                          "rel_res_true": ip.rel_res_true,
                                          "ms_per_iter": 1e3 * ip.seconds / max(ip.iters, 1),
                                          "ms_per_iter_classic": 1e3 * info.seconds / max(info.iters, 1)}
        extras["cg_matfree"] = cg

    # ---- vector Laplace (Eq. 5) on the elasticity workload's 160^3 mesh: matrix-free vs CSR
    if not args.no_vector:
        pv = inputs.vector_laplace_box(args.n_elasticity, sigma=0.5, layered=True, seed=0)
        mv = mf.Mesh.from_problem(pv, device=f"cuda:{local}")
        if args.variant == 0 and not args.no_tune:
            from paper_2308_09839_gb300 import autotune
            autotune.tune_apply(mv, use_cache=False)
        xv = torch.from_numpy(pv.x()).cuda()
        yv = torch.empty_like(xv)

        def timed(fn, reps):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            e0.record()
            for _ in range(reps):
                fn()
            e1.record()
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / 1e3 / reps

        tv = timed(lambda: mv.apply(xv, yv), max(10, K // 4))
        vec = {"mesh": f"vector Laplace {pv.nx}^3 Cartesian", "free_dof": pv.n_free, "ms_apply": 1e3 * tv,
               "gdofs_apply": pv.n_free / tv / 1e9}
        if not args.no_csr:
            Av = mv.assemble_csr()
            ts = timed(lambda: Av.spmv(xv, yv), max(10, K // 4))
            vec.update({"ms_csr": 1e3 * ts, "gdofs_csr": pv.n_free / ts / 1e9, "nnz": Av.info["nnz"],
                        "mf_over_csr": ts / tv})
            Av.close()
            del Av
        extras["vector_laplace"] = vec
        mv.close()
        del xv, yv
        torch.cuda.empty_cache()

    # ---- elements beyond Q1 (Sec. 7): P1 tetrahedra (Kuhn split of an n^3 box, 6 per box) and Q2
    # hexahedra (27 nodes, 3x3x3 Gauss), jitter 0.1h: matrix-free apply (FP64 and FP32) against the
    # CSR SpMV, and CG to 1e-8 both ways (tetrahedra, Laplace).  The FP64 kernels are bound by the
    # FP64 pipe: FP64 operations per element of their formulations (bytes_model.tet_apply_flops,
    # q2_apply_flops) against the measured 1.20 TFLOP/s of FP64 FMA.
    Q2_PA_FLOPS = {ph: bm.q2_apply_flops(ph, partial_assembly=True)["total"] for ph in ("laplace", "elasticity")}
    if not args.no_tet:
        tf_ = {ph: bm.tet_apply_flops(ph)["total"] for ph in ("laplace", "elasticity")}
        qf_ = {ph: bm.q2_apply_flops(ph)["total"] for ph in ("laplace", "elasticity")}
        cases = (("tetrahedra", inputs.tet_box, args.n_tet, tf_, "x 6 tetrahedra"),
                 ("q2_hexahedra", inputs.q2_box, args.n_q2, qf_, "Q2 hexahedra"))
        for key, make, nb, flops, what in cases:
            res = {}
            for phys in ("laplace", "elasticity"):
                pt = make(phys, nb, jitter=0.1, sigma=0.5, layered=True, seed=0)
                mt = mf.Mesh.from_problem(pt, device=f"cuda:{local}")
                xt = torch.from_numpy(pt.x()).cuda()
                yt = torch.empty_like(xt)
                x32, y32 = xt.float(), torch.empty_like(xt, dtype=torch.float32)

                def timed_t(fn, reps):
                    for _ in range(3):
                        fn()
                    torch.cuda.synchronize()
                    e0.record()
                    for _ in range(reps):
                        fn()
                    e1.record()
                    torch.cuda.synchronize()
                    return e0.elapsed_time(e1) / 1e3 / reps

                reps = 20 if key == "tetrahedra" else 5
                ta = timed_t(lambda: mt.apply(xt, yt), reps)
                t32 = timed_t(lambda: mt.apply(x32, y32), reps)
                pa = bool(mt.info["partial_assembly"])
                if pa:  # Q2: AUTO is the sum-factorised partial assembly; time the reference too
                    mt.set_variant(mf.MF_VARIANT_REFERENCE)
                    tref = timed_t(lambda: mt.apply(xt, yt), reps)
                    mt.set_variant(mf.MF_VARIANT_AUTO)
                tf = (Q2_PA_FLOPS[phys] if pa else flops[phys]) * pt.n_cells / ta / 1e12
                r = {"mesh": f"{nb}^3 boxes, {what}, jitter 0.1h", "cells": pt.n_cells, "free_dof": pt.n_free,
                     "colours": mt.info["n_colours"], "ms_apply": 1e3 * ta, "gdofs_apply": pt.n_free / ta / 1e9,
                     "ms_apply_f32": 1e3 * t32, "fp64_tflops": tf, "fp64_frac": tf / 1.20,
                     "fp64_peak_note": "of measured 1.20 TFLOP/s"}
                if pa:
                    r.update({"kernel": "sum-factorised partial assembly", "ms_apply_reference": 1e3 * tref,
                              "reference_fp64_tflops": flops[phys] * pt.n_cells / tref / 1e12})
                if not args.no_csr:
                    At = mt.assemble_csr()
                    ts = timed_t(lambda: At.spmv(xt, yt), reps)
                    r.update({"ms_csr": 1e3 * ts, "gdofs_csr": pt.n_free / ts / 1e9, "nnz": At.info["nnz"],
                              "mf_over_csr": ts / ta})
                    if phys == "laplace" and key == "tetrahedra" and not args.no_cg:
                        bt = torch.from_numpy(pt.b()).cuda()
                        _, im = mt.cg(bt, timeout_s=args.cg_timeout, ok=CG_OK)
                        _, ic = mt.cg(bt, csr=At, timeout_s=args.cg_timeout, ok=CG_OK)
                        r["cg"] = {"iters": im.iters, "seconds_matfree": im.seconds, "seconds_csr": ic.seconds,
                                   "status": [im.status, ic.status]}
                    At.close()
                    del At
                res[phys] = r
                mt.close()
                del xt, yt, x32, y32
                torch.cuda.empty_cache()
            extras[key] = res

    # ---- batched persistent CG: 64 independent Laplace problems, n ~ log-uniform [8, 96]
    if not args.no_batch:
        from paper_2308_09839_gb300 import autotune
        sizes = inputs.batch_sizes(64, 8, 96, seed=0)
        probs = [inputs.laplace_box(int(n), jitter=0.0, sigma=1.0, layered=False, seed=1000 + i)
                 for i, n in enumerate(sizes)]
        bm_meshes = [mf.Mesh.from_problem(q, device=f"cuda:{local}") for q in probs]
        bs = [torch.from_numpy(q.b()).cuda() for q in probs]
        xs = [torch.zeros_like(v) for v in bs]
        choice = autotune.tune(bm_meshes, [q.nz + 1 for q in probs], bs, xs, iters=10)
        o = mf.mf_solve_opts_default()
        batch = mf.mf_batch_create(bm_meshes, o)
        mf.mf_batch_solve(batch, bs, xs)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        infos = mf.mf_batch_solve(batch, bs, xs)
        t_batch = time.perf_counter() - t0
        mf.mf_batch_destroy(batch)
        dof_it = sum(q.n_free * i.iters for q, i in zip(probs, infos))
        for mm, v in zip(bm_meshes, bs):  # warm-up: graphs and workspaces
            mm.cg(v)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        single = [mm.cg(v)[1] for mm, v in zip(bm_meshes, bs)]
        torch.cuda.synchronize()
        t_single = time.perf_counter() - t0
        dof_it1 = sum(q.n_free * i.iters for q, i in zip(probs, single))
        extras["batched_cg"] = {
            "problems": len(probs), "sizes": [int(v) for v in sizes], "total_free_dof": int(sum(q.n_free for q in probs)),
            "seconds_batched": t_batch, "seconds_one_at_a_time": t_single,
            "gdofs_batched": dof_it / t_batch / 1e9, "gdofs_one_at_a_time": dof_it1 / t_single / 1e9,
            "speedup": t_single / t_batch, "all_converged": all(i.status == 0 for i in infos),
            "iters_total": int(sum(i.iters for i in infos)), "segments": {str(k): v for k, v in choice.items()}}
        for mm in bm_meshes:
            mm.close()

    # ---- multi right-hand-side block apply: 16 RHS on a 128^3 Cartesian elasticity mesh
    if not args.no_multi:
        pm = inputs.cartesian_elasticity_160(n=128)
        mm = mf.Mesh.from_problem(pm, device=f"cuda:{local}")
        R = 16
        X = torch.from_numpy(np.stack([pm.x(seed=s).reshape(-1, 3) for s in range(R)], axis=1).reshape(-1)).cuda()
        Y = torch.empty_like(X)
        xs1 = [torch.from_numpy(pm.x(seed=s)).cuda() for s in range(R)]
        ys1 = [torch.empty_like(v) for v in xs1]
        mm.apply_multi(X, R, Y)
        for v, w in zip(xs1, ys1):
            mm.apply(v, w)
        torch.cuda.synchronize()
        reps = 10
        e0.record()
        for _ in range(reps):
            mm.apply_multi(X, R, Y)
        e1.record()
        torch.cuda.synchronize()
        t_blk = e0.elapsed_time(e1) / 1e3 / reps
        e0.record()
        for _ in range(reps):
            for v, w in zip(xs1, ys1):
                mm.apply(v, w)
        e1.record()
        torch.cuda.synchronize()
        t_one = e0.elapsed_time(e1) / 1e3 / reps
        extras["multi_rhs"] = {"mesh": "elasticity 128^3 Cartesian", "nrhs": R, "ms_block": 1e3 * t_blk,
                               "ms_16_single": 1e3 * t_one, "gdofs_block": R * pm.n_free / t_blk / 1e9,
                               "gdofs_single": R * pm.n_free / t_one / 1e9, "speedup": t_one / t_blk}
        mm.close()
        del X, Y, xs1, ys1

    # ---- mixed precision: FP32 inner CG inside FP64 iterative refinement, 192^3 jittered elasticity
    if not args.no_mixed:
        p3 = inputs.jittered_elasticity_192()
        m3 = mf.Mesh.from_problem(p3, device=f"cuda:{local}")
        b3 = torch.from_numpy(p3.b()).cuda()
        xm, im = m3.cg(b3, precision=mf.MF_PREC_MIXED_IR, rtol=1e-10, inner_rtol=1e-4, timeout_s=args.cg_timeout,
                       ok=CG_OK)
        xd, idd = m3.cg(b3, rtol=1e-10, timeout_s=args.cg_timeout, ok=CG_OK)
        err = float(torch.linalg.norm(xm - xd) / torch.linalg.norm(xd)) if idd.status == 0 else None
        extras["mixed_precision"] = {
            "mesh": "elasticity 192^3, node jitter 0.1h", "free_dof": p3.n_free,
            "mixed": {"seconds": im.seconds, "outer": im.outer_iters, "inner_iters": im.iters, "status": im.status,
                      "rel_res_true": im.rel_res_true},
            "plain_fp64": {"seconds": idd.seconds, "iters": idd.iters, "status": idd.status,
                           "rel_res_true": idd.rel_res_true},
            "speedup": idd.seconds / im.seconds if im.status == 0 else None,
            "rel_err_vs_fp64_solution": err}
        m3.close()
        del xm, xd, b3

    # ---- learned preconditioner: 128^3 GRF Laplace, pairs from the FP64 solver, training, flexible CG
    if not args.no_learned:
        from paper_2308_09839_gb300 import learned
        p5 = inputs.grf_laplace_128(seed=0, n=args.n_learned)
        m5 = mf.Mesh.from_problem(p5, device=f"cuda:{local}")
        nzyx = (p5.nz + 1, p5.ny + 1, p5.nx + 1)
        t0 = time.perf_counter()
        Rp, Tp, cs = learned.generate_pairs(m5, p5, args.pairs, seed=1, k_range=(2, 150))
        torch.cuda.synchronize()
        t_pairs = time.perf_counter() - t0
        params, hist, t_train = learned.train(Rp, Tp, learned.node_logk(m5), nzyx, crop=nzyx[0],
                                              steps=args.train_steps, lr=args.lr)
        del Rp, Tp
        net5 = learned.make_inference_net(params, nzyx, cs)
        b5 = torch.from_numpy(p5.b()).cuda()
        _, i_cg = m5.cg(b5, timeout_s=args.cg_timeout, ok=CG_OK)
        _, i_j = m5.cg(b5, precond=mf.MF_PC_JACOBI, timeout_s=args.cg_timeout, ok=CG_OK)
        _, i_nn = m5.cg(b5, net=net5, timeout_s=args.cg_timeout, ok=CG_OK)
        extras["learned_preconditioner"] = {
            "mesh": f"Laplace {p5.nx}^3, GRF log-kappa (8 cells, sigma 1.5) + 8 layers", "pairs": args.pairs,
            "seconds_pairs": t_pairs, "train_steps": args.train_steps, "seconds_train": t_train,
            "loss_first": float(np.mean(hist[:20])), "loss_last": float(np.mean(hist[-50:])),
            "plain_cg": {"iters": i_cg.iters, "seconds": i_cg.seconds, "status": i_cg.status},
            "jacobi_pcg": {"iters": i_j.iters, "seconds": i_j.seconds, "status": i_j.status},
            "learned_fcg": {"iters": i_nn.iters, "seconds": i_nn.seconds, "status": i_nn.status,
                            "rel_res_true": i_nn.rel_res_true, "network_switched_off_at": i_nn.outer_iters}}
        net5.close()
        m5.close()

    # ---- CPU oracle on a bounded sample (rank 0, N = 1)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rate1, secs1, desc1 = oracle_sample_rate([pL, pE], [4, 2])
        workers = os.cpu_count() or 1
        rate_n, secs_n, desc_n = oracle_all_core_rate([pL, pE], [1, 1], workers)
        cpu = {"value": rate_n / 1e9, "unit": UNIT, "cores": workers, "kind": "oracle", "nproc": workers,
               "cpu_model": cpu_model(),
               "sample": f"all cores: {desc_n} ({secs_n:.1f} s wall, one slab per process)",
               "one_core": {"value": rate1 / 1e9, "unit": UNIT, "cores": 1,
                            "sample": desc1 + f" (bottom slabs of both workloads, {secs1:.1f} s of CPU time)"}}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_total / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32x2" if args.variant == 0 else "f64",
        "dtype_note": ("double-word FP32 arithmetic (pairs of floats), FP64 inputs and outputs, parity <= 1e-12 "
                       "relative 2-norm against the FP64 oracle" if args.variant == 0 else "FP64 arithmetic"),
        "data": "synthetic",
        "config": {"workload": workload_name(pL, pE),
                   "n_dof_total": [pL.n_dof, pE.n_dof], "parallelism": f"replicas{world}",
                   "l2": f"no flush: the FP64 x and y of one apply alone exceed the 129 MB L2 "
                         f"({16 * pL.n_dof / 1e9:.2f} GB Laplace, {16 * pE.n_dof / 1e9:.2f} GB elasticity)", "variant": args.variant,
                   "tile_segments": segs or None},
        "clocks": clk, "e2e": e2e, "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu,
        "extras": extras,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
