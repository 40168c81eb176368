#!/usr/bin/env python3
"""Benchmark of the matrix-free voxel finite-element elasticity PCG (ELAS3D-Xtal, Algorithm 2).

Workload (one step = one pass of the whole hot path): a 100^3 periodic polycrystal with 500
Voronoi grains (seeds uniform, seed 1), cubic grains C11/C12/C44 = 204.6/137.7/126.2 GPa with
uniform random orientations, 1% spherical pores (r ~ U[2,6]), applied eps_zz = 1e-3.  Each step
builds the point-block Jacobi preconditioner, the right-hand side, runs the PCG until the FP64
true relative residual is <= 1e-8, and computes the voxel stress, von Mises and macro stress.

Metric: PCG voxel-iterations per second (N voxels x iterations / time) of the plain FP64 solve,
plus the mixed-precision solve of the same problem, HBM GB/s of the iteration's algorithmic
traffic, the roofline of the dominant kernel, an end-to-end leg through host buffers and the
CPU oracle as a reported baseline.  Prints one JSON line (rank 0).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PCG voxel-iter/s + HBM GB/s at rel-res 1e-8 vs FP64 plain; served solves/s, p50/p99"
UNIT = "voxel-iter/s"
E6 = np.array([0.0, 0.0, 1e-3, 0.0, 0.0, 0.0])
TOL = 1e-8
# Algorithmic HBM bytes per voxel per PCG iteration (each vector read/written once per kernel):
#   FP64: apply 52 (h, ids, Ah) + update 216 (w,h,g,Ah,Minv in; w,g,z out) + direction 72 = 340
#   mixed: apply 28 + update 132 (w as a float pair, FP32 vectors and Minv) + direction 36 = 196
BYTES_PER_VOXEL_ITER = {"fp64": 340, "mixed": 196}
# Algorithmic flops per voxel of the modal element product + node gather: 30 MUL + 108 FMA in the
# 6x6/5x5/3x3 mode products, 186 adds (transform 72 + 72, strain/force assembly 21, gather 21)
APPLY_FLOPS_PER_VOXEL = 432
# The FP64 product in double-float arithmetic (ELAS_FP64_OP_PAIRED, the default) performs these
# FP32 operations per voxel (each FADD, FMUL and FFMA counted once): 126 pair sums x 8 (TwoSum 6 + 2),
# 138 terms of the 30 symmetric-product rows (first term of a row 4: product, its rounding error and
# two cross terms; every other term 12: those 4, TwoSum 6, 2 error sums), 30 row renormalisations x 3,
# and the h.Ah terms of the node (3 x 12)
PAIRED_OPS_PER_VOXEL = 126 * 8 + 30 * 4 + 108 * 12 + 30 * 3 + 3 * 12
APPLY_BYTES_PER_VOXEL = {"fp64": 52, "mixed": 28}
# FP64 pipe: 2 DFMA per clock per SM on GB300 (1.25 TFLOP/s nominal at 2070 MHz, 152 SMs)
FP64_FMA_PER_CLK_PER_SM = 2
FP32_FMA_PER_CLK_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--size", type=int, default=100)
    ap.add_argument("--grains", type=int, default=500)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the mixed and e2e legs")
    ap.add_argument("--serve-requests", type=int, default=2000, help="requests of the serving leg (the full stream)")
    ap.add_argument("--serve-low-rate", type=float, default=10.0,
                    help="arrival rate (req/s) of the second served stream, below the server's capacity")
    ap.add_argument("--serve-low-requests", type=int, default=500,
                    help="requests of the second served stream (0: skip it)")
    ap.add_argument("--batch-rves", type=int, default=64)
    ap.add_argument("--legs", default="fp64,mixed,e2e,r200,variants,batch,serve,large",
                    help="comma list of legs to run (the headline fp64 leg is always reported when present)")
    ap.add_argument("--profile-apply", choices=["f64", "f64native", "f32"], default=None,
                    help="only launch the operator product --reps times (for ncu captures); prints its timing")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--launcher-selftest", action="store_true",
                    help="check the replica launcher's rank bookkeeping and reductions (CPU, gloo) and exit")
    ap.add_argument("--kt-sweep", type=int, default=0, metavar="N",
                    help="the anisotropy sweep of Sec. 3.2 on an N^3 cell (generated on the GPU): K_t of the "
                         "central void for each Zener ratio; prints one JSON line per case")
    ap.add_argument("--large", action="store_true",
                    help="the large single solves: 500^3 (20,000 grains, 2%% mixed pores) FP64 and mixed, "
                         "800^3 mixed; prints one JSON line per solve")
    ap.add_argument("--mesh-study", default="", metavar="EDGES",
                    help="the Eshelby-void study of Sec. 3.1 / App. A at the given comma-separated grid edges "
                         "(e.g. 100,200,300,400,500): FP64 and mixed solve times and the App. C peak; one JSON "
                         "line per edge")
    return ap.parse_args()


def workload_name(a):
    return f"polycrystal {a.size}^3, {a.grains} grains, 1% pores, eps_zz=1e-3, true relres 1e-8"


def microstructure(a):
    from paper_2602_07354_gb300 import synth

    return synth.polycrystal(a.size, a.grains, pore_frac=0.01, seed=1)


# ---------------------------------------------------------------------------------------------
class Clocks:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.seek(0)
        rows = [r.split(", ") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.strip() == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def profile_traffic(name: str, a=None):
    """DRAM bytes per launch from the committed ncu summary (captured on the 100^3, 500-grain
    workload), if the kernel source is unchanged and the run is that workload."""
    if a is not None and (a.size != 100 or a.grains != 500):
        return None
    path = os.path.join(ROOT, "profiles", name)
    src = os.path.join(ROOT, "paper_2602_07354_gb300", "csrc", "apply.cu")
    try:
        txt = open(path).read()
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        m = re.search(r"traffic_bytes_per_launch_scaled:\s*([0-9.eE+]+)", txt)
        h = re.search(r"apply_cu_sha256_16:\s*([0-9a-f]+)", txt)
        if m and h and h.group(1) == sha:
            return float(m.group(1))
    except Exception:
        pass
    return None


# ---------------------------------------------------------------------------------------------
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def free_port() -> int:
    import socket

    sk = socket.socket()
    sk.bind(("127.0.0.1", 0))
    port = sk.getsockname()[1]
    sk.close()
    return port


def launch_ranks(n: int, argv, backend: str) -> int:
    """Start n ranks of this script on this node, rank r on GPU r (LOCAL_RANK = r), with a
    127.0.0.1 rendezvous, as torch.distributed.run would; rank 0's output is this process's
    output, the other ranks print nothing.  Returns the first non-zero exit code."""
    port = free_port()
    procs = []
    for r in range(n):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(n), LOCAL_WORLD_SIZE=str(n),
                   MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), ELAS_BENCH_BACKEND=backend)
        procs.append(subprocess.Popen([sys.executable, os.path.abspath(__file__), *argv], env=env,
                                      stdout=None if r == 0 else subprocess.DEVNULL))
    rc = 0
    for pr in procs:
        c = pr.wait()
        rc = rc or c
    return rc


def init_ranks(world: int):
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group(os.environ.get("ELAS_BENCH_BACKEND", "nccl"), init_method="env://")


def launcher_selftest(a, world, rank, local):
    """Rank bookkeeping of the replica launcher without a GPU: every rank reports its rank, local rank
    and the device it would drive, a fixed per-rank time and amount of work; rank 0 prints the
    reduction the benchmark applies (max of the times, sum of the work)."""
    import torch.distributed as dist

    init_ranks(world)
    me = {"rank": rank, "local_rank": local, "device": f"cuda:{local}", "world": world}
    ranks = [None] * world
    if world > 1:
        dist.all_gather_object(ranks, me)
    else:
        ranks = [me]
    t_max = allreduce(10.0 + rank, "max", world)
    work = allreduce(100.0 * (rank + 1), "sum", world)
    barrier(world)
    if rank == 0:
        print(json.dumps({"n_gpus": world, "ranks": ranks, "t_max_ms": t_max, "work": work}), flush=True)
    if world > 1:
        dist.destroy_process_group()


def allreduce(x: float, op: str, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def time_kernel(fn, torch, flush, reps=20):
    """Average device duration of one launch, CUDA events on the launching stream, L2 flushed."""
    st = torch.cuda.current_stream()
    tot = 0.0
    for _ in range(reps):
        flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn()
        e1.record(st)
        e1.synchronize()
        tot += e0.elapsed_time(e1)
    return tot / reps * 1e-3


def run_solver_leg(B, torch, ms, prec, a, flush, world, clocks=None, opts=None):
    ctx = B.create_from_micro(ms, precision=prec)
    opts = opts or {}
    N = ms.N
    w = torch.empty(3 * N, dtype=torch.float64, device="cuda")
    stress = torch.empty(6 * N, dtype=torch.float64, device="cuda")
    vm = torch.empty(N, dtype=torch.float64, device="cuda")

    def step():
        info = B.elas_pcg_solve(ctx, E6, TOL, 50000, w_out=w, stop_rule=B.STOP_TRUE, **opts)
        B.elas_stress(ctx, E6, None, stress, vm, want_macro=False)
        return info

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    st = torch.cuda.current_stream()
    t_ms, iters, launches, infos = 0.0, 0, 0, []
    for _ in range(a.steps):
        flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        info = step()
        e1.record(st)
        e1.synchronize()
        t_ms += e0.elapsed_time(e1)
        iters += info["iters"]
        launches += info["launches"] + 1  # + the stress kernel
        infos.append(info)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop() if clocks else None
    macro = B.elas_stress(ctx, E6, None, None, None)
    return dict(ctx=ctx, t_ms=t_ms, iters=iters, launches=launches, infos=infos, clocks=clk, macro=macro, w=w, vm=vm)


def solution_errors(torch, ms, w, vm, w_ref, vm_ref):
    """Relative errors of (w, vm) against a reference solution of the same problem: displacement
    (mean over the nodes of solid voxels removed), total voxel strain, and the peak von Mises
    stress over pore-edge voxels (solid voxels with a pore among their 26 neighbours)."""
    nz, ny, nx = ms.nz, ms.ny, ms.nx
    solid = torch.from_numpy(ms.phase >= 0).to("cuda").reshape(nz, ny, nx)
    node = torch.zeros_like(solid)
    for az in (0, 1):
        for ay in (0, 1):
            for ax in (0, 1):
                node |= torch.roll(solid, shifts=(az, ay, ax), dims=(0, 1, 2))
    node = node.reshape(-1)

    def disp(x):
        x = x.reshape(3, -1)[:, node]
        return x - x.mean(dim=1, keepdim=True)

    def strain(x):
        W = x.reshape(3, nz, ny, nx)
        G = torch.zeros(3, 3, nz, ny, nx, dtype=W.dtype, device=W.device)
        for a in range(8):
            ax, ay, az = a & 1, (a >> 1) & 1, (a >> 2) & 1
            Wa = torch.roll(W, shifts=(-az, -ay, -ax), dims=(1, 2, 3))
            for d, sd in enumerate((2 * ax - 1, 2 * ay - 1, 2 * az - 1)):
                G[:, d] += 0.25 * sd * Wa
        E = torch.tensor([[E6[0], E6[5], E6[4]], [E6[5], E6[1], E6[3]], [E6[4], E6[3], E6[2]]],
                         dtype=W.dtype, device=W.device)
        eps = 0.5 * (G + G.transpose(0, 1)) + E[:, :, None, None, None]
        return eps.reshape(9, -1)[:, solid.reshape(-1)]

    def rel(x, y):
        return float(torch.linalg.vector_norm(x - y) / torch.linalg.vector_norm(y))

    pore = ~solid
    edge = torch.zeros_like(solid)
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if dz or dy or dx:
                    edge |= torch.roll(pore, shifts=(dz, dy, dx), dims=(0, 1, 2))
    edge = (edge & solid).reshape(-1)
    peak_ref = float(vm_ref[edge].max())
    return {"displacement": rel(disp(w), disp(w_ref)), "strain": rel(strain(w), strain(w_ref)),
            "peak_pore_edge_von_mises": abs(float(vm[edge].max()) - peak_ref) / peak_ref,
            "pore_edge_voxels": int(edge.sum())}


def run_e2e(B, torch, ms, a, flush):
    """Public API from host buffers: per step the phase ids and stiffness go host->device
    (pinned), the solve and stress run, the fluctuation w comes back device->host."""
    N = ms.N
    phase_pinned = torch.from_numpy(ms.phase.astype(np.int32)).pin_memory()
    w_host = torch.empty(3 * N, dtype=torch.float64).pin_memory()
    C = B.materials_to_C(ms.materials)
    w = torch.empty(3 * N, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()

    def step():
        ctx = B.elas_create(ms.nx, ms.ny, ms.nz, phase_pinned.numpy(), C, ms.rho, B.PREC_FP64)
        info = B.elas_pcg_solve(ctx, E6, TOL, 50000, w_out=w, stop_rule=B.STOP_TRUE)
        macro = B.elas_stress(ctx, E6, None, None, None)
        w_host.copy_(w, non_blocking=True)
        st.synchronize()
        ctx.close()
        return info, macro

    for _ in range(max(1, a.warmup)):
        step()
    t, iters = 0.0, 0
    for _ in range(a.steps):
        flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        info, _ = step()
        e1.record(st)
        e1.synchronize()
        t += e0.elapsed_time(e1)
        iters += info["iters"]
    h2d = 4 * N + ms.n_phases * 36 * 8 + (0 if ms.rho is None else ms.n_phases * 3 * 8) + 6 * 8
    d2h = 3 * N * 8 + 6 * 8
    return dict(value=N * iters / (t * 1e-3), unit=UNIT, h2d_bytes_per_step=h2d, d2h_bytes_per_step=d2h,
                ms_per_step=t / a.steps)


def run_repeat_200(B, torch, flush):
    """The 100^3 workload repeated at 200^3 with 4,000 grains (seed 2): one timed FP64 solve and
    one timed mixed solve (replacement every 50) after a short warm-up solve of each."""
    from paper_2602_07354_gb300 import synth

    ms = synth.polycrystal(200, 4000, pore_frac=0.01, seed=2)
    out = {"workload": "polycrystal 200^3, 4000 grains, 1% pores, eps_zz=1e-3, true relres 1e-8",
           "pore_fraction": float(ms.meta.get("pore_frac", 0.0))}
    st = torch.cuda.current_stream()
    for name, prec in (("fp64", B.PREC_FP64), ("mixed", B.PREC_MIXED)):
        ctx = B.create_from_micro(ms, precision=prec)
        w = torch.empty(3 * ms.N, dtype=torch.float64, device="cuda")
        B.elas_pcg_solve(ctx, E6, TOL, 60, w_out=w, stop_rule=B.STOP_TRUE)  # warm-up, records the graph
        flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        info = B.elas_pcg_solve(ctx, E6, TOL, 100000, w_out=w, stop_rule=B.STOP_TRUE)
        e1.record(st)
        e1.synchronize()
        t = e0.elapsed_time(e1) * 1e-3
        ctx.close()
        out[name] = {"seconds": t, "iters": info["iters"], "relres_true": info["relres_true"],
                     "replacements": info["n_replacements"], "voxel_iter_per_s": ms.N * info["iters"] / t}
    out["mixed_speedup_vs_fp64"] = out["fp64"]["seconds"] / out["mixed"]["seconds"]
    return out


def run_variants(B, torch, ms, flush):
    """Table 4's comparison on this GPU: plain CG, point-Jacobi PCG and the paper's point-block
    Jacobi PCG, FP64, to true relres 1e-8 (the faster of two timed solves each, after a short
    warm-up solve, so that one disturbed solve does not decide the ratio), on
    Table 4's own workload (Sec. 3.1's spherical void, radius 2/50 of the box, isotropic matrix,
    eps_33 = 1e-3, 100^3) and on the 100^3 polycrystal."""
    from paper_2602_07354_gb300 import synth

    st = torch.cuda.current_stream()
    out = {}
    for key, m in (("eshelby_void_100", synth.eshelby_void(100)), ("polycrystal_100", ms)):
        ctx = B.create_from_micro(m, precision=B.PREC_FP64)
        w = torch.empty(3 * m.N, dtype=torch.float64, device="cuda")
        res = {}
        for name, pc in (("cg", B.PRECOND_NONE), ("point_jacobi", B.PRECOND_SCALAR),
                         ("block_jacobi", B.PRECOND_BLOCK)):
            B.elas_pcg_solve(ctx, E6, TOL, 60, w_out=w, stop_rule=B.STOP_TRUE, precond=pc)
            best = None
            for _ in range(2):
                flush()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                info = B.elas_pcg_solve(ctx, E6, TOL, 200000, w_out=w, stop_rule=B.STOP_TRUE, precond=pc)
                e1.record(st)
                e1.synchronize()
                t = e0.elapsed_time(e1) * 1e-3
                best = t if best is None else min(best, t)
            res[name] = {"seconds": best, "iters": info["iters"], "relres_true": info["relres_true"]}
        ctx.close()
        res["cg_over_block_time"] = res["cg"]["seconds"] / res["block_jacobi"]["seconds"]
        res["cg_over_block_iters"] = res["cg"]["iters"] / res["block_jacobi"]["iters"]
        out[key] = res
    out["stop"] = "FP64 true relative residual <= 1e-8, eps_33 = 1e-3"
    return out


def run_batch_leg(B, torch, a, flush):
    """64 uneven RVEs x 6 unit load cases in one batch (FP32 operator, FP64 residual replacement,
    autotuned per grid size), solved to true relres 1e-8."""
    from paper_2602_07354_gb300 import synth

    rves = synth.batch_rves(a.batch_rves)
    loads = synth.UNIT_LOAD_CASES
    b = B.elas_batch_create(rves, 6, B.PREC_MIXED)
    B.elas_batch_autotune(b, 6)
    strains = np.stack([loads for _ in rves])
    policy = {"replace_every": 1000, "replace_drop": 3}
    B.elas_batch_solve(b, strains, TOL, 50000, **policy)  # warm-up (records the graph)
    torch.cuda.synchronize()
    flush()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    infos = B.elas_batch_solve(b, strains, TOL, 50000, **policy)
    e1.record(st)
    e1.synchronize()
    t = e0.elapsed_time(e1) * 1e-3
    vi = sum(rv.N * infos[i * 6 + r]["iters"] for i, rv in enumerate(rves) for r in range(6))
    ok = sum(i["status"] == B.CONVERGED and i["relres_true"] <= TOL * 1.0001 for i in infos)
    b.close()
    return {"workload": f"{len(rves)} RVEs, edge in {{32,48,64,80,96}}, 1 grain/2000 voxels, 0-3% pores, "
                        "6 unit load cases each, mixed precision to true relres 1e-8, FP64 residual replacement "
                        "after each 3 decades of residual reduction",
            "voxels": int(sum(rv.N for rv in rves)), "problems": len(infos), "seconds": t,
            "voxel_iter_per_s": vi / t, "solves_per_s": len(infos) / t, "converged": int(ok),
            "max_iters": int(max(i["iters"] for i in infos))}


def generate_request_micro(B, torch, req, stream):
    """One request's own seeded polycrystal, generated on the device (on `stream`): Voronoi grains
    (Algorithm 4), spherical pores stamped in batches until the pore fraction is reached
    (Algorithm 5), random orientations (Algorithm 6); SS316L-like cubic constants.  The ids and
    orientations come back to the host, where the server's submit call takes them."""
    from paper_2602_07354_gb300 import synth

    n, ng = req["edge"], req["n_grains"]
    seeds, u, pore_batch = synth.polycrystal_draws(n, ng, req["pore_frac"], req["seed"])
    with torch.cuda.stream(stream):
        phase = B.elas_assign_grains((n, n, n), seeds, None, stream=stream)
        target, carved = req["pore_frac"] * n ** 3, 0
        while carved < target:
            carved = B.elas_stamp_pores((n, n, n), pore_batch(target - carved), phase, stream=stream)
        rho = B.elas_orientations(B.TEXTURE_RANDOM, torch.from_numpy(u).to("cuda"), stream=stream)
        ids, rho_h = phase.cpu().numpy(), rho.cpu().numpy()
    mats = np.broadcast_to(synth.cubic_mat(*synth.SS316L), (ng, 4)).copy()
    return synth.Microstructure(n, n, n, ids, mats, rho_h, dict(kind="polycrystal", seed=req["seed"]))


def run_serve_leg(B, torch, a, rate=20.0, n_requests=None, sequential=True):
    """Poisson stream at `rate` req/s through the solve server (150 GB budget): every request's own
    polycrystal is generated on the GPU once the request has arrived (a generator thread on its own
    stream), then submitted; p50/p99 latency from arrival to result (generation included), against
    sequential plain FP64 solves of a sample of the same requests on this GPU (`sequential`)."""
    import queue
    import threading

    from paper_2602_07354_gb300 import synth

    reqs = synth.request_stream(n_requests or a.serve_requests, rate=rate)
    n = len(reqs)
    budget = 150 * (1 << 30)
    # the server's solves on a high-priority stream, the generator's kernels on a normal one: the
    # block scheduler serves the solves first when both have work
    srv_stream = torch.cuda.Stream(priority=-10)  # (mapped to the device's highest priority)
    srv = B.elas_server_create(budget, 64, B.PREC_MIXED, stream=srv_stream)
    B.elas_server_set_replacement(srv, 1000, 3)
    torch.cuda.synchronize()
    ready = queue.Queue()
    gen_s = []
    t0 = time.perf_counter()
    errors = []

    def generator():
        stream = torch.cuda.Stream()
        try:
            for j, r in enumerate(reqs):
                wait = r["arrival"] - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(wait)
                tg = time.perf_counter()
                ms = generate_request_micro(B, torch, r, stream)
                gen_s.append(time.perf_counter() - tg)
                ready.put((j, ms))
        except Exception as ex:  # reported by the main loop
            errors.append(repr(ex))
            ready.put(None)

    th = threading.Thread(target=generator, daemon=True)
    th.start()
    lat, ids, done, submitted = {}, {}, 0, 0
    busy = 0.0
    while done < n and not errors:
        while True:
            try:
                item = ready.get_nowait()
            except queue.Empty:
                break
            if item is None:
                break
            j, ms = item
            r = reqs[j]
            ids[B.elas_server_submit(srv, ms, r["strain"], r["tol"], 50000)] = j
            submitted += 1
        st = B.elas_server_stats(srv)
        if st["active"] == 0 and st["queued"] == 0:
            time.sleep(0.002)
            continue
        tb = time.perf_counter()
        B.elas_server_step(srv)
        busy += time.perf_counter() - tb
        tnow = time.perf_counter() - t0
        for rid in [i for i in ids if ids[i] not in lat]:
            res = B.elas_server_poll(srv, rid)
            if res is not None:
                lat[ids[rid]] = (tnow - reqs[ids[rid]]["arrival"], res)
                done += 1
    wall = time.perf_counter() - t0
    th.join(timeout=60)
    srv.close()
    if errors:
        raise RuntimeError("request generation failed: " + errors[0])
    L = np.array([v[0] for v in lat.values()])
    conv = sum(v[1]["status"] == B.CONVERGED for v in lat.values())
    vox_iters = sum(reqs[j]["edge"] ** 3 * v[1]["iters"] for j, v in lat.items())
    out = {"workload": f"{n} requests, Poisson {rate:g} req/s, edge in {{48,64,96,128,160}}, each its own seeded "
                       "SS316L-like polycrystal (1 grain / 2000 voxels, 0-3% pores) generated on the GPU after "
                       "arrival, random strain |E|=1e-3, tol 1e-6/1e-8, 150 GB budget, mixed precision, FP64 "
                       "residual replacement after each 3 decades of residual reduction",
           "p50_s": float(np.percentile(L, 50)), "p99_s": float(np.percentile(L, 99)), "solves_per_s": n / wall,
           "wall_s": wall, "converged": int(conv), "requests": n,
           "capacity_solves_per_s": n / busy if busy > 0 else None,
           "server_voxel_iter_per_s": vox_iters / busy if busy > 0 else None,
           "sustained_arrival_rate_req_per_s": min(rate, n / busy) if busy > 0 else None,
           "generation_s_mean": float(np.mean(gen_s)), "generation_s_max": float(np.max(gen_s))}
    if not sequential:
        return out
    # sequential plain FP64 PCG of the first request of each grid edge (same microstructure, strain, tol)
    seq_t, seen = [], set()
    gstream = torch.cuda.Stream()
    for r in reqs:
        if r["edge"] in seen:
            continue
        seen.add(r["edge"])
        m = generate_request_micro(B, torch, r, gstream)
        ctx = B.create_from_micro(m, precision=B.PREC_FP64)
        B.elas_pcg_solve(ctx, r["strain"], r["tol"], 50, stop_rule=B.STOP_TRUE)  # warm-up (graph)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        B.elas_pcg_solve(ctx, r["strain"], r["tol"], 50000, stop_rule=B.STOP_TRUE)
        seq_t.append(time.perf_counter() - t1)
        ctx.close()
    mean_fp64 = float(np.mean(seq_t))
    out["sequential_fp64_solves_per_s"] = 1.0 / mean_fp64
    out["sequential_fp64_sample"] = f"first request of each grid edge (5 solves), mean {mean_fp64:.3f} s per solve"
    return out


def host_cpu():
    """The host the oracle runs on: model name and logical core count (the oracle uses one)."""
    model, arm = None, {}
    try:
        for line in open("/proc/cpuinfo"):
            key, _, val = line.partition(":")
            key = key.strip().lower()
            if key in ("model name", "cpu model") and model is None:
                model = val.strip()
            elif key in ("cpu implementer", "cpu part") and key not in arm:
                arm[key] = val.strip()
    except OSError:
        pass
    if model is None and arm:  # Arm hosts name the core by implementer and part codes
        model = f"Arm implementer {arm.get('cpu implementer', '?')}, part {arm.get('cpu part', '?')}"
    return {"model": model or platform.machine(), "logical_cores": os.cpu_count(), "machine": platform.machine()}


def cpu_oracle_rate(ms, budget_s: float, e6=E6):
    """The FP64 oracle as it stands: Algorithm 2 for a bounded number of iterations, one core."""
    from oracle import oracle as O

    p = O.Problem.from_micro(ms)
    t0 = time.perf_counter()
    p.pcg(e6, 0.0, 1)  # rhs + Jacobi + 1 iteration: sizes the sample
    t1 = time.perf_counter() - t0
    iters = max(2, int(budget_s / max(t1, 1e-3)))
    t0 = time.perf_counter()
    r = p.pcg(e6, 0.0, iters)
    dt = time.perf_counter() - t0
    return dict(value=ms.N * r["iters"] / dt, unit=UNIT, cores=1, kind="oracle",
                sample=f"{ms.nx}^3 workload: rhs + Jacobi build + {r['iters']} PCG iterations of Algorithm 2, "
                       f"FP64 C oracle (gcc -O2), single thread, {dt:.1f} s", host=host_cpu())


def eshelby_20(B, torch):
    """The 20^3 Eshelby-inclusion cell (eps_11 = 1e-3, Algorithm 2's stopping rule at 1e-10):
    the full oracle solve on one core next to the FP64 GPU solve of the same problem."""
    from oracle import oracle as O
    from paper_2602_07354_gb300 import synth

    ms = synth.eshelby_inclusion()
    e = np.array([1e-3, 0, 0, 0, 0, 0.0])
    p = O.Problem.from_micro(ms)
    t0 = time.perf_counter()
    ref = p.pcg(e, 1e-10, 5000)
    t_cpu = time.perf_counter() - t0
    ctx = B.create_from_micro(ms, precision=B.PREC_FP64)
    w = torch.empty(3 * ms.N, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    B.elas_pcg_solve(ctx, e, 1e-10, 5000, w_out=w, stop_rule=B.STOP_PRECOND)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    info = B.elas_pcg_solve(ctx, e, 1e-10, 5000, w_out=w, stop_rule=B.STOP_PRECOND)
    e1.record(st)
    e1.synchronize()
    ctx.close()
    return {"workload": "Eshelby inclusion 20^3, eps_11=1e-3, sqrt(z.g/z0.g0) < 1e-10",
            "oracle_seconds": t_cpu, "oracle_iters": ref["iters"], "oracle_cores": 1,
            "gpu_fp64_seconds": e0.elapsed_time(e1) * 1e-3, "gpu_fp64_iters": info["iters"]}


# ---------------------------------------------------------------------------------------------
def run_reference(a, world, rank):
    if rank != 0:
        return
    ms = microstructure(a)
    from oracle import oracle as O

    p = O.Problem.from_micro(ms)
    t0 = time.perf_counter()
    p.pcg(E6, 0.0, 1)
    t1 = time.perf_counter() - t0
    per_step_iters = max(1, int(min(20.0, 120.0 / max(1, a.steps + a.warmup)) / max(t1, 1e-3)))
    for _ in range(a.warmup):
        p.pcg(E6, 0.0, per_step_iters)
    t, iters = 0.0, 0
    for _ in range(a.steps):
        t0 = time.perf_counter()
        r = p.pcg(E6, 0.0, per_step_iters)
        t += time.perf_counter() - t0
        iters += r["iters"]
    value = ms.N * iters / t
    sample = (f"{a.size}^3 workload, each step rhs + Jacobi build + {per_step_iters} PCG iterations of the FP64 "
              f"oracle (Algorithm 2), single thread")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": t / a.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(a), "grid": [a.size] * 3, "grains": a.grains},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                         "host": host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_ours(a, world, rank, local):
    import torch

    from paper_2602_07354_gb300 import binding as B
    from paper_2602_07354_gb300 import build

    init_ranks(world)
    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        build.build()
    barrier(world)
    B.lib()
    ms = microstructure(a)
    N = ms.N
    flush_w = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    flush_r = torch.ones(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def flush():
        # write 256 MiB (evicts L2), then read another 256 MiB so the dirty lines are written
        # back here rather than inside the next timed launch
        flush_w.fill_(1.0)
        flush_r.sum()

    peaks = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    hbm_src = "measured" if "hbm_gbs" in peaks else "fallback"
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count

    legs = set(a.legs.split(","))
    if a.no_extras:
        legs &= {"fp64"}
    if world > 1:  # replicas of the headline workload only: the other legs are single-GPU studies
        legs &= {"fp64", "mixed", "e2e"}
    if legs == {"batch"}:  # the batched leg alone, for profiling
        print(json.dumps({"leg": "batch", "batched": run_batch_leg(B, torch, a, flush)}), flush=True)
        return
    if legs == {"serve"}:  # the served streams alone
        served = run_serve_leg(B, torch, a)
        if a.serve_low_requests > 0:
            served["below_capacity"] = run_serve_leg(B, torch, a, rate=a.serve_low_rate,
                                                     n_requests=a.serve_low_requests, sequential=False)
        print(json.dumps({"leg": "serve", "served": served}), flush=True)
        return
    if "fp64" not in legs:  # a single non-headline leg, for profiling
        prec = B.PREC_MIXED if "mixed" in legs else B.PREC_FP64
        lg = run_solver_leg(B, torch, ms, prec, a, flush, world)
        print(json.dumps({"leg": sorted(legs), "ms_per_solve": lg["t_ms"] / a.steps,
                          "iters": lg["infos"][-1]["iters"]}), flush=True)
        lg["ctx"].close()
        return
    # ---- headline: plain FP64 PCG -------------------------------------------------------------
    clocks = Clocks(local)
    leg = run_solver_leg(B, torch, ms, B.PREC_FP64, a, flush, world, clocks)
    t_max = allreduce(leg["t_ms"], "max", world)
    vi_total = allreduce(float(N * leg["iters"]), "sum", world)
    value = vi_total / (t_max * 1e-3)
    clk = leg["clocks"] or {}
    sm_mhz_peak = clk.get("sm_max_mhz") or 2070.0

    # dominant kernel: the FP64 operator product in double-float arithmetic (the kernel variant of
    # the solve), timed with events in a loop on the launching stream, L2 flushed between launches
    u = torch.randn(3 * N, dtype=torch.float64, device="cuda") * 1e-3
    y = torch.empty_like(u)
    for _ in range(3):
        B.elas_apply(leg["ctx"], u, y)
    t_apply = time_kernel(lambda: B.elas_apply(leg["ctx"], u, y), torch, flush)
    fp32_ops_peak = sm_count * FP32_FMA_PER_CLK_PER_SM * sm_mhz_peak * 1e6 / 1e12
    ach = N * PAIRED_OPS_PER_VOXEL / t_apply / 1e12
    fp64_peak = sm_count * FP64_FMA_PER_CLK_PER_SM * 2 * sm_mhz_peak * 1e6 / 1e12
    # the same product in native FP64 instructions, for comparison
    ctx_n = B.create_from_micro(ms, precision=B.PREC_FP64)
    B.elas_set_fp64_operator(ctx_n, B.FP64_OP_NATIVE)
    for _ in range(3):
        B.elas_apply(ctx_n, u, y)
    t_native = time_kernel(lambda: B.elas_apply(ctx_n, u, y), torch, flush)
    ctx_n.close()
    roof = {"bound": "alu", "achieved": ach, "peak": fp32_ops_peak, "unit": "Top/s", "frac": ach / fp32_ops_peak,
            "traffic": profile_traffic("apply_paired_100cube.md", a),
            "kernel": "k_apply<double, ff> (FP64 modal product in double-float arithmetic)",
            "ms_per_launch": t_apply * 1e3, "ops_per_voxel": PAIRED_OPS_PER_VOXEL,
            "peak_source": f"derived: {sm_count} SMs x 128 FP32 lanes x {sm_mhz_peak:.0f} MHz (one FP32 operation "
                           "per lane per clock, FMA counted once; an FADD/FFMA issue probe reaches 120-124 of the 128 lanes "
                           "per SM per clock)",
            "fp64_equivalent_tflops": N * APPLY_FLOPS_PER_VOXEL / t_apply / 1e12, "fp64_pipe_peak_tflops": fp64_peak,
            "native_fp64": {"ms_per_launch": t_native * 1e3,
                            "achieved_tflops": N * APPLY_FLOPS_PER_VOXEL / t_native / 1e12,
                            "frac_of_fp64_pipe": N * APPLY_FLOPS_PER_VOXEL / t_native / 1e12 / fp64_peak},
            "hbm_frac": N * APPLY_BYTES_PER_VOXEL["fp64"] / t_apply / 1e9 / hbm_peak}
    infos = leg["infos"]
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": t_max / a.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(a), "grid": [a.size] * 3, "grains": a.grains,
                   "pore_fraction": float(ms.meta.get("pore_frac", 0.0)), "load": "eps_zz=1e-3",
                   "stop": "FP64 true relative residual <= 1e-8",
                   "precision": "fp64: IEEE FP64 vectors, reductions and Jacobi blocks; operator products in "
                                "double-float arithmetic on the FP32 pipe (<= 1e-12 of the FP64 oracle per product)",
                   "l2": "256 MiB written + 256 MiB read between timed steps (outside the events); per-step working set "
                         f"{(N * (4 + 48 + 5 * 24)) / 1e9:.2f} GB > 129 MB L2",
                   "parallelism": "replicas (one independent solve per GPU)"},
        "iters_per_solve": infos[-1]["iters"], "relres_true": infos[-1]["relres_true"],
        "solves_per_s": world * a.steps / (t_max * 1e-3),
        "hbm": {"gbs": value / world * BYTES_PER_VOXEL_ITER["fp64"] / 1e9,
                "bytes_per_voxel_iter": BYTES_PER_VOXEL_ITER["fp64"], "peak_gbs": hbm_peak,
                "peak_source": hbm_src},
        "roofline": roof,
        "gpu_launches": leg["launches"],
        "clocks": clk or None,
    }

    # ---- mixed precision (FP32 operator + FP64 residual replacement) on the same problem -----
    if "mixed" in legs:
        mx = run_solver_leg(B, torch, ms, B.PREC_MIXED, a, flush, world)
        tm = allreduce(mx["t_ms"], "max", world)
        vm_val = allreduce(float(N * mx["iters"]), "sum", world) / (tm * 1e-3)
        u32 = torch.randn(3 * N, dtype=torch.float32, device="cuda")
        y32 = torch.empty_like(u32)
        t32 = time_kernel(lambda: B.elas_apply_f32(mx["ctx"], u32, y32), torch, flush)
        fp32_peak = sm_count * FP32_FMA_PER_CLK_PER_SM * 2 * sm_mhz_peak * 1e6 / 1e12
        ach32 = N * APPLY_FLOPS_PER_VOXEL / t32 / 1e12
        mi = mx["infos"][-1]
        errs = solution_errors(torch, ms, mx["w"], mx["vm"], leg["w"], leg["vm"])
        # the residual-drop replacement policy (after each 3 decades of residual reduction)
        md = run_solver_leg(B, torch, ms, B.PREC_MIXED, a, flush, world, opts={"replace_every": 1000, "replace_drop": 3})
        tmd = allreduce(md["t_ms"], "max", world)
        mdi = md["infos"][-1]
        md["ctx"].close()
        out["mixed"] = {
            "value": vm_val, "unit": UNIT, "ms_per_solve": tm / a.steps, "solves_per_s": world * a.steps / (tm * 1e-3),
            "iters_per_solve": mi["iters"], "relres_true": mi["relres_true"], "replacements": mi["n_replacements"],
            "speedup_vs_fp64_solves": (t_max / tm),
            "hbm": {"gbs": vm_val / world * BYTES_PER_VOXEL_ITER["mixed"] / 1e9,
                    "bytes_per_voxel_iter": BYTES_PER_VOXEL_ITER["mixed"]},
            "apply_roofline": {"bound": "alu", "achieved": ach32, "peak": fp32_peak, "unit": "TFLOP/s",
                               "frac": ach32 / fp32_peak, "ms_per_launch": t32 * 1e3,
                               "traffic": profile_traffic("apply_fp32_100cube.md", a),
                               "hbm_frac": N * APPLY_BYTES_PER_VOXEL["mixed"] / t32 / 1e9 / hbm_peak},
            "gpu_launches": mx["launches"],
            "replacement": "FP64 residual replacement every 50 iterations",
            "errors_vs_fp64": dict(errs, reference="FP64 GPU solve of the same problem, both at true relres 1e-8"),
            "residual_drop_policy": {
                "replacement": "after each 3 decades of residual reduction (at most every 1000 iterations)",
                "value": allreduce(float(N * md["iters"]), "sum", world) / (tmd * 1e-3), "ms_per_solve": tmd / a.steps,
                "iters_per_solve": mdi["iters"], "replacements": mdi["n_replacements"],
                "relres_true": mdi["relres_true"], "speedup_vs_fp64_solves": t_max / tmd},
        }
        out["gpu_launches"] += mx["launches"] + md["launches"]
        mx["ctx"].close()
    if "e2e" in legs:
        e2e = run_e2e(B, torch, ms, a, flush)
        e2e["value"] = allreduce(e2e["value"], "sum", world)
        out["e2e"] = e2e
    if "r200" in legs:
        out["repeat_200"] = run_repeat_200(B, torch, flush)
    if "variants" in legs:
        out["table4_solvers"] = run_variants(B, torch, ms, flush)
    if "batch" in legs:
        out["batched"] = run_batch_leg(B, torch, a, flush)
    if "serve" in legs:
        torch.cuda.empty_cache()
        out["served"] = run_serve_leg(B, torch, a)
        if a.serve_low_requests > 0:
            # the same kind of stream below the server's capacity: latency without a queue backlog
            torch.cuda.empty_cache()
            out["served"]["below_capacity"] = run_serve_leg(B, torch, a, rate=a.serve_low_rate,
                                                            n_requests=a.serve_low_requests, sequential=False)
    if "large" in legs:
        torch.cuda.empty_cache()
        out["large"] = run_large_leg(B, torch)
    leg["ctx"].close()

    # ---- CPU oracle baseline (rank 0, single GPU runs only) ------------------------------------
    if world == 1 and not a.no_cpu_baseline:
        out["cpu_baseline"] = cpu_oracle_rate(ms, a.cpu_seconds)
        out["cpu_baseline"]["eshelby_20"] = eshelby_20(B, torch)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def profile_apply(a):
    """Operator-product launches only, on the benchmark workload (a target for ncu captures)."""
    import torch

    from paper_2602_07354_gb300 import binding as B
    from paper_2602_07354_gb300 import build

    build.build()
    ms = microstructure(a)
    f32 = a.profile_apply == "f32"
    ctx = B.create_from_micro(ms, precision=B.PREC_MIXED if f32 else B.PREC_FP64)
    if a.profile_apply == "f64native":
        B.elas_set_fp64_operator(ctx, B.FP64_OP_NATIVE)
    dt = torch.float32 if f32 else torch.float64
    u = torch.randn(3 * ms.N, dtype=dt, device="cuda")
    y = torch.empty_like(u)
    flush_w = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    flush_r = torch.ones(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    fn = (lambda: B.elas_apply_f32(ctx, u, y)) if f32 else (lambda: B.elas_apply(ctx, u, y))
    fn()  # first launch (module load, shared-memory attribute) outside the timing
    torch.cuda.synchronize()
    t = time_kernel(fn, torch, lambda: (flush_w.fill_(1.0), flush_r.sum()), reps=a.reps)
    print(json.dumps({"profile_apply": a.profile_apply, "grid": [a.size] * 3, "ms_per_launch": t * 1e3,
                      "gvox_per_s": ms.N / t / 1e9}), flush=True)
    ctx.close()


def large_micro(B, torch, n, n_grains, pore_frac, seed):
    """The large-solve microstructure generated on the GPU: Voronoi grains of uniform seeds
    (Algorithm 4), mixed spherical / ellipsoidal pores stamped in batches until the pore fraction
    is reached (Algorithm 5), random orientations (Algorithm 6); cubic 204.6/137.7/126.2 GPa."""
    from paper_2602_07354_gb300 import synth

    rng = np.random.Generator(np.random.PCG64(seed))
    seeds = rng.random((n_grains, 3)) * n
    u = rng.random((n_grains, 3))
    phase = B.elas_assign_grains((n, n, n), seeds, None)
    target, carved = pore_frac * n ** 3, 0
    # mean pore volume of the recipe: spheres pi (8^4 - 2^4) / 18 = 712.5, ellipsoids
    # 4/3 pi E[a^3] E[b/a] E[c/a] = 4/3 pi 16.25 x 1.5 x 4.5 = 459.5 voxels; batches of about 70% of
    # the missing volume, so that the last one overshoots little
    mean_vol = 0.5 * (712.5 + 459.5)
    while carved < target:
        k = max(2, int(0.7 * (target - carved) / mean_vol))
        carved = B.elas_stamp_pores((n, n, n), synth.mixed_pore_draws(rng, n, k), phase)
    rho = B.elas_orientations(B.TEXTURE_RANDOM, torch.from_numpy(u).to("cuda")).cpu().numpy()
    ids = phase.cpu().numpy()
    del phase
    mats = np.broadcast_to(synth.cubic_mat(204.6, 137.7, 126.2), (n_grains, 4)).copy()
    return synth.Microstructure(n, n, n, ids, mats, rho,
                                dict(kind="polycrystal", seed=seed, pore_frac=float(carved) / n ** 3))


def run_large_leg(B, torch):
    """Large single solves: 500^3 voxels with 20,000 grains and 2% porosity (half spheres r 2-8,
    half randomly oriented ellipsoids), mixed precision and plain FP64 to true relres 1e-8; 800^3 in
    the mixed form only.  Microstructures are generated on the GPU (untimed); each solve is timed
    with CUDA events from its first kernel to the returned w."""
    out = []
    for n, seed, precs in ((500, 3, (B.PREC_MIXED, B.PREC_FP64)), (800, 4, (B.PREC_MIXED,))):
        t0 = time.perf_counter()
        ms = large_micro(B, torch, n, 20000, 0.02, seed)
        gen = time.perf_counter() - t0
        for prec in precs:
            torch.cuda.empty_cache()
            torch.cuda.reset_peak_memory_stats()
            ctx = B.create_from_micro(ms, precision=prec)
            tune_ms = B.elas_autotune(ctx, 8)
            st = torch.cuda.current_stream()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            info = B.elas_pcg_solve(ctx, E6, TOL, 100000, stop_rule=B.STOP_TRUE)
            e1.record(st)
            e1.synchronize()
            t = e0.elapsed_time(e1) * 1e-3
            out.append({"grid": f"{n}^3", "precision": "mixed" if prec == B.PREC_MIXED else "fp64", "grains": 20000,
                        "pore_fraction": ms.meta["pore_frac"], "generation_s": gen, "seconds": t,
                        "iters": info["iters"], "relres_true": info["relres_true"], "status": info["status"],
                        "replacements": info["n_replacements"], "voxel_iter_per_s": ms.N * info["iters"] / t,
                        "apply_ms_tuned": tune_ms, "device_gb": torch.cuda.max_memory_allocated() / 1e9})
            ctx.close()
            del ctx
        del ms
    return out


def large(a):
    """--large: the large single solves alone, one JSON line per solve."""
    import torch

    from paper_2602_07354_gb300 import binding as B
    from paper_2602_07354_gb300 import build

    build.build()
    for row in run_large_leg(B, torch):
        print(json.dumps({"large": row}), flush=True)


def kt_sweep(a):
    """Sec. 3.2's anisotropy sweep: a polycrystal with a central spherical void under eps_33 = 1e-3,
    solved (mixed precision, true relres 1e-8) for each Zener ratio of the material table; K_t =
    sigma_max / sigma_nom with sigma_max from App. C's extraction and sigma_nom = 8/3 G eps_33
    (G = 75.08 GPa)."""
    import torch

    from paper_2602_07354_gb300 import binding as B
    from paper_2602_07354_gb300 import build, synth

    build.build()
    n = a.kt_sweep
    t0 = time.perf_counter()
    seeds, semi, rho, void = synth.void_polycrystal_seeds(n)
    phase = B.elas_assign_grains((n, n, n), seeds, semi)
    B.elas_stamp_pores((n, n, n), void, phase)
    ph = phase.cpu().numpy()
    gen_s = time.perf_counter() - t0
    del phase
    e6 = np.array([0, 0, 1e-3, 0, 0, 0.0])
    sig_nom = 8.0 / 3.0 * 75.08 * 1e-3
    for A, c11, c12, c44 in synth.ANISOTROPY_CASES:
        C = B.materials_to_C(np.tile(synth.cubic_mat(c11, c12, c44), (len(seeds), 1)))
        ctx = B.elas_create(n, n, n, ph, C, rho, B.PREC_MIXED)
        t1 = time.perf_counter()
        info = B.elas_pcg_solve(ctx, e6, TOL, 100000, stop_rule=B.STOP_TRUE)
        vm = torch.empty(n ** 3, dtype=torch.float64, device="cuda")
        B.elas_stress(ctx, e6, None, None, vm)
        smax, at, sm = B.elas_hotspot(ctx, vm, 0.4)
        smax_solid = B.elas_hotspot(ctx, vm, 0.4, smoothed=sm, neighbours=B.HOTSPOT_SOLID)[0]
        dt = time.perf_counter() - t1
        ctx.close()
        del vm, sm
        torch.cuda.empty_cache()
        print(json.dumps({"kt_sweep": f"{n}^3", "A": A, "K_t": smax / sig_nom, "sigma_max_MPa": smax * 1e3,
                          "K_t_solid_neighbours": smax_solid / sig_nom,
                          "at": [int(at % n), int((at // n) % n), int(at // (n * n))], "iters": info["iters"],
                          "relres_true": info["relres_true"], "seconds": dt, "generation_s": gen_s,
                          "grains": len(seeds), "void_radius": n / 40.0}), flush=True)


def mesh_study(a):
    """Sec. 3.1's performance study and App. A's mesh sensitivity: the Eshelby void (isotropic
    matrix E = 194 GPa, nu = 0.2934, central spherical void of radius 2/50 of the edge, eps_33 =
    1e-3) at each grid edge of `--mesh-study`; FP64 with Algorithm 2's own criterion
    sqrt(z.g / z0.g0) < 1e-8 (the paper's timing rule) and mixed precision to the FP64 true relative
    residual 1e-8, each timed with CUDA events from the first kernel to the returned w; the App. C
    peak von Mises stress of the mixed solution and K_t = sigma_max / (8/3 G eps_33)."""
    import torch

    from paper_2602_07354_gb300 import binding as B
    from paper_2602_07354_gb300 import build, synth

    build.build()
    paper_s = {100: 1.0, 200: 15.0, 300: 73.0, 400: 233.0, 500: 555.0}
    e6 = np.array([0, 0, 1e-3, 0, 0, 0.0])
    for n in (int(v) for v in a.mesh_study.split(",")):
        ms = synth.eshelby_void(n)
        row = {"mesh_study": f"{n}^3", "void_radius": 2.0 / 50.0 * n, "pore_voxels": int(np.count_nonzero(ms.phase < 0)),
               "paper_openmp_pcg_s": paper_s.get(n)}
        for prec, rule, key in ((B.PREC_FP64, B.STOP_PRECOND, "fp64"), (B.PREC_MIXED, B.STOP_TRUE, "mixed")):
            torch.cuda.empty_cache()
            ctx = B.create_from_micro(ms, precision=prec)
            st = torch.cuda.current_stream()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            info = B.elas_pcg_solve(ctx, e6, TOL, 100000, stop_rule=rule)
            e1.record(st)
            e1.synchronize()
            t = e0.elapsed_time(e1) * 1e-3
            row[key] = {"seconds": t, "iters": info["iters"], "status": info["status"],
                        "relres_true": info["relres_true"], "voxel_iter_per_s": ms.N * info["iters"] / t}
            if prec == B.PREC_MIXED:
                vm = torch.empty(ms.N, dtype=torch.float64, device="cuda")
                B.elas_stress(ctx, e6, None, None, vm)
                smax, at, sm = B.elas_hotspot(ctx, vm, 0.4)
                smax_solid = B.elas_hotspot(ctx, vm, 0.4, smoothed=sm, neighbours=B.HOTSPOT_SOLID)[0]
                row["sigma_max_MPa"] = smax * 1e3
                row["K_t"] = smax / (8.0 / 3.0 * 75.08 * 1e-3)
                row["K_t_solid_neighbours"] = smax_solid / (8.0 / 3.0 * 75.08 * 1e-3)
                row["at"] = [int(at % n), int((at // n) % n), int(at // (n * n))]
                del vm, sm
            ctx.close()
            del ctx
        print(json.dumps(row), flush=True)


def main():
    a = parse()
    world, rank, local = dist_env()
    if a.gpus > 1 and "WORLD_SIZE" not in os.environ and (a.impl == "ours" or a.launcher_selftest):
        # one process per GPU, started here when no launcher (torchrun) did
        backend = "gloo" if a.launcher_selftest else "nccl"
        if not a.launcher_selftest:
            import torch

            if torch.cuda.device_count() < a.gpus:
                print(json.dumps({"error": f"--gpus {a.gpus} but {torch.cuda.device_count()} GPUs are visible"}),
                      flush=True)
                sys.exit(1)
        sys.exit(launch_ranks(a.gpus, sys.argv[1:], os.environ.get("ELAS_BENCH_BACKEND", backend)))
    if a.launcher_selftest:
        launcher_selftest(a, world, rank, local)
        return
    if a.mesh_study:
        mesh_study(a)
        return
    if a.kt_sweep:
        kt_sweep(a)
        return
    if a.large:
        large(a)
        return
    if a.profile_apply:
        profile_apply(a)
        return
    if a.impl == "reference":
        run_reference(a, world, rank)
        return
    run_ours(a, world, rank, local)


if __name__ == "__main__":
    main()
