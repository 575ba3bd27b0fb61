"""Benchmark of the multifrontal Cholesky hot path on one GB300 (per rank).

One step = one FP64 numeric factorization (assembly, extend-add, POTRF/TRSM/
SYRK fronts, level by level) plus one 1-RHS forward/backward solve, on the
extruded Q1 ice-sheet-like mesh (256 x 256 x 10 hexahedra, 2 dofs per node,
n = 1,453,078, horizontal nested dissection).  Inputs (values, RHS) are
resident in HBM when the timed region starts; the factor (~13 GB) is far
larger than L2, so no flush is needed between steps.

``value`` = sum_j c_j^2 (flops of the symbolic phase) * steps / time, in
TFLOP/s, max time over ranks.  Extra keys: factor-only TFLOP/s, solve
latency p50/p99 and solves/s, the FP32 + FP64-refinement path on the same
matrix, the end-to-end number through the C-ABI with host buffers, the
roofline of the dominant kernel and the oracle on the host cores.

Multi-GPU (torchrun): the path does not shard, so N ranks run N independent
replicas (weak scaling); no collective is on the data path.

``--impl reference`` times the FP64 CPU oracle (the reference arm of this
build) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "factor TFLOP/s (sum c_j^2 / step time; step = FP64 numeric factorization + 1-RHS solve)"


def metric_for(args):
    """The metric line names what one timed step does."""
    if args.ir:
        return ("factor TFLOP/s (sum c_j^2 / step time; step = FP32 tensor-core numeric "
                "factorization + %d-RHS solve refined in FP64 to berr <= 1e-13)" % args.nrhs)
    if args.prec == "fp32" or args.nrhs != 1:
        return ("factor TFLOP/s (sum c_j^2 / step time; step = %s numeric factorization + "
                "%d-RHS solve)" % (args.prec.upper(), args.nrhs))
    return METRIC


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--workload", default="q1",
                   choices=["q1", "lap3d", "jump3d", "batch", "serve", "fastilu", "dense", "lu"],
                   help="q1: extruded Q1 ice-sheet mesh (default); lap3d: 7-point Laplacian size^3 "
                        "(small cases for profiling); jump3d: 7-point Laplacian size^3 with "
                        "coefficients 1 / 1e3 on 8^3 blocks (seed 2); batch: 512 7-point Laplacian "
                        "boxes with sides U{8..48} (seed 4) as one block-diagonal forest")
    p.add_argument("--size", type=int, default=None,
                   help="q1: horizontal elements per side (256); lap3d: grid side (48); "
                        "jump3d: grid side (96)")
    p.add_argument("--layers", type=int, default=10)
    p.add_argument("--prec", default="fp64", choices=["fp64", "fp32"],
                   help="precision of the timed factorization + solve (fp64 is the benchmark; "
                        "fp32 runs the tensor-core path, for profiling)")
    p.add_argument("--ir", action="store_true",
                   help="step = FP32 factorization + solve refined in FP64 to berr 1e-13")
    p.add_argument("--autotune", action="store_true",
                   help="pick relaxation / small-front limit / tensor cores with mf_autotune first")
    p.add_argument("--count", type=int, default=512, help="batch: number of boxes")
    p.add_argument("--nrhs", type=int, default=1, help="right-hand sides per solve")
    p.add_argument("--sptrsv", type=int, default=2, choices=[1, 2, 3, 4],
                   help="pivot-block solve: 1 substitution, 2 stored diagonal-block inverses, "
                        "3 partitioned inverse (one product per level; computed inside the "
                        "timed factorization), 4 partitioned inverse of every front as one "
                        "sparse product per level and sweep")
    p.add_argument("--tile", type=int, default=0,
                   help="trailing-update tile of every front-size bucket (mf_options.update_tile "
                        "code: 0 default, 1 FMA 64, 2 FMA 128, 3 tcgen05 128, 4 FMA 32)")
    p.add_argument("--small-queue", type=int, default=1,
                   help="small fronts in one persistent launch: 0 off, 1 fronts of k+m <= 64 "
                        "(default), q >= 2 fronts of k+m <= q")
    p.add_argument("--serve-rates", default="25,100,400",
                   help="serve: Poisson arrival rates (requests/s) to sweep")
    p.add_argument("--serve-requests", type=int, default=240, help="serve: requests per rate")
    p.add_argument("--serve-workers", type=int, default=8)
    p.add_argument("--no-extras", action="store_true")
    p.add_argument("--solve-only-extras", action="store_true",
                   help="after the timed steps measure only the solve latency (p50/p99 over 200)")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    return p.parse_args()


def load_workload(args):
    import gen
    if args.workload == "lap3d":
        rp, ci, v = gen.laplacian_3d(args.size)
        perm = gen.nd_perm((args.size,) * 3)
    elif args.workload == "jump3d":
        rp, ci, v = gen.laplacian_3d(args.size, jump_block=8, jump_value=1e3, seed=2)
        perm = gen.nd_perm((args.size,) * 3)
    elif args.workload == "dense":
        rp, ci, v = gen.dense_spd(args.size, seed=0)
        perm = None
    elif args.workload == "batch":
        mats, _ = gen.box_batch(args.count, 8, 48, seed=4)
        rp, ci, v = gen.block_diag_csr([(a, b, c) for a, b, c, _ in mats])
        offs = np.cumsum([0] + [len(m[0]) - 1 for m in mats])
        perm = np.concatenate([m[3] + o for m, o in zip(mats, offs[:-1])]).astype(np.int32)
    else:
        rp, ci, v = gen.q1_extruded(args.size, args.size, args.layers, seed=1)
        perm = gen.nd_perm((args.size + 1, args.size + 1, args.layers + 1), split_axes=(0, 1),
                           dofs=2)
    n = len(rp) - 1
    b = gen.rhs(n, args.nrhs, seed=3)
    return rp, ci, v, perm, b


def workload_name(args):
    if args.workload == "lap3d":
        return "laplacian7_%d^3_nd" % args.size
    if args.workload == "jump3d":
        return "laplacian7_%d^3_jump1e3_8^3blocks_nd" % args.size
    if args.workload == "batch":
        return "batch_%d_laplacian7_boxes_8-48_seed4" % args.count
    if args.workload == "dense":
        return "dense_spd_%d" % args.size
    return "q1_extruded_%dx%dx%d_2dof_hnd" % (args.size, args.size, args.layers)


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, x):
    """Max of a host float over all ranks (NCCL on GPUs, gloo on CPU)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, steps, ws, ms_max):
    """Whole-job throughput: every rank processes `units_per_rank` per step
    (independent replicas, weak scaling); the slowest rank sets the time."""
    return units_per_rank * steps * ws / (ms_max / 1e3)


class ClockSampler:
    """nvidia-smi samples during the timed region (every 200 ms)."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        # raw samples go to BENCH_CLOCKS_DIR (default: the system temp dir);
        # the JSON line carries their summary
        out_dir = os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, "clocks_bench_%d.csv" % index)

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "samples": len(sm), "reasons": sorted(reasons)}


# DRAM traffic of the dominant FP64 kernel (k_syrk, 32 x 32 tiles): one ncu
# capture of the bulk trailing update of panel step 0 of a dense 8,192-column
# front (trailing matrix 264 MB, larger than L2 like the top fronts of the
# benchmark's meshes): 467.2 MB for 31,878 tiles, 14.66 KB per tile -- one
# read and one write of the 16 KB FP64 tile, the panel slices from L2.  A
# launch's traffic is that per-tile figure times the launch's tiles (the
# schedule's count); valid while the kernel's source text is the measured
# one (SHA-1 below) and the tile is 32.  Fronts whose trailing matrices fit
# in L2 move less, so on a whole factorization this is an upper estimate.
SYRK_TRAFFIC = {"kernel": "k_syrk<double, 32>", "workload": "dense_spd_8192",
                "bytes_per_tile": 467.206e6 / 31878,
                "source_sha1": "a937128192250b3e1851a88491328e14370b9c96"}


def kernel_source_sha1(path, signature):
    """SHA-1 of a kernel's text: from `signature` to its closing brace."""
    import hashlib
    try:
        src = open(path).read()
        i = src.index(signature)
        j = src.index("{", i)
    except (OSError, ValueError):
        return None
    depth = 0
    for k in range(j, len(src)):
        if src[k] == "{":
            depth += 1
        elif src[k] == "}":
            depth -= 1
            if depth == 0:
                return hashlib.sha1(src[i:k + 1].encode()).hexdigest()
    return None


# Oracle sample: the etree subtree with the most flops that stays within
# SAMPLE_FLOPS (sum c_j^2 over its columns).  Fixed flops, not a time budget,
# so the CPU-baseline leg and the reference arm pick the same columns on any
# host.  On the nested-dissection orders used here it holds a separator front
# of several hundred to a few thousand columns and everything below it.
SAMPLE_FLOPS = 2.5e10


def oracle_sample(orc, rp, ci, perm, budget=SAMPLE_FLOPS):
    """(sym, in_s mask, root, columns, flops) of the sample subtree."""
    n = len(rp) - 1
    so = orc.symbolic(rp, ci, perm)
    parent, cc = so["parent"], so["colcount"].astype(np.float64)
    sub = cc * cc
    for j in range(n):  # parent(j) > j: children are complete before parents
        p = parent[j]
        if p >= 0:
            sub[p] += sub[j]
    ok = np.nonzero(sub <= budget)[0]
    root = int(ok[np.argmax(sub[ok])])
    in_s = orc.descendant_closed(parent, [root])
    cols = np.nonzero(in_s)[0]
    return {"rows": so["rows"], "parent": parent}, in_s, root, cols, float(sub[root])


def host_info():
    """Core counts of this host (the oracle's cores) and the CPU model."""
    info = {"nproc": os.cpu_count()}
    try:
        info["affinity"] = len(os.sched_getaffinity(0))
    except AttributeError:
        pass
    try:
        out = subprocess.run(["lscpu"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                             text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            if k.strip() in ("Model name", "Architecture", "CPU(s)", "Socket(s)",
                             "Core(s) per socket", "Thread(s) per core"):
                info[k.strip()] = v.strip()
    except Exception:
        pass
    return info


def run_reference(args):
    """The oracle on all host cores, each step the fixed-flops etree subtree
    sample of the same matrix that the CPU-baseline leg times."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    oracle.build()
    rp, ci, v, perm, b = load_workload(args)
    n = len(rp) - 1
    sym, in_s, root, cols, sflops = oracle_sample(oracle, rp, ci, perm)
    threads = oracle.threads_available()
    for _ in range(args.warmup):
        oracle.factor(rp, ci, v, perm, in_s=in_s, sym=sym, threads=threads)
    t0 = time.perf_counter()
    fl = 0.0
    for _ in range(args.steps):
        F = oracle.factor(rp, ci, v, perm, in_s=in_s, sym=sym, threads=threads)
        fl += F.flops
    el = time.perf_counter() - t0
    val = fl / el / 1e12
    sample = ("etree subtree rooted at column %d: %d of %d columns, %.3g flops per step "
              "(the same sample as the CPU-baseline leg)" % (root, len(cols), n, F.flops))
    out = {
        "impl": "reference", "metric": metric_for(args), "value": val, "unit": "TFLOP/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args), "n": n, "l2_flush": "inputs larger than L2"},
        "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": F.threads, "kind": "oracle",
                         "sample": sample, "host": host_info()},
        "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def run_fastilu(args):
    """FastILU(k) and FastSpTRSV (paper Sec. 6) on the 3D Q1 elasticity
    matrix (27-point stencil, 3 dofs per node) of N^3 nodes, N = --size
    (default 32: n = 98,304): per level k = 0..3, the numeric phase (2
    out-of-place sweeps, no warm-up, as the paper's tables) and one
    preconditioner application (5 Jacobi sweeps per triangle), CUDA events,
    median of 10 after 3 warm-ups.  Bytes per triangular sweep: one read of
    the triangle's values, columns and levels (16 bytes per entry) plus the
    gathered x (8 per entry) and b, x (16 per row)."""
    import torch
    import paper_2506_05793_gb300 as mf
    import gen
    mf.build()
    N = args.size or 32
    rp, ci, v = gen.elasticity_3d(N)
    n = len(rp) - 1
    vd = torch.from_numpy(v).cuda()
    b = torch.from_numpy(gen.rhs(n, 1, seed=3)).cuda()
    x = torch.empty_like(b)
    st = torch.cuda.current_stream()
    h = mf.mf_create()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs") or 6800.0

    def timed(fn, reps=10):
        for _ in range(3):
            fn()
        ms = []
        for _ in range(reps):
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            fn()
            z.record(st)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(z))
        return float(np.median(ms))

    rows = []
    for K in range(4):
        ilu = mf.mf_ilu_symbolic(h, rp, ci, K)
        _, nnz = mf.mf_ilu_info(ilu)
        t_num = timed(lambda: mf.mf_ilu_numeric(ilu, vd, sweeps=2, stream=st))
        t_app = timed(lambda: mf.mf_ilu_apply(ilu, b, 5, x=x, stream=st))
        sweep_bytes = 24.0 * nnz / 2 + 16.0 * n  # one triangle
        gbs = 10 * sweep_bytes / (t_app / 1e3) / 1e9
        rows.append({"level": K, "nnz_per_row": nnz / n, "numeric_ms_2_sweeps": t_num,
                     "apply_ms_5_sweeps_per_triangle": t_app, "apply_GBs": gbs,
                     "apply_frac_of_hbm": gbs / hbm})
        mf.mf_ilu_free(ilu)
    mf.mf_destroy(h)
    print(json.dumps({"metric": "FastILU(k) numeric ms (2 sweeps) and FastSpTRSV apply ms",
                      "workload": "elasticity_q1_%d^3_nodes_3dof" % N, "n": n, "levels": rows,
                      "unit": "ms", "data": "synthetic",
                      "peak_source": "of measured" if peaks.get("hbm_gbs") else "of fallback"}))


def run_serve(args):
    """Serving stream: Poisson arrivals of factor+solve requests (90% boxes
    with sides U{8..48}, 10% 64^3 Laplacians) and solve-only requests with
    1..16 right-hand sides against resident factors; FP32 factors with FP64
    refinement to berr 1e-13; admission under a 120 GB factor budget."""
    import torch
    import paper_2506_05793_gb300 as mf
    import gen
    mf.build()
    rng = np.random.default_rng(5)
    h = mf.mf_create()
    pool = []
    for a, b, c in rng.integers(8, 49, size=(24, 3)):
        rp, ci, v = gen.laplacian_3d(int(a), int(b), int(c))
        pm = gen.nd_perm((int(a), int(b), int(c)))
        pool.append((rp, ci, v, mf.mf_symbolic_analyze(h, rp, ci, pm)))
    big = []
    for _ in range(1):
        rp, ci, v = gen.laplacian_3d(64)
        pm = gen.nd_perm((64, 64, 64))
        big.append((rp, ci, v, mf.mf_symbolic_analyze(h, rp, ci, pm)))
    results = []
    for rate in [float(x) for x in args.serve_rates.split(",")]:
        sv = mf.mf_server_create(h, workers=args.serve_workers, budget_bytes=120 * 10**9)
        t_arr = np.cumsum(rng.exponential(1.0 / rate, size=args.serve_requests))
        resident = []  # (factor_id, n)
        reqs = []
        t0 = time.perf_counter()
        for k in range(args.serve_requests):
            while time.perf_counter() - t0 < t_arr[k]:
                time.sleep(min(0.001, max(0.0, t_arr[k] - (time.perf_counter() - t0))))
            if resident and rng.random() < 0.4:
                fid, n = resident[rng.integers(len(resident))]
                nrhs = int(rng.integers(1, 17))
                req, X = mf.mf_server_submit_solve(sv, fid, gen.rhs(n, nrhs, seed=k))
                reqs.append(req)
            else:
                rp, ci, v, s = big[0] if rng.random() < 0.1 else pool[rng.integers(len(pool))]
                n = len(rp) - 1
                req, fid, X = mf.mf_server_submit_factor(sv, s, v, mf.MF_FP32, gen.rhs(n, 1, seed=k))
                reqs.append(req)
                resident.append((fid, n))
                if len(resident) > 48:  # keep the newest factors resident
                    old, _ = resident.pop(0)
                    mf.mf_server_release_factor(sv, old)
        bad = 0
        for r in reqs:
            st_, _ = mf.mf_server_wait(sv, r)
            bad += st_ != 0
        wall = time.perf_counter() - t0
        st = mf.mf_server_get_stats(sv)
        results.append({"rate_req_per_s": rate, "requests": len(reqs), "failed": int(bad),
                        "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "mean_ms": st["mean_ms"],
                        "solves_per_s": st["solves_per_s"], "wall_s": wall,
                        "peak_resident_GB": st["peak_resident_bytes"] / 1e9})
        mf.mf_server_free(sv)
    out = {"metric": "serving latency p50/p99 (ms) and solves/s under Poisson arrivals",
           "workload": "serve: 90% boxes U{8..48}^3 + 10% 64^3 factor+solve, 40% solve-only "
                       "1..16 RHS; FP32 + FP64 refinement to 1e-13; 120 GB budget",
           "workers": args.serve_workers, "sweep": results, "data": "synthetic"}
    print(json.dumps(out))
    for _, _, _, s in pool + big:
        mf.mf_symbolic_free(s)
    mf.mf_destroy(h)


def ldlt_piv_case(mf, gen, torch, st, timed, N):
    """Pivoted LDL^T (symmetric pivoting within the diagonal blocks) of the
    saddle point [K B^T; B 0] on N^3 nodes, multiplier first in each node
    (the unpivoted LDL^T stops at column 0), condensed analysis with 2 dofs
    per node: factorization ms (median of 5), the 1-RHS solve, berr."""
    import oracle
    rp, ci, v = gen.kkt_3d(N, N, N, delta=0.0, seed=12)
    perm = gen.nd_perm((N, N, N), dofs=2)
    perm = np.ascontiguousarray(perm.reshape(-1, 2)[:, ::-1].ravel()).astype(np.int32)
    n = len(rp) - 1
    h = mf.mf_create(mf.mf_options_default())
    s = mf.mf_symbolic_analyze_condensed(h, rp, ci, perm, block=2)
    info = mf.mf_symbolic_get_info(s)
    vd = torch.from_numpy(v).cuda()
    b = torch.from_numpy(gen.rhs(n, 1, seed=3)).cuda()
    out = {"workload": "saddle_kkt_%d^3_nodes_zero_block_multiplier_first" % N, "n": n,
           "flops": info["flops"]}
    f = mf.mf_factor_create_ldlt(h, s, mf.MF_FP64)
    try:
        mf.mf_factor_numeric(f, vd, stream=st)
        out["unpivoted"] = "factored"
    except mf.MFError as e:
        out["unpivoted"] = "zero pivot at column %d" % e.column
    mf.mf_factor_free(f)
    f = mf.mf_factor_create_ldlt_piv(h, s, mf.MF_FP64)
    out["ms"] = timed(lambda: mf.mf_factor_numeric(f, vd, stream=st, async_=1))
    out["tflops"] = info["flops"] / (out["ms"] / 1e3) / 1e12
    mf.mf_factor_numeric(f, vd, stream=st)
    x = mf.mf_solve(f, b, stream=st)
    out["solve_ms"] = timed(lambda: mf.mf_solve(f, b, stream=st), reps=20)
    torch.cuda.synchronize()
    out["berr"] = oracle.berr(rp, ci, v, x.cpu().numpy(), b.cpu().numpy())
    mf.mf_factor_free(f)
    mf.mf_symbolic_free(s)
    mf.mf_destroy(h)
    return out


def run_lu(args):
    """LU with a symmetric pattern (paper Sec. 5) on the 7-point
    convection-diffusion operator of N^3 nodes (N = --size, default 64),
    strong wind (U[-3, 3] per node and axis) and a tenth of the diagonal
    entries replaced by U[-0.5, 0.5], nested dissection: FP64 LU with
    pivoting within the diagonal blocks and without, FP32 LU + FP64
    refinement, and the Cholesky factorization of the same pattern (7-point
    Laplacian) for scale.  Factorization ms: median of 5 after 3 warm-ups
    (CUDA events); LU flops 2 sum c_j^2.  The trailing update's rate comes
    from one profiled factorization (per-launch events), separate from the
    timed ones.  Parity of the run: the same generator at 15 x 14 x 16
    (n = 3,360, fronts of up to 210 pivot columns) against the oracle's
    dense windowed LU, row order exactly and relF of L and U."""
    import torch
    import paper_2506_05793_gb300 as mf
    import gen
    mf.build()
    N = args.size or 64
    st = torch.cuda.current_stream()

    def timed(fn, reps=5):
        for _ in range(3):
            fn()
        ms = []
        for _ in range(reps):
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            fn()
            z.record(st)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(z))
        return float(np.median(ms))

    def case(rp, ci, v, perm, kind, prec=mf.MF_FP64, pivot=1, refine=False, profile=False,
             relax=1):
        opt = mf.mf_options_default()
        opt.profile = 1 if profile else 0
        opt.relax = relax
        h = mf.mf_create(opt)
        s = mf.mf_symbolic_analyze(h, rp, ci, perm)
        info = mf.mf_symbolic_get_info(s)
        f = (mf.mf_factor_create_lu(h, s, prec, pivot) if kind == "lu"
             else mf.mf_factor_create(h, s, prec))
        n = len(rp) - 1
        vd = torch.from_numpy(v).cuda()
        b = torch.from_numpy(gen.rhs(n, 1, seed=3)).cuda()
        out = {"flops": (2.0 if kind == "lu" else 1.0) * info["flops"]}
        if profile:
            mf.mf_factor_numeric(f, vd, stream=st)
            prof = mf.mf_factor_profile(f)
            syrk = prof["syrk"]
            out["syrk_ms"] = syrk["ms"]
            out["syrk_tflops"] = ((2.0 if kind == "lu" else 1.0) * syrk["flops"]
                                  / (syrk["ms"] / 1e3) / 1e12 if syrk["ms"] else None)
        else:
            out["ms"] = timed(lambda: mf.mf_factor_numeric(f, vd, stream=st, async_=1))
            out["tflops"] = out["flops"] / (out["ms"] / 1e3) / 1e12
            mf.mf_factor_numeric(f, vd, stream=st)
            if refine:
                x, rep = mf.mf_solve_refined(f, b, tol=1e-13, max_iter=30, stream=st)
                out["refined_solve_ms"] = timed(
                    lambda: mf.mf_solve_refined(f, b, tol=1e-13, max_iter=30, stream=st))
                out["refinement_steps"] = int(rep["iterations"])
                out["fell_back"] = bool(rep["fell_back"])
            else:
                x = mf.mf_solve(f, b, stream=st)
                out["solve_ms"] = timed(lambda: mf.mf_solve(f, b, stream=st), reps=20)
            torch.cuda.synchronize()
            out["berr"] = orc_berr(rp, ci, v, x.cpu().numpy(), b.cpu().numpy())
        mf.mf_factor_free(f)
        mf.mf_symbolic_free(s)
        mf.mf_destroy(h)
        return out

    def orc_berr(rp, ci, v, x, bb):
        import oracle
        return oracle.berr(rp, ci, v, x, bb)

    rp, ci, v = gen.nonsym_3d(N, N, N, wind=3.0, small_diag=0.1, seed=11)
    perm = gen.nd_perm((N, N, N))
    n = len(rp) - 1
    res = {"lu_pivot_fp64": case(rp, ci, v, perm, "lu", pivot=1),
           "lu_nopivot_fp64": case(rp, ci, v, perm, "lu", pivot=0),
           "lu_pivot_fp32_refined": case(rp, ci, v, perm, "lu", prec=mf.MF_FP32, pivot=1,
                                         refine=True),
           "lu_pivot_fp64_profiled": case(rp, ci, v, perm, "lu", pivot=1, profile=True)}
    lp, lc, lv = gen.laplacian_3d(N)
    res["cholesky_fp64_same_pattern"] = case(lp, lc, lv, perm, "chol")
    res["ldlt_piv_saddle_fp64"] = ldlt_piv_case(mf, gen, torch, st, timed, max(8, (N * 3) // 4))
    # parity of the run at a size the dense oracle factors in seconds
    import oracle as orc
    shape = (15, 14, 16)
    sp, sc, sv = gen.nonsym_3d(*shape, wind=3.0, small_diag=0.3, seed=1)
    sperm = gen.nd_perm(shape)
    sn = len(sp) - 1
    opt = mf.mf_options_default()
    opt.relax = 0
    h = mf.mf_create(opt)
    s = mf.mf_symbolic_analyze(h, sp, sc, sperm)
    f = mf.mf_factor_create_lu(h, s, mf.MF_FP64, 1)
    mf.mf_factor_numeric(f, sv)
    so = orc.symbolic(sp, sc, sperm)
    F = orc.lu_dense(sp, sc, sv, sperm, wend=orc.pivot_windows(so["sup_ptr"][:-1], sn))
    info = mf.mf_symbolic_get_info(s)
    Lp, Li = mf.mf_symbolic_pattern(s)
    Lx = mf.mf_factor_export_L(f, info["nnz_L"])
    Ux = mf.mf_factor_export_U(f, info["nnz_L"])
    rho = mf.mf_factor_export_pivots(f, sn)
    fronts = mf.mf_symbolic_fronts(s)
    cols = np.repeat(np.arange(sn), np.diff(Lp))
    rows = Li.astype(np.int64)
    fend = fronts[np.repeat(np.arange(len(fronts) - 1), np.diff(fronts)) + 1]
    pos = np.empty(sn, dtype=np.int64)
    pos[rho] = np.arange(sn)
    Ld = np.zeros((sn, sn))
    Ld[np.where(rows < fend[cols], rows, pos[rows]), cols] = Lx
    Ud = np.zeros((sn, sn))
    Ud[cols, rows] = Ux
    parity = {"workload": "convdiff7_15x14x16_wind3_nd", "n": sn,
              "rho_exact": bool(np.array_equal(rho, F.rho)),
              "rows_swapped": int(np.count_nonzero(F.rho != np.arange(sn))),
              "relF_L": float(np.linalg.norm(Ld - F.L) / np.linalg.norm(F.L)),
              "relF_U": float(np.linalg.norm(Ud - F.U) / np.linalg.norm(F.U))}
    mf.mf_factor_free(f)
    mf.mf_symbolic_free(s)
    mf.mf_destroy(h)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    dfma = mf.mf_diag_fp64_peak(0, stream=st)
    pr = res["lu_pivot_fp64_profiled"]
    print(json.dumps({
        "metric": "LU factor TFLOP/s (2 sum c_j^2 / factorization time)",
        "value": res["lu_pivot_fp64"]["tflops"], "unit": "TFLOP/s", "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "convdiff7_%d^3_wind3_smalldiag0.1_nd" % N, "n": n,
                   "nnz_A": int(rp[-1])},
        "cases": res,
        "roofline": {"kernel": "k_syrk<double, 32, LU>", "bound": "alu",
                     "achieved": pr.get("syrk_tflops"), "peak": dfma, "unit": "TFLOP/s",
                     "frac": (pr["syrk_tflops"] / dfma) if pr.get("syrk_tflops") else None,
                     "peak_source": "of measured: the DFMA probe (mf_diag_fp64_peak) on this GPU"},
        "parity": parity}))


def main():
    args = parse()
    if args.workload == "serve":
        run_serve(args)
        return
    if args.workload == "fastilu":
        run_fastilu(args)
        return
    if args.workload == "lu":
        run_lu(args)
        return
    if args.size is None:
        args.size = {"lap3d": 48, "jump3d": 96, "dense": 8192}.get(args.workload, 256)
    if args.impl == "reference":
        run_reference(args)
        return
    ws, rank, local = dist_setup()
    import torch
    import paper_2506_05793_gb300 as mf
    import gen
    mf.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rp, ci, v, perm, b = load_workload(args)
    n = len(rp) - 1
    if args.ir:
        args.prec = "fp32"
    prec = mf.MF_FP32 if args.prec == "fp32" else mf.MF_FP64
    opt = mf.mf_options_default()
    tuned = None
    if args.autotune:
        h0 = mf.mf_create()
        opt, tuned_ms = mf.mf_autotune(h0, rp, ci, perm, v, prec=prec, reps=2)
        mf.mf_destroy(h0)
        tuned = {"relax": opt.relax, "small_front_max": opt.small_front_max, "tc": opt.tc,
                 "small_queue": opt.small_queue, "update_tile": list(opt.update_tile),
                 "ms": tuned_ms}
    opt.profile = 1  # per-launch CUDA events: per-kernel-kind device time
    opt.sptrsv = args.sptrsv
    if not args.autotune:
        opt.small_queue = args.small_queue
        for bk in range(4):
            opt.update_tile[bk] = args.tile
    h = mf.mf_create(opt)
    t0 = time.perf_counter()
    s = mf.mf_symbolic_analyze(h, rp, ci, perm)
    t_sym = time.perf_counter() - t0
    info = mf.mf_symbolic_get_info(s)
    f = mf.mf_factor_create(h, s, prec)
    st = torch.cuda.current_stream(dev)
    vd = torch.from_numpy(v).to(dev)
    bd = torch.from_numpy(b).to(dev)
    xd = torch.empty_like(bd)
    nf_launch, ns_launch = mf.mf_factor_launch_counts(f)

    def step():
        mf.mf_factor_numeric(f, vd, stream=st, async_=True)
        if args.ir:
            mf.mf_solve_refined(f, bd, xd, tol=1e-13, max_iter=30, stream=st)
        else:
            mf.mf_solve(f, bd, xd, stream=st)

    for _ in range(args.warmup):
        step()
    mf.mf_factor_check(f, stream=st)
    torch.cuda.synchronize()
    fp64_peak = {"dfma": mf.mf_diag_fp64_peak(0, stream=st), "dmma": mf.mf_diag_fp64_peak(1, stream=st)}
    clk = ClockSampler(local)
    clk.start()
    barrier(ws)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        step()
    e1.record(st)
    torch.cuda.synchronize()
    barrier(ws)
    ms = e0.elapsed_time(e1)
    clocks = clk.stop()
    mf.mf_factor_check(f, stream=st)  # status of the last step; also reads the profile
    prof = mf.mf_factor_profile(f)
    ms_max = max_over_ranks(ws, ms)
    flops = info["flops"]
    value = job_value(flops, args.steps, ws, ms_max) / 1e12

    out = {
        "metric": metric_for(args), "value": value, "unit": "TFLOP/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.prec == "fp32" else "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(args), "n": n, "nnz_A": int(rp[-1]),
                   "nnz_L": info["nnz_L"],
                   "flops_per_factor": flops, "nsuper": info["nsuper"],
                   "levels": info["nlevels"], "max_front": info["max_front"], "nrhs": args.nrhs,
                   "sptrsv": args.sptrsv,
                   "parallelism": "replicas" if ws > 1 else "single",
                   "l2_flush": "inputs larger than L2 (factor %.1f GB)" % (
                       info["factor_bytes_fp64"] / 1e9),
                   "symbolic_s": t_sym},
        "step": ("FP32 factor + FP64-refined solve to berr 1e-13" if args.ir else
                 "%s factor + %s solve" % (args.prec.upper(), args.prec.upper())),
        "autotune": tuned,
        "gpu_launches": int((nf_launch + ns_launch) * args.steps),
        "clocks": clocks,
    }
    fac_ms = sum(p["ms"] for p in prof.values())
    out["factor_ms_sum_of_kernels"] = fac_ms
    out["kernels_note"] = ("per-kind sums of per-launch CUDA-event times; lookahead runs bulk "
                           "updates on a second stream, so kinds overlap and the sum can exceed "
                           "the step")
    out["factor_tflops_kernels"] = flops / (fac_ms / 1e3) / 1e12 if fac_ms > 0 else None
    out["kernels"] = prof
    # dominant kernel roofline.  split-TF32 tensor cores: the measured bf16
    # peak x nominal TF32/bf16 ratio, / 3 products per useful FMA.  FP64 and
    # FP32 FMA work runs on the ALU pipes: peaks from unit counts and clock
    # (152 SMs, 2.07 GHz; FP64: 2 FMA per clock per SM, the nominal
    # 1.25 TFLOP/s; FP32: 128 FMA lanes per SM).
    dom = max(prof, key=lambda k: prof[k]["ms"])
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    bf16 = peaks.get("bf16_tflops")
    bf16_src = "measured" if bf16 else "fallback"
    bf16 = bf16 or 1900.0
    ach = prof[dom]["flops"] / (prof[dom]["ms"] / 1e3) / 1e12 if prof[dom]["ms"] > 0 else 0.0
    if dom == "syrk_tc":
        bound = "tensor"
        peak = bf16 * (1100.0 / 2250.0) / 3.0
        src = ("of %s: bf16 %.0f TFLOP/s x nominal TF32/bf16 1100/2250, / 3 for split-TF32 "
               "(useful FP32 flops)" % (bf16_src, bf16))
    elif args.prec == "fp32":
        bound = "alu"
        peak = 152 * 128 * 2 * 2.07e9 / 1e12
        src = "derived: FP32 FMA, 152 SMs x 128 lanes x 2 flops x 2.07 GHz"
    else:
        # measured on this GPU by the two FP64 probes (register-resident
        # DFMA and DMMA loops); the faster one is the FP64 pipe's peak
        bound = "alu"
        out["fp64_peak_probe"] = fp64_peak
        peak = max(fp64_peak.values())
        src = ("of measured: best of the DFMA (%.3f) and DMMA (%.3f) TFLOP/s probes run by "
               "mf_diag_fp64_peak on this GPU before the timed region"
               % (fp64_peak["dfma"], fp64_peak["dmma"]))
    traffic = None
    items = mf.mf_factor_kind_items(f)
    if (dom == "syrk" and args.prec == "fp64" and args.tile in (0, 3, 4)
            and kernel_source_sha1(os.path.join(ROOT, "paper_2506_05793_gb300", "csrc",
                                                "factor_kernels.cu"), "k_syrk(FD<T> d")
            == SYRK_TRAFFIC["source_sha1"]):
        tiles, launches = items["syrk"]
        traffic = SYRK_TRAFFIC["bytes_per_tile"] * tiles / max(launches, 1)
    out["roofline"] = {"kernel": dom, "bound": bound, "achieved": ach, "peak": peak,
                       "unit": "TFLOP/s", "frac": ach / peak, "traffic": traffic,
                       "peak_source": src}
    if traffic is not None:
        out["roofline"]["traffic_source"] = (
            "bytes per launch = %.0f bytes per 32 x 32 tile (ncu dram__bytes_read.sum + "
            "dram__bytes_write.sum, bulk launch on a dense 8192-column front) x %.0f tiles per "
            "launch of this schedule; an upper estimate where trailing matrices fit in L2"
            % (SYRK_TRAFFIC["bytes_per_tile"], items["syrk"][0] / max(items["syrk"][1], 1)))
    if rank == 0 and args.solve_only_extras:
        solve_latency(args, out, mf, f, bd, st, info, len(rp) - 1)
    elif rank == 0 and not args.no_extras:
        extras(args, out, mf, h, s, f, rp, ci, v, b, vd, bd, xd, st, dev, info, perm)
    if rank == 0:
        print(json.dumps(out))
    mf.mf_factor_free(f)
    mf.mf_symbolic_free(s)
    mf.mf_destroy(h)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def solve_latency(args, out, mf, f, bd, st, info, n):
    """Solve latency (nrhs right-hand sides), p50 / p99 over 200 solves, and
    the solve's roofline: L read once per sweep plus the right-hand side /
    solution vectors (4 passes of n x nrhs values)."""
    import torch
    xs = torch.empty_like(bd)
    for _ in range(3):
        mf.mf_solve(f, bd, xs, stream=st)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(200)]
    for a, z in ev:
        a.record(st)
        mf.mf_solve(f, bd, xs, stream=st)
        z.record(st)
    torch.cuda.synchronize()
    mf.mf_solve_check(f, stream=st)
    lat = np.array([a.elapsed_time(z) for a, z in ev])
    out["solve_ms"] = {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "samples": len(lat)}
    out["solves_per_s"] = float(1e3 / np.mean(lat))
    out["solve_nrhs"] = args.nrhs
    # algorithmic bytes of one solve: L read once per sweep plus the
    # right-hand side / solution vectors (4 passes of n x nrhs values)
    es = 4 if args.prec == "fp32" else 8
    sbytes = 2.0 * es * info["nnz_L"] + 4.0 * es * n * args.nrhs
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = peaks.get("hbm_gbs") or 6800.0
    gbs = sbytes / (out["solve_ms"]["p50"] / 1e3) / 1e9
    out["solve_roofline"] = {"bound": "hbm", "bytes": sbytes, "achieved": gbs, "peak": hbm,
                             "unit": "GB/s", "frac": gbs / hbm,
                             "peak_source": "of measured" if peaks.get("hbm_gbs") else "of fallback"}


def extras(args, out, mf, h, s, f, rp, ci, v, b, vd, bd, xd, st, dev, info, perm):
    import torch
    n = len(rp) - 1
    solve_latency(args, out, mf, f, bd, st, info, n)
    # end to end through the C-ABI with host buffers (values H2D, B H2D, X D2H)
    K = 2
    xh = np.empty_like(b, order="F")
    t0 = time.perf_counter()
    for _ in range(K):
        mf.mf_factor_numeric(f, v)       # host values, sync + status read
        if args.ir:                      # the same step as the timed one
            mf.mf_solve_refined(f, b, xh, tol=1e-13, max_iter=30)
        else:
            mf.mf_solve(f, b, xh)        # host RHS and solution
    el = time.perf_counter() - t0
    out["e2e"] = {"value": info["flops"] * K / el / 1e12, "unit": "TFLOP/s",
                  "h2d_bytes_per_step": int(v.nbytes + b.nbytes),
                  "d2h_bytes_per_step": int(xh.nbytes + 16)}
    # FP32 factorization + FP64 refinement to berr 1e-13 on the same matrix:
    # 3 warm-up steps, then the median of 10; refined-solve p50 / p99 over
    # 200 calls
    f32 = None
    x32 = None
    try:
        f32 = mf.mf_factor_create(h, s, mf.MF_FP32)
        xr = torch.empty_like(bd)

        def step32():
            mf.mf_factor_numeric(f32, vd, stream=st, async_=True)
            return mf.mf_solve_refined(f32, bd, xr, tol=1e-13, max_iter=30, stream=st)[1]

        for _ in range(3):
            step32()
        torch.cuda.synchronize()
        ms32, reps = [], []
        for _ in range(10):
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            reps.append(step32())
            z.record(st)
            torch.cuda.synchronize()
            ms32.append(a.elapsed_time(z))
        mf.mf_factor_check(f32, stream=st)
        lat32 = []
        for _ in range(200):
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            mf.mf_solve_refined(f32, bd, xr, tol=1e-13, max_iter=30, stream=st)
            z.record(st)
            torch.cuda.synchronize()
            lat32.append(a.elapsed_time(z))
        x32 = xr.cpu().numpy()
        out["fp32_ir"] = {
            "ms_factor_plus_refined_solve": {"median": float(np.median(ms32)),
                                             "min": float(np.min(ms32)),
                                             "max": float(np.max(ms32)), "steps": len(ms32),
                                             "warmup": 3},
            "tflops_median": info["flops"] / (np.median(ms32) / 1e3) / 1e12,
            "refined_solve_ms": {"p50": float(np.percentile(lat32, 50)),
                                 "p99": float(np.percentile(lat32, 99)), "samples": len(lat32)},
            "report_last_step": reps[-1],
            "iterations": sorted(set(int(r["iterations"]) for r in reps)),
            "fell_back": any(r["fell_back"] for r in reps),
        }
        if not args.ir:
            out["fp32_ir"]["fp64_ms_per_step"] = out["ms_per_step"]
            out["fp32_ir"]["speedup_vs_fp64_step"] = out["ms_per_step"] / float(np.median(ms32))
    except Exception as e:  # report, do not hide the main number
        out["fp32_ir"] = {"error": str(e)}
    if int(os.environ.get("WORLD_SIZE", "1")) == 1:
        oracle_leg(args, out, mf, s, f, f32, rp, ci, v, b, xd, x32, perm)
    if f32 is not None:
        mf.mf_factor_free(f32)
    # the same solve with SpTRSV variant 4 (every front's partitioned
    # inverse as one sparse product per level and sweep): its own analysis
    # and factor; setup = the extra factorization time
    if args.sptrsv != 4:
        try:
            o4 = mf.mf_options_default()
            o4.sptrsv = 4
            h4 = mf.mf_create(o4)
            s4 = mf.mf_symbolic_analyze(h4, rp, ci, perm)
            f4 = mf.mf_factor_create(h4, s4, mf.MF_FP64 if args.prec == "fp64" else mf.MF_FP32)
            mf.mf_factor_numeric(f4, vd, stream=st)
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            mf.mf_factor_numeric(f4, vd, stream=st, async_=True)
            z.record(st)
            mf.mf_factor_check(f4, stream=st)
            sub = {}
            solve_latency(args, sub, mf, f4, bd, st, info, n)
            out["solve_variant4"] = {"solve_ms": sub["solve_ms"], "solves_per_s": sub["solves_per_s"],
                                     "solve_roofline": sub["solve_roofline"],
                                     "factor_ms_with_setup": a.elapsed_time(z)}
            mf.mf_factor_free(f4)
            mf.mf_symbolic_free(s4)
            mf.mf_destroy(h4)
        except Exception as e:
            out["solve_variant4"] = {"error": str(e)}


def oracle_leg(args, out, mf, s, f, f32, rp, ci, v, b, xd, x32, perm):
    """The CPU-baseline leg (rank 0, one GPU): the oracle times a fixed-flops
    etree subtree of the same matrix with one thread and with all host cores,
    and that exact factor checks the GPU factors' columns entry by entry; the
    backward errors of the timed step's solution and of the FP32 + refinement
    solution are the oracle's measure."""
    import oracle
    oracle.build()
    n = len(rp) - 1
    sym, in_s, root, cols, sflops = oracle_sample(oracle, rp, ci, perm)
    runs = {}
    for threads in (1, oracle.threads_available()):
        t0 = time.perf_counter()
        F = oracle.factor(rp, ci, v, perm, in_s=in_s, sym=sym, threads=threads)
        dt = time.perf_counter() - t0
        runs[F.threads] = (F, dt)
    F, dt = runs[max(runs)]
    F1, dt1 = runs[min(runs)]
    sample = ("etree subtree rooted at column %d: %d of %d columns, %.3g flops"
              % (root, len(cols), n, F.flops))
    out["cpu_baseline"] = {"value": F.flops / dt / 1e12, "unit": "TFLOP/s", "cores": F.threads,
                           "kind": "oracle", "sample": sample, "seconds": dt,
                           "one_thread": {"value": F1.flops / dt1 / 1e12, "cores": 1,
                                          "seconds": dt1},
                           "host": host_info()}
    # element-wise parity of the GPU factors on the sample's columns
    j0, j1 = int(cols[0]), int(cols[-1]) + 1
    cc = mf.mf_symbolic_colcounts(s)[j0:j1]  # column counts of the global pattern
    par = {"sample_columns": [j0, j1], "contiguous": bool(len(cols) == j1 - j0),
           "sample_max_column_count": int(cc.max())}
    ref = F.Lx[F.Lp[j0]:F.Lp[j1]]  # the oracle stores the sample's columns only
    mask = np.repeat(in_s[j0:j1].astype(bool), cc)
    for name, fac in (("fp64", f), ("fp32", f32)):
        if fac is None:
            continue
        got = mf.mf_factor_export_columns(fac, j0, j1, int(cc.sum()))[mask]
        assert len(got) == len(ref)
        par["relF_sample_" + name] = oracle.rel_fro(got, ref)
    x64 = xd.cpu().numpy()
    par["berr_step_solution"] = oracle.berr(rp, ci, v, x64, b)
    if x32 is not None:
        par["berr_fp32_ir"] = oracle.berr(rp, ci, v, x32, b)
        par["fwd_err_fp32_ir_vs_fp64"] = float(np.max(np.abs(x32 - x64)) / np.max(np.abs(x64)))
    out["parity"] = par


if __name__ == "__main__":
    main()
