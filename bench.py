"""Benchmark: MG-preconditioned CG solves of the 2D P2 workload on GB300.

Workload (one "step" = one solve, setup excluded): unit square, 1024^2 grid of squares
split into triangles, P2 elements (4,190,209 free DoFs), 6 non-nested independently
jittered levels (1024^2 .. 32^2), 32 seeded clusters of 2-8 needle/flattened cells (aspect
ratio 1e2-1e4) on the fine and on every intermediate level, right-hand side U[-1, 1],
V-cycle with the global-local combined smoother (sandwich S_c, Chebyshev degree 2 with the
adjusted lambda_max, S_c), CG to relative residual 1e-8.

`value` is the mixed-precision form (FP32 V-cycle inside FP64 CG); the plain FP64 form is
measured on the same GPU and reported under "fp64". Multi-GPU: independent replicas, one
problem per rank (weak scaling, no data-path collective).

--impl reference times the CPU oracle (NumPy/SciPy, the same algorithm in FP64) on a
bounded sample of the same workload family.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DoFs/s solved to rtol 1e-8 (mixed vs FP64, same GPU); SpMV HBM GB/s; p50/p99"
WORKLOAD = ("2D Poisson P2, unit square 1024^2 x 2 triangles (4,190,209 DoFs), 6 non-nested levels, "
            "32 needle/flattened clusters (AR 1e2-1e4) per fine/intermediate level, "
            "sandwich S_c-Chebyshev(2)-S_c with adjusted lambda, MG-PCG rtol 1e-8, RHS U[-1,1]")
WORKLOADS = {
    "c2": (WORKLOAD, 2),
    "c3": ("3D Poisson P1, unit cube 128^3 x 6 tets (2,048,383 DoFs), 5 non-nested levels, 64 cap slivers "
           "(1e-3 h) on the fine and 2nd-coarsest level, sandwich smoother, MG-PCG rtol 1e-8, RHS U[-1,1]", 1),
    "c4": ("3D Poisson P2, unit cube 64^3 x 6 tets (2,048,383 DoFs), 4 non-nested levels, 256 sliver clusters "
           "merged into 212 patches of 118-2053 DoFs, sandwich smoother, MG-PCG rtol 1e-8, RHS U[-1,1]", 2),
}
SAMPLE_N = 256   # CPU oracle sample: the same family at 256^2 (261,121 DoFs, 4 levels)
RTOL = 1e-8


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n-fine", type=int, default=1024)
    ap.add_argument("--levels", type=int, default=6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-oracle-check", action="store_true",
                    help="skip the oracle's solve of the same problem (error of each GPU solution against it)")
    ap.add_argument("--no-serve", action="store_true", help="skip the bounded serving stream and the batched solve of the default line")
    ap.add_argument("--no-graph", action="store_true",
                    help="launch every kernel individually instead of one CUDA graph per solve (profilers "
                         "cannot see kernel nodes of graphs with conditional nodes)")
    ap.add_argument("--workload", default="c2",
                    choices=["c2", "c3", "c4", "serve", "paper", "lattice", "dumbbell", "persistent"],
                    help="'serve': the mixed request stream through the continuous-batching server; "
                         "'paper': the Case A/B comparison and the residual history of the paper's examples")
    ap.add_argument("--reorder", default=None, choices=["none", "rcm", "spatial", "spatial-coarse"],
                    help="device-internal DoF order (default: the library's default)")
    ap.add_argument("--global-smoother", default="chebyshev", choices=["chebyshev", "sgs"],
                    help="S_g of the combined smoother (c2/c3/c4)")
    ap.add_argument("--requests", type=int, default=512)
    ap.add_argument("--rates", default="4,16,64", help="Poisson arrival rates (requests/s) to sweep")
    ap.add_argument("--precision", default="both", choices=["both", "mixed"],
                    help="'mixed' builds and times only the mixed-precision form (profiling runs)")
    return ap.parse_args()


def dist_env():
    from paper_2402_12947_gb300 import replicas
    return replicas.dist_env()


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, copy burst)"
    except Exception:
        return 6800.0, "fallback (6.8 TB/s)"


def profiled_traffic():
    """DRAM bytes per launch of the fine-level Chebyshev kernel from the committed ncu
    summary (a line 'traffic_bytes_per_launch: <int> kernel_rev: <rev>')."""
    path = os.path.join(ROOT, "profiles", "k_cheb_f32_c2_fine.md")
    try:
        for line in open(path):
            if line.startswith("traffic_bytes_per_launch:"):
                parts = line.split()
                rev = parts[3] if len(parts) > 3 else ""
                return float(parts[1]), rev
    except OSError:
        pass
    return None, None


KERNEL_REV = "v10"   # bump when the timed kernel changes (invalidates the profiled traffic)


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        # nvidia-smi samples go to a scratch file (NNMG_CLOCKS_DIR, default the temp directory)
        out = os.environ.get("NNMG_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out, f"nnmg_clocks_rank{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            p = [x.strip() for x in line.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx = max(mx, float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline_subprocess(n_fine: int, steps: int = 1, single_thread: bool = True) -> dict:
    """Time the CPU oracle's MG-PCG solve (setup excluded) in a fresh process, single-threaded
    or with the thread settings left to the libraries (all host cores)."""
    code = f"""
import json, time, os, sys
sys.path.insert(0, {ROOT!r})
from paper_2402_12947_gb300 import inputs
from oracle import hierarchy, mg
levels = max(2, ({n_fine}).bit_length() - 5)
meshes = inputs.config_c2(n_fine={n_fine}, levels=levels)
t0 = time.perf_counter()
H = hierarchy.build(meshes, 2)
setup = time.perf_counter() - t0
b = inputs.uniform_rhs(H.levels[0].n, 2)
times, its = [], []
for s in range({steps}):
    t0 = time.perf_counter()
    x, it, hist, tr = mg.pcg(H, b, {RTOL})
    times.append(time.perf_counter() - t0)
    its.append(it)
print(json.dumps({{"n": H.levels[0].n, "levels": levels, "setup_s": setup, "times": times, "iterations": its}}))
"""
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        if single_thread:
            env[k] = "1"
        else:
            env.pop(k, None)
    env.pop("CUDA_VISIBLE_DEVICES", None)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError("oracle baseline failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def export_for_oracle(H, b, path):
    """The FP64 hierarchy's operators, transfers, patches and eigenvalues (library numbering)
    and the right-hand side, for the oracle's V-cycle on the same data."""
    import numpy as np
    L = H.num_levels
    arrs = {"L": np.array(L), "b": b}
    for l in range(L):
        rp, ci, v = H.export_level(l)
        arrs.update({f"Ar{l}": rp, f"Ac{l}": ci, f"Av{l}": v})
        pt = H.export_patches(l)
        arrs[f"pp{l}"] = np.concatenate([[0], np.cumsum([len(p) for p in pt])]).astype(np.int64)
        arrs[f"pd{l}"] = np.concatenate(pt).astype(np.int32) if pt else np.zeros(0, np.int32)
        if l + 1 < L:
            rp, ci, v = H.export_transfer(l)
            arrs.update({f"Pr{l}": rp, f"Pc{l}": ci, f"Pv{l}": v})
    arrs["lam"] = np.array([H.eigs(l)[2] for l in range(L - 1)])
    np.savez(path, **arrs)


ORACLE_SOLVE = """
import json, sys, time
import numpy as np, scipy.sparse as sp
sys.path.insert(0, {root!r})
from oracle import hierarchy, mg
d = np.load({path!r})
L = int(d["L"])
n = [len(d[f"Ar{{l}}"]) - 1 for l in range(L)]
As = [sp.csr_matrix((d[f"Av{{l}}"], d[f"Ac{{l}}"], d[f"Ar{{l}}"]), shape=(n[l], n[l])) for l in range(L)]
Ps = [sp.csr_matrix((d[f"Pv{{l}}"], d[f"Pc{{l}}"], d[f"Pr{{l}}"]), shape=(n[l], n[l + 1])) for l in range(L - 1)]
pats = []
for l in range(L):
    pp, pd = d[f"pp{{l}}"], d[f"pd{{l}}"]
    pats.append([pd[pp[i]:pp[i + 1]] for i in range(len(pp) - 1)])
t0 = time.perf_counter()
H = hierarchy.from_matrices(As, Ps, pats, d["lam"])
t1 = time.perf_counter()
x, it, hist, tr = mg.pcg(H, d["b"], {rtol!r})
t2 = time.perf_counter()
np.save({out!r}, x)
print(json.dumps({{"iterations": it, "true_rel_residual": tr, "setup_s": t1 - t0, "solve_s": t2 - t1}}))
"""


def start_oracle_solve(H, b):
    """The oracle's MG-PCG on the exported FP64 hierarchy, started in the background
    (single-threaded SciPy); returns (process, output path, directory)."""
    tmp = tempfile.mkdtemp(prefix="nnmg_oracle_")
    path, out = os.path.join(tmp, "h.npz"), os.path.join(tmp, "x.npy")
    export_for_oracle(H, b, path)
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = "1"
    env.pop("CUDA_VISIBLE_DEVICES", None)
    code = ORACLE_SOLVE.format(root=ROOT, path=path, out=out, rtol=RTOL)
    proc = subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                            text=True, env=env)
    return proc, out, tmp


def finish_oracle_solve(handle, solutions, timeout=900):
    """Waits for the oracle; relative 2-norm errors of the GPU solutions against its solution."""
    import numpy as np
    import shutil
    proc, out, tmp = handle
    try:
        so, se = proc.communicate(timeout=timeout)
        if proc.returncode != 0:
            return {"error": se[-500:]}
        info = json.loads(so.strip().splitlines()[-1])
        xo = np.load(out)
        res = {k: float(np.linalg.norm(v - xo) / np.linalg.norm(xo)) for k, v in solutions.items()}
        res.update({"oracle_iterations": info["iterations"], "oracle_true_rel_residual": info["true_rel_residual"],
                    "oracle_solve_s": info["solve_s"],
                    "note": "relative 2-norm difference to the oracle's MG-PCG solution (FP64, rtol 1e-8) on the "
                            "exported operators; both solutions meet the residual test, so they may differ by up "
                            "to (||r_gpu|| + ||r_oracle||) / lambda_min(A)"})
        return res
    except subprocess.TimeoutExpired:
        proc.kill()
        return {"error": "oracle solve timed out"}
    finally:
        shutil.rmtree(tmp, ignore_errors=True)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    d = cpu_baseline_subprocess(SAMPLE_N, steps=args.warmup + args.steps, single_thread=False)
    t = d["times"][args.warmup:]
    mean = sum(t) / len(t)
    value = d["n"] / mean
    sample = (f"oracle MG-PCG solve (setup excluded) on the same workload family at {SAMPLE_N}^2 "
              f"({d['n']} DoFs, {d['levels']} levels), {d['iterations'][-1]} iterations")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "DoFs/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": "DoFs/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample + " (thread settings left to NumPy/SciPy on all host cores; the sparse "
                                                "products run on one of them)", "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": "DoFs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def solve_bytes_per_iteration(H, nnmg, vbytes, cheb_degree=2, nu=1):
    """Algorithmic bytes of one MG-PCG iteration (each matrix once per pass, each vector once
    per pass, int32 indices, value size vbytes in the V-cycle, FP64 in CG), for the passes the
    method needs: per smoothed level and side nu smoother applications of (S_c, Chebyshev,
    S_c) where the first pre-smoothing Chebyshev step from the zero iterate needs no SpMV, one
    residual + restriction, one prolongation, the coarsest dense solve, and the CG update.
    S_c reads each patch's dense FP64 inverse once per application."""
    import numpy as np
    L = H.num_levels
    s, tot = vbytes, 0.0
    for l in range(L - 1):
        n, nc = H.num_dofs(l), H.num_dofs(l + 1)
        nnz = int(nnmg.lib.mg_level_nnz(H._h, l))
        nnz_p = int(nnmg.lib.mg_transfer_nnz(H._h, l))
        a_pass = nnz * (s + 4) + n * 6 * s
        sweeps = 2 * nu * cheb_degree - 1                 # A-passes of the smoother per cycle
        tot += sweeps * a_pass + n * 4 * s                # + the zero-iterate first step
        tot += nnz * (s + 4) + n * 3 * s + nnz_p * (s + 4) + nc * 2 * s + n * s   # residual + restriction
        tot += nnz_p * (s + 4) + n * 2 * s + nc * s                               # prolongation
        sizes = np.array([len(p) for p in H.export_patches(l)], dtype=np.float64)
        tot += 4 * nu * 8.0 * float((sizes ** 2).sum())                          # S_c applications
    nL = H.num_dofs(L - 1)
    tot += 8.0 * nL * nL
    n0 = H.num_dofs(0)
    tot += int(nnmg.lib.mg_level_nnz(H._h, 0)) * 12 + n0 * 16                 # CG: q = A p (FP64)
    tot += n0 * (9 * 8 + 4 * s)                                               # CG vector updates
    return tot


def run_ours(args):
    """C2 (the headline), C3 or C4: mixed and FP64 MG-PCG solves to rtol 1e-8."""
    import numpy as np
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2402_12947_gb300 import build, inputs, nnmg, replicas
    build.build()

    workload, degree = WORKLOADS[args.workload]
    if args.global_smoother == "sgs":
        workload = workload.replace("Chebyshev(2)", "multicolour SGS")
    if args.workload == "c2":
        meshes = inputs.config_c2(n_fine=args.n_fine, levels=args.levels, seed=replicas.mesh_seed(2, rank))
    elif args.workload == "c3":
        meshes = inputs.config_c3(seed=replicas.mesh_seed(3, rank))
    else:
        meshes = inputs.config_c4(seed=replicas.mesh_seed(4, rank))
    both = args.precision == "both"
    t0 = time.perf_counter()
    graph = 0 if args.no_graph else 1
    opts = dict(use_graph=graph, global_smoother=args.global_smoother)
    if args.reorder is not None:
        opts["reorder"] = {"none": 0, "rcm": 1, "spatial": 2, "spatial-coarse": 3}[args.reorder]
    sgs = args.global_smoother == "sgs"
    H64 = nnmg.Hierarchy.from_meshes(meshes, degree, 0.1, **opts) if both else None
    setup64 = time.perf_counter() - t0
    lam = [H64.eigs(l)[2] for l in range(H64.num_levels - 1)] if both and not sgs else None
    t0 = time.perf_counter()
    H32 = nnmg.Hierarchy.from_meshes(meshes, degree, 0.1, precision="mixed", lambda_override=lam, **opts)
    setup32 = time.perf_counter() - t0
    n = H32.num_dofs(0)
    b_host = inputs.uniform_rhs(n, replicas.rhs_seed(2, rank))
    b = torch.from_numpy(b_host).cuda()

    x = torch.zeros_like(b)
    stream = torch.cuda.current_stream()

    barrier = replicas.barrier

    def timed(H, steps, warmup):
        for _ in range(warmup):
            info = H.solve(b, x, rtol=RTOL, maxit=500)
        per = []
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            s0 = torch.cuda.Event(enable_timing=True)
            s1 = torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            info = H.solve(b, x, rtol=RTOL, maxit=500)
            s1.record(stream)
            per.append((s0, s1))
        e1.record(stream)
        barrier()
        total = e0.elapsed_time(e1) / steps
        # latency percentiles over at least 30 solves (extra solves after the timed region)
        for _ in range(max(0, 30 - steps)):
            s0 = torch.cuda.Event(enable_timing=True)
            s1 = torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            H.solve(b, x, rtol=RTOL, maxit=500)
            s1.record(stream)
            per.append((s0, s1))
        torch.cuda.synchronize()
        lat = sorted(a.elapsed_time(c) for a, c in per)
        return total, lat, info

    clocks = ClockSampler(local)
    clocks.start()
    ms32, lat32, info32 = timed(H32, args.steps, max(3, args.warmup))
    clk = clocks.stop()
    x32 = x.clone()
    ms64, lat64, info64 = timed(H64, args.steps, max(3, args.warmup)) if both else (float("nan"), [float("nan")], {})
    # error of the mixed-precision result against the FP64 result (both solved to rtol)
    err_vs_fp64 = float((x32 - x).norm() / x.norm()) if both else None
    ms32, ms64 = replicas.max_over_ranks([ms32, ms64], device="cuda")

    # end to end through the C ABI with host buffers (copies inside the timed region)
    pin_b = torch.from_numpy(b_host).pin_memory()
    pin_x = torch.empty_like(pin_b).pin_memory()
    H32.solve_host(pin_b.numpy(), rtol=RTOL, out=pin_x.numpy())
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        H32.solve_host(pin_b.numpy(), rtol=RTOL, out=pin_x.numpy())
    barrier()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    e2e_ms = replicas.max_over_ranks([e2e_ms], device="cuda")[0]

    x64 = x.clone()
    # the dominant kernel: fine-level fused Chebyshev SpMV of the FP32 V-cycle
    kms, kbytes = H32.time_smoother_kernel(reps=50)
    # the second: the FP64 CG product q = A p with its p.q reduction
    ap_ms, ap_bytes = H32.time_cg_product(reps=50)
    # the local correction's solve launch on the fine level (FP64-ALU bound where FP64) and the
    # device's FP64 FMA rate
    fp64_fma = nnmg.measure_fp64_fma()
    ps32 = H32.time_patch_solve(0, reps=20)
    ps64 = H64.time_patch_solve(0, reps=20) if both else None
    kms64, kbytes64 = H64.time_smoother_kernel(reps=50) if both else (float("nan"), float("nan"))
    peak, peak_src = measured_peak()
    traffic, rev = profiled_traffic()
    if rev != KERNEL_REV or sgs:
        traffic = None
    per_vc, per_it = H32.launch_counts()
    nnz0 = int(nnmg.lib.mg_level_nnz(H32._h, 0))
    launches = per_it * info32["iterations"] + 4   # ABI gather/scatter and the true-residual check
    if rank != 0:
        return 0
    cpu = None
    if not args.no_cpu_baseline and args.workload == "c2":
        ncores = os.cpu_count()
        d1 = cpu_baseline_subprocess(SAMPLE_N, steps=1, single_thread=True)
        dn = cpu_baseline_subprocess(SAMPLE_N, steps=1, single_thread=False)
        sample = (f"oracle MG-PCG solve (setup excluded) on the same family at {SAMPLE_N}^2 ({dn['n']} DoFs, "
                  f"{dn['levels']} levels, {dn['iterations'][0]} iterations)")
        cpu = {"value": dn["n"] / dn["times"][0], "unit": "DoFs/s", "cores": ncores, "kind": "oracle",
               "sample": sample + f", {dn['times'][0]:.1f} s with the thread settings left to NumPy/SciPy on "
                         f"all {ncores} host cores (the sparse products run on one of them, BLAS on all)",
               "cpu_model": cpu_model(),
               "single_thread": {"value": d1["n"] / d1["times"][0], "cores": 1,
                                 "sample": sample + f", {d1['times'][0]:.1f} s single-threaded"}}
    serve = None if (args.no_serve or world > 1 or args.workload != "c2") else serve_bounded(nnmg, inputs)
    batch = None if (args.no_serve or world > 1 or args.workload != "c2") else batch_bounded(nnmg, inputs)
    # the oracle solves the same problem on the exported operators (after every GPU timing)
    oracle_check = None
    if both and not args.no_oracle_check and not sgs:
        oracle_check = finish_oracle_solve(start_oracle_solve(H64, b_host),
                                           {"mixed": x32.cpu().numpy(), "fp64": x64.cpu().numpy()})
    value = replicas.job_throughput(n, world, ms32)
    bpi32 = solve_bytes_per_iteration(H32, nnmg, 4)
    ideal32 = bpi32 * info32["iterations"] / (peak * 1e9) * 1e3
    solve_roof = {"bytes_per_iteration": bpi32, "iterations": info32["iterations"], "ideal_ms": ideal32,
                  "measured_ms": ms32, "frac": ideal32 / ms32, "peak_gbs": peak,
                  "note": "every pass of a CG iteration at the measured copy peak vs the measured solve"}
    if both:
        bpi64 = solve_bytes_per_iteration(H64, nnmg, 8)
        ideal64 = bpi64 * info64["iterations"] / (peak * 1e9) * 1e3
        solve_roof["fp64"] = {"bytes_per_iteration": bpi64, "ideal_ms": ideal64, "measured_ms": ms64,
                              "frac": ideal64 / ms64}
    order = args.reorder or "library"
    kernel_name = (f"fine-level multicolour SGS application, FP32 (k_gs, one launch per colour and sweep, "
                   f"autotuned layouts, {order} order)" if sgs else
                   f"fine-level fused Chebyshev SpMV, FP32 (k_cheb, autotuned layout, {order} order, 16-bit "
                   f"column offsets where a slice spans < 2^16 columns)")
    line = {
        "metric": METRIC, "value": value, "unit": "DoFs/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms32, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": workload, "parallelism": f"replicas x{world}", "rtol": RTOL,
                   "launch": "per-kernel launches" if args.no_graph else "one CUDA graph per solve (conditional while)",
                   "l2": f"inputs larger than L2 (A_0 alone {12e-9 * nnz0:.2f} GB FP64 / {8e-9 * nnz0:.2f} GB FP32 "
                         "with 32-bit indices)",
                   "dofs_per_gpu": n, "levels": H32.num_levels, "global_smoother": args.global_smoother,
                   "internal_order": order},
        "iterations": {"mixed": info32["iterations"], "fp64": info64.get("iterations")},
        "p50_ms": lat32[len(lat32) // 2], "p99_ms": lat32[min(len(lat32) - 1, int(0.99 * len(lat32)))],
        "fp64": {"value": replicas.job_throughput(n, world, ms64), "ms_per_step": ms64, "iterations": info64.get("iterations"),
                 "p50_ms": lat64[len(lat64) // 2], "p99_ms": lat64[min(len(lat64) - 1, int(0.99 * len(lat64)))],
                 "true_rel_residual": info64.get("true_rel_residual")} if both else None,
        "true_rel_residual": info32["true_rel_residual"],
        "mixed_rel_error_vs_fp64": err_vs_fp64,
        "solve_roofline": solve_roof,
        "e2e": {"value": replicas.job_throughput(n, world, e2e_ms), "unit": "DoFs/s", "h2d_bytes_per_step": 8 * n,
                "d2h_bytes_per_step": 8 * n},
        "gpu_launches": launches * args.steps,
        "roofline": {"bound": "hbm", "achieved": kbytes / (kms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": kbytes / (kms * 1e-3) / 1e9 / peak, "traffic": traffic,
                     "kernel": kernel_name,
                     "bytes_per_launch": kbytes, "ms_per_launch": kms, "peak_source": peak_src,
                     "fp64_kernel": {"achieved": kbytes64 / (kms64 * 1e-3) / 1e9, "ms_per_launch": kms64,
                                     "bytes_per_launch": kbytes64},
                     "cg_product": {"kernel": "FP64 CG product q = A_0 p with its p.q reduction (k_ap + k_finish)",
                                    "bound": "hbm", "achieved": ap_bytes / (ap_ms * 1e-3) / 1e9, "peak": peak,
                                    "frac": ap_bytes / (ap_ms * 1e-3) / 1e9 / peak, "ms_per_launch": ap_ms,
                                    "bytes_per_launch": ap_bytes}},
        "patch_solve": {
            "kernel": "S_c solve launch on level 0 (k_patch_solve: lane per row, columns split over 8 warps)",
            "bound": "alu (FP64 FMA) where the inverses are FP64", "fp64_fma_per_s_measured": fp64_fma,
            "mixed": {"ms_per_launch": ps32[0], "fma_fp64": ps32[1], "fma_fp32": ps32[2], "bytes": ps32[3],
                      "frac_fp64_alu": (ps32[1] / (ps32[0] * 1e-3)) / fp64_fma if ps32[0] > 0 else None,
                      "hbm_gbs": ps32[3] / (ps32[0] * 1e-3) / 1e9 if ps32[0] > 0 else None},
            "fp64": {"ms_per_launch": ps64[0], "fma_fp64": ps64[1], "bytes": ps64[3],
                     "frac_fp64_alu": (ps64[1] / (ps64[0] * 1e-3)) / fp64_fma if ps64[0] > 0 else None,
                     "hbm_gbs": ps64[3] / (ps64[0] * 1e-3) / 1e9 if ps64[0] > 0 else None} if ps64 else None},
        "rel_error_vs_oracle": oracle_check,
        "serve": serve,
        "batch": batch,
        "cpu_baseline": cpu,
        "clocks": clk,
        "setup_s": {"fp64": setup64 if both else None, "mixed": setup32},
        "device_bytes": {"fp64": H64.device_bytes() if both else None, "mixed": H32.device_bytes()},
    }
    print(json.dumps(line), flush=True)
    if H64 is not None:
        H64.close()
    H32.close()
    return 0


def serve_stream(n_requests: int, seed: int = 5):
    """The seeded request stream: (meshes, degree, rhs, label) per request."""
    import numpy as np
    from paper_2402_12947_gb300 import inputs
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_requests):
        meshes, degree, label = inputs.serving_request(rng, seed * 100000 + k)
        n = meshes[0].n
        dim = meshes[0].dim
        nfree = (n - 1) ** dim if degree == 1 else (2 * n - 1) ** dim
        out.append((meshes, degree, inputs.uniform_rhs(nfree, seed * 100000 + k), label))
    return out


def serve_once(nnmg, stream, prec, rate, budget, max_active=16, setup_threads=12, arrival_seed=7):
    """One pass of a request stream through the continuous-batching server: Poisson arrivals
    at `rate` per second; per-request latency (submit to done) and device time (admission to
    done), throughput over the wall time of the pass."""
    import numpy as np
    arrivals = np.cumsum(np.random.default_rng(arrival_seed).exponential(1.0 / rate, len(stream)))
    with nnmg.Server(hbm_budget_bytes=budget, max_active=max_active, setup_threads=setup_threads) as srv:
        t0 = time.perf_counter()
        ids = []
        for (meshes, degree, b, _), ta in zip(stream, arrivals):
            now = time.perf_counter() - t0
            if ta > now:
                time.sleep(ta - now)
            ids.append(srv.submit(meshes, degree, b=b, rtol=RTOL, precision=prec))
        res = [srv.wait(i, timeout=3600) for i in ids]
        wall = time.perf_counter() - t0
        for i, r in zip(ids, res):
            srv.fetch(i, r["n"])
        st = srv.stats()
    lat = np.array([r["t_total_ms"] for r in res])
    dev = np.array([r["t_device_ms"] for r in res])
    sol = np.array([r["t_solve_ms"] for r in res])
    ok = [r for r in res if r["status"] == 0]
    dofs = sum(r["n"] for r in ok)
    return {"throughput_dofs_per_s": dofs / wall, "requests_per_s": len(ok) / wall,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "p50_device_ms": float(np.percentile(dev, 50)), "p99_device_ms": float(np.percentile(dev, 99)),
            "mean_device_ms": float(dev.mean()),
            "p50_solve_ms": float(np.percentile(sol, 50)), "p99_solve_ms": float(np.percentile(sol, 99)),
            "sum_solve_ms": float(sol.sum()),
            "failed": len(res) - len(ok), "peak_active": st["peak_active"],
            "peak_bytes": st["peak_bytes"],
            "max_true_rel_residual": max(r["true_rel_residual"] for r in ok) if ok else None,
            "mean_iterations": float(np.mean([r["iterations"] for r in ok])) if ok else None}


def batch_bounded(nnmg, inputs, n_problems=16, reps=5):
    """The default line's batch measurement: n_problems requests of the serving family (2D
    P1/P2 32^2-128^2, 3D P1 16^3-32^3, 0-16 clusters, random right-hand sides, rtol 1e-8) set
    up once, then solved together by mg_solve_batch (each problem's solve graph on its own
    stream, overlapping on the device), mixed precision vs FP64 on the same GPU: GPU time per
    batch (CUDA events on the calling stream, best of reps after one warm-up batch) and the
    largest true relative residual."""
    import numpy as np
    import torch
    rng = np.random.default_rng(5)
    specs, k = [], 0
    while len(specs) < n_problems:
        m, degree, label = inputs.serving_request(rng, 1000 + k)
        k += 1
        if (m[0].dim == 2 and m[0].n <= 128) or (m[0].dim == 3 and m[0].n <= 32):
            specs.append((m, degree, label))
    out = {"problems": n_problems, "mix": "2D P1/P2 32^2-128^2 and 3D P1 16^3-32^3, 0-16 clusters, RHS U[-1,1], "
           "rtol 1e-8", "launch": "mg_solve_batch: one solve graph per problem on its own stream"}
    for prec in ("mixed", "fp64"):
        hs = [nnmg.Hierarchy.from_meshes(m, d, 0.1, precision=prec) for m, d, _ in specs]
        try:
            bs = [torch.from_numpy(inputs.uniform_rhs(h.num_dofs(0), 3)).cuda() for h in hs]
            xs = [torch.zeros_like(v) for v in bs]
            infos = nnmg.solve_batch(hs, bs, xs, rtol=RTOL)
            torch.cuda.synchronize()
            best = None
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                infos = nnmg.solve_batch(hs, bs, xs, rtol=RTOL)
                e1.record()
                torch.cuda.synchronize()
                t = e0.elapsed_time(e1)
                best = t if best is None else min(best, t)
            dofs = sum(h.num_dofs(0) for h in hs)
            out[prec] = {"ms_per_batch": best, "dofs_per_s": dofs / (best * 1e-3), "dofs": dofs,
                         "iterations": [i["iterations"] for i in infos],
                         "max_true_rel_residual": max(i["true_rel_residual"] for i in infos),
                         "converged": all(i["converged"] for i in infos)}
        finally:
            for h in hs:
                h.close()
    return out


def serve_bounded(nnmg, inputs, n_requests=64, rate=32.0):
    """The default line's serving measurement: a bounded seeded stream of the serving family
    (2D P1/P2 32^2-256^2, 3D P1 16^3-32^3, 0-16 clusters each, random right-hand sides,
    rtol 1e-8) at one Poisson arrival rate, mixed precision and FP64 on the same GPU."""
    import numpy as np
    import torch
    rng = np.random.default_rng(11)
    stream, k = [], 0
    while len(stream) < n_requests:
        meshes, degree, label = inputs.serving_request(rng, 700000 + k)
        k += 1
        n = meshes[0].n
        if (meshes[0].dim == 2 and n > 256) or (meshes[0].dim == 3 and n > 32):
            continue
        nfree = (n - 1) ** meshes[0].dim if degree == 1 else (2 * n - 1) ** meshes[0].dim
        stream.append((meshes, degree, inputs.uniform_rhs(nfree, 700000 + k), label))
    free, _ = torch.cuda.mem_get_info()
    budget = int(0.25 * free)
    out = {"requests": n_requests, "arrival_rate_per_s": rate, "hbm_budget_bytes": budget, "max_active": 16,
           "mix": "2D P1/P2 32^2-256^2 and 3D P1 16^3-32^3, 0-16 clusters, RHS U[-1,1], rtol 1e-8",
           "dofs_total": int(sum((m[0].n - 1) ** m[0].dim if d == 1 else (2 * m[0].n - 1) ** m[0].dim
                                 for m, d, _, _ in stream))}
    for prec in ("mixed", "fp64"):
        out[prec] = serve_once(nnmg, stream, prec, rate, budget)
    return out


def run_serve(args):
    """Continuous-batching server on the mixed stream at several Poisson arrival rates."""
    import torch
    from paper_2402_12947_gb300 import build, nnmg
    build.build()
    torch.cuda.set_device(0)
    stream = serve_stream(args.requests)
    free, total = torch.cuda.mem_get_info()
    budget = int(0.5 * free)
    results = {}
    for prec in ("mixed", "fp64"):
        for rate in [float(r) for r in args.rates.split(",")]:
            results[f"{prec}@{rate:g}/s"] = serve_once(nnmg, stream, prec, rate, budget)
    best = max(results.values(), key=lambda d: d["throughput_dofs_per_s"])
    line = {"metric": METRIC, "value": best["throughput_dofs_per_s"], "unit": "DoFs/s", "n_gpus": 1,
            "steps": args.requests, "warmup": 0, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"serving: {args.requests} seeded requests, Poisson arrivals, mixed 2D P1/P2 "
                                   "32^2-512^2 and 3D P1 16^3-64^3 with 0-16 clusters, rtol 1e-8",
                       "hbm_budget_bytes": budget, "max_active": 16},
            "serve": results}
    print(json.dumps(line), flush=True)
    return 0


def run_persistent(args):
    """The persistent cooperative path against the default launches: (1) the C2 solve with the
    cycle from the first level of at most small_level_dofs DoFs down in one persistent launch
    per cycle, for several split points (0 = off), with the V-cycle time from each level;
    (2) 16 small requests of the serving family solved one by one and as one batch, with CUDA
    graphs on their own streams (small_level_dofs = 0) and as one persistent launch
    (small_level_dofs >= n_0)."""
    import numpy as np
    import torch
    from paper_2402_12947_gb300 import build
    build.build()
    from paper_2402_12947_gb300 import inputs, nnmg
    torch.cuda.set_device(0)

    def timed(f, reps):
        f()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            f()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {"workload": "persistent", "c2": [], "batch": {}}
    meshes = inputs.config_c2()
    b = torch.from_numpy(inputs.uniform_rhs(2047 ** 2, 2)).cuda()
    lam = None
    for thr in (0, 20000, 100000):
        H = nnmg.Hierarchy.from_meshes(meshes, 2, 0.1, precision="mixed", small_level_dofs=thr, lambda_override=lam)
        if lam is None:
            lam = [H.eigs(l)[2] for l in range(H.num_levels - 1)]
        x = torch.zeros_like(b)
        info = H.solve(b, x, rtol=RTOL)
        ms = timed(lambda: H.solve(b, x, rtol=RTOL), 5)
        out["c2"].append({"small_level_dofs": thr, "ms_per_solve": ms, "iterations": info["iterations"],
                          "vcycle_us_from_level": [round(H.time_vcycle(l, reps=30) * 1e3, 1)
                                                   for l in range(H.num_levels)]})
        H.close()
    rng = np.random.default_rng(5)
    specs, k = [], 0
    while len(specs) < 16:
        m, degree, label = inputs.serving_request(rng, 1000 + k)
        k += 1
        if (m[0].dim == 2 and m[0].n <= 128) or (m[0].dim == 3 and m[0].n <= 32):
            specs.append((m, degree, label))
    for mode, thr in (("graphs", 0), ("persistent", 1 << 30)):
        hs = [nnmg.Hierarchy.from_meshes(m, d, 0.1, precision="mixed", small_level_dofs=thr) for m, d, _ in specs]
        bs = [torch.from_numpy(inputs.uniform_rhs(h.num_dofs(0), 3)).cuda() for h in hs]
        xs = [torch.zeros_like(v) for v in bs]
        seq = timed(lambda: [h.solve(v, x, rtol=RTOL) for h, v, x in zip(hs, bs, xs)], 3)
        bat = timed(lambda: nnmg.solve_batch(hs, bs, xs, rtol=RTOL), 3)
        out["batch"][mode] = {"sequential_ms": seq, "batch_ms": bat}
        for h in hs:
            h.close()
    out["batch"]["requests"] = [lab for _, _, lab in specs]
    print(json.dumps(out), flush=True)
    return 0


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def run_paper(args):
    """Sec. 6 comparisons on synthetic hierarchies (the paper's meshes are not available):
    CG iterations (one V-cycle per iteration) and stationary V-cycles to 1e-10 for the clean
    reference, Case A (clusters on every level) and Case B (every level but the finest),
    without correction, with correction and the unadjusted lambda_max, and with correction
    and the adjusted lambda_max (the layout of Table number_struct); and the residual
    history of a two-level cycle on f = 0 from u0 = sin(10 pi x) sin(10 pi y) (Sec. 6.1.1)."""
    import numpy as np
    import torch
    from paper_2402_12947_gb300 import build, inputs, nnmg
    build.build()
    torch.cuda.set_device(0)
    problems = [("2D P1 256^2", 2, 1, 256, 4), ("2D P2 256^2", 2, 2, 256, 4),
                ("3D P1 32^3", 3, 1, 32, 3), ("3D P2 16^3", 3, 2, 16, 3)]
    table = {}
    for label, dim, degree, n, levels in problems:
        amp = 0.2 if dim == 2 else 0.15
        kw = dict(n_clusters=8 if dim == 2 else 6, moves_per_cluster=(2, 4), kinds=("cap",), eps=1e-3)
        meshes = {"reference": inputs.hierarchy_meshes(dim, n, levels, amp, 11),
                  "A": inputs.hierarchy_meshes(dim, n, levels, amp, 11, cluster_levels=tuple(range(levels)), **kw),
                  "B": inputs.hierarchy_meshes(dim, n, levels, amp, 11, cluster_levels=tuple(range(1, levels)), **kw)}
        nfree = (n - 1) ** dim if degree == 1 else (2 * n - 1) ** dim
        b = torch.from_numpy(inputs.uniform_rhs(nfree, 3)).cuda()
        variants = {"reference": ("reference", dict())}
        for case in ("A", "B"):
            variants[f"{case} without correction"] = (case, dict(smoother="global", adjusted_lambda=0))
            variants[f"{case} correction, unadjusted lambda"] = (case, dict(adjusted_lambda=0))
            variants[f"{case} correction, adjusted lambda"] = (case, dict(adjusted_lambda=1))
        row = {}
        for name, (case, opt) in variants.items():
            with nnmg.Hierarchy.from_meshes(meshes[case], degree, 0.1, **opt) as H:
                x = torch.zeros_like(b)
                cg = H.solve(b, x, rtol=1e-10, maxit=300, raise_on_fail=False)
                x.zero_()
                st = H.solve_stationary(b, x, rtol=1e-10, maxit=300)
                row[name] = {"cg": cg["iterations"] if cg["converged"] else f">{cg['iterations']}",
                             "stationary": st["iterations"] if st["converged"] else f">{st['iterations']}",
                             "lambda_used_L0": H.eigs(0)[2]}
        table[label] = row
    # residual history, two levels (Sec. 6.1.1 shape): 64^2 fine with one cluster, 32^2 coarse
    hist = {}
    base = inputs.hierarchy_meshes(2, 64, 2, 0.2, 21)
    bad = inputs.hierarchy_meshes(2, 64, 2, 0.2, 21, cluster_levels=(0,), n_clusters=1, moves_per_cluster=(3, 3),
                                  kinds=("cap",), eps=1e-3)
    for name, ms, opt in (("high quality", base, dict()), ("low quality, no correction", bad,
                          dict(smoother="global", adjusted_lambda=0)), ("low quality, correction", bad, dict())):
        with nnmg.Hierarchy.from_meshes(ms, 1, 0.1, **opt) as H:
            pts = H.dof_coords(0, 2)
            x = torch.from_numpy(np.sin(10 * np.pi * pts[:, 0]) * np.sin(10 * np.pi * pts[:, 1])).cuda()
            zero = torch.zeros_like(x)
            ax = torch.zeros_like(x)
            H.apply_A(0, x, ax)
            r0 = float(ax.norm())
            h = []
            for _ in range(12):
                H.vcycle(zero, x)
                H.apply_A(0, x, ax)
                h.append(float(ax.norm()) / r0)
            hist[name] = h
    print(json.dumps({"workload": "paper", "iterations_to_1e-10": table, "residual_history_two_level": hist}),
          flush=True)
    return 0


def run_lattice(args):
    """Sec. 6.3 elasticity comparison on the synthetic clamped lattice (four non-nested
    levels, 1/h = 13, 6, 3, 2; E = 6.9e10, nu = 0.33; traction (1e3, 0, 0) on x = 6): MG-PCG
    iterations to rtol 1e-8 with the multicolour SGS global smoother applied twice before
    and after the coarse correction, for the clean reference, Case A (sliver clusters on
    every level) and Case B (every level but the finest), without and with the local
    correction; and the solve time and DoFs/s of the corrected Case A hierarchy (FP64 and
    mixed precision)."""
    import torch
    from paper_2402_12947_gb300 import build, inputs, nnmg
    build.build()
    torch.cuda.set_device(0)
    ns = (13, 6, 3, 2)
    meshes = {"reference": inputs.config_lattice(ns=ns, n_clusters=0),
              "A": inputs.config_lattice(ns=ns, n_clusters=16),
              "B": inputs.config_lattice(ns=ns, n_clusters=16, cluster_levels=(1, 2, 3))}
    out = {}
    for degree in (1, 2):
        row = {}
        for name, case, opt in (("reference", "reference", {}), ("A without correction", "A", dict(smoother="global")),
                                ("A with correction", "A", {}), ("B without correction", "B", dict(smoother="global")),
                                ("B with correction", "B", {})):
            ms, masks = meshes[case]
            t0 = time.perf_counter()
            with nnmg.Hierarchy.from_meshes(ms, degree, 0.1, pde="elasticity", dirichlet_masks=masks,
                                            global_smoother="sgs", nu=2, **opt) as H:
                setup = time.perf_counter() - t0
                b = torch.from_numpy(H.load_traction(0, 6.0, [1e3, 0.0, 0.0])).cuda()
                x = torch.zeros_like(b)
                info = H.solve(b, x, rtol=RTOL, maxit=500, raise_on_fail=False)
                entry = {"dofs": H.num_dofs(0), "iterations": info["iterations"], "converged": info["converged"],
                         "true_rel_residual": info["true_rel_residual"], "setup_s": round(setup, 2)}
                if name == "A with correction":
                    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    for _ in range(2):
                        x.zero_()
                        H.solve(b, x, rtol=RTOL, maxit=500)
                    ev0.record()
                    for _ in range(5):
                        x.zero_()
                        H.solve(b, x, rtol=RTOL, maxit=500)
                    ev1.record()
                    torch.cuda.synchronize()
                    ms_solve = ev0.elapsed_time(ev1) / 5
                    entry.update(ms_per_solve=ms_solve, dofs_per_s=H.num_dofs(0) / (ms_solve * 1e-3))
                row[name] = entry
            if name == "A with correction":
                with nnmg.Hierarchy.from_meshes(ms, degree, 0.1, pde="elasticity", dirichlet_masks=masks,
                                                global_smoother="sgs", nu=2, precision="mixed") as H:
                    x = torch.zeros_like(b)
                    info = H.solve(b, x, rtol=RTOL, maxit=500, raise_on_fail=False)
                    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    ev0.record()
                    for _ in range(5):
                        x.zero_()
                        H.solve(b, x, rtol=RTOL, maxit=500)
                    ev1.record()
                    torch.cuda.synchronize()
                    ms_solve = ev0.elapsed_time(ev1) / 5
                    row["A with correction, mixed"] = {"iterations": info["iterations"],
                                                       "true_rel_residual": info["true_rel_residual"],
                                                       "ms_per_solve": ms_solve,
                                                       "dofs_per_s": H.num_dofs(0) / (ms_solve * 1e-3)}
        out[f"P{degree}"] = row
    print(json.dumps({"workload": "lattice elasticity (Sec. 6.3)", "rtol": RTOL, "results": out}), flush=True)
    return 0


def run_dumbbell(args):
    """The paper's four-way comparison (Table number_struct: Case A / Case B x no correction /
    correction with unadjusted lambda_max / correction with adjusted lambda_max, against the
    clean reference) on the synthetic dumbbell-like elasticity structure: Chebyshev(2) global
    smoother applied twice before and after the coarse correction, MG-PCG to 1e-10, body force
    (0, 0, -1e3), traction (1e3, 0, 0) on x = 6, clamped at x = 0."""
    import torch
    from paper_2402_12947_gb300 import build, inputs, nnmg
    build.build()
    torch.cuda.set_device(0)
    out = {}
    for degree, ns in ((1, (24, 8, 4, 2)), (2, (16, 8, 4, 2))):
        meshes = {"reference": inputs.config_dumbbell(ns=ns, n_clusters=0),
                  "A": inputs.config_dumbbell(ns=ns),
                  "B": inputs.config_dumbbell(ns=ns, cluster_levels=tuple(range(1, len(ns))))}
        variants = [("reference", "reference", {})]
        for case in ("A", "B"):
            variants += [(f"{case} without correction", case, dict(smoother="global", adjusted_lambda=0)),
                         (f"{case} correction, unadjusted lambda", case, dict(adjusted_lambda=0)),
                         (f"{case} correction, adjusted lambda", case, dict(adjusted_lambda=1))]
        row = {}
        for name, case, opt in variants:
            ms, masks = meshes[case]
            with nnmg.Hierarchy.from_meshes(ms, degree, 0.1, pde="elasticity", dirichlet_masks=masks, nu=2,
                                            **opt) as H:
                b = H.load_body([0.0, 0.0, -1e3]) + H.load_traction(0, 6.0, [1e3, 0.0, 0.0])
                bt = torch.from_numpy(b).cuda()
                x = torch.zeros_like(bt)
                info = H.solve(bt, x, rtol=1e-10, maxit=300, raise_on_fail=False)
                row[name] = {"iterations": info["iterations"] if info["converged"] else f">{info['iterations']}",
                             "dofs": H.num_dofs(0), "lambda_used_L0": H.eigs(0)[2],
                             "true_rel_residual": info["true_rel_residual"]}
        out[f"P{degree}"] = row
    print(json.dumps({"workload": "dumbbell-like elasticity (Table number_struct layout)", "rtol": 1e-10,
                      "results": out}), flush=True)
    return 0


def main():
    args = parse()
    if args.workload == "persistent":
        return run_persistent(args)
    if args.workload == "paper":
        return run_paper(args)
    if args.workload == "lattice":
        return run_lattice(args)
    if args.workload == "dumbbell":
        return run_dumbbell(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serve":
        return run_serve(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
