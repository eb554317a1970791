"""Benchmark of the matrix-free Galerkin single-layer apply on GB300.

One step = one gyps_sl_apply of the whole operator (interpolation W_y Phi X,
the dense kernel product G u, the projection Phi^T W_x v / 4pi and the CSR
singular correction C X) on the workload sphere10242_k16_q7: icosphere with
20480 triangles (10242 vertices), 7-point rule (143360 points), k = 16, one
right-hand side, FP32 kernel products and FP64 correction.

Metric: GPairs/s = Nq^2 (target point, source point) pairs per apply divided
by the apply's device time.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gyps|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

WORKLOAD = "sphere10242_k16_q7"
METRIC = "GPairs/s single-layer apply (%FP32+SFU roof); GMRES time-to-1e-6 vs plain FP64"
UNIT = "GPairs/s"
MUFU_PER_PAIR = 3          # rsqrt, sin, cos
MUFU_PER_CLK_PER_SM = 16   # special-function results per clock per SM
PROFILE = os.path.join(ROOT, "profiles", "far32_sphere10242_k16_q7.md")
FAR_SRC = os.path.join(ROOT, "paper_1804_00995_gb300", "csrc", "far.cu")
FAR_TILE_SRC = os.path.join(ROOT, "paper_1804_00995_gb300", "csrc", "far_tile.cuh")


def read_text(path):
    with open(path) as f:
        return f.read()


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="gyps", choices=["gyps", "reference"])
    p.add_argument("--workload", default=WORKLOAD,
                   choices=[WORKLOAD, "batch12_r64", "precond_ellipsoids", "sphere163842_k64_q3_r16",
                            "assemble_sphere10242", "field_sphere10242_k16", "dl_sphere10242_k16_q7",
                            "efie_sphere10242_k8_q3", "hmat_sphere163842_k64_q3_r16"])
    p.add_argument("--precond-meshes", type=int, default=125, help="training meshes (16 solves each)")
    p.add_argument("--precond-steps", type=int, default=3000)
    p.add_argument("--precond-test", type=int, default=50, help="held-out meshes (4 plane waves each)")
    p.add_argument("--precond-krylov-steps", default="5,15,40",
                   help="GMRES steps m of the iterates whose errors make the Krylov pairs")
    p.add_argument("--precond-data", default="krylov", choices=["noise", "krylov", "both"],
                   help="training pairs: white-noise residuals, Krylov-iteration errors, or both")
    p.add_argument("--save-precond", default="", help="write the trained network here")
    p.add_argument("--nrhs", type=int, default=1, help="right-hand sides per apply (the workload has 1)")
    p.add_argument("--prec", default="fp32", choices=["fp32", "tc_bf16x3", "auto"],
                   help="kernel-product arithmetic (tc_bf16x3: tensor cores, needs nrhs >= 16)")
    p.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle baseline sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--solve", action=argparse.BooleanOptionalAction, default=None,
                   help="also time GMRES to 1e-6 (FP32 / tensor-core operator, double-float true-residual "
                        "checks); on by default for the default workload, off for the others")
    p.add_argument("--solve-fp64", action="store_true", help="also time the plain FP64 GMRES (minutes)")
    p.add_argument("--precond-file", default="",
                   help="sphere163842_k64_q3_r16 --solve: learned preconditioner saved by --save-precond")
    p.add_argument("--solve-maxit", type=int, default=1500)
    p.add_argument("--hmat-eps", type=float, default=1e-5, help="hmat workload: tolerance of the low-rank blocks")
    p.add_argument("--hmat-leaf", type=int, default=8, help="hmat workload: vertex tiles per cluster")
    p.add_argument("--hmat-eta", type=float, default=0.5, help="hmat workload: admissibility parameter")
    p.add_argument("--hmat-level", type=int, default=0,
                   help="hmat workload: icosphere level of a smaller case (0: the workload's level 7)")
    p.add_argument("--hmat-k", type=float, default=0.0, help="hmat workload: wavenumber of a smaller case (0: 64)")
    return p.parse_args()


def workload():
    cfg = synth.WORKLOADS[WORKLOAD]
    v, t = synth.icosphere(cfg["level"])
    return v, t, cfg


# ---------------------------------------------------------------- clocks
def smi_id_of(props, local_rank=0):
    """nvidia-smi id of the device: its UUID where torch reports one."""
    if getattr(props, "uuid", None) is not None:
        return "GPU-" + str(props.uuid)
    return str(local_rank)


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.idx = device_index
        self.proc = None
        self.path = os.path.join("/tmp", f"gyps_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader", "-lms", "100"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
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
        self.fh.close()
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in read_text(self.path).splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1].split()[0]))
                mx.append(float(f[2].split()[0]))
                pw.append(float(f[3].split()[0]))
            except ValueError:
                continue
            for n, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- roofline
def far_traffic_per_launch():
    """DRAM bytes per far-kernel launch from the committed ncu summary, if it
    was taken on the current far-kernel source (else None)."""
    if not os.path.exists(PROFILE):
        return None
    text = read_text(PROFILE)
    m_sha = re.search(r"far_source_sha256:\s*([0-9a-f]{64})", text)
    m_b = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)
    if not m_sha or not m_b:
        return None
    sha = far_kernel_sha()
    if sha != m_sha.group(1):
        return None
    return float(m_b.group(1))


def far_kernel_sha():
    """sha256 of the FP32 far-kernel code the counters describe: the tile body
    in far_tile.cuh and the FP32 section of far.cu."""
    tile = read_text(FAR_TILE_SRC)
    src = read_text(FAR_SRC)
    a = src.index("// ---------------------------------------------------------------- a3: far, FP32")
    b = src.index("// ---------------------------------------------------------------- a3: far, FP64")
    return hashlib.sha256((tile + src[a:b]).encode()).hexdigest()


def sm_peak_pairs(num_sms, mhz):
    return num_sms * MUFU_PER_CLK_PER_SM / MUFU_PER_PAIR * mhz * 1e6


def far_roofline(achieved_gpairs, prec, nrhs, num_sms, mhz):
    """Roofline of the dense kernel product.  CUDA cores: the MUFU bound (3
    special-function results per pair).  Tensor cores: the lower of that bound
    and the tensor-pipe bound of the three split products, 3 x 8 R flop per pair
    for a pass of R right-hand sides (measured bf16 burst rate); when the tensor
    pipe binds, achieved and peak are stated in TFLOP/s."""
    sfu = sm_peak_pairs(num_sms, mhz) / 1e9
    out = {"bound": "alu", "achieved": achieved_gpairs, "peak": sfu, "unit": UNIT, "frac": achieved_gpairs / sfu,
           "peak_basis": f"{num_sms} SMs x {MUFU_PER_CLK_PER_SM}/{MUFU_PER_PAIR} pairs/clk x {mhz:.0f} MHz "
                         f"(measured sm_max_mhz)"}
    if prec == "fp32" or nrhs < 16:
        return out
    r_pass = 64 if nrhs >= 64 else (32 if nrhs > 16 else 16)
    flop_per_pair = 24.0 * r_pass
    try:
        tflops = json.loads(read_text(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"]
        basis = "measured bf16 burst"
    except Exception:
        tflops, basis = 1900.0, "fallback bf16 burst"
    tensor = tflops * 1e12 / flop_per_pair / 1e9
    out["tensor_peak_gpairs"] = tensor
    if tensor < sfu:
        out.update({"bound": "tensor", "achieved": achieved_gpairs * flop_per_pair / 1e3, "peak": tflops,
                    "unit": "TFLOP/s", "frac": achieved_gpairs / tensor,
                    "peak_basis": f"{basis} {tflops:.0f} TFLOP/s; 3 split products x 8 x {r_pass} flop per pair "
                                  f"(the MUFU bound, {sfu:.0f} GPairs/s, is higher)"})
    return out


# ---------------------------------------------------------------- CPU baseline
def oracle_sample(v, t, cfg, seconds, seed=1804):
    """Times the oracle's apply restricted to a sample of output rows: all
    source points, the target points in the support of the sampled vertices.
    Returns (pairs/s, cores, description, seconds)."""
    import oracle
    om = oracle.Mesh(v, t, cfg["q"])
    _ = om.near  # correction built outside the timing (k-independent, once per mesh)
    x = synth.random_complex(np.random.default_rng(seed), om.nv, 1)
    rng = np.random.default_rng(seed)
    order = rng.permutation(om.nv)
    n = 8
    t0 = time.perf_counter()
    om.apply(cfg["k"], x, rows=np.sort(order[:n]))
    dt = time.perf_counter() - t0
    npts = len(om.quad_ids_of_vertices(order[:n]))
    per_target = dt / max(npts, 1)
    want = int(max(n, min(om.nv, n * seconds / max(dt, 1e-6))))
    rows = np.sort(order[:want])
    tids = om.quad_ids_of_vertices(rows)
    t0 = time.perf_counter()
    om.apply(cfg["k"], x, rows=rows)
    dt = time.perf_counter() - t0
    pairs = len(tids) * om.nq
    desc = (f"{want} of {om.nv} output rows ({len(tids)} of {om.nq} target points x all {om.nq} sources, "
            f"plus their correction rows), {dt:.1f} s")
    del per_target
    return pairs / dt, oracle.num_threads(), desc, dt


# ---------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return
    v, t, cfg = workload()
    import oracle
    om = oracle.Mesh(v, t, cfg["q"])
    _ = om.near
    x = synth.random_complex(np.random.default_rng(0), om.nv, 1)
    rng = np.random.default_rng(1804)
    # size one step so that warm-up + timed steps take about two minutes of CPU work
    per_step = min(2.5, 120.0 / max(args.steps + args.warmup, 1))
    probe = np.sort(rng.choice(om.nv, 8, replace=False))
    t0 = time.perf_counter()
    om.apply(cfg["k"], x, rows=probe)
    dt = time.perf_counter() - t0
    nrows = int(max(8, min(om.nv, 8 * per_step / max(dt, 1e-6))))
    times, pairs = [], []
    for i in range(args.warmup + args.steps):
        rows = np.sort(rng.choice(om.nv, nrows, replace=False))
        ntgt = len(om.quad_ids_of_vertices(rows))
        t0 = time.perf_counter()
        om.apply(cfg["k"], x, rows=rows)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
            pairs.append(ntgt * om.nq)
    value = sum(pairs) / sum(times) / 1e9
    desc = f"each step {nrows} random output rows of {om.nv} (all {om.nq} sources)"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "mesh": "icosphere level 5", "nv": om.nv, "nq": om.nq, "k": cfg["k"],
                   "quad_points": cfg["q"], "nrhs": 1},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
def triangle_range(rank, world, nt):
    """Contiguous test-triangle range of a rank: the ranges of all ranks partition [0, nt)."""
    return (rank * nt // world, (rank + 1) * nt // world)


def run_gyps(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_1804_00995_gb300 import build as gb
    if local_rank == 0:
        gb.build()
    if world > 1:
        dist.barrier()
    import paper_1804_00995_gb300 as g

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    props = torch.cuda.get_device_properties(dev)
    v, t, cfg = workload()
    k = cfg["k"]
    mesh = g.Mesh(v, t, cfg["q"])
    nq, nv = mesh.nq, mesh.nv
    pairs = float(nq) * nq
    # one operator apply per step, sharded over the ranks by contiguous ranges of test
    # triangles (their target points), then one all-reduce (sum) of Y: the row blocks of
    # Phi^T W G W Phi are independent, so the partial applies add up to the full apply
    nrhs, prec = args.nrhs, args.prec
    tr = triangle_range(rank, world, mesh.nt)
    x = torch.as_tensor(synth.random_complex(np.random.default_rng(1000), nv, nrhs)).to(dev)
    y = g.sl_apply(mesh, k, x, prec=prec, tri_range=tr)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2
    stream = torch.cuda.current_stream(dev)

    def step(xin, yout):
        g.sl_apply(mesh, k, xin, prec=prec, out=yout, tri_range=tr)
        if world > 1:
            dist.all_reduce(torch.view_as_real(yout.t()))  # (nrhs, nv) is contiguous

    for _ in range(args.warmup):
        flush.zero_()
        step(x, y)
    torch.cuda.synchronize(dev)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(smi_id_of(props, local_rank))
    mesh.profile(True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    time.sleep(0.3)
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        step(x, y)
        ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - wall0
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    prof = mesh.profile_read()
    mesh.profile(False)
    step_ms = sum(a.elapsed_time(b) for a, b in ev)
    t_max = step_ms
    if world > 1:
        tt = torch.tensor([step_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_max = float(tt.item())
    ms_per_step = t_max / args.steps
    value = pairs / (ms_per_step * 1e-3) / 1e9  # the whole operator per step, over all ranks

    # roofline of the dominant kernel (dense G u), from its own events
    far_ms = prof["far_ms"] / max(prof["far_launches"], 1)
    # one launch covers all right-hand sides of a pass: pairs per launch = Nq^2 x (passes per apply)^-1
    launches_per_apply = prof["far_launches"] / max(prof["applies"], 1)
    rank_pairs = pairs * (tr[1] - tr[0]) / mesh.nt  # this rank's target points x all sources
    achieved = rank_pairs / (far_ms * launches_per_apply * 1e-3) / 1e9
    peak_mhz = None
    try:
        peak_mhz = json.loads(read_text(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"]
    except Exception:
        peak_mhz = clk.get("sm_max_mhz") or 2070.0
    traffic = far_traffic_per_launch() if (prec == "fp32" and nrhs == 1 and world == 1) else None

    # end to end through the public API with host buffers (pinned), copies inside: X from the
    # host into the library's staging, the (partial) apply, the all-reduce, Y back to the host
    xh = torch.as_tensor(synth.random_complex(np.random.default_rng(2000), nv, nrhs)).t().contiguous().t()
    xh = xh.pin_memory().t().contiguous().t() if nrhs == 1 else xh
    yh = torch.empty((nrhs, nv), dtype=torch.complex128).pin_memory().t()
    yd = torch.empty((nrhs, nv), dtype=torch.complex128, device=dev).t()

    def e2e_step():
        if world == 1:
            g.sl_apply(mesh, k, xh, prec=prec, out=yh)  # returns once Y is back on the host
            return
        step(xh, yd)
        yh.copy_(yd)

    e2e_step()
    e2e_t = []
    for i in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        e2e_step()
        e2e_t.append(time.perf_counter() - t0)
    e2e_mean = sum(e2e_t) / len(e2e_t)
    if world > 1:
        tt = torch.tensor([e2e_mean], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_mean = float(tt.item())
    e2e_value = pairs / e2e_mean / 1e9

    solve = None
    if world == 1 and (args.solve is not False or args.solve_fp64):
        f = g.rhs_planewave(mesh, k, [cfg["dirs"][0]])
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        xs, rep = g.gmres_solve(mesh, k, f, tol=cfg["tol"], restart=200, maxit=2000, prec="fp32",
                                check_prec="df64", max_refine=4)
        torch.cuda.synchronize(dev)
        t_solve = time.perf_counter() - t0
        # after the timed solve: the residual with the FP64 operator
        r64 = f - g.sl_apply(mesh, k, xs, prec="fp64")
        solve = {"tol": cfg["tol"], "fp32_refined_s": t_solve, "iterations": rep.iterations,
                 "refinements": rep.refinements, "check": "df64", "check_applies": rep.check_applies,
                 "true_residual_df64": float(rep.true_residual[0]),
                 "true_residual_fp64": float(torch.linalg.norm(r64) / torch.linalg.norm(f)), "status": rep.status}
        # the same scattering problem in the combined-field (Brakhage-Werner) form
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        _, repb = g.gmres_solve(mesh, k, -f, tol=cfg["tol"], restart=200, maxit=2000, prec="fp32",
                                check_prec="df64", max_refine=4, formulation="bw", eta=k)
        torch.cuda.synchronize(dev)
        solve["brakhage_werner"] = {"s": time.perf_counter() - t0, "eta": k, "iterations": repb.iterations,
                                    "refinements": repb.refinements,
                                    "true_residual_df64": float(repb.true_residual[0]), "status": repb.status}
        # The plain FP64 GPU form (FP64 operator and checks) takes minutes here, so the default
        # line times it over a bounded number of iterations and takes its iteration count from
        # GMRES with the double-float operator (within 1e-13 of the FP64 operator, so it follows
        # the same Krylov path); --solve-fp64 runs it to the end instead.
        def timed_fp64(maxit):
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            g.gmres_solve(mesh, k, f, tol=cfg["tol"], restart=200, maxit=maxit, prec="fp64", check_prec="fp64",
                          max_refine=0)
            torch.cuda.synchronize(dev)
            return time.perf_counter() - t0
        t1, t5 = timed_fp64(1), timed_fp64(5)
        t_iter = (t5 - t1) / 4.0
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        _, repd = g.gmres_solve(mesh, k, f, tol=cfg["tol"], restart=200, maxit=2000, prec="df64",
                                check_prec="df64", max_refine=0)
        torch.cuda.synchronize(dev)
        t_df = time.perf_counter() - t0
        fp64_est = t1 + (repd.iterations - 1) * t_iter
        solve.update({"fp64_s_est": fp64_est, "fp64_per_iteration_s": t_iter, "fp64_iterations_est": repd.iterations,
                      "fp64_est_basis": "plain FP64 GMRES timed over 1 and 5 iterations; iterations of the "
                                        "double-float-operator solve (FP64-class operator, same Krylov path)",
                      "df64_s": t_df, "df64_iterations": repd.iterations,
                      "df64_true_residual": float(repd.true_residual[0]), "df64_status": repd.status,
                      "speedup_vs_fp64_est": fp64_est / t_solve})
        if args.solve_fp64:
            t0 = time.perf_counter()
            _, rep64 = g.gmres_solve(mesh, k, f, tol=cfg["tol"], restart=200, maxit=2000, prec="fp64",
                                     check_prec="fp64", max_refine=0)
            torch.cuda.synchronize(dev)
            solve.update({"fp64_s": time.perf_counter() - t0, "fp64_iterations": rep64.iterations,
                          "fp64_true_residual": float(rep64.true_residual[0]), "fp64_status": rep64.status})

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pv, cores, desc, _ = oracle_sample(v, t, cfg, args.cpu_seconds)
        cpu = {"value": pv / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32" if prec == "fp32" else "bf16x3+f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "mesh": "icosphere level 5 (20480 triangles)", "nv": nv, "nq": nq,
                       "k": k, "quad_points": cfg["q"], "nrhs": nrhs, "far": prec, "near": "fp64",
                       "l2": "flushed (512 MB write) before every step", "pairs_per_step": pairs,
                       "ranks": f"one operator sharded over {world} rank(s) by contiguous test-triangle ranges, "
                                f"one all-reduce of Y (nv x nrhs complex) per step",
                       "triangles_per_rank": mesh.nt // world},
            "roofline": dict(far_roofline(achieved, prec, nrhs, props.multi_processor_count, peak_mhz),
                             traffic=traffic,
                             kernel="far32_kernel<1,4,false>" if prec == "fp32" else "far_tc_kernel",
                             far_ms_per_launch=far_ms),
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nv * 16 * nrhs,
                    "d2h_bytes_per_step": nv * 16 * nrhs},
            "pair_rhs_per_s": pairs * nrhs / (ms_per_step * 1e-3),
            "gpu_launches": int(prof["launches"]),
            "clocks": clk,
            "wall_s_timed_region": wall,
        }
        if solve is not None:
            line["solve"] = solve
        print(json.dumps(line), flush=True)
    mesh.close()


def run_batch(args):
    """Workload batch12_r64: 12 meshes (icospheres levels 2-6 and 7 random
    ellipsoids, 320-81920 triangles, q = 3), k_i ~ U[2, 24], 64 right-hand
    sides each, one graph replay per step (one persistent far launch)."""
    import torch

    import paper_1804_00995_gb300 as g
    from paper_1804_00995_gb300 import build as gb
    gb.build()
    dev = torch.device("cuda", 0)
    items, _ = synth.batch_workload(nrhs=64)
    meshes = [g.Mesh(it["vtx"], it["tri"], 3) for it in items]
    t0 = time.perf_counter()
    b = g.Batch([(m, it["k"]) for m, it in zip(meshes, items)], 64, graph=True, autotune=True)
    t_create = time.perf_counter() - t0
    for i, m in enumerate(meshes):
        b.X[i].copy_(torch.as_tensor(synth.random_complex(np.random.default_rng(i), m.nv, 64)))
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        b.apply()
    torch.cuda.synchronize(dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(smi_id_of(torch.cuda.get_device_properties(0)))
    clocks.start()
    time.sleep(0.3)
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        b.apply()
        ev[i][1].record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    ms = sum(a.elapsed_time(c) for a, c in ev) / args.steps
    pairs = b.info["pairs"]
    line = {
        "metric": "GPairs/s batched single-layer apply", "value": pairs / (ms * 1e-3) / 1e9, "unit": UNIT,
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "dtype": "bf16x3+f32" if b.info["tensor_cores"] else "f32", "data": "synthetic",
        "pair_rhs_per_s": pairs * 64 / (ms * 1e-3), "clocks": clk,
        "config": {"workload": "batch12_r64", "meshes": [(it["kind"], it["level"], int(it["tri"].shape[0]),
                                                             round(float(it["k"]), 3)) for it in items],
                   "nq_total": int(sum(m.nq for m in meshes)), "nrhs": 64, "quad_points": 3,
                   "pairs_per_rhs": pairs, "l2": "flushed (512 MB write) before every step"},
        "batch": dict(b.info), "create_s": t_create,
    }
    print(json.dumps(line), flush=True)
    b.close()


def run_precond(args):
    """Workload precond_ellipsoids: learned message-passing preconditioner.
    Training pairs come from the library's own solves on random ellipsoids of
    5120-20480 triangles (q = 3) at k ~ U[4, 16] (seed 995): by default the
    errors of GMRES iterates on plane-wave right-hand sides with their
    residuals (Krylov pairs), optionally also white-noise residuals r with
    their corrections e = V^{-1} r (16 GMRES solves per mesh); the network is trained by the
    library's kernels; held-out ellipsoids (seed 996) with 4 plane-wave
    right-hand sides each are solved to 1e-6 (FP64 residual) by flexible
    GMRES + network and by plain GMRES."""
    import torch

    import paper_1804_00995_gb300 as g
    from paper_1804_00995_gb300 import build as gb
    from paper_1804_00995_gb300 import precond_train as pt
    gb.build()
    t0 = time.perf_counter()
    train_meshes = pt.random_meshes(995, args.precond_meshes, levels=(4, 5))
    pairs, stats = [], []
    if args.precond_data in ("noise", "both"):
        p_n, s_n = pt.make_pairs(train_meshes, nrhs=16, tol=1e-3, maxit=300, seed=1)
        pairs += p_n
        stats += s_n
    if args.precond_data in ("krylov", "both"):
        ksteps = tuple(int(v) for v in args.precond_krylov_steps.split(","))
        p_k, s_k = pt.make_krylov_pairs(train_meshes, ndirs=4, steps=ksteps, tol=1e-5, maxit=600, seed=3)
        pairs += p_k
        stats += s_k
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    P = g.Precond(64, 4, seed=995)
    log = pt.train(P, pairs, steps=args.precond_steps, lr=2e-3, batch=16, seed=2, lr_final=2e-4,
                   log_every=max(args.precond_steps // 10, 1))
    if args.save_precond:
        P.save(args.save_precond)
    test_meshes = pt.random_meshes(996, args.precond_test, levels=(4, 5))
    rows = pt.evaluate(P, test_meshes, tol=1e-6, ndirs=4, restart=100, maxit=1500)
    both = [r for r in rows if r["gmres"]["status"] == "OK" and r["fgmres_mpnn"]["status"] == "OK"]
    it_g = sum(r["gmres"]["iterations"] for r in both)
    it_p = sum(r["fgmres_mpnn"]["iterations"] for r in both)
    s_g = sum(r["gmres"]["seconds"] for r in both)
    s_p = sum(r["fgmres_mpnn"]["seconds"] for r in both)
    kept = [r for r in both if r["fgmres_mpnn"]["fallback"] == 0]

    def tot(rs, solver, key):
        return sum(r[solver][key] for r in rs)
    line = {
        "metric": "GMRES to 1e-6: flexible GMRES + learned preconditioner vs plain GMRES (iterations, seconds)",
        "value": (s_g / s_p) if s_p > 0 else None, "unit": "x (plain seconds / preconditioned seconds)",
        "higher_is_better": True, "data": "synthetic", "dtype": "bf16 weights, f32 activations",
        "config": {"workload": "precond_ellipsoids", "train_meshes": len(train_meshes), "train_data": args.precond_data, "krylov_steps": args.precond_krylov_steps,
                   "pairs_kept": int(sum(s["kept"] for s in stats)),
                   "levels": [4, 5], "k_range": [4, 16], "hidden": 64, "layers": 4, "steps": args.precond_steps,
                   "test_meshes": len(test_meshes), "rhs_per_test_mesh": 4, "restart": 100},
        "data_seconds": t_data, "train_seconds": log.seconds,
        "train_loss": log.losses,
        "both_converged": len(both), "iterations_plain": it_g, "iterations_precond": it_p,
        "seconds_plain": s_g, "seconds_precond": s_p,
        "all_meshes": {"seconds_plain": tot(rows, "gmres", "seconds"), "seconds_precond": tot(rows, "fgmres_mpnn", "seconds"),
                       "iterations_plain": tot(rows, "gmres", "iterations"),
                       "iterations_precond": tot(rows, "fgmres_mpnn", "iterations")},
        "network_kept": {"meshes": len(kept), "seconds_plain": tot(kept, "gmres", "seconds"),
                         "seconds_precond": tot(kept, "fgmres_mpnn", "seconds"),
                         "iterations_plain": tot(kept, "gmres", "iterations"),
                         "iterations_precond": tot(kept, "fgmres_mpnn", "iterations")},
        "rows": [{k: (v if not isinstance(v, float) else round(v, 4)) for k, v in r.items()} for r in rows],
    }
    print(json.dumps(line), flush=True)


def mie_density_sphere(k, d, pts):
    """Density of the sound-soft unit sphere for p_inc = exp(ik d.x) (Mie series,
    the exact solution the discrete one converges to): sum_n (2n+1) i^n
    P_n(d.x) / (i k h_n(k)); measurement only."""
    from scipy.special import eval_legendre, spherical_jn, spherical_yn
    d = np.asarray(d, dtype=np.float64)
    d = d / np.linalg.norm(d)
    c = (pts / np.linalg.norm(pts, axis=1, keepdims=True)) @ d
    lam = np.zeros(pts.shape[0], dtype=np.complex128)
    for n in range(int(np.ceil(k + 4.0 * k ** (1.0 / 3.0) + 10)) + 1):
        lam += (2 * n + 1) * (1j ** n) * eval_legendre(n, c) / (1j * k * (spherical_jn(n, k) + 1j * spherical_yn(n, k)))
    return lam


def mie_scattered_sphere(k, d, pts):
    """Field scattered by the sound-soft unit sphere for p_inc = exp(ik d.x), outside it:
    -sum_n (2n+1) i^n j_n(k)/h_n(k) h_n(k r) P_n(d.x/r); measurement only."""
    from scipy.special import eval_legendre, spherical_jn, spherical_yn
    d = np.asarray(d, dtype=np.float64)
    d = d / np.linalg.norm(d)
    r = np.linalg.norm(pts, axis=1)
    c = (pts / r[:, None]) @ d
    s = np.zeros(pts.shape[0], dtype=np.complex128)
    for n in range(int(np.ceil(k + 4.0 * k ** (1.0 / 3.0) + 12)) + 1):
        hk = spherical_jn(n, k) + 1j * spherical_yn(n, k)
        hr = spherical_jn(n, k * r) + 1j * spherical_yn(n, k * r)
        s -= (2 * n + 1) * (1j ** n) * spherical_jn(n, k) / hk * hr * eval_legendre(n, c)
    return s


def run_field(args):
    """Workload field_sphere10242_k16: the total field of the sound-soft sphere
    (the listing of Sec. 5.4: Pdom = PW - Sdom lambda) on a 300 x 300 grid of the
    plane y = 0, x, z in [-2.5, 2.5], from the GMRES density of
    sphere10242_k16_q7 (icosphere 20480 triangles, q = 7, k = 16, d = (1, 0, 0)).
    One step = one potential evaluation (FP32 far sum, FP64 [1/r]
    regularisation) at the 90000 points; error against the Mie total field at
    the points more than 0.1 from the surface."""
    import torch

    import paper_1804_00995_gb300 as g
    from paper_1804_00995_gb300 import build as gb
    gb.build()
    cfg = synth.WORKLOADS[WORKLOAD]
    v, t = synth.icosphere(cfg["level"])
    mesh = g.Mesh(v, t, cfg["q"])
    k, d = cfg["k"], np.asarray(cfg["dirs"][0], dtype=np.float64)
    f = g.rhs_planewave(mesh, k, [d])
    t0 = time.perf_counter()
    lam, rep = g.gmres_solve(mesh, k, f, tol=cfg["tol"], restart=200, maxit=2000, prec="fp32", check_prec="df64")
    torch.cuda.synchronize()
    t_solve = time.perf_counter() - t0
    n = 300
    a = np.linspace(-2.5, 2.5, n)
    X, Z = np.meshgrid(a, a, indexing="ij")
    pts = np.stack([X.ravel(), np.zeros(n * n), Z.ravel()], axis=1)
    pd = torch.as_tensor(pts).cuda()
    for _ in range(args.warmup):
        g.sl_potential(mesh, k, pd, lam, prec="fp32")
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(smi_id_of(torch.cuda.get_device_properties(0)))
    clocks.start()
    time.sleep(0.3)
    for i in range(args.steps):
        ev[i][0].record(stream)
        p = g.sl_potential(mesh, k, pd, lam, prec="fp32")
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = sum(x.elapsed_time(y) for x, y in ev) / args.steps
    p = p.cpu().numpy()[:, 0]
    total = np.exp(1j * k * pts @ d) - p
    r = np.linalg.norm(pts, axis=1)
    inside, outside = r < 0.9, r > 1.1
    mie_total = np.exp(1j * k * pts[outside] @ d) + mie_scattered_sphere(k, d, pts[outside])
    pairs = float(len(pts)) * mesh.nq
    line = {
        "metric": "GPairs/s single-layer potential at points (total field of the solved sphere)",
        "value": pairs / (ms * 1e-3) / 1e9, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "field_sphere10242_k16", "points": len(pts), "grid": "300 x 300, y = 0, [-2.5, 2.5]^2",
                   "nq": mesh.nq, "k": k, "near": "fp64 [1/r] regularisation"},
        "solve": {"seconds": t_solve, "iterations": rep.iterations, "status": rep.status,
                  "true_residual_df64": float(rep.true_residual[0])},
        "field_error": {"inside_max_abs_total": float(np.abs(total[inside]).max()),
                        "outside_max_abs": float(np.abs(total[outside] - mie_total).max()),
                        "outside_median_abs": float(np.median(np.abs(total[outside] - mie_total))),
                        "points_inside": int(inside.sum()), "points_outside": int(outside.sum())},
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def run_dl(args):
    """Workload dl_sphere10242_k16_q7: the Galerkin double layer K on the mesh of
    sphere10242_k16_q7 (icosphere 20480 triangles, q = 7, k = 16).  One step =
    one FP32 apply of K to one random column (persistent tile kernel, FP64
    correction); once each: the double-float and FP64 applies and the
    Brakhage-Werner operator 1/2 M + K - i k V; then GMRES to 1e-6 (FP32
    operator, double-float checks) for the plane wave d = (1, 0, 0) in the
    first-kind (V), the indirect combined-field (Brakhage-Werner) and the direct
    combined-field (1/2 M + K' - i k V) form, at k = 16 and at k = 3 pi, where
    j_0(k) = 0 and V is singular on the unit sphere; the first-kind and direct
    solutions are both du/dn and are compared with the Mie series at 2048
    vertices."""
    import torch

    import paper_1804_00995_gb300 as g
    from paper_1804_00995_gb300 import build as gb
    gb.build()
    cfg = synth.WORKLOADS[WORKLOAD]
    v, t = synth.icosphere(cfg["level"])
    mesh = g.Mesh(v, t, cfg["q"])
    k = cfg["k"]
    x = torch.as_tensor(synth.random_complex(np.random.default_rng(1), mesh.nv, 1)).cuda()
    for _ in range(args.warmup):
        g.dl_apply(mesh, k, x, prec="fp32")
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(smi_id_of(torch.cuda.get_device_properties(0)))
    mesh.profile(True)
    clocks.start()
    time.sleep(0.3)
    for i in range(args.steps):
        ev[i][0].record(stream)
        y32 = g.dl_apply(mesh, k, x, prec="fp32")
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    prof = mesh.profile_read()
    mesh.profile(False)
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    far_ms = prof["far_ms"] / max(prof["far_launches"], 1)
    once = {}
    for name, fn in (("df64", lambda: g.dl_apply(mesh, k, x, prec="df64")),
                     ("fp64", lambda: g.dl_apply(mesh, k, x, prec="fp64")),
                     ("bw_fp32", lambda: g.bw_apply(mesh, k, k, x, prec="fp32"))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        y = fn()
        torch.cuda.synchronize()
        once[name] = {"ms": (time.perf_counter() - t0) * 1e3}
        if name != "bw_fp32":
            once[name]["y"] = y
    y64 = once["fp64"].pop("y")
    once["df64"]["rel_diff_vs_fp64"] = float(torch.linalg.norm(once["df64"].pop("y") - y64) / torch.linalg.norm(y64))
    rel32 = float(torch.linalg.norm(y32 - y64) / torch.linalg.norm(y64))
    solves = []
    d = np.asarray(cfg["dirs"][0], dtype=np.float64)
    samp = np.sort(np.random.default_rng(7).choice(mesh.nv, 2048, replace=False))
    for kk in (k, 3.0 * np.pi):
        f = g.rhs_planewave(mesh, kk, [d])
        fc = g.rhs_planewave_cfie(mesh, kk, kk, [d])
        mie = mie_density_sphere(kk, d, v[samp])
        for form in ("sl", "bw", "cfie"):
            rhs = {"sl": f, "bw": -f, "cfie": fc}[form]
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            x, rep = g.gmres_solve(mesh, kk, rhs, tol=cfg["tol"], restart=200, maxit=2000, prec="fp32",
                                   check_prec="df64", max_refine=4, formulation=form, eta=kk)
            torch.cuda.synchronize()
            row = {"k": kk, "form": {"sl": "V", "bw": "1/2 M + K - i k V", "cfie": "1/2 M + K' - i k V"}[form],
                   "seconds": time.perf_counter() - t0, "iterations": rep.iterations,
                   "true_residual_df64": float(rep.true_residual[0]), "status": rep.status}
            if form != "bw":  # both solve for du/dn, the Mie density
                xs = x.cpu().numpy()[samp, 0]
                row["mie_rel_error_2048_vertices"] = float(np.linalg.norm(xs - mie) / np.linalg.norm(mie))
            solves.append(row)
    pairs = float(mesh.nq) ** 2
    achieved = pairs / (far_ms * 1e-3) / 1e9
    props = torch.cuda.get_device_properties(0)
    try:
        peak_mhz = json.loads(read_text(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"]
    except Exception:
        peak_mhz = clk.get("sm_max_mhz") or 2070.0
    roof = sm_peak_pairs(props.multi_processor_count, peak_mhz) / 1e9
    line = {
        "metric": "GPairs/s double-layer apply (Gauss-point pairs per second)", "value": pairs / (ms * 1e-3) / 1e9,
        "unit": UNIT,
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "dl_sphere10242_k16_q7", "nv": mesh.nv, "nq": mesh.nq, "k": k, "nrhs": 1,
                   "near": "fp64 closed-form grady[1/r] correction", "l2": "inputs 5 MB, not flushed (alu bound)"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": roof, "unit": "GPairs/s", "frac": achieved / roof,
                     "traffic": None, "kernel": "far_dl32_kernel<1,4,false>", "far_ms_per_launch": far_ms,
                     "peak_basis": "3 MUFU results per pair at 16 per clock per SM, measured sm_max_mhz"},
        "fp32_rel_diff_vs_fp64": rel32, "once": once, "solves": solves, "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def mie_pec_sphere(k, cos_theta):
    """S1, S2 of the perfectly conducting unit sphere (Mie series, a_n = psi_n'/xi_n',
    b_n = psi_n/xi_n); measurement only."""
    from scipy.special import spherical_jn, spherical_yn
    mu = np.asarray(cos_theta, dtype=np.float64)
    s1 = np.zeros(mu.shape, dtype=np.complex128)
    s2 = np.zeros(mu.shape, dtype=np.complex128)
    p0, p1 = np.zeros_like(mu), np.ones_like(mu)
    for n in range(1, int(np.ceil(k + 4.0 * k ** (1.0 / 3.0) + 10)) + 1):
        if n > 1:
            p0, p1 = p1, ((2 * n - 1) * mu * p1 - n * p0) / (n - 1)
        tau = n * mu * p1 - (n + 1) * p0
        j, jp = spherical_jn(n, k), spherical_jn(n, k, derivative=True)
        h, hp = j + 1j * spherical_yn(n, k), jp + 1j * spherical_yn(n, k, derivative=True)
        an, bn = (j + k * jp) / (h + k * hp), j / h
        c = (2 * n + 1) / (n * (n + 1))
        s1 += c * (an * p1 + bn * tau)
        s2 += c * (an * tau + bn * p1)
    return s1, s2


def rwg_current_at_points(g, mesh, v, t, x):
    """The surface current sum_e x_e phi_e at the mesh's Gauss points (numpy, from the
    RWG definition: local edge j of a triangle joins vertices j+1 and j+2, sign +1
    where it runs from the smaller to the larger index, phi = s l/(2A) (y - P_j));
    measurement only."""
    ne, edges = g.rwg_edges(mesh)
    key = edges[:, 0].astype(np.int64) * mesh.nv + edges[:, 1]
    qp = mesh.quad_points().cpu().numpy()
    P = v[t]
    two_a = np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1)
    J = np.zeros((mesh.nt, mesh.q, 3), dtype=np.complex128)
    y = qp[:, :3].reshape(mesh.nt, mesh.q, 3)
    for j in range(3):
        a, b = t[:, (j + 1) % 3].astype(np.int64), t[:, (j + 2) % 3].astype(np.int64)
        e = np.searchsorted(key, np.minimum(a, b) * mesh.nv + np.maximum(a, b))
        c = np.where(a < b, 1.0, -1.0) * np.linalg.norm(P[:, (j + 2) % 3] - P[:, (j + 1) % 3], axis=1) / two_a
        J += (x[e] * c)[:, None, None] * (y - P[:, None, j, :])
    return qp, J.reshape(-1, 3)


def run_efie(args):
    """Workload efie_sphere10242_k8_q3: the EFIE of the electromagnetic listing
    of Sec. 5.5 with RWG functions on the icosphere of 20480 triangles (30720
    edges), q = 3 (61440 Gauss points), k = 8.  One step = one FP32 apply of T to
    one random current (four density columns through the FP32 far kernel, FP64
    correction); once each: the FP64 and double-float applies; then GMRES to 1e-6
    on -T J = int phi . E_inc (x-polarised plane wave along z; FP32 operator,
    double-float checks) and the far field of J against the Mie amplitudes of the
    perfectly conducting sphere (E- and H-plane, 24 directions); then the listing's
    combined system -beta T + (1 - beta)(Id/2 - nxK) at beta = 0.5 for the same wave
    (the MFIE part in FP64 for its double-float check)."""
    import torch

    import paper_1804_00995_gb300 as g
    from paper_1804_00995_gb300 import build as gb
    gb.build()
    cfg = synth.WORKLOADS["efie_sphere10242_k8_q3"]
    v, t = synth.icosphere(cfg["level"])
    mesh = g.Mesh(v, t, cfg["q"])
    k = cfg["k"]
    ne, _ = g.rwg_edges(mesh)
    x = torch.as_tensor(synth.random_complex(np.random.default_rng(1), ne, 1)).cuda()
    for _ in range(args.warmup):
        g.efie_apply(mesh, k, x, prec="fp32")
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = ClockSampler(smi_id_of(torch.cuda.get_device_properties(0)))
    mesh.profile(True)
    clocks.start()
    time.sleep(0.3)
    for i in range(args.steps):
        ev[i][0].record(stream)
        y32 = g.efie_apply(mesh, k, x, prec="fp32")
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    prof = mesh.profile_read()
    mesh.profile(False)
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    far_ms = prof["far_ms"] / max(prof["far_launches"], 1)
    once = {}
    for prec in ("fp64", "df64"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        y = g.efie_apply(mesh, k, x, prec=prec)
        torch.cuda.synchronize()
        once[prec] = {"ms": (time.perf_counter() - t0) * 1e3, "y": y}
    y64 = once["fp64"].pop("y")
    once["df64"]["rel_diff_vs_fp64"] = float(torch.linalg.norm(once["df64"].pop("y") - y64) / torch.linalg.norm(y64))
    rel32 = float(torch.linalg.norm(y32 - y64) / torch.linalg.norm(y64))
    d, p = np.asarray(cfg["dirs"][0]), np.asarray(cfg["pols"][0])
    F = g.rhs_planewave_efie(mesh, k, d[None, :], p[None, :])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    J, rep = g.gmres_solve(mesh, k, F, tol=cfg["tol"], restart=300, maxit=3000, prec="fp32", check_prec="df64",
                           max_refine=4, formulation="efie")
    torch.cuda.synchronize()
    t_solve = time.perf_counter() - t0
    th = np.linspace(0.05, np.pi - 0.05, 12)
    s1, s2 = mie_pec_sphere(k, np.cos(th))

    def far_field_error(Jc):
        qp, Jq = rwg_current_at_points(g, mesh, v, t, Jc)
        e = 0.0
        for xd, s in ((np.stack([np.sin(th), 0 * th, np.cos(th)], 1), s2),
                      (np.stack([0 * th, np.sin(th), np.cos(th)], 1), s1)):
            I = np.exp(-1j * k * (xd @ qp[:, :3].T)) @ (qp[:, 3:4] * Jq)
            amp = k / (4.0 * np.pi) * np.linalg.norm(I - np.sum(I * xd, axis=1)[:, None] * xd, axis=1)
            e = max(e, float(np.abs(amp / (np.abs(s) / k) - 1.0).max()))
        return e

    err = far_field_error(J.cpu().numpy()[:, 0])
    # the listing's combined system at beta = 0.5 (EFIE + MFIE), same wave
    for _ in range(2):
        g.mfie_apply(mesh, k, x, prec="fp32")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(5):
        g.mfie_apply(mesh, k, x, prec="fp32")
    torch.cuda.synchronize()
    mfie_ms = (time.perf_counter() - t0) / 5 * 1e3
    Fc = g.rhs_planewave_emcfie(mesh, k, 0.5, d[None, :], p[None, :])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Jc, repc = g.gmres_solve(mesh, k, Fc, tol=cfg["tol"], restart=300, maxit=3000, prec="fp32", check_prec="df64",
                             max_refine=4, formulation="emcfie", eta=0.5)
    torch.cuda.synchronize()
    t_cfie = time.perf_counter() - t0
    cfie = {"beta": 0.5, "seconds": t_cfie, "iterations": repc.iterations, "refinements": repc.refinements,
            "true_residual": float(repc.true_residual[0]), "status": repc.status,
            "far_field_max_rel_error_vs_mie": far_field_error(Jc.cpu().numpy()[:, 0]),
            "mfie_fp32_apply_ms": mfie_ms}
    pairs = float(mesh.nq) ** 2
    achieved = pairs / (far_ms * 1e-3) / 1e9
    props = torch.cuda.get_device_properties(0)
    try:
        peak_mhz = json.loads(read_text(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"]
    except Exception:
        peak_mhz = clk.get("sm_max_mhz") or 2070.0
    roof = sm_peak_pairs(props.multi_processor_count, peak_mhz) / 1e9
    line = {
        "metric": "GPairs/s EFIE apply (Gauss-point pairs per second, 4 density columns each)",
        "value": pairs / (ms * 1e-3) / 1e9, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "efie_sphere10242_k8_q3", "nt": mesh.nt, "ne": ne, "nq": mesh.nq, "k": k,
                   "columns_per_apply": 4, "near": "fp64 '[1/r]' correction (RWG from the P1 closed form)",
                   "l2": "inputs 4 MB, not flushed (alu bound)"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": roof, "unit": "GPairs/s", "frac": achieved / roof,
                     "traffic": None, "kernel": "far32_kernel<4,2,false>", "far_ms_per_launch": far_ms,
                     "peak_basis": "3 MUFU results per pair at 16 per clock per SM, measured sm_max_mhz"},
        "fp32_rel_diff_vs_fp64": rel32, "once": once,
        "solve": {"seconds": t_solve, "iterations": rep.iterations, "refinements": rep.refinements,
                  "true_residual_df64": float(rep.true_residual[0]), "status": rep.status,
                  "far_field_max_rel_error_vs_mie": err},
        "combined_field_solve": cfie,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)


def solve_large(g, mesh, v, t, k, F, dirs, args, hmat=None):
    """Workload sphere163842_k64_q3_r16, --solve: (flexible) GMRES to 1e-6 on all
    16 plane waves, tensor-core working operator, double-float operator for the
    true residual (the FP64 pipe would take about three minutes per check here);
    then the FP64 residual on the exact rows of the vertices inside a patch of
    4096 triangles and the error against the Mie series at 4096 sampled
    vertices."""
    import torch
    P = None
    if args.precond_file:
        P = g.Precond(64, 4)
        P.load(args.precond_file)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    working = "hmat" if hmat is not None else "tc_bf16x3"
    X, rep = g.gmres_solve(mesh, k, F, tol=1e-6, restart=300, maxit=args.solve_maxit, prec=working,
                           check_prec="df64", max_refine=3, precond=P, hmat=hmat)
    torch.cuda.synchronize()
    seconds = time.perf_counter() - t0
    patch = 4096
    tot = np.bincount(t.ravel(), minlength=mesh.nv)
    inside = np.bincount(t[:patch].ravel(), minlength=mesh.nv)
    rows = np.flatnonzero((inside == tot) & (tot > 0))
    t1 = time.perf_counter()
    Y = g.sl_apply(mesh, k, X, prec="fp64", tri_range=(0, patch))
    torch.cuda.synchronize()
    t_fp64 = time.perf_counter() - t1
    Fr, Yr = F.cpu().numpy()[rows], Y.cpu().numpy()[rows]
    res64 = np.linalg.norm(Fr - Yr, axis=0) / np.linalg.norm(Fr, axis=0)
    samp = np.sort(np.random.default_rng(7).choice(mesh.nv, 4096, replace=False))
    Xs = X.cpu().numpy()[samp]
    mie = []
    for j in range(len(dirs)):
        lam = mie_density_sphere(k, dirs[j], v[samp])
        mie.append(float(np.linalg.norm(Xs[:, j] - lam) / np.linalg.norm(lam)))
    return {"tol": 1e-6, "seconds": seconds, "iterations": rep.iterations, "applies": rep.applies,
            "check_applies": rep.check_applies, "refinements": rep.refinements, "status": rep.status,
            "precond": "learned (flexible GMRES)" if P is not None else "none",
            "precond_dropped": bool(rep.precond_fallback), "restart": 300,
            "working": working, "check": "df64",
            "residual_check_max": float(np.max(rep.true_residual)),
            "fp64_rows": int(rows.size), "fp64_patch_triangles": patch, "fp64_check_s": t_fp64,
            "fp64_residual_rows_max": float(res64.max()), "fp64_residual_rows_median": float(np.median(res64)),
            "mie_vertices": int(samp.size), "mie_rel_err_max": max(mie), "mie_rel_err_median": float(np.median(mie))}


def run_large(args):
    """Workload sphere163842_k64_q3_r16: icosphere with 327680 triangles,
    q = 3 (983040 points), k = 64, 16 plane waves (directions seed 7); one step
    = one tensor-core apply of all 16 columns (kernel products on tensor cores,
    FP64 correction); inputs (983040 x 16 density panel) exceed L2."""
    import torch

    import paper_1804_00995_gb300 as g
    from paper_1804_00995_gb300 import build as gb
    gb.build()
    cfg = synth.WORKLOADS["sphere163842_k64_q3_r16"]
    v, t = synth.icosphere(cfg["level"])
    mesh = g.Mesh(v, t, cfg["q"])
    dirs = synth.plane_wave_dirs(np.random.default_rng(cfg["seed"]), cfg["ndirs"])
    x = g.rhs_planewave(mesh, cfg["k"], dirs)
    y = g.sl_apply(mesh, cfg["k"], x, prec=args.prec if args.prec != "fp32" else "tc_bf16x3")
    prec = args.prec if args.prec != "fp32" else "tc_bf16x3"
    for _ in range(args.warmup):
        g.sl_apply(mesh, cfg["k"], x, prec=prec, out=y)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    props = torch.cuda.get_device_properties(0)
    clocks = ClockSampler(smi_id_of(props))
    mesh.profile(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks.start()
    time.sleep(0.3)
    for i in range(args.steps):
        ev[i][0].record(stream)
        g.sl_apply(mesh, cfg["k"], x, prec=prec, out=y)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    prof = mesh.profile_read()
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    pairs = float(mesh.nq) ** 2
    far_ms = prof["far_ms"] / max(prof["far_launches"], 1) * prof["far_launches"] / max(prof["applies"], 1)
    line = {
        "metric": "GPairs/s single-layer apply, 16 right-hand sides", "value": pairs / (ms * 1e-3) / 1e9,
        "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "dtype": "bf16x3+f32" if prec == "tc_bf16x3" else "f32", "data": "synthetic",
        "pair_rhs_per_s": pairs * 16 / (ms * 1e-3),
        "config": {"workload": "sphere163842_k64_q3_r16", "nv": mesh.nv, "nq": mesh.nq, "k": cfg["k"], "nrhs": 16,
                   "far": prec, "near": "fp64", "l2": "inputs larger than L2"},
        "roofline": dict(far_roofline(pairs / (far_ms * 1e-3) / 1e9, prec, 16, props.multi_processor_count, 2070.0),
                         traffic=None, kernel="far_tc_kernel" if prec != "fp32" else "far32_kernel"),
        "gpu_launches": int(prof["launches"]), "clocks": clk,
    }
    if args.solve:
        line["solve"] = solve_large(g, mesh, v, t, cfg["k"], x, dirs, args)
    print(json.dumps(line), flush=True)


def run_hmat(args):
    """Workload hmat_sphere163842_k64_q3_r16: the compressed far field of the
    icosphere with 327680 triangles (q = 3, 983040 points) at k = 64 (eps 1e-5,
    clusters of 8 vertex tiles, eta 0.5 by default), 16 plane waves.  One step = one apply
    of H + C to all 16 columns.  Reported: build time, stored bytes against the
    dense matrix, ranks, the apply time next to one tensor-core all-pairs apply
    of the same columns, and the difference to the FP32 all-pairs apply on two
    full columns (norm and largest element, relative)."""
    import torch

    import paper_1804_00995_gb300 as g
    from paper_1804_00995_gb300 import build as gb
    gb.build()
    cfg = synth.WORKLOADS["sphere163842_k64_q3_r16"]
    level = args.hmat_level if args.hmat_level > 0 else cfg["level"]
    v, t = synth.icosphere(level)
    mesh = g.Mesh(v, t, cfg["q"])
    k = args.hmat_k if args.hmat_k > 0 else cfg["k"]
    dirs = synth.plane_wave_dirs(np.random.default_rng(cfg["seed"]), cfg["ndirs"])
    x = g.rhs_planewave(mesh, k, dirs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = g.Hmat(mesh, k, eps=args.hmat_eps, leaf_tiles=args.hmat_leaf, eta=args.hmat_eta)
    build_s = time.perf_counter() - t0
    y = h.apply(x)
    for _ in range(args.warmup):
        h.apply(x, out=y)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    props = torch.cuda.get_device_properties(0)
    clocks = ClockSampler(smi_id_of(props))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks.start()
    time.sleep(0.3)
    for i in range(args.steps):
        ev[i][0].record(stream)
        h.apply(x, out=y)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    # the all-pairs forms for comparison: one tensor-core apply of the 16 columns, FP32 on two columns
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ytc = g.sl_apply(mesh, k, x, prec="tc_bf16x3")
    e0.record(stream)
    g.sl_apply(mesh, k, x, prec="tc_bf16x3", out=ytc)
    e1.record(stream)
    y32 = g.sl_apply(mesh, k, x[:, :2].contiguous(), prec="fp32")
    torch.cuda.synchronize()
    tc_ms = e0.elapsed_time(e1)
    a, b = y[:, :2].cpu().numpy(), y32.cpu().numpy()
    err_norm = max(np.linalg.norm(a[:, c] - b[:, c]) / np.linalg.norm(b[:, c]) for c in range(2))
    err_elem = max(np.abs(a[:, c] - b[:, c]).max() / np.abs(b[:, c]).max() for c in range(2))
    info = h.info
    pairs = float(mesh.nq) ** 2
    line = {
        "metric": "compressed far field: ms per 16-column apply", "value": ms, "unit": "ms",
        "higher_is_better": False, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "data": "synthetic",
        "dtype": "f32 blocks, f64 correction and output",
        "config": {"workload": "hmat_sphere163842_k64_q3_r16" if level == cfg["level"] and k == cfg["k"]
                   else f"hmat_icosphere{level}_k{k:g}_q3_r16 (smaller case)", "nv": mesh.nv, "nq": mesh.nq, "k": k, "nrhs": 16,
                   "eps": args.hmat_eps, "leaf_tiles": args.hmat_leaf, "eta": args.hmat_eta,
                   "l2": "blocks (tens of GB) larger than L2"},
        "build_s": build_s, "hmat": info, "compression": info["bytes"] / info["dense_bytes"],
        "stream_gbs": info["bytes"] / (ms * 1e-3) / 1e9,
        "roofline": hmat_roofline(info, ms, clk),
        "equivalent_gpairs_per_s": pairs / (ms * 1e-3) / 1e9,
        "tensor_core_all_pairs_ms": tc_ms, "speedup_vs_tensor_core_all_pairs": tc_ms / ms,
        "diff_vs_fp32_all_pairs": {"columns": 2, "norm": err_norm, "element": err_elem},
        "clocks": clk,
    }
    if args.solve:
        line["solve"] = solve_large(g, mesh, v, t, k, x, dirs, args, hmat=h)
    print(json.dumps(line), flush=True)
    h.close()


def hmat_roofline(info, ms, clk):
    """Roofline of the compressed apply, timed whole (gather, projections, rows, correction):
    every stored complex FP32 value meets the 16 columns once in the rows kernel (16 complex
    multiply-adds = 64 FP32 FMAs); the CUDA-core FMA peak is 152 SMs x 128 lanes x the measured
    maximum SM clock.  The HBM view (stored bytes per apply over the measured copy bandwidth) is
    given beside it."""
    try:
        peaks = json.loads(read_text(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        peaks = {}
    mhz = (clk or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz") or 2070.0
    fma = info["bytes"] / 8.0 * 64.0
    achieved = fma / (ms * 1e-3) / 1e12
    peak = 152 * 128 * mhz * 1e6 / 1e12
    hbm = peaks.get("hbm_gbs")
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFMA/s", "frac": achieved / peak,
            "peak_basis": f"152 SMs x 128 FP32 lanes x {mhz:g} MHz (of measured clock)",
            "kernel": "hm_rows16_kernel (whole apply timed)", "traffic": None,
            "hbm_frac": (info["bytes"] / (ms * 1e-3) / 1e9) / hbm if hbm else None}


def run_assemble(args):
    """Workload assemble_sphere10242: dense Galerkin matrix (a6) of the icosphere
    with 20480 triangles (10242 vertices), q = 3, k = 16: Nv^2 complex entries
    (1.68 GB) plus the correction.  FP32 kernel values: vertex-tile blocks, each
    entry written once (the complex-symmetric Gauss-Gauss part computed for tile
    pairs I <= J); FP64: triangle-pair blocks with FP64 atomics.  Reported:
    assembly time, Gauss pairs per second (Nq^2 / t, the algorithmic count) against
    the MUFU roof, and the bytes of V written per second (16 Nv^2 / t)."""
    import torch

    import paper_1804_00995_gb300 as g
    from paper_1804_00995_gb300 import build as gb
    gb.build()
    v, t = synth.icosphere(5)
    mesh = g.Mesh(v, t, 3)
    k = 16.0
    props = torch.cuda.get_device_properties(0)
    out = {}
    for prec in ("fp32", "fp64"):
        V = g.sl_assemble(mesh, k, prec=prec)  # warm-up (first FP32 call builds the vertex tiles)
        for _ in range(max(args.warmup - 1, 0)):
            g.sl_assemble(mesh, k, prec=prec, out=V)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        stream = torch.cuda.current_stream()
        clocks = ClockSampler(smi_id_of(props))
        clocks.start()
        time.sleep(0.3)
        for i in range(args.steps):
            ev[i][0].record(stream)
            g.sl_assemble(mesh, k, prec=prec, out=V)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
        out[prec] = {"ms": ms, "v_write_gbs": 16.0 * mesh.nv ** 2 / (ms * 1e-3) / 1e9,
                     "gauss_pairs_per_s": float(mesh.nq) ** 2 / (ms * 1e-3), "clocks": clk}
        del V
    try:
        peak_mhz = json.loads(read_text(os.path.join(ROOT, "MEASURED_PEAKS.json")))["sm_max_mhz"]
    except Exception:
        peak_mhz = 2070.0
    sfu = sm_peak_pairs(props.multi_processor_count, peak_mhz) / 1e9
    gp = out["fp32"]["gauss_pairs_per_s"] / 1e9
    line = {
        "metric": "dense single-layer assembly (a6): ms, V bytes written per second", "value": out["fp32"]["ms"],
        "unit": "ms", "higher_is_better": False, "n_gpus": 1, "steps": args.steps, "data": "synthetic",
        "dtype": "f32 kernel values and sums, f64 output",
        "roofline": {"bound": "alu", "achieved": gp, "peak": sfu, "unit": UNIT, "frac": gp / sfu,
                     "peak_basis": f"{props.multi_processor_count} SMs x 16/3 pairs/clk x {peak_mhz:.0f} MHz",
                     "kernel": "tile_block_kernel<3,false,true,double2>", "traffic": None},
        "config": {"workload": "assemble_sphere10242", "nv": mesh.nv, "nt": mesh.nt, "q": 3, "k": k,
                   "v_bytes": 16 * mesh.nv ** 2},
        "fp32": out["fp32"], "fp64": out["fp64"],
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.workload == "assemble_sphere10242":
        run_assemble(args)
        return
    if args.workload == "field_sphere10242_k16":
        run_field(args)
        return
    if args.workload == "dl_sphere10242_k16_q7":
        run_dl(args)
        return
    if args.workload == "efie_sphere10242_k8_q3":
        run_efie(args)
        return
    if args.workload == "sphere163842_k64_q3_r16":
        run_large(args)
        return
    if args.workload == "hmat_sphere163842_k64_q3_r16":
        run_hmat(args)
        return
    if args.workload == "batch12_r64":
        run_batch(args)
        return
    if args.workload == "precond_ellipsoids":
        run_precond(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    run_gyps(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
