"""Benchmark of the matrix-free P1 hot path on one GB300 (or N replicas).

Workload (default): unit cube split into 6 Kuhn macro-tetrahedra, refined to
level 7 (129^3 = 2 146 689 vertex DoFs), P1 Laplacian with constant-coefficient
15-point stencils, FP32.  One step = one operator application y = A x through
the C ABI, including the ghost-layer exchange between macro primitives.
Inputs are seeded U[-1,1] vectors (zero Dirichlet values); 32 distinct (x, y)
pairs rotate between steps so the working set (563 MB) exceeds 4x L2.

Printed: one JSON line (rank 0) with the value in GDoF/s (unique DoFs per
second, all ranks), the roofline of the apply against the measured HBM peak,
the oracle's CSR SpMV timed on the host cores (cpu_baseline), an end-to-end
number through host buffers (e2e), and the SM clocks seen during timing.

``--impl reference`` times the CPU oracle (the only other arm this task has)
on the same metric: CSR SpMV of the same operator on a bounded sample.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthgen as sg  # noqa: E402

WORKLOAD = "cube6_L7_p1_laplace_apply_f32"
LEVEL = 7
N_PAIRS = 32
METRIC = "matvec GDoF/s (% HBM roofline); GMG time to 1e-8 resid, learned vs plain"
BYTES_PER_DOF = 8            # FP32: x read once + y written once per unique DoF
SAMPLE_LEVEL = 6             # oracle sample: same mesh one level coarser


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _kernel_source_sha():
    """Hash of the headline kernel's sources (the plane-window kernel and the
    interface items it includes)."""
    h = hashlib.sha256()
    for f in ("hg_p1.cu", "hg_p1dev.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2308_01792_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def _profiled_traffic():
    """DRAM bytes per apply from the committed ncu summary, if it matches the source."""
    path = os.path.join(ROOT, "profiles", "p1_apply_cube6_L7_f32.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    m = re.search(r"source_sha256_16:\s*([0-9a-f]+)", txt)
    t = re.search(r"traffic_bytes_per_apply:\s*([0-9.eE+]+)", txt)
    if not m or not t or m.group(1) != _kernel_source_sha():
        return None
    return float(t.group(1))


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.gpu_id = None
        self.path = os.path.join(tempfile.gettempdir(), f"hytet_clocks_{os.getpid()}.csv")

    @staticmethod
    def smi_gpu_id(device_index, run=subprocess.run):
        """The nvidia-smi --id of torch device `device_index`.  torch numbers
        only the devices CUDA_VISIBLE_DEVICES exposes, while nvidia-smi numbers
        every GPU of the machine, so the index can name another GPU; the
        device's UUID names the same one in both.  The UUID is used when torch
        reports it and nvidia-smi accepts it, else the index."""
        try:
            import torch
            u = str(torch.cuda.get_device_properties(device_index).uuid)
        except Exception:
            return str(device_index)
        gid = u if u.startswith("GPU-") else f"GPU-{u}"
        try:
            p = run(["nvidia-smi", f"--id={gid}", "--query-gpu=index", "--format=csv,noheader"],
                    capture_output=True, text=True, timeout=30)
            if p.returncode == 0 and p.stdout.strip():
                return gid
        except Exception:
            pass
        return str(device_index)

    def start(self):
        try:
            self.gpu_id = self.smi_gpu_id(self.dev)
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu_id}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
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
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        r = {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
             "samples": len(sm)}
        if self.gpu_id is not None:
            r["gpu"] = self.gpu_id
        return r


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate_replicas(ms, units_per_rank, steps, pg=None, device="cuda"):
    """Whole-job figures of N independent replicas: the timed region is the
    maximum over ranks (all_reduce MAX of each rank's CUDA-event time, ms) and
    every rank processed units_per_rank per step.  Returns (ms per step,
    units per second in units of 1e9)."""
    import torch
    ws = 1
    if pg is not None:
        t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms = float(t.item())
        ws = pg.get_world_size()
    ms_step = ms / steps
    return ms_step, units_per_rank * ws / (ms_step * 1e-3) / 1e9


def cpu_baseline_spmv(seconds=10.0):
    """Oracle CSR SpMV (SciPy, single thread) on the same mesh at SAMPLE_LEVEL."""
    from oracle import fem
    from oracle.mesh import RefinedMesh
    macro = sg.kuhn_cube(1)
    rm = RefinedMesh(macro, SAMPLE_LEVEL)
    A = fem.assemble(rm.cells, fem.p1_stiffness(rm.cell_xyz), rm.n_vertices)
    ii = rm.interior
    AII = A[ii][:, ii].tocsr()
    x = sg.uniform_vector(0, rm.n_vertices)[ii]
    y = AII @ x
    reps, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        y = AII @ x
        reps += 1
    dt = time.perf_counter() - t0
    return {"value": rm.n_vertices * reps / dt / 1e9, "unit": "GDoF/s", "cores": 1,
            "kind": "oracle", "host_cores": _host_cores(),
            "sample": f"SciPy CSR SpMV of the same P1 operator on the same mesh at level "
                      f"{SAMPLE_LEVEL} ({rm.n_vertices} DoFs), {reps} reps in {dt:.1f} s"}


ORACLE_GMG_LEVEL = 4          # oracle GMG sample: the GMG workload's mesh two levels coarser


def cpu_baseline_gmg(level=ORACLE_GMG_LEVEL):
    """The oracle's FP64 GMG (SciPy CSR, V(3,3) weighted Jacobi omega = 2/3,
    exact coarse solve on level 0) on the GMG workload's problem: 4x4x4 Kuhn
    cube, P1 -div(k grad) with the same log-normal k (seed 1000) and the same
    seeded right-hand side, to 1e-8 relative residual, at `level` instead of
    6.  Assembly is timed apart from the solve.  The level-6 figure is
    extrapolated linearly in the DoFs at the sample's V-cycle count, and
    labelled so."""
    from oracle import gmg as og
    macro = sg.kuhn_cube(4)
    p = sg.rff_params(1000)
    t0 = time.perf_counter()
    H = og.Hierarchy(macro, 0, level, kind="divkgrad", coeff=lambda xyz: sg.rff_eval(p, xyz))
    setup_s = time.perf_counter() - t0
    lev = H.levels[level]
    b = sg.uniform_vector(9, lev.n)[lev.interior]
    t0 = time.perf_counter()
    _, it, hist = og.solve(H, b, tol=1e-8, max_iter=200)
    solve_s = time.perf_counter() - t0
    n6 = (4 * 64 + 1) ** 3
    return {"kind": "oracle", "cores": 1, "host_cores": _host_cores(), "level": level,
            "unique_dofs": int(lev.n),
            "assembly_s": setup_s, "solve_s": solve_s, "v_cycles": it, "rel_res": hist[-1],
            "level6_solve_s_extrapolated": solve_s * n6 / lev.n,
            "sample": f"oracle GMG (SciPy CSR, single thread) of the GMG workload's problem at level "
                      f"{level} ({lev.n} DoFs); the level-6 time is extrapolated linearly in the "
                      f"DoFs at {it} V-cycles"}


GMG_WORKLOAD = "cube384_L6_p1_lognormal_gmg_to_1e-8"
# FP32 V-cycles per FP64 refinement step of the mixed solves (one FP64
# residual per step; measured on GB300: 3 beats 1 and 2 for both the P1
# div-k-grad and the P2 problem, whose FP64 residuals cost 8 ms and 26 ms).
# Plain FP64 solves do one V-cycle per residual as before.
INNER_CYCLES = 3
# The same for the 17 M-DoF log-normal problem of the multigrid and stencil
# legs, measured on GB300 over 2..6: Jacobi V(3,3) 0.169 / 0.143 / 0.144 /
# 0.135 / 0.117 s (9 / 6 / 5 / 4 / 3 steps), Chebyshev(2) V(1,1) 0.133 /
# 0.123 / 0.099 / 0.113 / 0.097 s: six FP32 cycles per FP64 residual (8 ms
# each on the fly) reach 1e-8 in 3 steps.
LOGNORMAL_INNER_CYCLES = 6
WEIGHTS = os.path.join(ROOT, "paper_2308_01792_gb300", "weights", "learned_smoother_cube384.npy")


def gmg_comparison(stream):
    """Time to 1e-8 relative residual on the 4x4x4 Kuhn cube (384 macro cells),
    level 6 (17 M DoFs), P1 -div(k grad), k = exp(g) log-normal (seed 1000),
    seeded U[-1,1] right-hand side: plain FP64 V(3,3) cycles vs FP32 V-cycles
    in FP64 refinement, without and with the learned smoother."""
    import torch
    import paper_2308_01792_gb300 as hg
    from paper_2308_01792_gb300 import learned
    macro = sg.kuhn_cube(4)
    t0 = time.perf_counter()
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), 0, 6)
    _, xyz, dirich = H.canonical_info(6)
    k = sg.rff_eval_torch(sg.rff_params(1000), xyz, dtype=torch.float32)
    op = hg.Operator(H, hg.HG_OP_P1_DIVKGRAD, coeff=k)
    bc = sg.uniform_vector(9, len(xyz))
    bc[dirich] = 0.0
    b = H.from_canonical(6, torch.tensor(bc, device="cuda"))
    setup_s = time.perf_counter() - t0
    if os.path.exists(WEIGHTS):
        net, trained = hg.MLP(np.load(WEIGHTS)), "loaded " + os.path.relpath(WEIGHTS, ROOT)
    else:
        X, t, npairs = learned.make_noise_pairs(macro, 0, 4, range(1, 25), 4, 2)
        net, loss = learned.train(X, t, steps=3000, batch=65536, lr=1e-3)
        trained = f"trained in bench: {npairs} noise pairs, loss {loss:.4g}"
    out = {"workload": GMG_WORKLOAD, "unique_dofs": int(len(xyz)), "tol": 1e-8,
           "setup_s": setup_s, "weights": trained,
           "fp32_cycles_per_refinement_step": LOGNORMAL_INNER_CYCLES}
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for name, prec, use in (("plain_f64", hg.HG_PREC_F64, False),
                            ("mixed_f32_ir", hg.HG_PREC_MIXED, False),
                            ("learned_mixed", hg.HG_PREC_MIXED, True)):
        G = hg.GMG(op, inner_cycles=LOGNORMAL_INNER_CYCLES)
        G.set_learned(net if use else None)
        x = H.zeros(6, torch.float64)
        G.solve(x, b, tol=1e-8, max_iter=200, precision=prec, stream=stream)   # warm-up
        torch.cuda.synchronize()
        e0.record(stream)
        it, rel = G.solve(x, b, tol=1e-8, max_iter=200, precision=prec, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        out[name] = {"s": e0.elapsed_time(e1) / 1e3, "iters": it, "rel_res": rel}
        if use:
            out[name]["fallbacks"] = G.learned_fallbacks()
        del G
    # fewer smoothing steps per level: Jacobi and learned V(2,2) and V(1,1)
    for nu in (2, 1):
        for name, use in ((f"mixed_f32_ir_v{nu}{nu}", False), (f"learned_mixed_v{nu}{nu}", True)):
            G = hg.GMG(op, nu1=nu, nu2=nu, inner_cycles=LOGNORMAL_INNER_CYCLES)
            G.set_learned(net if use else None)
            x = H.zeros(6, torch.float64)
            G.solve(x, b, tol=1e-8, max_iter=200, precision=hg.HG_PREC_MIXED, stream=stream)
            torch.cuda.synchronize()
            e0.record(stream)
            it, rel = G.solve(x, b, tol=1e-8, max_iter=200, precision=hg.HG_PREC_MIXED,
                              stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            out[name] = {"s": e0.elapsed_time(e1) / 1e3, "iters": it, "rel_res": rel}
            if use:
                out[name]["fallbacks"] = G.learned_fallbacks()
            del G
    out["learned_vs_plain_f64_speedup"] = out["plain_f64"]["s"] / out["learned_mixed"]["s"]
    out["learned_vs_mixed_speedup"] = out["mixed_f32_ir"]["s"] / out["learned_mixed"]["s"]
    # Chebyshev-accelerated Jacobi of order 2, V(1,1), FP32 cycles in FP64
    # refinement; then full multigrid with 5 V(1,1) Chebyshev cycles per level
    G = hg.GMG(op, nu1=1, nu2=1, inner_cycles=LOGNORMAL_INNER_CYCLES, smoother=hg.HG_SMOOTH_CHEB)
    x = H.zeros(6, torch.float64)
    G.solve(x, b, tol=1e-8, max_iter=200, precision=hg.HG_PREC_MIXED, stream=stream)
    torch.cuda.synchronize()
    e0.record(stream)
    it, rel = G.solve(x, b, tol=1e-8, max_iter=200, precision=hg.HG_PREC_MIXED, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    out["cheb2_v11_mixed_f32_ir"] = {"s": e0.elapsed_time(e1) / 1e3, "iters": it, "rel_res": rel}
    bb = H.dot(6, b, b)
    for name, dt in (("fmg_f32", torch.float32), ("fmg_f64", torch.float64)):
        xf = H.zeros(6, dt)
        bf = b.to(dt)
        G.fmg(6, xf, bf, cycles=5, stream=stream)
        torch.cuda.synchronize()
        e0.record(stream)
        G.fmg(6, xf, bf, cycles=5, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        r = H.zeros(6, torch.float64)
        op.residual(6, xf.double(), b, r)
        out[name] = {"s": e0.elapsed_time(e1) / 1e3, "cycles_per_level": 5,
                     "rel_res": float(np.sqrt(H.dot(6, r, r) / bb))}
    del G
    return out


BATCH_WORKLOAD = "batch512_p1_poisson_to_1e-8"


def batch_comparison(stream, count=512):
    """512 independent P1 Poisson problems (unit cube as m^3 sub-cubes x 6
    Kuhn tetrahedra, m in {1,2,3}, level in {3..6}, drawn with seed 42),
    seeded U[-1,1] right-hand sides, each solved to 1e-8 relative residual:
    one batched solve (a persistent launch per V-cycle stage over all
    problems, CUDA-graph replay, autotuned variant) against the same problems
    solved one after another."""
    import torch
    import paper_2308_01792_gb300 as hg
    draw = sg.batched_problem_draw(42, count)
    t0 = time.perf_counter()
    shared = {}
    Gs, xs, bs = [], [], []
    dofs = 0
    for p, (m, L) in enumerate(draw):
        if (m, L) not in shared:
            macro = sg.kuhn_cube(m)
            H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), 0, L)
            op = hg.Operator(H)
            _, xyz, dirich = H.canonical_info(L)
            shared[(m, L)] = [H, op, hg.GMG(op, inner_cycles=INNER_CYCLES), False, len(xyz),
                              dirich]
        H, op, G0, used, nu, dirich = shared[(m, L)]
        Gs.append(G0.clone() if used else G0)
        shared[(m, L)][3] = True
        bc = sg.uniform_vector(1000 + p, nu)
        bc[dirich] = 0.0
        bs.append(H.from_canonical(L, torch.tensor(bc, device="cuda")))
        xs.append(H.zeros(L, torch.float64))
        dofs += nu
    B = hg.Batch(Gs, xs, bs, graph=True, autotune=True)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    B.solve(tol=1e-8, max_iter=100, stream=stream)        # warm-up
    times = []
    for _ in range(3):
        e0.record(stream)
        it, rel = B.solve(tol=1e-8, max_iter=100, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    rows, gf, us = B.tuning()
    t_batch = float(np.median(times))
    # the same problems, one solve at a time (same kernels, no batching)
    x1 = [torch.zeros_like(v) for v in xs]
    Gs[0].solve(x1[0], bs[0], tol=1e-8, max_iter=100, precision=hg.HG_PREC_MIXED, stream=stream)
    torch.cuda.synchronize()
    e0.record(stream)
    its1 = []
    for p in range(count):
        i1, _ = Gs[p].solve(x1[p], bs[p], tol=1e-8, max_iter=100, precision=hg.HG_PREC_MIXED,
                            stream=stream)
        its1.append(i1)
    e1.record(stream)
    torch.cuda.synchronize()
    t_seq = e0.elapsed_time(e1) / 1e3
    return {"workload": BATCH_WORKLOAD, "problems": count, "unique_dofs_total": int(dofs),
            "fp32_cycles_per_refinement_step": INNER_CYCLES,
            "hierarchies": len(shared), "tol": 1e-8, "setup_s": setup_s,
            "batched": {"s": t_batch, "s_all": times, "iters_max": int(it.max()),
                        "iters_mean": float(it.mean()), "rel_res_max": float(rel.max()),
                        "gdof_per_s_solved": dofs / t_batch / 1e9,
                        "tuned_rows": rows, "tuned_grid_blocks_per_sm": 4 * gf,
                        "tuned_stage_us": us},
            "one_at_a_time": {"s": t_seq, "iters_max": int(max(its1)),
                              "iters_equal": bool(np.array_equal(np.array(its1), it))},
            "batched_vs_one_at_a_time_speedup": t_seq / t_batch}


P2_WORKLOAD = "cube48_L6_p2_sinprod"
# FP32 operations per micro-cell of the P2 stiffness apply: per quadrature point
# 6 (k: three separable sines) + 2 (kq) + 8 (C_q factors) + 16 (u = C^T x)
# + 20 (v = kq H u) + 16 (y += C v) multiply-add pairs or singles, counted as
# flops: 2 per FMA.
P2_FLOPS_PER_CELL = 14 * 2 * (3 + 1 + 4 + 16 + 20 + 16)
# FP32 CUDA-core peak: 152 SMs x 128 FP32 lanes x 2 flops per FMA x max SM clock
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# FP32 operations per micro-cell of the element-wise P1 -div(k grad) apply
# (scatter form, the minimum): k_T = mean of 4 vertex values (4), y_T = K x_T
# (16 FMA = 32), scaled by k_T (4)
DIVKGRAD_FLOPS_PER_CELL = 4 + 32 + 4


def p2_comparison(stream, level=6, solve=True):
    """P2 -div(k grad), k = 1 + 0.5 sin(2 pi x) sin(2 pi y) sin(2 pi z), on the
    unit cube as 2x2x2 sub-cubes x 6 Kuhn tetrahedra (48 macro cells), P2
    level 6 (257^3 DoFs): FP32 element-wise apply (on-the-fly quadrature), and
    the manufactured problem u = sin(pi x) sin(pi y) sin(pi z) solved to 1e-10
    by FP32 V-cycles in FP64 refinement and by FP64 V-cycles."""
    import torch
    import paper_2308_01792_gb300 as hg
    P2 = hg.HG_SPACE_P2
    macro = sg.kuhn_cube(2)
    t0 = time.perf_counter()
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), 0, level + 1)
    stiff = hg.Operator(H, hg.HG_OP_P2_DIVKGRAD, coeff=sg.SINPROD_AB)
    mass = hg.Operator(H, hg.HG_OP_P2_MASS)
    ns, nu, ni, _ = H.size(level, space=P2)
    _, xyz, dirich = H.canonical_info(level, space=P2)
    setup_s = time.perf_counter() - t0
    n_cells_micro = len(macro.cells) * 8 ** level
    # apply throughput, 4 rotating pairs (4 x 2 x 70 MB > L2)
    xs = [H.from_canonical(level, torch.tensor(sg.uniform_vector(300 + q, nu), dtype=torch.float32,
                                               device="cuda"), space=P2) for q in range(4)]
    ys = [torch.zeros_like(v) for v in xs]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for q in range(3):
        stiff.apply(level, xs[q % 4], ys[q % 4], stream=stream)
    torch.cuda.synchronize()
    K = 20
    e0.record(stream)
    for q in range(K):
        stiff.apply(level, xs[q % 4], ys[q % 4], stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t_apply = e0.elapsed_time(e1) / K * 1e-3
    tflops = P2_FLOPS_PER_CELL * n_cells_micro / t_apply / 1e12
    out = {"workload": P2_WORKLOAD, "unique_dofs": int(nu), "interior_dofs": int(ni),
           "fp32_cycles_per_refinement_step": INNER_CYCLES,
           "micro_cells": int(n_cells_micro), "setup_s": setup_s,
           "apply_f32": {"us": t_apply * 1e6, "gdof_per_s": nu / t_apply / 1e9,
                         "tflops": tflops, "roofline": {"bound": "alu", "achieved": tflops,
                                                        "peak": FP32_PEAK_TFLOPS,
                                                        "unit": "TFLOP/s",
                                                        "frac": tflops / FP32_PEAK_TFLOPS}}}
    del xs, ys
    if not solve:
        return out
    u, f = sg.sinprod_manufactured(xyz, *sg.SINPROD_AB)
    b = H.zeros(level, torch.float64, space=P2)
    mass.apply(level, H.from_canonical(level, torch.tensor(f, device="cuda"), space=P2), b,
               stream=stream)
    sol = {}
    for name, prec in (("mixed_f32_ir", hg.HG_PREC_MIXED), ("plain_f64", hg.HG_PREC_F64)):
        G = hg.GMG(stiff, lmin=0, inner_cycles=INNER_CYCLES)
        x = H.zeros(level, torch.float64, space=P2)
        torch.cuda.synchronize()
        e0.record(stream)
        it, rel = G.solve(x, b, tol=1e-10, max_iter=100, precision=prec, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        xc = H.to_canonical(level, x, space=P2).cpu().numpy()
        sol[name] = xc
        out[name] = {"s": e0.elapsed_time(e1) / 1e3, "iters": it, "rel_res": rel,
                     "max_err_vs_u": float(np.max(np.abs(xc - u)))}
        del G
    out["mixed_vs_f64_rel_diff"] = float(np.linalg.norm(sol["mixed_f32_ir"] - sol["plain_f64"]) /
                                         np.linalg.norm(sol["plain_f64"]))
    out["mixed_vs_f64_speedup"] = out["plain_f64"]["s"] / out["mixed_f32_ir"]["s"]
    return out


N1_WORKLOAD = "cube48_L6_n1_curlcurl_apply"


def n1_comparison(stream, level=6):
    """Lowest-order Nedelec alpha curl curl + beta I (alpha = 1, beta = 0.3) on
    the unit cube as 2x2x2 sub-cubes x 6 Kuhn tetrahedra (48 macro cells),
    N1 level 6 (one DoF per micro-edge): FP32 and FP64 element-wise apply
    (colour phases + finish pass), CUDA-event time per apply, 4 rotating
    input vectors (> L2)."""
    import torch
    import paper_2308_01792_gb300 as hg
    P2 = hg.HG_SPACE_P2
    macro = sg.kuhn_cube(2)
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), level, level + 1)
    op = hg.Operator(H, hg.HG_OP_N1_CURLCURL, coeff=(1.0, 0.3))
    ns, nu, _, _ = H.size(level, space=P2)
    n = 1 << level
    cells = len(macro.cells)
    # unique micro-edges = doubled-lattice points of the cube (2 * 2n + 1 per
    # side for 2 sub-cubes per side) minus its vertex points (2n + 1 per side)
    edges = (4 * n + 1) ** 3 - (2 * n + 1) ** 3
    peak, kind = _peaks()
    out = {"workload": N1_WORKLOAD, "edge_dofs": int(edges), "micro_cells": int(cells * 8 ** level)}
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for dt, w in ((torch.float32, 4), (torch.float64, 8)):
        xs = [torch.rand(ns, dtype=dt, device="cuda") for _ in range(4)]
        ys = [torch.zeros_like(v) for v in xs]
        for q in range(3):
            op.apply(level, xs[q], ys[q], stream=stream)
        torch.cuda.synchronize()
        K = 20
        e0.record(stream)
        for q in range(K):
            op.apply(level, xs[q % 4], ys[q % 4], stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / K * 1e-3
        gbs = 2 * w * edges / t / 1e9
        out["apply_f32" if w == 4 else "apply_f64"] = {
            "us": t * 1e6, "gdof_per_s": edges / t / 1e9,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                         "frac": gbs / peak, "peak_source": f"{kind} hbm_gbs",
                         "algorithmic_bytes_per_launch": 2 * w * edges}}
        del xs, ys
    return out


N1_SOLVE_WORKLOAD = "cube48_L6_n1_curlcurl_hiptmair_gmg_to_1e-8"


def n1_solve_comparison(stream, level=6, m=2):
    """The Nedelec problem alpha curl curl u + beta u = f (alpha = 1,
    beta = 0.3) on the same 48-cell cube at N1 level 6 (14.8 M edge DoFs),
    seeded U[-1,1] right-hand side on the interior edges: multigrid with
    Hiptmair's hybrid smoother (weighted Jacobi, omega = 1/2, in the edge and
    the potential space), coarsest level 1.  Solves to 1e-8 relative residual
    with FP32 V(2,2) cycles in FP64 refinement and with FP64 V(2,2) cycles,
    and one FP32 FMG pass with 5 V(1,1) per level; then the paper's
    smoother, order-2 Chebyshev in both spaces: the mixed solve with V(1,1)
    and one FP32 FMG pass with 5 V(1,1) per level."""
    import torch
    import paper_2308_01792_gb300 as hg
    P2 = hg.HG_SPACE_P2
    macro = sg.kuhn_cube(m)
    t0 = time.perf_counter()
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), 0, level + 1)
    op = hg.Operator(H, hg.HG_OP_N1_CURLCURL, coeff=(1.0, 0.3))
    _, xyz, dirich = H.canonical_info(level, space=P2)
    # edge DoFs: points of the level+1 lattice with an odd coordinate
    q = np.rint(xyz * (m << (level + 1))).astype(np.int64)
    edge = np.any(q % 2 == 1, axis=1)
    bc = sg.uniform_vector(11, len(xyz))
    bc[dirich | ~edge] = 0.0
    b = H.from_canonical(level, torch.tensor(bc, device="cuda"), space=P2)
    setup_s = time.perf_counter() - t0
    out = {"workload": N1_SOLVE_WORKLOAD, "edge_dofs": int(edge.sum()),
           "interior_edge_dofs": int((edge & ~dirich).sum()), "tol": 1e-8, "setup_s": setup_s,
           "smoother": "Hiptmair, weighted Jacobi omega = 0.5 in both spaces",
           "fp32_cycles_per_refinement_step": INNER_CYCLES}
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    G = hg.GMG(op, nu1=2, nu2=2, omega=0.5, lmin=1, inner_cycles=INNER_CYCLES)
    for name, prec in (("mixed_f32_ir", hg.HG_PREC_MIXED), ("plain_f64", hg.HG_PREC_F64)):
        x = H.zeros(level, torch.float64, space=P2)
        G.solve(x, b, tol=1e-8, max_iter=100, precision=prec, stream=stream, check=False)
        torch.cuda.synchronize()                                  # warm-up, then from x = 0
        x.zero_()
        e0.record(stream)
        it, rel = G.solve(x, b, tol=1e-8, max_iter=100, precision=prec, stream=stream, check=False)
        e1.record(stream)
        torch.cuda.synchronize()
        out[name] = {"s": e0.elapsed_time(e1) / 1e3, "iters": it, "rel_res": rel,
                     "timed_after_warmup": True}
    out["mixed_vs_f64_speedup"] = out["plain_f64"]["s"] / out["mixed_f32_ir"]["s"]
    del G
    # the paper's smoother: order-2 Chebyshev in both spaces, V(1,1)
    G = hg.GMG(op, nu1=1, nu2=1, lmin=1, inner_cycles=INNER_CYCLES, smoother=hg.HG_SMOOTH_CHEB)
    x = H.zeros(level, torch.float64, space=P2)
    G.solve(x, b, tol=1e-8, max_iter=100, precision=hg.HG_PREC_MIXED, stream=stream, check=False)
    torch.cuda.synchronize()
    x.zero_()
    e0.record(stream)
    it, rel = G.solve(x, b, tol=1e-8, max_iter=100, precision=hg.HG_PREC_MIXED, stream=stream,
                      check=False)
    e1.record(stream)
    torch.cuda.synchronize()
    out["mixed_f32_ir_cheb2_v11"] = {"s": e0.elapsed_time(e1) / 1e3, "iters": it, "rel_res": rel,
                                     "timed_after_warmup": True}
    xf = H.zeros(level, torch.float32, space=P2)
    bf = b.float()
    G.fmg(level, xf, bf, cycles=5, stream=stream)
    torch.cuda.synchronize()
    e0.record(stream)
    G.fmg(level, xf, bf, cycles=5, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    r = H.zeros(level, torch.float64, space=P2)
    op.residual(level, xf.double(), b, r)
    out["fmg_f32_cheb2"] = {"s": e0.elapsed_time(e1) / 1e3, "cycles_per_level": 5,
                            "rel_res": float(np.sqrt(H.dot(level, r, r, space=P2) /
                                                     H.dot(level, b, b, space=P2)))}
    del G
    G = hg.GMG(op, nu1=1, nu2=1, omega=0.5, lmin=1)
    xf = H.zeros(level, torch.float32, space=P2)
    bf = b.float()
    G.fmg(level, xf, bf, cycles=5, stream=stream)
    torch.cuda.synchronize()
    e0.record(stream)
    G.fmg(level, xf, bf, cycles=5, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    r = H.zeros(level, torch.float64, space=P2)
    op.residual(level, xf.double(), b, r)
    out["fmg_f32"] = {"s": e0.elapsed_time(e1) / 1e3, "cycles_per_level": 5,
                      "rel_res": float(np.sqrt(H.dot(level, r, r, space=P2) /
                                               H.dot(level, b, b, space=P2)))}
    del G
    return out


KERNELS_WORKLOAD = "cube384_L6_p1_laplace_kernels"


def kernels_comparison(stream):
    """Every P1 multigrid kernel on its own, HBM-cold: the 4x4x4 Kuhn cube
    (384 macro cells), level 6 (17 M DoFs, vectors of 70 MB FP32 > L2),
    constant-coefficient P1 Laplacian; plus the headline apply L2-hot (the
    6-cell level-7 x and y reused every rep).  Per kernel: CUDA-event time
    per launch (mean of 20 after 3 warm-up), algorithmic bytes (unique DoFs
    of the level, the transfers per fine DoF) and the fraction of the measured
    HBM bandwidth."""
    import torch
    import paper_2308_01792_gb300 as hg
    macro = sg.kuhn_cube(4)
    L = 6
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), L - 1, L)
    op = hg.Operator(H)
    ns, nu, _, _ = H.size(L)
    nuc = H.size(L - 1)[1]
    peak, kind = _peaks()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def tm(f, K=20):
        for _ in range(3):
            f()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(K):
            f()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / K * 1e-3

    out = {"workload": KERNELS_WORKLOAD, "unique_dofs": int(nu), "peak_gbs": peak,
           "peak_source": f"{kind} hbm_gbs"}

    def rec(name, t, nbytes, note=None):
        gbs = nbytes / t / 1e9
        out[name] = {"us": t * 1e6, "gb_per_s": gbs, "frac": gbs / peak, "bytes": int(nbytes)}
        if note:
            out[name]["note"] = note

    for dt, w in ((torch.float32, 4), (torch.float64, 8)):
        tag = "f32" if dt == torch.float32 else "f64"
        x = H.from_canonical(L, torch.tensor(sg.uniform_vector(21, nu), dtype=dt, device="cuda"))
        b = H.from_canonical(L, torch.tensor(sg.uniform_vector(22, nu), dtype=dt, device="cuda"))
        y = torch.zeros_like(x)
        rec(f"apply_{tag}", tm(lambda: op.apply(L, x, y, stream=stream)), 2 * w * nu,
            None if w == 4 else "FP64 arithmetic binds on GB300")
        rec(f"residual_{tag}", tm(lambda: op.residual(L, x, b, y, stream=stream)), 3 * w * nu)
        rec(f"jacobi_{tag}", tm(lambda: op.jacobi(L, x, b, y, stream=stream)), 3 * w * nu)
        if w == 4:
            xc = torch.zeros(H.size(L - 1)[0], dtype=dt, device="cuda")
            # restriction: fine residual read, coarse written; prolongation: coarse
            # read, fine read and written
            rec("restrict_f32", tm(lambda: H.restrict(L, x, xc, stream=stream)), w * (nu + nuc))
            rec("prolong_f32", tm(lambda: H.prolong_add(L, xc, y, stream=stream)),
                w * (2 * nu + nuc))
            rec("dot_f32", tm(lambda: H.dot(L, x, b, stream=stream), 10), 2 * w * nu,
                "includes the host read of the result")
        del x, b, y
    # the three constant-stencil kernels on the same applies (FP32 and FP64;
    # the 384-cell vectors of this leg, then the headline mesh with 16
    # rotating pairs)
    modes = {"windows": hg.HG_P1_KERNEL_WINDOWS, "stream": hg.HG_P1_KERNEL_STREAM,
             "march": hg.HG_P1_KERNEL_MARCH}
    m6 = sg.kuhn_cube(1)
    H6 = hg.Hierarchy(hg.Mesh(m6.xyz, m6.cells), LEVEL, LEVEL)
    op6 = hg.Operator(H6)
    nu6 = H6.size(LEVEL)[1]
    for dt, w in ((torch.float32, 4), (torch.float64, 8)):
        tag = "f32" if w == 4 else "f64"
        x = H.from_canonical(L, torch.tensor(sg.uniform_vector(21, nu), dtype=dt, device="cuda"))
        y = torch.zeros_like(x)
        xs6 = [H6.from_canonical(LEVEL, torch.tensor(sg.uniform_vector(40 + q, nu6), dtype=dt,
                                                     device="cuda")) for q in range(16)]
        ys6 = [torch.zeros_like(v) for v in xs6]
        for name, mode in modes.items():
            hg.set_p1_kernel(mode)
            rec(f"apply_{tag}_{name}", tm(lambda: op.apply(L, x, y, stream=stream)), 2 * w * nu)
            it6 = iter(range(1 << 30))

            def ap6():
                q = next(it6) % 16
                op6.apply(LEVEL, xs6[q], ys6[q], stream=stream)
            rec(f"apply_{tag}_{name}_cube6_L7", tm(ap6, 64), 2 * w * nu6)
        hg.set_p1_kernel(hg.HG_P1_KERNEL_AUTO)
        del x, y, xs6, ys6
    # the copy ceiling: a device-to-device copy moving the apply's algorithmic
    # bytes (4 B read + 4 B written per unique DoF) at both sizes, HBM-cold
    # (rotating buffers), CUDA events over 20 copies after 3 warm-up
    n1u = (1 * (1 << LEVEL) + 1) ** 3
    for name, cnt in (("copy_ceiling_cube6_L7", n1u), ("copy_ceiling_cube384_L6", nu)):
        nb = max(2, int(np.ceil(4 * 129e6 / (8 * cnt))))         # > 4x L2 in all
        src = [torch.empty(cnt, dtype=torch.float32, device="cuda").fill_(1.0) for _ in range(nb)]
        dst = [torch.empty_like(v) for v in src]
        it = iter(range(1 << 30))

        def cp():
            q = next(it) % nb
            dst[q].copy_(src[q])
        rec(name, tm(cp), 8 * cnt, "torch copy_ (library kernel) of the apply's bytes: the "
                                   "device-side ceiling at this size")
        del src, dst
    # the headline apply with x and y resident in L2
    m1 = sg.kuhn_cube(1)
    H1 = hg.Hierarchy(hg.Mesh(m1.xyz, m1.cells), LEVEL, LEVEL)
    op1 = hg.Operator(H1)
    nu1 = H1.size(LEVEL)[1]
    x = H1.from_canonical(LEVEL, torch.tensor(sg.uniform_vector(23, nu1), dtype=torch.float32,
                                              device="cuda"))
    y = torch.zeros_like(x)
    rec("apply_f32_l2hot_cube6_L7", tm(lambda: op1.apply(LEVEL, x, y, stream=stream), 200),
        8 * nu1, "x and y (17 MB) stay in L2; not an HBM figure")
    return out


STENCIL_WORKLOAD = "cube384_L6_p1_lognormal_stored_vs_onthefly"


def stencil_comparison(stream, m=4, L=6, solve=True):
    """P1 -div(k grad) on the 4x4x4 Kuhn cube (384 macro cells), level 6
    (17 M DoFs), k = exp(g) log-normal (seed 1000): FP32 apply with element
    matrices on the fly against the stored-stencil form (grid-aware
    precomputation: 15 weights per stored point streamed from HBM), and the
    mixed-precision GMG solve to 1e-8 with each (Jacobi V(3,3); the stored form
    also with Chebyshev(2) V(1,1))."""
    import torch
    import paper_2308_01792_gb300 as hg
    macro = sg.kuhn_cube(m)
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), 0, L)
    _, xyz, dirich = H.canonical_info(L)
    k = sg.rff_eval_torch(sg.rff_params(1000), xyz, dtype=torch.float32)
    t0 = time.perf_counter()
    fly = hg.Operator(H, hg.HG_OP_P1_DIVKGRAD, coeff=k)
    t1 = time.perf_counter()
    st = hg.Operator(H, hg.HG_OP_P1_DIVKGRAD_STORED, coeff=k)
    t2 = time.perf_counter()
    ns, nu, _, _ = H.size(L)
    n = 1 << L
    lattice = len(macro.cells) * (n + 1) * (n + 2) * (n + 3) // 6
    bytes_st = lattice * (15 * 4 + 4 + 4)       # weights, x and y of every stored point
    x = H.from_canonical(L, torch.tensor(sg.uniform_vector(5, nu), dtype=torch.float32,
                                         device="cuda"))
    y = torch.zeros_like(x)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    out = {"workload": STENCIL_WORKLOAD if (m, L) == (4, 6) else f"cube{6 * m ** 3}_L{L}",
           "unique_dofs": int(nu), "stored_points": int(lattice),
           "setup_s": {"onthefly": t1 - t0, "stored": t2 - t1},
           "stored_stencil_gb_per_level_f32": 15 * 4 * ns / 1e9,
           "l2": "x, y and the 1.1 GB of weights exceed L2; no flush needed"}
    peak, kind = _peaks()
    for name, op in (("onthefly", fly), ("stored", st)):
        for _ in range(5):
            op.apply(L, x, y, stream=stream)
        torch.cuda.synchronize()
        K = 50
        e0.record(stream)
        for _ in range(K):
            op.apply(L, x, y, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / K * 1e-3
        out[name] = {"apply_us": t * 1e6, "gdof_per_s": nu / t / 1e9}
    ach = bytes_st / (out["stored"]["apply_us"] * 1e-6) / 1e9
    out["stored"]["roofline"] = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                                 "frac": ach / peak, "peak_source": f"{kind} hbm_gbs",
                                 "algorithmic_bytes_per_launch": bytes_st}
    # on the fly: x, y and k (FP32) once per unique DoF; per micro-cell the
    # element-wise form's k_T (3 adds + 1 multiply), the 4x4 element row
    # products (16 FMA) and the scaling of the 4 results by k_T
    t_fly = out["onthefly"]["apply_us"] * 1e-6
    micro = len(macro.cells) * 8 ** L
    gbs_fly = 12 * nu / t_fly / 1e9
    tf_fly = DIVKGRAD_FLOPS_PER_CELL * micro / t_fly / 1e12
    out["onthefly"]["roofline"] = {
        "bound": "alu", "achieved": tf_fly, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
        "frac": tf_fly / FP32_PEAK_TFLOPS, "flops_per_micro_cell": DIVKGRAD_FLOPS_PER_CELL,
        "hbm": {"achieved": gbs_fly, "peak": peak, "unit": "GB/s", "frac": gbs_fly / peak,
                "algorithmic_bytes_per_launch": 12 * nu, "peak_source": f"{kind} hbm_gbs"}}
    out["stored_vs_onthefly_apply_speedup"] = out["onthefly"]["apply_us"] / out["stored"]["apply_us"]
    # polynomial surrogates of degree 2 and 3: apply time, and the distance of
    # their result from the exact operator's on the same x (INNER rows)
    y_ex = torch.zeros_like(x)
    fly.apply(L, x, y_ex, stream=stream)
    for q in (2, 3):
        t0 = time.perf_counter()
        sur = hg.Operator(H, hg.HG_OP_P1_DIVKGRAD_SURROGATE, coeff=k, degree=q)
        t_setup = time.perf_counter() - t0
        for _ in range(5):
            sur.apply(L, x, y, stream=stream)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(50):
            sur.apply(L, x, y, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) / 50 * 1e-3
        err = float((y - y_ex).abs().max() / y_ex.abs().max())
        gbs = 8 * nu / t / 1e9
        out[f"surrogate_q{q}"] = {
            "apply_us": t * 1e6, "gdof_per_s": nu / t / 1e9, "setup_s": t_setup,
            "rel_max_diff_vs_exact": err,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                         "frac": gbs / peak, "algorithmic_bytes_per_launch": 8 * nu,
                         "peak_source": f"{kind} hbm_gbs"}}
        del sur
    if not solve:
        return out
    bc = sg.uniform_vector(9, nu)
    bc[dirich] = 0.0
    b = H.from_canonical(L, torch.tensor(bc, device="cuda"))
    for name, op, cheb in (("onthefly", fly, False), ("stored", st, False), ("stored", st, True)):
        inner = LOGNORMAL_INNER_CYCLES
        G = (hg.GMG(op, nu1=1, nu2=1, inner_cycles=inner, smoother=hg.HG_SMOOTH_CHEB) if cheb
             else hg.GMG(op, inner_cycles=inner))
        xs = H.zeros(L, torch.float64)
        G.solve(xs, b, tol=1e-8, max_iter=200, precision=hg.HG_PREC_MIXED, stream=stream)
        torch.cuda.synchronize()
        e0.record(stream)
        it, rel = G.solve(xs, b, tol=1e-8, max_iter=200, precision=hg.HG_PREC_MIXED, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        out[name]["mixed_solve_cheb2_v11" if cheb else "mixed_solve"] = {
            "s": e0.elapsed_time(e1) / 1e3, "iters": it, "rel_res": rel}
        del G
    return out


LEARNED_WORKLOAD = "learned_smoother_kernels"
# Tensor-core work of the network per sample: layer 1 (16 x 32) and layer 2
# (32 x 32) multiply-adds, 2 flops each; the gradient adds dW2, dH1 and dW1
# (32 x 32, 32 x 32, 16 x 32 multiply-adds).
MLP_FWD_TC_FLOPS = 2 * (16 * 32 + 32 * 32)
MLP_GRAD_TC_FLOPS = MLP_FWD_TC_FLOPS + 2 * (32 * 32 + 32 * 32 + 16 * 32)


def _bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def learned_kernels_comparison(stream, m=4, L=6, samples=1 << 22):
    """The learned smoother's BF16 tensor-core kernels on their own: the
    forward pass over `samples` FP32 feature rows (16 per sample), the
    gradient over as many BF16 rows (with its partial sums and the host read
    of the 1568 gradient values), and one learned smoothing step on the
    m^3 x 6 Kuhn cube at level L (FP32 x, r and the inverse diagonal of the
    log-normal -div(k grad) operator).  Per kernel: CUDA-event time per call
    (mean of 10 after 3 warm-up), bytes that must cross HBM and tensor-core
    flops against the measured bf16 peak."""
    import torch
    import paper_2308_01792_gb300 as hg
    peak_hbm, kind = _peaks()
    peak_tc, kind_tc = _bf16_peak()
    g = torch.Generator(device="cuda")
    g.manual_seed(5)
    net = hg.MLP(np.load(WEIGHTS)) if os.path.exists(WEIGHTS) else hg.MLP(
        sg.uniform_vector(3, hg.N_MLP_PARAMS) * 0.2)
    X = torch.rand(samples, 16, device="cuda", generator=g) * 2 - 1
    Xb = X.to(torch.bfloat16)
    t = torch.rand(samples, device="cuda", generator=g)
    out_f = torch.empty(samples, device="cuda")
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def tm(f, K=10):
        for _ in range(3):
            f()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(K):
            f()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / K * 1e-3

    def rec(tsec, nbytes, tc_flops):
        gbs, tf = nbytes / tsec / 1e9, tc_flops / tsec / 1e12
        return {"us": tsec * 1e6, "hbm": {"achieved": gbs, "peak": peak_hbm, "unit": "GB/s",
                                          "frac": gbs / peak_hbm, "bytes": int(nbytes)},
                "tensor": {"achieved": tf, "peak": peak_tc, "unit": "TFLOP/s",
                           "frac": tf / peak_tc, "flops": int(tc_flops),
                           "peak_source": f"{kind_tc} bf16_tflops"}}

    out = {"workload": LEARNED_WORKLOAD, "samples": samples,
           "mma": "mma.sync m16n8k16 bf16 -> f32"}
    out["mlp_forward"] = rec(tm(lambda: net.forward(X, out=out_f, stream=stream)),
                             samples * (64 + 4), samples * MLP_FWD_TC_FLOPS)
    out["mlp_grad"] = rec(tm(lambda: net.grad(Xb, t, stream=stream)), samples * (32 + 4),
                          samples * MLP_GRAD_TC_FLOPS)
    out["mlp_grad"]["note"] = "includes the partial-sum pass and the host read of the gradient"
    del X, Xb, t, out_f
    macro = sg.kuhn_cube(m)
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), L, L)
    _, xyz, _ = H.canonical_info(L)
    k = sg.rff_eval_torch(sg.rff_params(1000), xyz, dtype=torch.float32)
    op = hg.Operator(H, hg.HG_OP_P1_DIVKGRAD, coeff=k)
    ns, nu, _, _ = H.size(L)
    x = H.from_canonical(L, torch.tensor(sg.uniform_vector(41, nu), dtype=torch.float32,
                                         device="cuda"))
    r = H.from_canonical(L, torch.tensor(sg.uniform_vector(42, nu), dtype=torch.float32,
                                         device="cuda"))
    xo = torch.empty_like(x)
    n = 1 << L
    interior = len(macro.cells) * (n - 1) * (n - 2) * (n - 3) // 6     # cell-interior DoFs
    ts = tm(lambda: hg.learned_step(op, net, L, x, r, xo, 2.0 / 3.0, stream=stream))
    out["learned_step"] = rec(ts, 16 * ns, interior * MLP_FWD_TC_FLOPS)
    out["learned_step"].update({"mesh": f"cube{len(macro.cells)}_L{L}", "stored_points": int(ns),
                                "cell_interior_dofs": int(interior)})
    return out


def _host_cores():
    """Cores of this host as the process sees them (affinity), and in all."""
    try:
        usable = len(os.sched_getaffinity(0))
    except AttributeError:
        usable = os.cpu_count()
    return {"usable": usable, "total": os.cpu_count()}


def _oracle_threads():
    """Threads the oracle's SciPy/NumPy calls use: CSR products are single
    threaded; dense BLAS (the coarse solve) may use the BLAS pool."""
    return 1


def _manufactured_rhs(H, mass, level, stream, dtype=None):
    """b = M I_h f (interior rows, Dirichlet rows 0) of f = 3 pi^2 sin(pi x)
    sin(pi y) sin(pi z), with the library's P1 mass operator; returns
    (b stored FP64, u = I_h u canonical, xyz, dirichlet mask)."""
    import torch
    _, xyz, dirich = H.canonical_info(level)
    u = np.prod(np.sin(np.pi * xyz), axis=1)
    f = 3 * np.pi ** 2 * u
    b = H.zeros(level, torch.float64)
    mass.apply(level, H.from_canonical(level, torch.tensor(f, device="cuda")), b, stream=stream)
    return b, u, xyz, dirich


REFTET_WORKLOAD = "reftet_L4_p1_poisson_f64"


def reftet_comparison(stream, level=4, reps=100):
    """The reference tetrahedron (0,0,0),(1,0,0),(0,1,0),(0,0,1) refined to
    level 4 (n = 16, 969 vertex DoFs), P1 Poisson with zero Dirichlet values,
    FP64: (a) 100 operator applications to a seeded U[-1,1] vector (CUDA
    events around the 100 launches; the apply is launch-bound at this size),
    (b) GMG V(3,3), weighted Jacobi 2/3, coarsest level 2, from x = 0 to 1e-10
    relative residual with b = M I_h f, f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z)
    (not zero on the slanted face; the solve is defined all the same).  The
    oracle (SciPy CSR, one thread) does the same work on the host, timed
    beside it, and gives the parity of both results."""
    import torch
    import paper_2308_01792_gb300 as hg
    from oracle import gmg as og
    macro = sg.reference_tet()
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), 2, level)
    op = hg.Operator(H)
    mass = hg.Operator(H, hg.HG_OP_P1_MASS)
    ns, nu, ni, _ = H.size(level)
    _, xyz, dirich = H.canonical_info(level)
    xc = sg.uniform_vector(31, nu)
    xc[dirich] = 0.0
    x = H.from_canonical(level, torch.tensor(xc, device="cuda"))
    y = H.zeros(level, torch.float64)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for _ in range(10):
        op.apply(level, x, y, stream=stream)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        op.apply(level, x, y, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t_mv = e0.elapsed_time(e1) * 1e-3
    yg = H.to_canonical(level, y).cpu().numpy()
    Ho = og.Hierarchy(macro, 2, level)
    lev = Ho.levels[level]
    ii = lev.interior
    xi = xc[ii]
    yo = lev.A @ xi
    t0 = time.perf_counter()
    for _ in range(reps):
        yo = lev.A @ xi
    t_mv_cpu = time.perf_counter() - t0
    out = {"workload": REFTET_WORKLOAD, "unique_dofs": int(nu), "interior_dofs": int(ni),
           "matvecs": {"count": reps, "gpu_s": t_mv, "us_per_matvec": t_mv / reps * 1e6,
                       "gdof_per_s": nu * reps / t_mv / 1e9,
                       "max_rel_err_vs_oracle": float(np.abs(yg[ii] - yo).max() / np.abs(yo).max()),
                       "oracle_s": t_mv_cpu, "oracle_threads": _oracle_threads(),
                       "note": "launch-bound: 969 DoFs per launch"}}
    b, u, _, _ = _manufactured_rhs(H, mass, level, stream)
    G = hg.GMG(op)
    xs = H.zeros(level, torch.float64)
    G.solve(xs, b, tol=1e-10, max_iter=100, stream=stream)          # warm-up
    torch.cuda.synchronize()
    xs.zero_()
    e0.record(stream)
    it, rel = G.solve(xs, b, tol=1e-10, max_iter=100, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    xg = H.to_canonical(level, xs).cpu().numpy()[ii]
    bo = H.to_canonical(level, b).cpu().numpy()[ii]
    t0 = time.perf_counter()
    xo, ito, _ = og.solve(Ho, bo, tol=1e-10)
    t_cpu = time.perf_counter() - t0
    out["vcycle_solve"] = {"s": e0.elapsed_time(e1) / 1e3, "iters": it, "rel_res": rel,
                           "smoother": "weighted Jacobi 2/3, V(3,3), coarsest level 2",
                           "rel_diff_vs_oracle_solution": float(np.linalg.norm(xg - xo) /
                                                                np.linalg.norm(xo)),
                           "oracle_s": t_cpu, "oracle_iters": ito,
                           "oracle_threads": _oracle_threads()}
    out["host_cores"] = _host_cores()
    return out


CUBE6_WORKLOAD = "cube6_L7_p1_poisson_sweeps_and_solve"


def cube6_comparison(stream, level=LEVEL, series=(3, 4, 5, 6, 7), oracle_levels=(3, 4, 5)):
    """The headline mesh (unit cube as 6 Kuhn macro-tetrahedra, level 7,
    129^3 DoFs, P1 Poisson, zero Dirichlet values): the FP64 apply sweep
    HBM-cold (32 rotating x/y pairs, 1.1 GB), the GMG V(3,3) solve of the
    manufactured problem u = sin(pi x) sin(pi y) sin(pi z) to 1e-10 (FP64
    cycles, and FP32 cycles in FP64 refinement), and the discretisation
    error ||I_h u - u_h||_M for levels 3..7 (ratios near 4 for O(h^2)), the
    oracle's errors beside it on the levels it finishes in seconds."""
    import torch
    import paper_2308_01792_gb300 as hg
    from oracle import gmg as og
    macro = sg.kuhn_cube(1)
    mesh = hg.Mesh(macro.xyz, macro.cells)
    peak, kind = _peaks()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    H = hg.Hierarchy(mesh, 1, level)
    op = hg.Operator(H)
    mass = hg.Operator(H, hg.HG_OP_P1_MASS)
    ns, nu, ni, _ = H.size(level)
    _, _, dirich = H.canonical_info(level)
    out = {"workload": CUBE6_WORKLOAD, "unique_dofs": int(nu), "stored_dofs": int(ns)}
    xs, ys = [], []
    for p in range(N_PAIRS):
        c = sg.uniform_vector(2000 + p, nu)
        c[dirich] = 0.0
        xs.append(H.from_canonical(level, torch.tensor(c, device="cuda")))
        ys.append(H.zeros(level, torch.float64))
    for q in range(3):
        op.apply(level, xs[q], ys[q], stream=stream)
    torch.cuda.synchronize()
    K = 64
    e0.record(stream)
    for q in range(K):
        op.apply(level, xs[q % N_PAIRS], ys[q % N_PAIRS], stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / K * 1e-3
    gbs = 16 * nu / t / 1e9
    out["apply_f64"] = {"us": t * 1e6, "gdof_per_s": nu / t / 1e9,
                        "l2": f"{N_PAIRS} rotating x/y pairs, {N_PAIRS * 2 * ns * 8 / 1e9:.1f} GB",
                        "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                                     "frac": gbs / peak, "peak_source": f"{kind} hbm_gbs",
                                     "algorithmic_bytes_per_launch": 16 * nu}}
    del xs, ys
    b, u, _, _ = _manufactured_rhs(H, mass, level, stream)
    for name, prec in (("plain_f64", hg.HG_PREC_F64), ("mixed_f32_ir", hg.HG_PREC_MIXED)):
        G = hg.GMG(op, inner_cycles=INNER_CYCLES)
        x = H.zeros(level, torch.float64)
        G.solve(x, b, tol=1e-10, max_iter=100, precision=prec, stream=stream)   # warm-up
        torch.cuda.synchronize()
        x.zero_()
        e0.record(stream)
        it, rel = G.solve(x, b, tol=1e-10, max_iter=100, precision=prec, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        out[name + "_solve"] = {"s": e0.elapsed_time(e1) / 1e3, "iters": it, "rel_res": rel,
                                "smoother": "weighted Jacobi 2/3, V(3,3), coarsest level 1",
                                "timed_after_warmup": True}
        del G
    del H, op, mass
    # discretisation error series
    errs = {}
    for L in series:
        HL = hg.Hierarchy(mesh, 1, L)
        opL = hg.Operator(HL)
        mL = hg.Operator(HL, hg.HG_OP_P1_MASS)
        bL, uL, _, _ = _manufactured_rhs(HL, mL, L, stream)
        G = hg.GMG(opL)
        x = HL.zeros(L, torch.float64)
        G.solve(x, bL, tol=1e-10, max_iter=100, stream=stream)
        e = x - HL.from_canonical(L, torch.tensor(uL, device="cuda"))
        Me = HL.zeros(L, torch.float64)
        mL.apply(L, e, Me, mask=hg.HG_MASK_ALL, stream=stream)
        errs[L] = float(np.sqrt(max(HL.dot(L, e, Me, mask=hg.HG_MASK_ALL), 0.0)))
        del G, HL, opL, mL
    ser = {"levels": list(series), "l2_mass_norm_err": [errs[L] for L in series],
           "ratios": [errs[a] / errs[b] for a, b in zip(series[:-1], series[1:])]}
    oerr, t0 = [], time.perf_counter()
    for L in oracle_levels:
        Ho = og.Hierarchy(macro, 1, L)
        lev = Ho.levels[L]
        uo = np.prod(np.sin(np.pi * lev.xyz), axis=1)
        bo = (lev.M_full @ (3 * np.pi ** 2 * uo))[lev.interior]
        xo, _, _ = og.solve(Ho, bo, tol=1e-10)
        eo = -uo
        eo[lev.interior] += xo
        oerr.append(float(np.sqrt(eo @ (lev.M_full @ eo))))
    ser["oracle"] = {"levels": list(oracle_levels), "l2_mass_norm_err": oerr,
                     "s": time.perf_counter() - t0, "threads": _oracle_threads()}
    ser["max_rel_diff_vs_oracle"] = float(max(abs(errs[L] - e) / e for L, e in
                                              zip(oracle_levels, oerr)))
    out["l2_error_series"] = ser
    out["host_cores"] = _host_cores()
    return out


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    from oracle import fem
    from oracle.mesh import RefinedMesh
    rm = RefinedMesh(sg.kuhn_cube(1), SAMPLE_LEVEL)
    A = fem.assemble(rm.cells, fem.p1_stiffness(rm.cell_xyz), rm.n_vertices)
    ii = rm.interior
    AII = A[ii][:, ii].tocsr()
    x = sg.uniform_vector(0, rm.n_vertices)[ii]
    inner = 20                            # SpMVs per step: a bounded sample of the workload
    for _ in range(args.warmup):
        for _ in range(inner):
            y = AII @ x
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for _ in range(inner):
            y = AII @ x
    dt = time.perf_counter() - t0
    val = rm.n_vertices * inner * args.steps / dt / 1e9
    sample = (f"SciPy CSR SpMV (single thread) of the same P1 operator on the same mesh at level "
              f"{SAMPLE_LEVEL} ({rm.n_vertices} DoFs), {inner} SpMVs per step")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "GDoF/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "oracle_level": SAMPLE_LEVEL},
        "cpu_baseline": {"value": val, "unit": "GDoF/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": val, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))
    sys.stdout.flush()


def make_parser():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-gmg", action="store_true")
    ap.add_argument("--no-reftet", action="store_true")
    ap.add_argument("--no-learned-kernels", action="store_true")
    ap.add_argument("--learned-samples", type=int, default=1 << 22,
                    help="samples of the learned-kernel leg (smaller for profiling)")
    ap.add_argument("--only", default=None,
                    help="comma-separated legs to run besides the headline apply (e.g. "
                         "learned_kernels,cube6); the others are skipped")
    ap.add_argument("--no-cube6", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-p2", action="store_true")
    ap.add_argument("--no-stencil", action="store_true")
    ap.add_argument("--no-kernels", action="store_true")
    ap.add_argument("--no-n1", action="store_true")
    ap.add_argument("--no-n1-solve", action="store_true")
    ap.add_argument("--stencil-case", type=int, nargs=2, default=[4, 6], metavar=("M", "LEVEL"),
                    help="stencil leg mesh (m^3 sub-cubes x 6 cells) and level (smaller for profiling)")
    ap.add_argument("--no-stencil-solve", action="store_true")
    ap.add_argument("--no-p2-solve", action="store_true",
                    help="P2 leg: apply only (for profiling)")
    ap.add_argument("--p2-level", type=int, default=6,
                    help="P2 level of the P2 leg (6 = the 17 M DoF workload; smaller for profiling)")
    return ap


LEGS = ("gmg", "batch", "p2", "stencil", "kernels", "n1", "n1_solve", "reftet", "cube6",
        "learned_kernels", "cpu_baseline")


def apply_only(args):
    """--only a,b: skip every leg not named (the headline apply and its e2e
    pass always run)."""
    if args.only is not None:
        keep = set(args.only.split(","))
        for leg in LEGS:
            if leg not in keep:
                setattr(args, "no_" + leg, True)
    return args


def main():
    args = apply_only(make_parser().parse_args())
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_2308_01792_gb300 as hg

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist

    macro = sg.kuhn_cube(1)
    H = hg.Hierarchy(hg.Mesh(macro.xyz, macro.cells), LEVEL, LEVEL)
    op = hg.Operator(H)
    ns, nu, ni, stride = H.size(LEVEL)
    _, _, dirich = H.canonical_info(LEVEL)
    dt = torch.float32
    xs, ys = [], []
    for p in range(N_PAIRS):
        c = sg.uniform_vector(1000 + p, nu)
        c[dirich] = 0.0
        xs.append(H.from_canonical(LEVEL, torch.tensor(c, dtype=dt, device="cuda")))
        ys.append(H.zeros(LEVEL, dt))
    stream = torch.cuda.current_stream()

    def step(s):
        op.apply(LEVEL, xs[s % N_PAIRS], ys[s % N_PAIRS], stream=stream)

    for s in range(max(args.warmup, 3)):
        step(s)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    # the timed region lasts milliseconds, far below the 100 ms sampling
    # interval: keep the GPU under the same apply load (untimed) for 0.5 s so
    # that the samples show the clocks of this workload
    t_load, s_extra = time.perf_counter(), 0
    while time.perf_counter() - t_load < 0.5:
        for _ in range(64):
            step(s_extra)
            s_extra += 1
        torch.cuda.synchronize()
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for s in range(args.steps):
        step(s)
    e1.record(stream)
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    if clk is not None:
        clk["window"] = (f"0.5 s of the same apply (untimed) before the timed region "
                         f"({ms:.1f} ms) and the region itself")
    ms_step, value = aggregate_replicas(ms, nu, args.steps, pg, "cuda")
    # the same bytes moved by a plain device copy (torch copy_, a library
    # kernel) over the same rotation of buffers: the ceiling at this size
    cp_src = [torch.empty(nu, dtype=dt, device="cuda").fill_(1.0) for _ in range(N_PAIRS)]
    cp_dst = [torch.empty_like(v) for v in cp_src]
    for q in range(3):
        cp_dst[q].copy_(cp_src[q])
    torch.cuda.synchronize()
    e0.record(stream)
    for q in range(args.steps):
        cp_dst[q % N_PAIRS].copy_(cp_src[q % N_PAIRS])
    e1.record(stream)
    torch.cuda.synchronize()
    copy_us = e0.elapsed_time(e1) / args.steps * 1e3
    del cp_src, cp_dst

    # end to end through the public API with host buffers: every step copies
    # its canonical input from pinned host memory into a function of the
    # library (hg_function_copy_canonical: host -> device, then every stored
    # copy set), applies the operator to the functions (hg_apply_function)
    # and copies the result back (one value per DoF gathered, device -> host).
    # Steps rotate over three streams, each with its own pair of functions
    # and host buffers, so that one step's copies overlap the neighbouring
    # steps' kernels.
    NB = 3
    e2e_streams = [torch.cuda.Stream() for _ in range(NB)]
    x0 = sg.uniform_vector(7, nu).astype(np.float32)
    x0[dirich] = 0.0
    bufs = []
    for _ in range(NB):
        bufs.append({"xh": torch.from_numpy(x0.copy()).pin_memory(),
                     "yh": torch.empty(nu, dtype=dt).pin_memory(),
                     "x": hg.Function(H, dt, levels=[LEVEL]), "y": hg.Function(H, dt, levels=[LEVEL])})
    e2e_steps = max(12, args.steps // 4)

    def e2e_step(q):
        b, s = bufs[q % NB], e2e_streams[q % NB]
        b["x"].copy_from_host(LEVEL, b["xh"], stream=s)
        op.apply_function(LEVEL, b["x"], b["y"], stream=s)
        b["y"].copy_to_host(LEVEL, b["yh"], stream=s)

    for q in range(2 * NB):
        e2e_step(q)
    torch.cuda.synchronize()
    e0.record(stream)
    for s in e2e_streams:
        s.wait_event(e0)
    for q in range(e2e_steps):
        e2e_step(q)
    for s in e2e_streams:
        ev = torch.cuda.Event()
        ev.record(s)
        stream.wait_event(ev)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1) / e2e_steps
    ref_y = torch.zeros(nu, dtype=dt, device="cuda")
    H.to_canonical(LEVEL, bufs[0]["y"][LEVEL], out=ref_y)
    if not torch.equal(bufs[0]["yh"], ref_y.cpu()):
        raise RuntimeError("e2e: host result differs from the device result")

    peak, peak_kind = _peaks()
    achieved = BYTES_PER_DOF * nu / (ms_step * 1e-3) / 1e9
    traffic = _profiled_traffic()
    out = {
        "metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": ws, "steps": args.steps,
        "warmup": max(args.warmup, 3), "ms_per_step": ms_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "mesh": "unit cube, 6 Kuhn macro-tetrahedra",
                   "level": LEVEL, "unique_dofs": nu, "stored_dofs": ns, "operator": "P1 Laplacian",
                   "l2": f"{N_PAIRS} rotating x/y pairs, {N_PAIRS * 2 * ns * 4 / 1e6:.0f} MB > 4x L2",
                   "parallelism": f"replicas{ws}"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "p1_fused_kernel<float,APPLY,kPat7> (plane windows, one launch "
                               "per apply)",
                     "peak_source": f"{peak_kind} hbm_gbs", "algorithmic_bytes_per_launch":
                         BYTES_PER_DOF * nu,
                     "copy_same_bytes": {
                         "us": copy_us, "frac_of_peak": BYTES_PER_DOF * nu / (copy_us * 1e-6) / 1e9
                         / peak, "apply_rate_over_copy_rate": copy_us / (ms_step * 1e3),
                         "note": "torch copy_ of the apply's 8 B per DoF, same rotation: the "
                                 "ceiling of a launch of this size"}},
        "e2e": {"value": nu / (e2e_ms * 1e-3) / 1e9, "unit": "GDoF/s",
                "h2d_bytes_per_step": 4 * nu, "d2h_bytes_per_step": 4 * nu,
                "path": "hg_function_copy_canonical (pinned host -> device) + hg_apply_function "
                        "+ hg_function_copy_canonical (device -> pinned host), 3 streams"},
        "gpu_launches": args.steps,
        "clocks": clk,
    }
    if rank == 0 and not args.no_reftet:
        out["reftet"] = reftet_comparison(stream)
    if rank == 0 and not args.no_cube6:
        out["cube6"] = cube6_comparison(stream)
    if rank == 0 and not args.no_gmg:
        out["gmg"] = gmg_comparison(stream)
    if rank == 0 and not args.no_learned_kernels:
        out["learned_kernels"] = learned_kernels_comparison(stream, samples=args.learned_samples)
    if rank == 0 and not args.no_batch:
        out["batch"] = batch_comparison(stream)
    if rank == 0 and not args.no_p2:
        out["p2"] = p2_comparison(stream, args.p2_level, solve=not args.no_p2_solve)
    if rank == 0 and not args.no_n1:
        out["n1"] = n1_comparison(stream)
    if rank == 0 and not args.no_kernels:
        out["kernels"] = kernels_comparison(stream)
    if rank == 0 and not args.no_stencil:
        out["stencil"] = stencil_comparison(stream, *args.stencil_case,
                                            solve=not args.no_stencil_solve)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_spmv()
        out["cpu_baseline"]["gmg"] = cpu_baseline_gmg()
    if rank == 0 and not args.no_n1_solve:
        # last leg; an error here is recorded in the line instead of ending the run
        try:
            out["n1_solve"] = n1_solve_comparison(stream)
        except Exception as e:                                    # noqa: BLE001
            out["n1_solve"] = {"workload": N1_SOLVE_WORKLOAD, "error": f"{type(e).__name__}: {e}"}
    if rank == 0:
        print(json.dumps(out))
        sys.stdout.flush()
    if pg:
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
