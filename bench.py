"""Benchmark of the dense fractional-Laplacian hot path on GB300.

One step = one pass of the hot path on the quasi-uniform unit-disc workload
(25 rings, 3929 triangles, 1887 interior DOFs, s = 0.75, f = 1):
  assemble A^s (float32 separated pairs, float64 touching pairs / boundary /
  reductions) -> float32 copy -> load vector -> float64-refined Jacobi-PCG on the
  float32 copy to ||b - A u|| <= 1e-8 ||b||.
value = element pairs per second over the whole step: N_el^2 ordered pairs (K, K')
of the double sum of Section 5 per step, times steps, divided by the timed device
time (max over ranks).  Side figures: assembly-only pair rate in both precisions,
the float64 / float32 dense matvec bandwidth on the assembled matrix, and the time
to 1e-8 of the refined solve against plain float64 Jacobi-PCG.

--impl reference times the CPU oracle (oracle/) on a bounded sample of the same
workload (element-pair rows), on this machine's host cores.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
# the oracle's numpy runs with the thread count reported as cpu_baseline's cores (one unless the
# caller sets OMP_NUM_THREADS); set before numpy's BLAS is loaded
for _var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_var, os.environ.get("OMP_NUM_THREADS", "1"))

WORKLOAD = {"workload": "disc-quasi-uniform-25-rings", "domain": "unit disc", "rings": 25, "triangles": 3929,
            "dofs": 1887, "s": 0.75, "f": "1", "dtype_assembly": "f32 separated pairs + f64 near/boundary",
            "solve": "f64-refined Jacobi-PCG on f32 copy to 1e-8", "l2": "flushed between timed steps (512 MiB write)"}
METRIC = "element pairs/s assembled; matvec HBM GB/s; solve time to 1e-8 vs plain FP64"
# the L-shape workload: nested levels 1..4 of the corner- and boundary-refined L-shape
LSHAPE = {"level": 4, "s": 0.5}
# the batched workload: 4 orders x 64 loads on the disc graded toward the boundary
BATCH = {"rings": 30, "mu": 2.0, "s": [0.25, 0.5, 0.75, 0.9], "nrhs": 64}
# DRAM bytes (read 1.434 MB + write 2.044 MB) per launch of far_tile_kernel<2,float,16,0> on this
# workload, from one ncu capture of the current kernel; reset to None whenever that kernel changes.
FAR_KERNEL_DRAM_BYTES = 3.478e6
UNIT = "element pairs/s"


def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while active."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return

        def rd():
            for line in self.proc.stdout:
                self.rows.append([x.strip() for x in line.split(",")])

        self.thread = threading.Thread(target=rd, daemon=True)
        self.thread.start()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm = [float(r[1]) for r in self.rows if len(r) > 8 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 8 and r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            if len(r) > 8:
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def job_rate(total_ms, steps, units_per_step, world, dist=None, device="cpu"):
    """Whole-job rate over replicas: every rank processed `units_per_step` units in each of
    `steps` timed steps; the job time is the maximum of the ranks' timed totals (ms).
    Returns (max time in ms, units of all ranks per second)."""
    t_max = float(total_ms)
    if dist is not None and world > 1:
        import torch

        t = torch.tensor([t_max], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    return t_max, world * steps * units_per_step / (t_max / 1000.0)


def oracle_sample(seconds_target=15.0):
    """Time the CPU oracle on element-pair rows of the same workload.  Returns
    (ordered element pairs evaluated per second, threads, sample description)."""
    import numpy as np

    from oracle import OracleMesh, assemble_matrix
    from paper_1708_03912_gb300 import synth

    V, T = synth.disc(WORKLOAD["rings"])
    om = OracleMesh(V, T)
    s = WORKLOAD["s"]
    n = len(om.dofs(s)[0])
    rows = synth.random_rows(n, 4)
    # ordered pairs covered: each active cell against every cell (both orders of each unordered pair)
    active = set()
    vod = om.dofs(s)[0]
    for r in rows:
        active.update(om.cells_of_vertex[vod[r]])
    t0 = time.perf_counter()
    assemble_matrix(om, s, rows=rows)
    dt = time.perf_counter() - t0
    pairs = 2 * len(active) * om.nc - len(active) ** 2  # unordered pairs touching the active set, x2 ordered
    threads = int(os.environ.get("OMP_NUM_THREADS", "1"))
    return pairs / dt, dt, threads, f"{len(rows)} seeded rows = {len(active)} cells x {om.nc} partner cells"


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    vals = []
    for _ in range(args.warmup):
        oracle_sample()
    t_all = 0.0
    for _ in range(args.steps):
        v, dt, threads, desc = oracle_sample()
        vals.append(v)
        t_all += dt
    value = statistics.mean(vals)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * t_all / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": dict(WORKLOAD),
            "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": desc + ", numpy float64, host cores of the GPU box"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def build_problems(F, synth, m, svals, nrhs, nslices, V):
    """Batched-solve problems on mesh m: for every s the mixed-mode matrix, its bf16 slices and
    f = 1 plus nrhs - 1 seeded Gaussian nodal loads."""
    import torch

    f = torch.tensor(synth.gaussian_nodal(len(V), nrhs - 1, seed=synth.SEED + 1), device="cuda") if nrhs > 1 else None
    probs = []
    for s in svals:
        n = m.num_dofs(s)
        A = m.assemble(s, "mixed")
        S, d = F.split_bf16(A, nslices)
        B = torch.empty((n, nrhs), dtype=torch.float64, device="cuda")
        F.fl_load_vector(m.h, s, None, B[:, :1])
        if nrhs > 1:
            F.fl_load_vector(m.h, s, f, B[:, 1:])
        probs.append({"A": A, "S": S, "nslices": nslices, "dscale": d, "B": B, "U": torch.empty_like(B)})
    return probs


# small named workloads for profilers (`--case`): rings, grading exponent, s
CASES = {"disc25": (25, 1.0, 0.75), "gdisc30": (30, 2.0, 0.75), "disc10": (10, 1.0, 0.75)}


def run_case(args):
    """One untimed warm-up step and `--steps` profiled steps of assemble -> float32 copy -> load
    vector -> refined Jacobi-PCG on a small named disc workload; prints the stage times."""
    import torch

    from paper_1708_03912_gb300 import fraclap as F
    from paper_1708_03912_gb300 import synth

    M, mu, s = CASES[args.case]
    V, T = synth.disc(M, mu)
    m = F.Mesh(V, T)
    n = m.num_dofs(s)
    A = torch.empty((n, n), dtype=torch.float64, device="cuda")
    A32 = torch.empty((n, n), dtype=torch.float32, device="cuda")

    def step():
        m.assemble(s, args.precision, out=A)
        if not args.no_solve:
            F.fl_convert(A, F.FL_F32, A32)
            b = m.load_vector(s)
            m.solve(A, b, tol=1e-8, A_lo=A32, inner_tol=1e-3)

    step()
    F.fl_set_profiling(m.h, True)
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    st = F.fl_stage_ms(m.h)
    print(f"case {args.case}: cells {len(T)} dofs {n} precision {args.precision}; stage ms " +
          " ".join(f"{k}={v:.3f}" for k, v in st.items()))
    m.close()
    return 0


def lshape_section(F, synth, timed, dev):
    """L-shape level LSHAPE["level"] (s = 1/2): Jacobi-PCG, multigrid-preconditioned CG on the nested
    levels below it, and flexible CG with the learned stencil trained on a coarser level."""
    import torch

    s = LSHAPE["s"]
    lev = LSHAPE["level"]
    meshes = [synth.lshape(0.25, l) for l in range(lev, 0, -1)]  # fine to coarse
    hs = [F.fl_create(V, T) for V, T in meshes]
    mf = F.Mesh(*meshes[0])
    A = mf.assemble(s, "mixed")
    n = A.shape[0]
    b = mf.load_vector(s)
    u = torch.empty_like(b)
    out = {"workload": f"L-shape [0,2]^2 minus [1,2]^2, level {lev} (refined towards (1,1) and the boundary), "
                       f"n = {n}, s = {s}, f = 1, tol 1e-8, float64 matvec", "n": n}
    _, ij = mf.solve(A, b, tol=1e-8)
    out["jacobi_pcg"] = {"ms": timed(lambda: mf.solve(A, b, tol=1e-8), reps=2), "iterations": ij.iterations}
    # multigrid on the nested levels
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mg = F.Multigrid(A)
    for k in range(len(hs) - 1):
        ptr, col, val = F.fl_prolongation(hs[k], hs[k + 1], s)
        mg.add_level(ptr, col, val, F.fl_num_dofs(hs[k + 1], s))
    mg.setup(nu=2)
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1000
    im = mg.solve(b, u, tol=1e-8, maxit=500)
    out["mg_pcg"] = {"ms": timed(lambda: mg.solve(b, u, tol=1e-8, maxit=500), reps=2), "iterations": im.iterations,
                     "setup_ms": setup_ms, "levels": [F.fl_num_dofs(h, s) for h in hs]}
    # learned stencil: trained on level 2 from noise-started CG pairs, transferred to this level
    V2, T2 = synth.lshape(0.25, 2)
    m2 = F.Mesh(V2, T2)
    A2 = m2.assemble(s, "mixed")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lp2 = F.LearnedPreconditioner(m2.h, s, seed=1)
    lp2.collect_noise(A2, 8, [0, 1, 2, 4])
    loss = lp2.train(2000, batch=8192, lr=1e-3)
    torch.cuda.synchronize()
    train_ms = (time.perf_counter() - t0) * 1000
    lp = F.LearnedPreconditioner(mf.h, s, seed=1)
    lp.set_params(lp2.params())
    il = F.fl_fcg_solve(mf.h, A, b, u, lp=lp, mg=mg, tol=1e-8)
    out["learned_fcg"] = {"ms": timed(lambda: F.fl_fcg_solve(mf.h, A, b, u, lp=lp, mg=mg, tol=1e-8), reps=2),
                          "iterations": il.iterations, "fallback_at": il.fallback_at,
                          "rel_residual_f64": il.rel_residual, "train_ms": train_ms, "train_loss": loss,
                          "note": "stencil network trained on level 2 (2000 Adam steps, batch 8192), weights "
                                  "transferred; multigrid as fallback"}
    ij2 = F.fl_fcg_solve(mf.h, A, b, u, mg=mg, tol=1e-8)
    out["mg_fcg_iterations"] = ij2.iterations
    for obj in (lp, lp2, mg):
        obj.close()
    m2.close()
    mf.close()
    for h in hs:
        F.fl_destroy(h)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tune-file", default=None, help="load/save the autotuner's table (JSON)")
    ap.add_argument("--case", default=None, choices=sorted(CASES),
                    help="profiling mode: run a small named workload and print stage times (no JSON line)")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"], help="assembly precision of --case")
    ap.add_argument("--no-solve", action="store_true", help="--case: assembly only")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.case:
        return run_case(args)

    import numpy as np
    import torch

    from paper_1708_03912_gb300 import fraclap as F
    from paper_1708_03912_gb300 import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    s = WORKLOAD["s"]
    V, T = synth.disc(WORKLOAD["rings"])
    n_el = len(T)
    m = F.Mesh(V, T)
    n = m.num_dofs(s)
    stats = F.fl_get_stats(m.h, s)
    A = torch.empty((n, n), dtype=torch.float64, device=dev)
    A32 = torch.empty((n, n), dtype=torch.float32, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        m.assemble(s, "mixed", out=A)
        F.fl_convert(A, F.FL_F32, A32)
        b = m.load_vector(s)
        u, info = m.solve(A, b, tol=1e-8, A_lo=A32, inner_tol=1e-3)
        return info

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = F.fl_launch_count()
    total_ms = 0.0
    infos = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        infos.append(step())
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    launches = F.fl_launch_count() - launches0
    if dist:
        dist.barrier()
    clk = clocks.stop()
    t_max, value = job_rate(total_ms, args.steps, n_el * n_el, world, dist, dev)

    # ---- side measurements (untimed for the headline) ----
    def timed(fn, reps=5, flush_between=True):
        ts = []
        for _ in range(reps):
            if flush_between:
                flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b_ = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b_.record(stream)
            b_.synchronize()
            ts.append(a.elapsed_time(b_))
        return statistics.median(ts)

    peaks = load_peaks()
    asm_mixed_ms = timed(lambda: m.assemble(s, "mixed", out=A))
    asm_fp64_ms = timed(lambda: m.assemble(s, "fp64", out=A), reps=3)
    # dominant kernel: the far-field tile kernel, timed by the library's events on this stream
    F.fl_set_profiling(m.h, True)
    far_ms = []
    stage_tot = {k: 0.0 for k in F.STAGES}
    for _ in range(5):
        flush.zero_()
        m.assemble(s, "mixed", out=A)
        st = F.fl_stage_ms(m.h)
        far_ms.append(st["far"])
        for k in st:
            stage_tot[k] += st[k] / 5
    F.fl_set_profiling(m.h, False)
    far_avg = statistics.mean(far_ms)
    q = 16  # collapsed rule of order 4
    evals = stats["n_far_pairs"] * q * q
    # dense matvec bandwidth on an HBM-resident matrix of the graded-disc size (n = 8195:
    # 537 MB float64, 269 MB float32, both larger than L2), L2 flushed between products
    nb = 8195
    Ab = torch.randn(nb, nb, dtype=torch.float64, device=dev)
    Ab32 = Ab.float()
    xb = torch.randn(nb, 1, dtype=torch.float64, device=dev)
    xb1 = xb[:, 0].contiguous()
    yb = torch.empty(nb, 1, dtype=torch.float64, device=dev)
    yb1 = torch.empty(nb, dtype=torch.float64, device=dev)
    # blocks per SM of the staged product from the project's autotuner, for both storage types
    def tune_mv(dt, M):
        try:
            return F.fl_tune_matvec(dt, M, xb1, yb1, reps=5)
        except F.FlError as e:  # FL_ENOTIMPL: the staged product is not used at this size
            if e.code != F.FL_ENOTIMPL:
                raise
            return (None, None)

    mv_tuned = {"f64": tune_mv(F.FL_F64, Ab), "f32": tune_mv(F.FL_F32, Ab32)}
    mv64 = timed(lambda: F.fl_matvec(F.FL_F64, Ab, xb, yb), reps=10)
    mv32 = timed(lambda: F.fl_matvec(F.FL_F32, Ab32, xb, yb), reps=10)
    mv32s = timed(lambda: F.fl_matvec_f32_static(Ab32, xb1, yb1), reps=10)
    Ab2 = torch.empty(nb, 2 * nb, dtype=torch.float32, device=dev)  # hi + lo float32 pairs
    F.fl_convert(Ab, F.FL_F32X2, Ab2)
    mvx2 = timed(lambda: F.fl_matvec(F.FL_F32X2, Ab2, xb, yb), reps=10)
    del Ab2
    del Ab, Ab32
    # time to 1e-8: refined float32 solve vs plain float64 Jacobi-PCG on the same matrix
    m.assemble(s, "fp64", out=A)
    F.fl_convert(A, F.FL_F32, A32)
    b = m.load_vector(s)
    sol_mixed = timed(lambda: m.solve(A, b, tol=1e-8, A_lo=A32, inner_tol=1e-3), reps=3)
    sol_fp64 = timed(lambda: m.solve(A, b, tol=1e-8), reps=3)
    _, inf64 = m.solve(A, b, tol=1e-8)
    _, infmx = m.solve(A, b, tol=1e-8, A_lo=A32, inner_tol=1e-3)

    # ---- batched: 4 orders x 64 right-hand sides on the graded disc (n = 8195) ----
    Vg, Tg = synth.disc(BATCH["rings"], BATCH["mu"])
    mg = F.Mesh(Vg, Tg)
    probs = build_problems(F, synth, mg, BATCH["s"], BATCH["nrhs"], 2, Vg)
    # launch shape of the tensor-core product from the project's autotuner (persisted if asked)
    if args.tune_file and os.path.exists(args.tune_file):
        F.fl_tune_load(args.tune_file)
    tuned, tuned_ms = F.fl_tune_batch(mg.h, probs, reps=5)
    if args.tune_file:
        F.fl_tune_save(args.tune_file)
    ob = F.fl_default_batch_opts()
    ob.inner_tol = 1e-4
    binfo = {}

    def batched():
        r_, inf_, rel_, st_ = F.fl_batch_solve(mg.h, probs, ob)
        binfo.update(status=int(r_), outer=inf_.outer_iterations, inner=inf_.inner_iterations,
                     max_rel=float(rel_.max()), ctas=inf_.ctas, stages=inf_.stages)

    batched()
    batch_ms = timed(batched, reps=3)
    # plain float64 Jacobi-PCG on the same systems: f = 1 and the first Gaussian load for every s,
    # the per-column mean extrapolated to all columns
    plain_cols = []
    for q in probs:
        for j in (0, 1):
            bj = q["B"][:, j].contiguous()
            mg.solve(q["A"], bj)
            plain_cols.append(timed(lambda: mg.solve(q["A"], bj), reps=1, flush_between=True))
    plain_total = statistics.mean(plain_cols) * BATCH["nrhs"] * len(BATCH["s"])
    # the tensor-core product alone, from the autotuner's CUDA-event timing of the GEMM kernel over all
    # four matrices (two bf16 slices each, 64 columns): bytes = slice tiles streamed once
    nbg = probs[2]["A"].shape[0]
    gemm_bytes = sum(F.fl_split_bf16_bytes(q["A"].shape[0], 2) for q in probs)
    gemm_flops = sum(2 * 3 * q["A"].shape[0] ** 2 * BATCH["nrhs"] for q in probs)
    batch_line = {
        "workload": f"graded disc {BATCH['rings']} rings mu {BATCH['mu']}, n = {nbg}, s = {BATCH['s']}, "
                    f"{BATCH['nrhs']} right-hand sides (f = 1 and seeded Gaussian nodal loads)",
        "ms_to_1e-8": batch_ms, "systems": BATCH["nrhs"] * len(BATCH["s"]),
        "plain_f64_ms_extrapolated": plain_total,
        "plain_f64_note": "mean of 2 timed single-column float64 Jacobi-PCG solves per s, times 64 columns",
        "speedup_vs_plain_f64": plain_total / batch_ms, **binfo,
        "autotune": {"stages": tuned.stages, "ctas": tuned.ctas, "gemm_ms": tuned_ms,
                     "note": "fl_tune_batch sweep of pipeline depth x CTA count on these slices"},
        "tc_gemm": {"ms": tuned_ms, "bytes": gemm_bytes, "gbs": gemm_bytes / (tuned_ms / 1000) / 1e9,
                    "frac_of_measured_hbm": gemm_bytes / (tuned_ms / 1000) / 1e9 / peaks.get("hbm_gbs", 6660.3),
                    "tflops": gemm_flops / (tuned_ms / 1000) / 1e12,
                    "note": "tcgen05 GEMM kernel alone (autotuner timing), 4 matrices x 2 bf16 slices x 64 columns "
                            "(3 bf16 products), HBM-bound: 48 flop/byte"},
    }
    del probs
    mg.close()

    # ---- L-shape refined towards the corner and the boundary: preconditioners, time to 1e-8 ----
    lsh = lshape_section(F, synth, timed, dev)

    # ---- end to end through the public API with host buffers ----
    def e2e_step():
        mm = F.Mesh(V, T)
        AA = mm.assemble(s, "mixed")
        AL = torch.empty((n, n), dtype=torch.float32, device=dev)
        F.fl_convert(AA, F.FL_F32, AL)
        bb = mm.load_vector(s)
        uu, _ = mm.solve(AA, bb, tol=1e-8, A_lo=AL, inner_tol=1e-3)
        host = uu.cpu()
        st_ = F.fl_get_stats(mm.h, s)
        mm.close()
        return host, st_

    e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = max(1, min(args.steps, 3))
    for _ in range(e2e_steps):
        _, st_e = e2e_step()
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    h2d = int(st_e["h2d_bytes"] + V.nbytes + T.nbytes)
    d2h = n * 8

    sm_clock = clk.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    # far kernel (float32, s = 3/4): one MUFU.LG2 (16 results/clk/SM) and one MUFU.EX2 (32/clk/SM on GB300,
    # measured) per kernel evaluation -> 1 / (1/16 + 1/32) = 10.67 evaluations/clk/SM
    evals_per_clk_sm = 1.0 / (1.0 / 16 + 1.0 / 32)
    peak_evals = 152 * evals_per_clk_sm * (peaks.get("sm_max_mhz", 2070.0) * 1e6)
    achieved = evals / (far_avg / 1000.0)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": dict(WORKLOAD, cells=n_el, parallelism=f"replicas x{world}"),
        "roofline": {"bound": "alu", "kernel": "far_tile_kernel<2,float,16,0>", "achieved": achieved / 1e9,
                     "peak": peak_evals / 1e9, "unit": "Geval/s", "frac": achieved / peak_evals,
                     "traffic": FAR_KERNEL_DRAM_BYTES,
                     "note": "kernel evaluations |x-y|^{-2-2s}; peak = 152 SMs x 10.67 evals/clk (MUFU lg2 16/clk + "
                             "ex2 32/clk per SM) x max SM clock; evals = far pairs x 16 x 16"},
        "stage_ms": stage_tot,
        "assembly_pairs_per_s": {"mixed": n_el * n_el / (asm_mixed_ms / 1000), "fp64": n_el * n_el / (asm_fp64_ms / 1000)},
        "matvec": {"n": nb, "f64_gbs": nb * nb * 8 / (mv64 / 1000) / 1e9, "f32_gbs": nb * nb * 4 / (mv32 / 1000) / 1e9,
                   "f64_ms": mv64, "f32_ms": mv32, "f32_static_gbs": nb * nb * 4 / (mv32s / 1000) / 1e9,
                   "f32x2_gbs": nb * nb * 8 / (mvx2 / 1000) / 1e9, "f32x2_ms": mvx2,
                   "tuned_blocks_per_sm": {k: v[0] for k, v in mv_tuned.items()},
                   "hbm_peak_gbs": peaks.get("hbm_gbs"),
                   "note": "bytes of A per product / device time of fl_matvec (x staged in shared memory per block; "
                           "the float32 call includes the rounding of x); L2 flushed; f32_static: the allocation-free "
                           "fl_matvec_f32_static; f32x2: hi + lo float32 pairs (8 bytes per entry) multiplied in double-float "
                           "arithmetic on the float32 pipe"},
        "solve_ms_to_1e-8": {"f32_refined": sol_mixed, "plain_f64": sol_fp64, "iters_f64": inf64.iterations,
                             "iters_refined": infmx.iterations, "outer": infmx.outer_iterations},
        "batched": batch_line,
        "lshape": lsh,
        "gpu_launches": int(launches),
        "clocks": clk,
        "e2e": {"value": n_el * n_el / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "note": "Mesh(host arrays) -> planner -> table upload -> assemble -> solve -> u to host"},
    }
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        v, dt, threads, desc = oracle_sample()
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc}
    m.close()
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
