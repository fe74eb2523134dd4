"""Batched solves on the graded disc, for profilers and quick timing.

python -m paper_1708_03912_gb300.profile_batch [--s 0.25 0.5 0.75 0.9] [--nrhs 64] [--rings 30]
    [--slices 2] [--residual df|f64] [--reps 1] [--inner-tol 1e-4]

Assembles A^s for every s on the disc graded toward the boundary (mu = 2), splits
each into bf16 slices, loads f = 1 plus nrhs - 1 seeded Gaussian nodal loads, runs
one untimed batched solve and then `reps` timed ones (CUDA events), and prints the
time, the refinement and CG step counts and the worst final residual.
"""
import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def build_problems(m, svals, nrhs, nslices, V):
    import torch

    from paper_1708_03912_gb300 import fraclap as F
    from paper_1708_03912_gb300 import synth

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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--s", type=float, nargs="+", default=[0.25, 0.5, 0.75, 0.9])
    ap.add_argument("--nrhs", type=int, default=64)
    ap.add_argument("--rings", type=int, default=30)
    ap.add_argument("--slices", type=int, default=2)
    ap.add_argument("--residual", default="df", choices=["df", "f64"])
    ap.add_argument("--reps", type=int, default=1)
    ap.add_argument("--inner-tol", type=float, default=1e-4)
    a = ap.parse_args()
    import torch

    from paper_1708_03912_gb300 import fraclap as F
    from paper_1708_03912_gb300 import synth

    V, T = synth.disc(a.rings, 2.0)
    m = F.Mesh(V, T)
    probs = build_problems(m, a.s, a.nrhs, a.slices, V)
    o = F.fl_default_batch_opts()
    o.inner_tol = a.inner_tol
    o.residual = F.FL_RESID_DF if a.residual == "df" else F.FL_RESID_F64
    F.fl_batch_solve(m.h, probs, o)
    torch.cuda.synchronize()
    for _ in range(a.reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        r, info, rel, st = F.fl_batch_solve(m.h, probs, o)
        e1.record()
        torch.cuda.synchronize()
        print(f"n {probs[0]['A'].shape[0]} s {a.s} nrhs {a.nrhs}: {e0.elapsed_time(e1):.2f} ms status {r} "
              f"outer {info.outer_iterations} inner {info.inner_iterations} max rel {rel.max():.2e}")
    m.close()


if __name__ == "__main__":
    main()
