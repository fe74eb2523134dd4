"""One warm step of the hot path on a named workload, for profilers.

python -m paper_1708_03912_gb300.profile_case [--case disc25|gdisc30|disc10] [--precision mixed|fp64]
    [--steps N] [--no-solve]

Runs one untimed warm-up step, then N steps of: assemble -> float32 copy -> load
vector -> refined Jacobi-PCG to 1e-8.  Prints the stage times of the last assembly.
"""
import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

CASES = {"disc25": (25, 1.0, 0.75), "gdisc30": (30, 2.0, 0.75), "disc10": (10, 1.0, 0.75)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="disc25", choices=sorted(CASES))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--no-solve", action="store_true")
    a = ap.parse_args()
    import torch

    from paper_1708_03912_gb300 import fraclap as F
    from paper_1708_03912_gb300 import synth

    M, mu, s = CASES[a.case]
    V, T = synth.disc(M, mu)
    m = F.Mesh(V, T)
    n = m.num_dofs(s)
    A = torch.empty((n, n), dtype=torch.float64, device="cuda")
    A32 = torch.empty((n, n), dtype=torch.float32, device="cuda")

    def step():
        m.assemble(s, a.precision, out=A)
        if not a.no_solve:
            F.fl_convert(A, F.FL_F32, A32)
            b = m.load_vector(s)
            m.solve(A, b, tol=1e-8, A_lo=A32, inner_tol=1e-3)

    step()
    F.fl_set_profiling(m.h, True)
    for _ in range(a.steps):
        step()
    torch.cuda.synchronize()
    st = F.fl_stage_ms(m.h)
    print(f"case {a.case}: cells {len(T)} dofs {n} precision {a.precision}; stage ms " +
          " ".join(f"{k}={v:.3f}" for k, v in st.items()))
    m.close()


if __name__ == "__main__":
    main()
