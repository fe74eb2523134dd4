"""Writes the stored expected values under tests/golden/ (calls only oracle/).

interval16_exact.json : exact stiffness matrix of the 15 interior hats of the
    uniform 16-element mesh of (-1,1), from the closed form
    a(u,v) = c ∬ |x-y|^{3-2s} u'' v'' (Section 2 Fourier form; 1D, s != 1/2),
    evaluated with 40-digit arithmetic.
square4_exact.json : exact matrix of the interior hats of the jittered 4x4
    square mesh (paper_1708_03912_gb300.synth.square(4, 0.2)), from the
    edge-pair form a(u,v) = c ∬ |x-y|^{2-2s} dΔu dΔv (2D).

Run:  python tests/golden/make_golden.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import OracleMesh, exact  # noqa: E402
from paper_1708_03912_gb300 import synth  # noqa: E402


def main():
    V, T = synth.interval(16)
    out = {"citation": "Section 2 (Fourier form of a(u,v)); 1D closed form through phi''",
           "mesh": "synth.interval(16)", "matrices": {}}
    for s in (0.25, 0.75):
        out["matrices"][str(s)] = exact.exact_matrix_1d(V[:, 0], s).tolist()
    with open(os.path.join(HERE, "interval16_exact.json"), "w") as f:
        json.dump(out, f, indent=0)
    V, T = synth.square(4, 0.2)
    m = OracleMesh(V, T)
    out = {"citation": "Section 2 (Fourier form of a(u,v)); 2D edge-pair form through Δphi",
           "mesh": "synth.square(4, 0.2)", "matrices": {}}
    for s in (0.25, 0.5, 0.75):
        out["matrices"][str(s)] = exact.exact_matrix_2d(m, s).tolist()
    with open(os.path.join(HERE, "square4_exact.json"), "w") as f:
        json.dump(out, f, indent=0)


if __name__ == "__main__":
    main()
