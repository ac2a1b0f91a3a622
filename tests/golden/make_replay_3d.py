"""Writes replay_3d_128cube_f8.txt: the oracle's run of the 3D 128^3 workload
(anisotropic ln K field, lognormal S_s, 4 preconditioner shifts cycled, centre
source) with 8 of its 200 shifts spread over the period range, for the GPU's
replay parity test at the full grid size.

The record holds what the GPU replays (the inner-cycle count of every flexible
Arnoldi step, Algorithm 3 with the inexact inner solve of Section 4, and each
shift's freeze step m_j, Algorithm 4) and what it is compared with: every
shift's ||x_j|| and x_j at 1024 seeded cells (plus the source cell). This
script calls only the oracle and the seeded input generator.

    python tests/golden/make_replay_3d.py      (about ten minutes on one core)
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from oracle.gmg import GMGInner, Hierarchy  # noqa: E402
from paper_1212_3660_gb300 import synth  # noqa: E402

OUT = os.path.join(HERE, "replay_3d_128cube_f8.txt")
SHIFT_IDX = np.linspace(0, 199, 8).round().astype(int)
EPS, RELAX, SAMPLES = 1e-10, 0.003, 1024


def main():
    pr = synth.workload(3, m_max=100)
    sigma = pr.sigma[SHIFT_IDX]
    op = oracle.assemble(pr.shape, pr.h, pr.cond, pr.ss, pr.dirichlet_mask)
    b = pr.rhs()[:, 0]
    ref = oracle.shifted_solve(op, b, sigma, pr.tau_bar, pr.schedule, pr.tol, pr.m_max,
                               GMGInner(Hierarchy(op, pr.tau_bar), EPS), inner_relax=RELAX, eps=EPS)
    cells = np.sort(np.unique(np.concatenate([np.random.default_rng(4242).choice(pr.n, SAMPLES, replace=False),
                                              pr.src_cells])))
    with open(OUT, "w") as f:
        f.write("# oracle replay record: workload 3 (3D 128^3), shifts " + " ".join(map(str, SHIFT_IDX))
                + f" of 200, inner eps {EPS:g}, relaxed l = {RELAX:g}\n")
        f.write(f"steps {ref.steps}\n")
        f.write("cycles " + " ".join(str(int(c)) for c in ref.cycles[:ref.steps]) + "\n")
        f.write("m_j " + " ".join(str(int(m)) for m in ref.m_j) + "\n")
        f.write("xnorm " + " ".join(repr(float(np.linalg.norm(ref.x[:, j]))) for j in range(len(sigma))) + "\n")
        f.write("cells " + " ".join(str(int(c)) for c in cells) + "\n")
        for j in range(len(sigma)):
            xs = ref.x[cells, j]
            f.write(f"x{j} " + " ".join(f"{float(v.real)!r} {float(v.imag)!r}" for v in xs) + "\n")


if __name__ == "__main__":
    main()
