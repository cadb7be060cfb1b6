"""Writes the symbolic size fixtures in this folder from the oracle alone.

Run from the repository root:  python tests/golden/make_golden.py
The values are sizes of the elimination tree built by recursive bisection
(Sec. 2.4 of the paper) for the seeded structured workloads; they serve as
regression values for the product library's analysis.
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import fem_inputs as F  # noqa: E402
import oracle as O  # noqa: E402

CASES = {
    "poisson2d_q1_16": ((16, 16), 1),
    "diffusion2d_q3_64": ((64, 64), 3),
    "diffusion2d_q3_512": ((512, 512), 3),
    "diffusion3d_q1_16": ((16, 16, 16), 1),
    "diffusion3d_q1_64": ((64, 64, 64), 1),
    "poisson2d_q1_1024": ((1024, 1024), 1),
}


def main():
    for name, (nel, p) in CASES.items():
        mesh = F.structured_mesh(nel, p)
        s = O.OracleSolver(mesh.n_nodes, mesh.elem_nodes, O.tree_bisection(nel))
        rows = {
            "n_dof": mesh.n_nodes, "n_front": s.n_front, "n_classes": s.n_classes, "max_m": s.max_m,
            "root_m": int(s.m[-1]), "max_k": s.max_k, "sum_k": s.sum_k, "nnz_lu": s.nnz_lu,
            "sum_cb": s.sum_cb, "flops": s.flops,
        }
        with open(os.path.join(HERE, f"symbolic_{name}.txt"), "w") as f:
            for k, v in rows.items():
                f.write(f"{k}={v}\n")
        print(name, rows)


if __name__ == "__main__":
    main()
