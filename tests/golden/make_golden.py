"""Writes the stored expected values under tests/golden/ from the oracle only.

Run:  python tests/golden/make_golden.py
Each fixture is a small case from ``cases`` solved by the CPU oracle
(dense Cholesky), stored as hex floats so the per-face quantities can be
compared bit for bit.  The inputs (alpha, phi) are stored too: the case
generator calls libm (cos, cosh), whose last bits differ between machines,
so tests read the stored inputs instead of regenerating them.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import cases  # noqa: E402
import oracle  # noqa: E402

FIXTURES = {
    "tank_8x4": lambda: cases.box_case(8, 4, 1, seed=3, ka=0.15),
    "box_6x4x3_perm": lambda: cases.box_case(6, 4, 3, seed=4, permute=True, alpha_noise=0.1),
}


def write(name, c):
    p, fc, sy, info = oracle.solve(c, direct=True)
    q = oracle.corrected_flux(c, fc, p)
    path = os.path.join(HERE, f"{name}.txt")
    with open(path, "w") as fh:
        fh.write(f"# {name}: oracle output (dense Cholesky) for cases recipe {name}\n")
        fh.write(f"# n {c.n} F {c.F} ref_cell {c.ref_cell}\n")
        fh.write("# face: f phi lambda gamma jump corrected_flux (hex floats)\n")
        for f in range(c.F):
            fh.write(f"F {f} {c.phi[f].hex()} {fc.lam[f].hex()} {fc.gamma[f].hex()} {fc.jump[f].hex()} {q[f].hex()}\n")
        fh.write("# cell: i alpha diag b p (hex floats)\n")
        for i in range(c.n):
            fh.write(f"C {i} {c.alpha[i].hex()} {sy.diag[i].hex()} {sy.b[i].hex()} {p[i].hex()}\n")


def read(name):
    faces, cells = [], []
    with open(os.path.join(HERE, f"{name}.txt")) as fh:
        for line in fh:
            t = line.split()
            if not t or t[0] == "#":
                continue
            vals = [float.fromhex(v) for v in t[2:]]
            (faces if t[0] == "F" else cells).append(vals)
    fa, ca = np.array(faces), np.array(cells)
    return {"phi": fa[:, 0], "lam": fa[:, 1], "lambda": fa[:, 1], "gamma": fa[:, 2], "jump": fa[:, 3],
            "flux": fa[:, 4], "alpha": ca[:, 0], "diag": ca[:, 1], "b": ca[:, 2], "p": ca[:, 3]}


def case(name):
    """The fixture's case with its stored inputs (machine independent)."""
    c = FIXTURES[name]()
    g = read(name)
    c.alpha = g["alpha"].copy()
    c.phi = g["phi"].copy()
    return c, g


if __name__ == "__main__":
    for nm, mk in FIXTURES.items():
        write(nm, mk())
        print("wrote", nm)
