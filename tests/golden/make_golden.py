"""Write tests/golden/oracle_n8.txt: the FP64 oracle's A h, A^T g and two
iterations of Algorithm 8 (Sec. 3.2; the operator of Sec. 2.1, eq. (1)-(4))
on an 8^3 problem drawn with the seeded generators, so that GPU tests can
compare against stored values and any later change of the oracle's arithmetic
shows up as a diff of this file.  The paper prints no worked example for this
path (its only numbers are the 2D experiment errors of Sec. 5 on a phantom
that is not published), so the stored values are the oracle's.

  python tests/golden/make_golden.py

Calls only the oracle and the input generators.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

N, NTH, T, LAM, STEP, ITERS, SEED = 8, 6, 0.6, 1e-3, 0.05, 2, 808


def case():
    from paper_1901_06503_gb300.inputs import config
    w = config(1, n=N, seed=SEED)
    noise = np.random.default_rng(SEED + 1).standard_normal((NTH, N, N))
    return w.c, w.h, noise


def compute():
    import oracle.oracle as o
    c, h, noise = case()
    g = o.forward(c, h, T, NTH)
    from paper_1901_06503_gb300.inputs import add_noise
    gd = add_noise(g, noise, 0.01)
    a = o.adjoint(c, gd, T)
    hk, _, k = o.fb(c, gd, T, LAM, STEP, ITERS)
    assert k == ITERS
    return {"A_h": g, "At_g": a, "fb_h2": hk}


def main():
    out = compute()
    path = os.path.join(HERE, "oracle_n8.txt")
    with open(path, "w") as f:
        f.write(f"# FP64 oracle, N={N}, angles={NTH}, T={T}, lambda={LAM}, step={STEP}, "
                f"iters={ITERS}, seed={SEED}\n")
        f.write("# inputs: config(1, n=8, seed=808) sound speed and source, 1 % noise from "
                "default_rng(809); written by tests/golden/make_golden.py\n")
        for name, arr in out.items():
            f.write(f"{name} {' '.join(str(d) for d in arr.shape)}\n")
            for v in arr.ravel():
                f.write(f"{float(v)!r}\n")
    print(path)


def load():
    path = os.path.join(HERE, "oracle_n8.txt")
    res, lines = {}, [ln for ln in open(path) if not ln.startswith("#")]
    i = 0
    while i < len(lines):
        head = lines[i].split()
        shape = tuple(int(d) for d in head[1:])
        size = int(np.prod(shape))
        res[head[0]] = np.array([float(v) for v in lines[i + 1:i + 1 + size]]).reshape(shape)
        i += 1 + size
    return res


if __name__ == "__main__":
    main()
