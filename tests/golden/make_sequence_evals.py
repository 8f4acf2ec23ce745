"""Writes tests/golden/seq_n2000_evals.txt: the lowest nev + nex + 1 eigenvalues of every
problem of the seeded n = 2000 sequence (20 steps, nev = 200, nex = 40), computed with the
oracle's direct solver (O1) only.  Inputs come from the seeded generator.

Run:  python tests/golden/make_sequence_evals.py  (about half an hour on 8 cores)."""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import direct  # noqa: E402
from paper_1305_5120_gb300 import synth  # noqa: E402


def main():
    w = synth.SEQ_N2000
    count = w.nev + w.nex + 1
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "seq_n2000_evals.txt")
    lines = [f"# lowest {count} eigenvalues of H_l x = lam S x, n={w.n}, seed={w.seed}, "
             f"steps={w.steps} (oracle O1: Cholesky, Householder tridiagonalisation, implicit QR)"]
    L = None
    for step, p in synth.sequence(w.n, w.n_low, w.high, w.steps, w.seed):
        t = time.time()
        if L is None:
            L = direct.cholesky(p.S)
        Hs = direct.reduce_to_standard(p.H, L)
        lam = direct.hermitian_eig(Hs, vectors=False)[:count]
        if p.lam is not None:
            print(f"step 0 vs prescribed: {np.abs(lam - p.lam[:count]).max():.3e}", flush=True)
        lines.append(f"{step} " + " ".join(f"{x:.17e}" for x in lam))
        print(f"step {step} done in {time.time() - t:.1f}s", flush=True)
        with open(out, "w") as f:
            f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
