"""Writes config3_det_mod.txt: det A mod eight primes just below 2^62 for the
dense random matrix of the n = 10007 Smith-form workload (entries uniform in
[-100, 100], inputs.smith_dense_matrix(10007, 100, seed 0)).

The values come from the oracle alone (oracle.det_mod: Gaussian elimination
over GF(q) in plain C); the primes are sympy's prevprime chain below 2^62.
Section 2: the invariant factors of a nonsingular A multiply to |det A|, so a
Smith form of this matrix must satisfy prod s_i = +-det A mod every q, with
one sign for all of them.  The GPU test of that Smith form reads this file.

Run once from the repository root (about five minutes per prime on 8 cores):
    python tests/golden/config3_det.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

N, BOUND, SEED, COUNT = 10007, 100, 0, 8
OUT = os.path.join(HERE, "config3_det_mod.txt")


def main():
    import sympy

    import oracle
    from paper_2605_19254_gb300 import inputs

    A = inputs.smith_dense_matrix(N, BOUND, SEED)
    primes, q = [], 1 << 62
    while len(primes) < COUNT:
        q = int(sympy.prevprime(q))
        primes.append(q)
    lines = [f"# det A mod q for inputs.smith_dense_matrix({N}, {BOUND}, {SEED}); written by config3_det.py "
             "from oracle.det_mod", f"n {N} bound {BOUND} seed {SEED}"]
    for q in primes:
        d = oracle.det_mod(A, q)
        lines.append(f"{q} {d}")
        print(q, d, flush=True)
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
