"""Writes tests/golden/hashes_seed1.txt and tests/golden/hashes_order_p_seed3.txt from the
oracle alone (oracle.hashing.cs_hashes, oracle.orderp.cs_hashes_p).

The fixture freezes the hash convention (Carter-Wegman polynomials over GF(2^61 - 1) with
SplitMix64 coefficients; the paper fixes only the independence the family must have,
Sec. 2 and Prop. 2).  Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))
import oracle  # noqa: E402


def main():
    seed, B, log2b, dims = 1, 2, 10, [3, 5, 4]
    h, g = oracle.cs_hashes(seed, B, log2b, dims)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "hashes_seed1.txt")
    with open(out, "w") as f:
        f.write(f"# cs_hashes(seed={seed}, B={B}, log2b={log2b}, dims={dims}) from oracle.hashing\n")
        f.write("# columns: sketch m, mode j, index i, h, g\n")
        for m in range(B):
            for j, n in enumerate(dims):
                for i in range(n):
                    f.write(f"{m} {j} {i} {h[m, j, i]} {g[m, j, i]}\n")
    # order-p hashes: h from the degree-(2p-1) polynomial, g reduced mod m (8 for p = 4..6)
    seed, B, log2b, n = 3, 2, 12, 6
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "hashes_order_p_seed3.txt")
    with open(out, "w") as f:
        f.write(f"# cs_hashes_p(seed={seed}, B={B}, log2b={log2b}, p, n={n}) from oracle.orderp\n")
        f.write("# columns: order p, sketch m, index i, h, g\n")
        for p in (4, 6):
            h, g = oracle.orderp.cs_hashes_p(seed, B, log2b, p, n)
            for m in range(B):
                for i in range(n):
                    f.write(f"{p} {m} {i} {h[m, i]} {g[m, i]}\n")


if __name__ == "__main__":
    main()
