"""Oracle: hash functions h: [n] -> [b] and complex Rademacher signs (Sec. 3.3, Prop. 2).

The paper asks for a 2-wise independent H = h1 + h2 + h3 (Sec. 2, tensor sketch) and, for
the colliding symmetric sketch, a 6-wise independent h (Prop. 2 with p = 3, q = 2).  It
does not fix a family.  The reading used here (and by the CUDA path, independently
written) is the Carter-Wegman polynomial family over GF(P), P = 2^61 - 1:

    h(i) = ((a_0 + a_1 i + ... + a_5 i^5) mod P) mod b        (degree 5: 6-wise independent)
    g(i) = ((c_0 + c_1 i + ... + c_11 i^11) mod P) mod 4      (degree 11: 12-wise independent)

and sigma(i) = sqrt(-1)^g(i), i.e. uniform on the 4th roots of unity {1, i, -1, -i}
(Sec. 3.3 takes m = 4).  For the asymmetric sketch the real sign is xi(i) = 1 - 2 (g(i) & 1).

Coefficients come from the SplitMix64 generator (Steele, Lea & Flood, OOPSLA 2014):
state_c = seed + (c + 1) * 0x9E3779B97F4A7C15 (mod 2^64), output_c = mix64(state_c).
Coefficient e of (sketch m, mode j, table w) uses counter c = ((m * M + j) * 2 + w) * 16 + e,
with w = 0 for h and w = 1 for g, reduced mod P.

TEST INFRASTRUCTURE ONLY -- imported by tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline legs; the product path never calls it.
"""
from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1
P61 = (1 << 61) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15
H_DEGREE = 5      # 6-wise independent bucket hash
G_DEGREE = 11     # 12-wise independent sign hash


def mix64(z: int) -> int:
    """SplitMix64 output function (published constants)."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def splitmix64_output(seed: int, counter: int) -> int:
    """Output number `counter` (0-based) of the SplitMix64 stream started at `seed`."""
    return mix64((seed + (counter + 1) * GOLDEN_GAMMA) & MASK64)


def coefficients(seed: int, m: int, mode: int, M: int, which: int, count: int) -> list[int]:
    base = ((m * M + mode) * 2 + which) * 16
    return [splitmix64_output(seed, base + e) % P61 for e in range(count)]


def poly_mod_p(coefs: list[int], x: int) -> int:
    """sum_e coefs[e] * x^e mod P, by Horner's rule with exact integers."""
    acc = 0
    for c in reversed(coefs):
        acc = (acc * x + c) % P61
    return acc


def cs_hashes(seed: int, B: int, log2b: int, dims: list[int]):
    """Return (h, g): int64 arrays of shape [B][M][nmax] with h in [0, b) and g in {0,1,2,3}.

    M = len(dims) is 1 for the colliding (symmetric) sketch and 3 for the asymmetric one.
    Entries beyond dims[j] in mode j are left at 0.
    """
    M = len(dims)
    b = 1 << log2b
    nmax = max(dims) if dims else 0
    h = np.zeros((B, M, nmax), dtype=np.int64)
    g = np.zeros((B, M, nmax), dtype=np.int64)
    for m in range(B):
        for j in range(M):
            a = coefficients(seed, m, j, M, 0, H_DEGREE + 1)
            c = coefficients(seed, m, j, M, 1, G_DEGREE + 1)
            for i in range(dims[j]):
                h[m, j, i] = poly_mod_p(a, i) % b
                g[m, j, i] = poly_mod_p(c, i) % 4
    return h, g


def sigma_of(g: np.ndarray) -> np.ndarray:
    """Complex Rademacher variable sigma = sqrt(-1)^g (Sec. 3.3, m = 4)."""
    return np.array([1.0 + 0j, 1j, -1.0 + 0j, -1j])[np.asarray(g) % 4]


def xi_of(g: np.ndarray) -> np.ndarray:
    """Real Rademacher sign xi = 1 - 2 (g & 1) used by the asymmetric sketch (Eq. 1)."""
    return 1.0 - 2.0 * (np.asarray(g) & 1)
