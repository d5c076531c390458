"""Oracle: sketched tensor contractions T^(I,u,u) and T^(u,u,u) (Sec. 3.2, Prop. 1, App. B).

Exact contractions (Sec. 2):
    T(I,u,u)_i = sum_{j,k} T_ijk u_j u_k ,    T(u,u,u) = sum_{i,j,k} T_ijk u_i u_j u_k.

Definition-level sketched estimates (App. B, Eq. (11)), for one colliding sketch S = s~_T:
    T^(u,u,u)   = Re <S, s~_{X~}>          X   = u (x) u (x) u
    T^(I,u,u)_i = Re <S, s~_{Z~_i}> / 3    Z_i = e_i(x)u(x)u + u(x)e_i(x)u + u(x)u(x)e_i
(<A, Y_i> = <A, Z_i>/3 for symmetric A, footnote in App. B), where ~ keeps only i <= j <= k.

Fast forms (App. B, Eq. (13)-(14)).  With s_u = s~_u, s_2 = s~_{2,u o u}, s_3 = s~_{3,u o u o u},
w = s_u * s_u, and corr(x, y) = F^{-1}(F x o conj F y) (Prop. 1):
    s~_{X~} = 1/6 s_u*s_u*s_u + 1/2 s_2*s_u + 1/3 s_3
    T^(u,u,u) = Re[ 1/6 <S, w*s_u> + 1/2 <S, s_2*s_u> + 1/3 <S, s_3> ]
    T^(I,u,u)_i = Re[ 1/6 conj(sigma_i) (corr(S,w) + corr(S,s_2))[h_i]
                      + 1/3 conj(sigma_i)^2 u_i corr(S,s_u)[2 h_i mod b]
                      + 1/3 conj(sigma_i)^3 u_i^2 S[3 h_i mod b] ]
Reading: Eq. (14) as printed carries coefficients (1, 1/6, 1/6, 1); expanding the printed
sketch of Z~_i and dividing by 3 gives (1/3, 1/6, 1/6, 1/3), used here.  The collision-free
tests (where the estimate must equal the exact contraction) decide between the two.
Eq. (13) mixes frequency- and time-domain inner products; everything here is in the time
domain (an unnormalised DFT would scale the frequency-domain ones by b).

TEST INFRASTRUCTURE ONLY -- imported by tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline legs; the product path never calls it.
"""
from __future__ import annotations

import numpy as np

from .conv import conv_direct, conv_fft, corr_direct, corr_fft, inner
from .hashing import sigma_of, xi_of
from .sketch import count_sketch, count_sketch_asym, sketch_truncated_sym

ENGINES = {
    "direct": (conv_direct, corr_direct),
    "fft": (conv_fft, corr_fft),
}


# ---------------------------------------------------------------- exact (Sec. 2)
def exact_iuu(T: np.ndarray, u: np.ndarray) -> np.ndarray:
    T = np.asarray(T, dtype=np.float64)
    return np.einsum("ijk,j,k->i", T, u, u)


def exact_uuu(T: np.ndarray, u: np.ndarray) -> float:
    return float(np.dot(exact_iuu(T, u), u))


def exact_ivw(T: np.ndarray, v: np.ndarray, w: np.ndarray) -> np.ndarray:
    return np.einsum("ijk,j,k->i", np.asarray(T, dtype=np.float64), v, w)


# ---------------------------------------------------------------- definition level (App. B)
def contract_uuu_def(S: np.ndarray, u: np.ndarray, h, g, b: int) -> float:
    """Re <S, s~_{X~}> with X~ the truncated u(x)u(x)u sketched by definition (O(n^3))."""
    X = np.einsum("i,j,k->ijk", u, u, u)
    return float(np.real(inner(S, sketch_truncated_sym(X, h, g, b))))


def contract_iuu_def(S: np.ndarray, u: np.ndarray, h, g, b: int) -> np.ndarray:
    """Re <S, s~_{Z~_i}> / 3 with Z~_i sketched by definition (O(n^4): tiny n only)."""
    n = u.shape[0]
    out = np.zeros(n)
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        Z = (np.einsum("i,j,k->ijk", e, u, u) + np.einsum("i,j,k->ijk", u, e, u)
             + np.einsum("i,j,k->ijk", u, u, e))
        out[i] = np.real(inner(S, sketch_truncated_sym(Z, h, g, b))) / 3.0
    return out


# ---------------------------------------------------------------- fast forms (App. B)
def contract_uuu(S: np.ndarray, u: np.ndarray, h, g, b: int, engine: str = "direct") -> float:
    conv, _ = ENGINES[engine]
    su = count_sketch(u, h, g, b, 1)
    s2 = count_sketch(u, h, g, b, 2)
    s3 = count_sketch(u, h, g, b, 3)
    w = conv(su, su)
    val = inner(S, conv(w, su)) / 6.0 + inner(S, conv(s2, su)) / 2.0 + inner(S, s3) / 3.0
    return float(np.real(val))


def contract_iuu(S: np.ndarray, u: np.ndarray, h, g, b: int, engine: str = "direct") -> np.ndarray:
    conv, corr = ENGINES[engine]
    n = u.shape[0]
    hh = np.asarray(h[:n], dtype=np.int64)
    csig = np.conj(sigma_of(g[:n]))
    su = count_sketch(u, h, g, b, 1)
    s2 = count_sketch(u, h, g, b, 2)
    w = conv(su, su)
    g0 = corr(S, su)
    g1 = corr(S, s2)
    g2 = corr(S, w)
    v = ((g2[hh] + g1[hh]) * csig / 6.0
         + g0[(2 * hh) % b] * csig ** 2 * u / 3.0
         + S[(3 * hh) % b] * csig ** 3 * u * u / 3.0)
    return np.real(v)


def contract_ivw_asym(S: np.ndarray, v: np.ndarray, w: np.ndarray, h, g, b: int, n1: int,
                      engine: str = "direct") -> np.ndarray:
    """Asymmetric T^(I,v,w)_i = xi_1(i) [F^{-1}(F s_T o conj F s_{2,v} o conj F s_{3,w})]_{h_1(i)}
    (Prop. 1 with Alg. 1's read-off rule).  h, g have shape [3][nmax]; S is the Eq. (1) sketch."""
    _, corr = ENGINES[engine]
    s2 = count_sketch_asym(v, h[1], g[1], b)
    s3 = count_sketch_asym(w, h[2], g[2], b)
    c = corr(corr(S, s2), s3)
    return np.real(xi_of(g[0][:n1]) * c[np.asarray(h[0][:n1], dtype=np.int64)])
