"""Oracle: order-p symmetric (colliding) tensor sketches, p >= 3 -- the extension of Sec. 3.3
that the paper mentions without details (it attributes the higher-order recovery coefficients to
Young tableaux).

Readings (all of them this module's, written from the paper's definitions):

1. Sketch (Eq. 7 with p indices): s~_T(t) = sum over ordered p-tuples (i_1..i_p) with
   (h(i_1) + ... + h(i_p)) mod b = t of T_{i_1..i_p} sigma(i_1) ... sigma(i_p).
2. Signs: sigma uniform on the m-th roots of unity (Sec. 3.3).  E[sigma^k] = 0 unless m | k, and
   two p-tuples' sign products differ by sigma(i)^(c - c') with |c - c'| <= p, so m > p removes
   every repeated-entry alias; m = 4 for p = 3 (the paper's choice) and m = 8 for p = 4..7.
   With m = 4 and p = 4, sigma^4 = 1 aliases T_iiii onto u_j^4 (pinned in the tests).
3. Hash: h (2p)-wise independent (Prop. 2 with q = 2): the Carter-Wegman family of
   oracle.hashing with degree 2p - 1 for h (degree 5 at p = 3, the same hashes); the sign index
   keeps degree 11 (12-wise) and is reduced mod m.
4. Estimators.  The colliding sketch sums each multiset of indices once per ordering, so
   <s~_T, Y> with Y the sketch of the complete homogeneous polynomial h_p in the variables
   sigma(i) u_i x^{h(i)} gives T(u,...,u).  In power sums, h_p = sum over partitions lambda of
   p of p_lambda / z_lambda (z_lambda = prod_k k^{m_k} m_k!, m_k the multiplicity of part k), and
   the power sum p_k is the count sketch s_k[(k h(i)) mod b] += sigma(i)^k u_i^k.  So
       T^(u,...,u) = Re < S, sum_lambda (1/z_lambda) (s_{lambda_1} * ... * s_{lambda_l}) >.
   T^(I,u,...,u) is its gradient / p.  With R_k = sum over lambda containing k of
   (m_k(lambda) / z_lambda) times the convolution of lambda's other parts (R_p = delta / p) and
   G_k = corr(S, R_k):
       T^(I,u,...,u)_i = (1/p) Re sum_{k=1..p} k conj(sigma(i))^k u_i^(k-1) G_k[(k h(i)) mod b].
   At p = 3 these are App. B's Eq. 13 and the corrected Eq. 14 (pinned in the tests); with
   hashes whose p-fold sums never collide they are exact for every p (pinned).
5. Deflation: the sketch of u^{(x)p} is the p-fold convolution of s_1 (by definition), so
   S <- S - lambda^ s_1^{*p}.
6. Alg. 1 for order p: the power update v = median_m T^(m)(I,u,...,u), u <- v / ||v||; the
   selection lambda_tau = median_m T^(m)(u,...,u), tau* = first argmax; deflation as in 5.

TEST INFRASTRUCTURE ONLY -- imported by tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline legs; the product path never calls it.
"""
from __future__ import annotations

import math
from collections import Counter

import numpy as np

from .conv import conv_direct, conv_fft, corr_direct, corr_fft, inner
from .hashing import coefficients, poly_mod_p, G_DEGREE
from .rtpm import median, median_rows, normalise

ENGINES = {"direct": (conv_direct, corr_direct), "fft": (conv_fft, corr_fft)}


def roots_order(p: int) -> int:
    """m of reading 2: the smallest power of two above p (4 for p = 3, 8 for p = 4..7)."""
    m = 4
    while m <= p:
        m *= 2
    return m


def cs_hashes_p(seed: int, B: int, log2b: int, p: int, n: int):
    """Reading 3: h [B][n] in [0, b) from the degree-(2p-1) polynomial, g [B][n] in [0, m)."""
    b = 1 << log2b
    m_roots = roots_order(p)
    h = np.zeros((B, n), dtype=np.int64)
    g = np.zeros((B, n), dtype=np.int64)
    for s in range(B):
        a = coefficients(seed, s, 0, 1, 0, 2 * p)
        c = coefficients(seed, s, 0, 1, 1, G_DEGREE + 1)
        for i in range(n):
            h[s, i] = poly_mod_p(a, i) % b
            g[s, i] = poly_mod_p(c, i) % m_roots
    return h, g


def sigma_p(g, p: int) -> np.ndarray:
    """sigma = exp(2 pi i g / m), m = roots_order(p) (reading 2)."""
    m = roots_order(p)
    return np.exp(2j * np.pi * (np.asarray(g, dtype=np.int64) % m) / m)


def sketch_sym_p(T: np.ndarray, h, g, b: int, p: int) -> np.ndarray:
    """Reading 1 by its definition: every ordered p-tuple of the dense order-p tensor T."""
    n = T.shape[0]
    idx = np.indices((n,) * p).reshape(p, -1)
    hh = np.asarray(h[:n], dtype=np.int64)
    gg = np.asarray(g[:n], dtype=np.int64)
    H = hh[idx].sum(axis=0) % b
    val = T.reshape(-1).astype(np.complex128) * sigma_p(gg[idx].sum(axis=0), p)
    return (np.bincount(H, weights=val.real, minlength=b)
            + 1j * np.bincount(H, weights=val.imag, minlength=b))


def power_sketch(u: np.ndarray, h, g, b: int, p: int, k: int) -> np.ndarray:
    """s_k[(k h(i)) mod b] += sigma(i)^k u_i^k (the power sum p_k of reading 4)."""
    n = u.shape[0]
    hh = np.asarray(h[:n], dtype=np.int64)
    w = sigma_p(g[:n], p) ** k * np.asarray(u, dtype=np.float64) ** k
    return (np.bincount((k * hh) % b, weights=w.real, minlength=b)
            + 1j * np.bincount((k * hh) % b, weights=w.imag, minlength=b))


def partitions(p: int):
    """All partitions of p as non-increasing tuples (recursive enumeration)."""
    out = []

    def rec(rest, largest, prefix):
        if rest == 0:
            out.append(tuple(prefix))
            return
        for part in range(min(rest, largest), 0, -1):
            rec(rest - part, part, prefix + [part])

    rec(p, p, [])
    return out


def z_of(lam) -> int:
    """z_lambda = prod_k k^{m_k} m_k! (the size of the centraliser of a permutation of type lambda)."""
    z = 1
    for k, mk in Counter(lam).items():
        z *= k ** mk * math.factorial(mk)
    return z


def _conv_all(parts, sk, b, conv):
    """Circular convolution of the power sketches sk[k] over the parts (delta for no parts)."""
    acc = np.zeros(b, dtype=np.complex128)
    acc[0] = 1.0
    for k in parts:
        acc = conv(acc, sk[k])
    return acc


def estimate_uuu_p(S: np.ndarray, u: np.ndarray, h, g, b: int, p: int, engine: str = "fft") -> float:
    """Reading 4: T^(u,...,u) = Re <S, sum_lambda s_lambda / z_lambda>."""
    conv, _ = ENGINES[engine]
    sk = {k: power_sketch(u, h, g, b, p, k) for k in range(1, p + 1)}
    Y = np.zeros(b, dtype=np.complex128)
    for lam in partitions(p):
        Y += _conv_all(lam, sk, b, conv) / z_of(lam)
    return float(np.real(inner(S, Y)))


def estimate_iuu_p(S: np.ndarray, u: np.ndarray, h, g, b: int, p: int, engine: str = "fft") -> np.ndarray:
    """Reading 4: T^(I,u,...,u)_i = (1/p) Re sum_k k conj(sigma_i)^k u_i^(k-1) G_k[k h_i]."""
    conv, corr = ENGINES[engine]
    n = u.shape[0]
    hh = np.asarray(h[:n], dtype=np.int64)
    cs = np.conj(sigma_p(g[:n], p))
    sk = {k: power_sketch(u, h, g, b, p, k) for k in range(1, p + 1)}
    v = np.zeros(n, dtype=np.complex128)
    for k in range(1, p + 1):
        R = np.zeros(b, dtype=np.complex128)
        for lam in partitions(p):
            mk = lam.count(k)
            if mk == 0:
                continue
            rest = list(lam)
            rest.remove(k)
            R += mk / z_of(lam) * _conv_all(rest, sk, b, conv)
        G = corr(S, R)
        v += k * cs ** k * np.asarray(u, dtype=np.float64) ** (k - 1) * G[(k * hh) % b]
    return np.real(v) / p


def exact_uuu_p(T: np.ndarray, u: np.ndarray) -> float:
    """T(u,...,u): every mode contracted with u."""
    X = np.asarray(T, dtype=np.float64)
    for _ in range(X.ndim):
        X = X @ u
    return float(X)


def exact_iuu_p(T: np.ndarray, u: np.ndarray) -> np.ndarray:
    """T(I,u,...,u): every mode but the first contracted with u."""
    X = np.asarray(T, dtype=np.float64)
    for _ in range(X.ndim - 1):
        X = X @ u
    return X


def sketch_rank1_p(u: np.ndarray, h, g, b: int, p: int, engine: str = "fft") -> np.ndarray:
    """Reading 5: the sketch of u^{(x)p} = the p-fold convolution of s_1."""
    conv, _ = ENGINES[engine]
    s1 = power_sketch(u, h, g, b, p, 1)
    acc = s1
    for _ in range(p - 1):
        acc = conv(acc, s1)
    return acc


def symmetric_rank1_sum(lam: np.ndarray, A: np.ndarray, p: int) -> np.ndarray:
    """sum_r lam_r a_r^{(x)p} for the columns a_r of A (dense, order p)."""
    n, k = A.shape
    T = np.zeros((n,) * p)
    for r in range(k):
        X = np.asarray(A[:, r], dtype=np.float64)
        for _ in range(p - 1):
            X = np.multiply.outer(X, A[:, r])
        T += lam[r] * X
    return T


def power_step_p(S: np.ndarray, u: np.ndarray, h, g, b: int, p: int, engine: str = "fft"):
    """Reading 6: v^(m) = T^(m)(I,u,...,u) for every sketch, v_bar = median, u' = v_bar / ||v_bar||."""
    V = np.stack([estimate_iuu_p(S[m], u, h[m], g[m], b, p, engine) for m in range(S.shape[0])])
    return normalise(median_rows(V)), V


def eigenvalue_p(S: np.ndarray, u: np.ndarray, h, g, b: int, p: int, engine: str = "fft"):
    """Reading 6: lambda = median_m T^(m)(u,...,u).  Returns (lambda, per-sketch values)."""
    lam = np.array([estimate_uuu_p(S[m], u, h[m], g[m], b, p, engine) for m in range(S.shape[0])])
    return median(lam), lam


def deflate_p(S: np.ndarray, lam: float, u: np.ndarray, h, g, b: int, p: int,
              engine: str = "fft") -> np.ndarray:
    """Reading 5 for every sketch: S^(m) <- S^(m) - lam s~^(m)_{u^{(x)p}}."""
    return np.stack([S[m] - lam * sketch_rank1_p(u, h[m], g[m], b, p, engine)
                     for m in range(S.shape[0])])


def rtpm_sketched_p(S: np.ndarray, h, g, b: int, p: int, U0: np.ndarray, T_iters: int,
                    engine: str = "fft", tau_choice=None):
    """Alg. 1 for order p (reading 6).  U0: [k][L][n].  Returns lam, V, tau, U_final, lam_all,
    S_deflated as oracle.rtpm.rtpm_sketched does for p = 3."""
    k, L, n = U0.shape
    S = np.array(S, dtype=np.complex128, copy=True)
    lam_out, V_out = np.zeros(k), np.zeros((k, n))
    tau_out = np.zeros(k, dtype=np.int64)
    U_final, lam_all = np.zeros((k, L, n)), np.zeros((k, L))
    for r in range(k):
        U = np.stack([normalise(U0[r, tau]) for tau in range(L)])
        for _ in range(T_iters):
            U = np.stack([power_step_p(S, U[tau], h, g, b, p, engine)[0] for tau in range(L)])
        lam = np.array([eigenvalue_p(S, U[tau], h, g, b, p, engine)[0] for tau in range(L)])
        tau_star = int(np.argmax(lam)) if tau_choice is None else int(tau_choice[r])
        lam_out[r], V_out[r], tau_out[r] = lam[tau_star], U[tau_star], tau_star
        U_final[r], lam_all[r] = U, lam
        S = deflate_p(S, lam[tau_star], U[tau_star], h, g, b, p, engine)
    return {"lam": lam_out, "V": V_out, "tau": tau_out, "U_final": U_final,
            "lam_all": lam_all, "S_deflated": S}


def rtpm_exact_p(T: np.ndarray, U0: np.ndarray, T_iters: int):
    """The plain robust tensor power method of Sec. 2 for an order-p tensor (exact contractions,
    dense deflation), for the collision-free pin of rtpm_sketched_p."""
    k, L, n = U0.shape
    p = T.ndim
    T = np.array(T, dtype=np.float64, copy=True)
    lam_out, V_out = np.zeros(k), np.zeros((k, n))
    for r in range(k):
        U = np.stack([normalise(U0[r, tau]) for tau in range(L)])
        for _ in range(T_iters):
            U = np.stack([normalise(exact_iuu_p(T, U[tau])) for tau in range(L)])
        lam = np.array([exact_uuu_p(T, U[tau]) for tau in range(L)])
        t = int(np.argmax(lam))
        lam_out[r], V_out[r] = lam[t], U[t]
        T = T - symmetric_rank1_sum(np.array([lam[t]]), U[t][:, None], p)
    return {"lam": lam_out, "V": V_out}
