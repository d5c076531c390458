"""Oracle: sketched CP loss and its gradient; the sketched ALS update (Alg. 2 with Eq. 15).

Sketched CP loss for B asymmetric sketches S[m] of T (Eq. 1) and a rank-R model:
    L = (1/B) sum_m || S[m] - sum_r lam_r s^(m)_{a_r (x) b_r (x) c_r} ||^2,
    s_{a (x) b (x) c} = s_1,a * s_2,b * s_3,c                                  (Eq. 4)
All sketches are real (xi = +-1).  The gradient is obtained from linearity of the sketch in each
factor (s_1,a = sum_i a_i s_1,e_i, Sec. 3.1) and Prop. 1:
    dL/dlam_r = -(2/B) sum_m < R^(m), s^(m)_r >,  R^(m) = S[m] - sum_r lam_r s^(m)_r
    dL/da_r[i] = -(2 lam_r / B) sum_m xi_1(i) corr(corr(R^(m), s_2,b_r), s_3,c_r)[h_1(i)]
and likewise for b_r (with s_1,a_r, s_3,c_r read at h_2) and c_r (s_1,a_r, s_2,b_r at h_3).
This loss and gradient are not printed in the paper; they follow from Eq. 4 and Prop. 1.

Sketched ALS (Alg. 2): column r of T_(1)(C (.) B) is T(I, b_r, c_r) (Eq. 16-17), estimated by
the median over sketches of the asymmetric T^(I, b_r, c_r); the update applies the Gram
pseudo-inverse of Eq. 15, A = T_(1)(C (.) B) (C^T C o B^T B)^+, which the printed Alg. 2 omits.
Then lam_r = ||a_r|| and a_r is normalised.

TEST INFRASTRUCTURE ONLY -- imported by tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline legs; the product path never calls it.
"""
from __future__ import annotations

import numpy as np

from .contract import ENGINES
from .hashing import xi_of
from .rtpm import median_rows
from .sketch import count_sketch_asym


def _other_modes(mode: int):
    return [j for j in range(3) if j != mode]


def _rank1(factors, r, h, g, b, conv):
    s = [count_sketch_asym(factors[j][r], h[j], g[j], b) for j in range(3)]
    return conv(conv(s[0], s[1]), s[2]), s


def cp_sketch_loss(S, h, g, b, lam, A, Bf, C, engine="fft") -> float:
    """S: [B][b] real sketches; h, g: [B][3][nmax]; A: [R][n1], Bf: [R][n2], C: [R][n3]."""
    conv, _ = ENGINES[engine]
    factors = (A, Bf, C)
    total = 0.0
    for m in range(S.shape[0]):
        model = np.zeros(b)
        for r in range(len(lam)):
            s_r, _ = _rank1(factors, r, h[m], g[m], b, conv)
            model += lam[r] * np.real(s_r)
        R = np.real(S[m]) - model
        total += float(np.dot(R, R))
    return total / S.shape[0]


def cp_sketch_grad(S, h, g, b, lam, A, Bf, C, engine="fft"):
    """Closed-form gradient of cp_sketch_loss: (g_lam [R], g_A, g_B, g_C)."""
    conv, corr = ENGINES[engine]
    factors = (A, Bf, C)
    Bn = S.shape[0]
    R_ = len(lam)
    g_lam = np.zeros(R_)
    grads = [np.zeros_like(np.asarray(f, dtype=np.float64)) for f in factors]
    for m in range(Bn):
        parts = [_rank1(factors, r, h[m], g[m], b, conv) for r in range(R_)]
        model = sum(lam[r] * np.real(parts[r][0]) for r in range(R_))
        Res = np.real(S[m]) - model
        for r in range(R_):
            s_r, sk = parts[r]
            g_lam[r] += -2.0 * float(np.dot(Res, np.real(s_r)))
            for j in range(3):
                p, q = _other_modes(j)
                c = np.real(corr(corr(Res, sk[p]), sk[q]))
                n_j = factors[j].shape[1]
                hj = np.asarray(h[m][j][:n_j], dtype=np.int64)
                grads[j][r] += -2.0 * lam[r] * xi_of(g[m][j][:n_j]) * c[hj]
    return g_lam / Bn, grads[0] / Bn, grads[1] / Bn, grads[2] / Bn


def cp_exact_loss(T, lam, A, Bf, C) -> float:
    model = np.einsum("r,ri,rj,rk->ijk", lam, A, Bf, C)
    D = np.asarray(T, dtype=np.float64) - model
    return float(np.sum(D * D))


def contract_ivw_mode(S, h, g, b, mode: int, V, W, n_o: int, engine="fft"):
    """Asymmetric T^(.)(I at `mode`, V on the lower other mode, W on the higher), one sketch:
    xi_mode(i) corr(corr(S, s_p,V), s_q,W)[h_mode(i)] (Prop. 1)."""
    _, corr = ENGINES[engine]
    p, q = _other_modes(mode)
    sp = count_sketch_asym(V, h[p], g[p], b)
    sq = count_sketch_asym(W, h[q], g[q], b)
    c = np.real(corr(corr(np.asarray(S, dtype=np.complex128), sp), sq))
    hm = np.asarray(h[mode][:n_o], dtype=np.int64)
    return xi_of(g[mode][:n_o]) * c[hm]


def als_sketched_columns(S, h, g, b, mode: int, factors, engine="fft"):
    """M[r] = median_m T^(m)(I, x_r, y_r) for the two other factors (Alg. 2)."""
    p, q = _other_modes(mode)
    n_o = factors[mode].shape[1]
    K = factors[p].shape[0]
    M = np.zeros((K, n_o))
    for r in range(K):
        V = np.stack([contract_ivw_mode(S[m], h[m], g[m], b, mode, factors[p][r], factors[q][r], n_o, engine)
                      for m in range(S.shape[0])])
        M[r] = median_rows(V)
    return M


def als_solve(M, P, Q):
    """Eq. 15: rows of out = (G^+ M) with G = (P P^T) o (Q Q^T); lam = row norms; rows normalised."""
    G = (P @ P.T) * (Q @ Q.T)
    out = np.linalg.pinv(G) @ M
    lam = np.linalg.norm(out, axis=1)
    return out / lam[:, None], lam
