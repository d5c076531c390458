"""Oracle: robust tensor power method, plain (Sec. 2) and sketched (Alg. 1 with the colliding
sketch of Sec. 3.3 and the contractions of App. B).

Readings where Alg. 1 is silent:
* median of an even number of values = mean of the two middle order statistics, taken over
  the real parts (Alg. 1, footnote to the median step);
* every deflation round draws fresh initial vectors; they are inputs here (U0[r][tau]) and are
  normalised before use (Alg. 1 draws u_0 uniformly from the unit sphere);
* tau* = first index attaining the maximum of the signed lambda_tau (selection step);
* no extra refinement iterations from tau* (the printed Alg. 1 has none);
* deflation subtracts lambda^ times the full colliding sketch of u^(x)3 from every sketch
  (deflation step; Sec. 3.3: s~_{u^(x)3} = s~_u * s~_u * s~_u);
* a zero or non-finite ||v_bar|| is an error (Alg. 1 divides by it).

`tau_choice` lets a caller force the selection of each round (used by parity tests to follow a
decision the other side took among near-ties); by default the argmax above is used.

TEST INFRASTRUCTURE ONLY -- imported by tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline legs; the product path never calls it.
"""
from __future__ import annotations

import numpy as np

from .contract import contract_iuu, contract_uuu, exact_iuu, exact_uuu
from .sketch import count_sketch
from .conv import conv_direct, conv_fft


class NonFiniteError(ArithmeticError):
    pass


def median(values: np.ndarray) -> float:
    """Median of a 1-D sequence; mean of the two middle values when the length is even."""
    x = np.sort(np.asarray(values, dtype=np.float64))
    m = x.shape[0]
    if m % 2 == 1:
        return float(x[m // 2])
    return float(0.5 * (x[m // 2 - 1] + x[m // 2]))


def median_rows(V: np.ndarray) -> np.ndarray:
    """Elementwise median over axis 0 (the B sketches)."""
    return np.array([median(V[:, i]) for i in range(V.shape[1])])


def normalise(v: np.ndarray) -> np.ndarray:
    nrm = float(np.sqrt(np.dot(v, v)))
    if not np.isfinite(nrm) or nrm == 0.0:
        raise NonFiniteError("zero or non-finite norm in the power update")
    return v / nrm


def power_step_sketched(S: np.ndarray, u: np.ndarray, h, g, b: int, engine: str = "fft"):
    """One power update of Alg. 1: v^(m) = T^(m)(I,u,u) for every sketch m, v_bar = median,
    u' = v_bar / ||v_bar||.  Returns (u', V) with V of shape [B][n]."""
    B = S.shape[0]
    V = np.stack([contract_iuu(S[m], u, h[m], g[m], b, engine) for m in range(B)])
    return normalise(median_rows(V)), V


def eigenvalue_sketched(S: np.ndarray, u: np.ndarray, h, g, b: int, engine: str = "fft"):
    """lambda = median_m T^(m)(u,u,u) (selection step of Alg. 1).  Returns (lambda, per-sketch)."""
    lam = np.array([contract_uuu(S[m], u, h[m], g[m], b, engine) for m in range(S.shape[0])])
    return median(lam), lam


def deflate_sketches(S: np.ndarray, lam: float, u: np.ndarray, h, g, b: int,
                     engine: str = "fft") -> np.ndarray:
    """S^(m) <- S^(m) - lam * s~^(m)_{u^(x)3} for every m (deflation step of Alg. 1)."""
    conv = conv_fft if engine == "fft" else conv_direct
    out = S.copy()
    for m in range(S.shape[0]):
        su = count_sketch(u, h[m], g[m], b, 1)
        out[m] = S[m] - lam * conv(conv(su, su), su)
    return out


def rtpm_sketched(S: np.ndarray, h, g, b: int, U0: np.ndarray, T_iters: int,
                  engine: str = "fft", tau_choice=None):
    """Alg. 1 on B colliding sketches S[m] (complex, time domain).

    U0: [k][L][n] initial vectors.  Returns dict with lam [k], V [k][n], tau [k], the final
    iterates of every round (U_final [k][L][n]) and their eigenvalues (lam_all [k][L])."""
    k, L, n = U0.shape
    S = np.array(S, dtype=np.complex128, copy=True)
    lam_out = np.zeros(k)
    V_out = np.zeros((k, n))
    tau_out = np.zeros(k, dtype=np.int64)
    U_final = np.zeros((k, L, n))
    lam_all = np.zeros((k, L))
    for r in range(k):
        U = np.stack([normalise(U0[r, tau]) for tau in range(L)])
        for _ in range(T_iters):
            U = np.stack([power_step_sketched(S, U[tau], h, g, b, engine)[0] for tau in range(L)])
        lam = np.array([eigenvalue_sketched(S, U[tau], h, g, b, engine)[0] for tau in range(L)])
        tau_star = int(np.argmax(lam)) if tau_choice is None else int(tau_choice[r])
        lam_out[r] = lam[tau_star]
        V_out[r] = U[tau_star]
        tau_out[r] = tau_star
        U_final[r] = U
        lam_all[r] = lam
        S = deflate_sketches(S, lam[tau_star], U[tau_star], h, g, b, engine)
    return {"lam": lam_out, "V": V_out, "tau": tau_out, "U_final": U_final,
            "lam_all": lam_all, "S_deflated": S}


def rtpm_exact(T: np.ndarray, U0: np.ndarray, T_iters: int, tau_choice=None):
    """The plain robust tensor power method (Sec. 2) with exact contractions and dense deflation
    T <- T - lam u(x)u(x)u."""
    k, L, n = U0.shape
    T = np.array(T, dtype=np.float64, copy=True)
    lam_out = np.zeros(k)
    V_out = np.zeros((k, n))
    tau_out = np.zeros(k, dtype=np.int64)
    for r in range(k):
        U = np.stack([normalise(U0[r, tau]) for tau in range(L)])
        for _ in range(T_iters):
            U = np.stack([normalise(exact_iuu(T, U[tau])) for tau in range(L)])
        lam = np.array([exact_uuu(T, U[tau]) for tau in range(L)])
        tau_star = int(np.argmax(lam)) if tau_choice is None else int(tau_choice[r])
        lam_out[r] = lam[tau_star]
        V_out[r] = U[tau_star]
        tau_out[r] = tau_star
        u = U[tau_star]
        T = T - lam[tau_star] * np.einsum("i,j,k->ijk", u, u, u)
    return {"lam": lam_out, "V": V_out, "tau": tau_out}


def rtpm_sketched_asym(S: np.ndarray, h, g, b: int, U0: np.ndarray, T_iters: int,
                       engine: str = "fft", tau_choice=None):
    """Alg. 1 exactly as printed: B asymmetric sketches S[m] (Eq. 1, real, time domain) built
    with three independent hashes h[m][j], xi[m][j] (j = 0, 1, 2 for modes 1, 2, 3).

    Power update: v^(m)_i = xi_1(i) [F^-1(F s_T o conj F s_{2,u} o conj F s_{3,u})]_{h_1(i)},
    u <- median_m Re v^(m) / ||.||.  Selection: lambda^(m)_tau = T^(m)(u,u,u), which by
    Prop. 1's linearity is sum_i u_i v^(m)_i(u); lambda_tau = median_m, tau* = first argmax.
    Deflation: every sketch loses lambda^ s_{1,u^} * s_{2,u^} * s_{3,u^} (Eq. 4).
    Same readings as rtpm_sketched (median, fresh inputs U0[r][tau], no refinement)."""
    from .contract import contract_ivw_asym
    from .sketch import sketch_rank1_asym
    k, L, n = U0.shape
    B = S.shape[0]
    S = np.array(np.real(S), dtype=np.float64, copy=True)
    lam_out = np.zeros(k)
    V_out = np.zeros((k, n))
    tau_out = np.zeros(k, dtype=np.int64)
    U_final = np.zeros((k, L, n))
    lam_all = np.zeros((k, L))

    def per_sketch(u):
        return np.stack([contract_ivw_asym(S[m], u, u, h[m], g[m], b, n, engine) for m in range(B)])

    for r in range(k):
        U = np.stack([normalise(U0[r, tau]) for tau in range(L)])
        for _ in range(T_iters):
            U = np.stack([normalise(median_rows(per_sketch(U[tau]))) for tau in range(L)])
        lam = np.array([median(per_sketch(U[tau]) @ U[tau]) for tau in range(L)])
        tau_star = int(np.argmax(lam)) if tau_choice is None else int(tau_choice[r])
        lam_out[r] = lam[tau_star]
        V_out[r] = U[tau_star]
        tau_out[r] = tau_star
        U_final[r] = U
        lam_all[r] = lam
        u = U[tau_star]
        for m in range(B):
            S[m] = S[m] - lam[tau_star] * np.real(sketch_rank1_asym(u, u, u, h[m], g[m], b))
    return {"lam": lam_out, "V": V_out, "tau": tau_out, "U_final": U_final,
            "lam_all": lam_all, "S_deflated": S}
