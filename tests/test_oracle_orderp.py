"""Pins of the order-p oracle (oracle/orderp.py) against facts fixed by the paper or by
mathematics: the class equation of the partitions, the p = 3 case of App. B, exactness with
hashes whose p-fold sums never collide, the rank-1 sketch by definition, the sign alias that
m > p removes (exact enumeration), unbiasedness over hash draws, and Alg. 1 for order p."""
import itertools

import numpy as np
import pytest

import oracle as O
import synth

P = O.orderp


def random_symmetric_p(n: int, p: int, seed: int) -> np.ndarray:
    """Average of a Gaussian order-p tensor over all permutations of its modes."""
    X = synth.rng(seed).standard_normal((n,) * p)
    perms = list(itertools.permutations(range(p)))
    return sum(np.transpose(X, q) for q in perms) / len(perms)


def collision_free(n: int, p: int, seed: int):
    """h(i) = (p+1)^i: a multiset of p indices is its base-(p+1) digit counts, so p-fold sums
    never collide; b is the next power of two above (p+1)^n.  Signs random on the m-th roots."""
    b = 1 << int(np.ceil(np.log2((p + 1) ** n)))
    h = np.array([(p + 1) ** i for i in range(n)], dtype=np.int64)
    g = synth.rng(seed).integers(0, P.roots_order(p), n)
    return h, g, b


def test_partitions_and_class_equation():
    """p(4), p(5), p(6) = 5, 7, 11, and sum_lambda 1/z_lambda = 1 (the class equation of S_p)."""
    for p, count in ((3, 3), (4, 5), (5, 7), (6, 11)):
        lam = P.partitions(p)
        assert len(lam) == count and len(set(lam)) == count
        assert all(sum(x) == p and list(x) == sorted(x, reverse=True) for x in lam)
        assert sum(1.0 / P.z_of(x) for x in lam) == pytest.approx(1.0, abs=1e-15)
    assert P.z_of((1, 1, 1)) == 6 and P.z_of((2, 1)) == 2 and P.z_of((3,)) == 3


def test_roots_order():
    assert [P.roots_order(p) for p in (3, 4, 5, 6, 7, 8)] == [4, 8, 8, 8, 8, 16]


def test_order3_reduces_to_app_b():
    """At p = 3 the power-sum estimators are App. B's Eq. 13 and the corrected Eq. 14 (the
    coefficients 1/6, 1/6, 1/3, 1/3 that the collision-free pins of the p = 3 oracle fix)."""
    n, b = 23, 256
    h, g = P.cs_hashes_p(11, 1, 8, 3, n)
    r = synth.rng(12)
    S = r.standard_normal(b) + 1j * r.standard_normal(b)
    u = r.standard_normal(n)
    for engine in ("fft", "direct"):
        assert P.estimate_uuu_p(S, u, h[0], g[0], b, 3, engine) == pytest.approx(
            O.contract_uuu(S, u, h[0], g[0], b, engine), rel=1e-12, abs=1e-12)
        np.testing.assert_allclose(P.estimate_iuu_p(S, u, h[0], g[0], b, 3, engine),
                                   O.contract_iuu(S, u, h[0], g[0], b, engine), rtol=1e-11, atol=1e-11)


def test_order3_hashes_are_the_colliding_hashes():
    h, g = P.cs_hashes_p(5, 3, 10, 3, 40)
    h3, g3 = O.cs_hashes(5, 3, 10, [40])
    np.testing.assert_array_equal(h, h3[:, 0])
    np.testing.assert_array_equal(g, g3[:, 0])


@pytest.mark.parametrize("p,n", [(3, 5), (4, 4), (4, 5), (5, 4), (6, 3)])
def test_collision_free_hashes_make_the_estimators_exact(p, n):
    T = random_symmetric_p(n, p, 100 + p)
    h, g, b = collision_free(n, p, 200 + p)
    S = P.sketch_sym_p(T, h, g, b, p)
    u = synth.rng(300 + p).standard_normal(n)
    for engine in ("fft", "direct"):
        assert P.estimate_uuu_p(S, u, h, g, b, p, engine) == pytest.approx(P.exact_uuu_p(T, u), rel=1e-9)
        np.testing.assert_allclose(P.estimate_iuu_p(S, u, h, g, b, p, engine), P.exact_iuu_p(T, u),
                                   rtol=1e-9, atol=1e-9)


def test_a_dropped_term_breaks_exactness():
    """Guard of the pin above: leaving out the single-part partition (p) of the power-sum
    expansion changes the p = 4 estimate (so every term is exercised)."""
    p, n = 4, 4
    T = random_symmetric_p(n, p, 7)
    h, g, b = collision_free(n, p, 8)
    S = P.sketch_sym_p(T, h, g, b, p)
    u = synth.rng(9).standard_normal(n)
    sk = {k: P.power_sketch(u, h, g, b, p, k) for k in range(1, p + 1)}
    Y = sum(P._conv_all(lam, sk, b, O.conv.conv_fft) / P.z_of(lam) for lam in P.partitions(p) if lam != (p,))
    assert abs(np.real(O.conv.inner(S, Y)) - P.exact_uuu_p(T, u)) > 1e-3


@pytest.mark.parametrize("p", [4, 5])
def test_rank1_sketch_is_the_definition(p):
    n, log2b = 7, 9
    h, g = P.cs_hashes_p(3, 1, log2b, p, n)
    u = synth.rng(40 + p).standard_normal(n)
    X = u
    for _ in range(p - 1):
        X = np.multiply.outer(X, u)
    for engine in ("fft", "direct"):
        np.testing.assert_allclose(P.sketch_rank1_p(u, h[0], g[0], 1 << log2b, p, engine),
                                   P.sketch_sym_p(X, h[0], g[0], 1 << log2b, p), atol=1e-10)


def test_fourth_roots_alias_at_order_four_and_eighth_roots_do_not():
    """T = e_0^{(x)4}, u = e_1: T(u,u,u,u) = 0.  When 4 h_0 = 4 h_1 (mod b) the estimate is
    sigma_0^4 conj(sigma_1)^4.  Averaged exactly over all sign pairs it is 1 if the signs are 4th
    roots (sigma^4 = 1: biased) and 0 if they are 8th roots (reading 2: m > p)."""
    p, n, b = 4, 2, 64
    T = np.zeros((n,) * p)
    T[0, 0, 0, 0] = 1.0
    u = np.array([0.0, 1.0])
    h = np.array([3, 3 + b // 4])               # 4 h_0 = 4 h_1 mod b, h_0 != h_1
    def mean_over(signs):
        vals = []
        for g0 in signs:
            for g1 in signs:
                g = np.array([g0, g1])
                vals.append(P.estimate_uuu_p(P.sketch_sym_p(T, h, g, b, p), u, h, g, b, p, "direct"))
        return float(np.mean(vals))
    assert mean_over([0, 2, 4, 6]) == pytest.approx(1.0, abs=1e-12)     # 4th roots of unity
    assert mean_over(range(8)) == pytest.approx(0.0, abs=1e-12)         # 8th roots of unity
    assert P.exact_uuu_p(T, u) == 0.0


@pytest.mark.parametrize("p,n,draws", [(4, 6, 600), (5, 4, 400)])
def test_order_p_estimate_unbiased_over_hash_draws(p, n, draws):
    """Lemma 1's unbiasedness at p = 4 and 5: the mean of T^(u,...,u) over independent hash
    draws matches T(u,...,u) within 4 standard errors."""
    log2b = 5
    T = random_symmetric_p(n, p, 55)
    u = synth.rng(56).standard_normal(n)
    u /= np.linalg.norm(u)
    est = []
    for d in range(draws):
        h, g = P.cs_hashes_p(1000 + d, 1, log2b, p, n)
        S = P.sketch_sym_p(T, h[0], g[0], 1 << log2b, p)
        est.append(P.estimate_uuu_p(S, u, h[0], g[0], 1 << log2b, p))
    est = np.array(est)
    se = est.std(ddof=1) / np.sqrt(draws)
    assert abs(est.mean() - P.exact_uuu_p(T, u)) < 4 * se


@pytest.mark.parametrize("p", [4, 5])
def test_exact_order_p_rtpm_recovers_planted_components(p):
    n, k = 8, 3
    A = synth.orthonormal_columns(n, k, 60 + p)
    lam = np.array([2.0, 1.5, 1.0])
    T = P.symmetric_rank1_sum(lam, A, p)
    res = P.rtpm_exact_p(T, synth.gaussian_inits(k, 6, n, 70 + p), 40)
    np.testing.assert_allclose(res["lam"], lam, rtol=1e-8)
    for r in range(k):
        assert min(np.linalg.norm(res["V"][r] - A[:, r]), np.linalg.norm(res["V"][r] + A[:, r])) < 1e-6


@pytest.mark.parametrize("p,n", [(4, 4), (5, 4)])
def test_sketched_order_p_rtpm_with_collision_free_hashes_is_the_plain_method(p, n):
    k = 2
    A = synth.orthonormal_columns(n, k, 80 + p)
    T = P.symmetric_rank1_sum(np.array([2.0, 1.0]), A, p) + 0.01 * random_symmetric_p(n, p, 81)
    h, g, b = collision_free(n, p, 82)
    S = P.sketch_sym_p(T, h, g, b, p)[None, :]
    U0 = synth.gaussian_inits(k, 3, n, 83)
    res = P.rtpm_sketched_p(S, h[None, :], g[None, :], b, p, U0, 8)
    ref = P.rtpm_exact_p(T, U0, 8)
    np.testing.assert_allclose(res["lam"], ref["lam"], rtol=1e-8)
    np.testing.assert_allclose(res["V"], ref["V"], atol=1e-8)


def test_order_p_hash_golden_fixture():
    """Frozen order-p hash values (tests/golden/hashes_order_p_seed3.txt, written by
    tests/golden/make_golden.py from the oracle alone): guards the degree-(2p-1) bucket
    polynomial and the mod-8 sign index against drift."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "hashes_order_p_seed3.txt")
    rows = [line.split() for line in open(path) if not line.startswith("#")]
    assert len(rows) == 2 * 2 * 6
    for p in (4, 6):
        h, g = P.cs_hashes_p(3, 2, 12, p, 6)
        for ps, ms, i_s, hv, gv in rows:
            if int(ps) == p:
                assert h[int(ms), int(i_s)] == int(hv) and g[int(ms), int(i_s)] == int(gv)
    assert all(0 <= int(r[4]) < 8 for r in rows)
