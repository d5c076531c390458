"""Pins for the FP64 oracle: facts fixed by the paper or by mathematics, not by the oracle itself.

Each test names the passage it pins.  A plausible mistake in the oracle (a dropped term, a
wrong coefficient, sign, conjugate or index, a transposed operand) fails at least one of them:
* collision-free hashes make every sketched estimate exact (proof of Lemma 1: with no
  collisions only matching multisets survive), which fixes all App. B coefficients;
* Prop. 1 and the convolution theorem tie the FFT engine to direct sums;
* Lemma 1's unbiasedness and variance bound and Thm. 1's 1/sqrt(b) error scaling;
* planted orthonormal components are recovered by the plain power method (Sec. 2).
"""
import numpy as np
import pytest

import oracle as O
import synth
from oracle import conv as C
from oracle import hashing as Hh


def injective_sym_hash(n):
    """h(i) = 4^i, b = 4^n: sums of three hashes encode the multiset in base 4 (no collisions)."""
    return np.array([4 ** i for i in range(n)], dtype=np.int64), 4 ** n


# ------------------------------------------------------------------ Prop. 1 / convolution theorem
@pytest.mark.parametrize("b", [16, 64, 1024, 4096])
def test_fft_engine_matches_direct_sums(b):
    r = synth.rng(b)
    x = r.standard_normal(b) + 1j * r.standard_normal(b)
    y = r.standard_normal(b) + 1j * r.standard_normal(b)
    y[r.random(b) < 0.7] = 0.0
    np.testing.assert_allclose(C.conv_fft(x, y), C.conv_direct(x, y), rtol=0, atol=1e-10 * b)
    np.testing.assert_allclose(C.corr_fft(x, y), C.corr_direct(x, y), rtol=0, atol=1e-10 * b)


def test_direct_convolution_small_closed_form():
    # (a*c)[t] = sum_{(i+j) mod b = t} a_i c_j, worked by hand for b = 3.
    a = np.array([1.0, 2.0, 3.0])
    c = np.array([4.0, 5.0, 6.0])
    # t=0: a0c0 + a1c2 + a2c1 = 4 + 12 + 15; t=1: a0c1 + a1c0 + a2c2 = 5 + 8 + 18; t=2: 6 + 10 + 12
    np.testing.assert_allclose(C.conv_direct(a, c).real, [31.0, 31.0, 28.0])
    # corr(x, y)[s] = sum_d x[(d+s) mod b] conj(y[d])
    np.testing.assert_allclose(C.corr_direct(a, c).real, [1 * 4 + 2 * 5 + 3 * 6,
                                                          2 * 4 + 3 * 5 + 1 * 6,
                                                          3 * 4 + 1 * 5 + 2 * 6])


def test_prop1_statement_asymmetric():
    """Prop. 1: <s_T, s_{1,e_i} * s_{2,u} * s_{3,u}> = <F^-1(F s_T o conj F s_2 o conj F s_3), s_{1,e_i}>."""
    b = 64
    n = 7
    h, g = O.cs_hashes(3, 1, 6, [n, n, n])
    h, g = h[0], g[0]
    r = synth.rng(5)
    S = r.standard_normal(b) + 1j * r.standard_normal(b)
    u = r.standard_normal(n)
    s2 = O.count_sketch_asym(u, h[1], g[1], b)
    s3 = O.count_sketch_asym(u, h[2], g[2], b)
    left_op = C.ifft(C.fft(S) * np.conj(C.fft(s2)) * np.conj(C.fft(s3)))
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        s1 = O.count_sketch_asym(e, h[0], g[0], b)
        lhs = C.inner(S, C.conv_direct(C.conv_direct(s1, s2), s3))
        rhs = C.inner(left_op, s1)
        assert abs(lhs - rhs) < 1e-12 * max(1.0, abs(lhs))


# ------------------------------------------------------------------ collision-free exactness
@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_collision_free_sym_contractions_are_exact(n):
    h, b = injective_sym_hash(n)
    T = synth.random_symmetric(n, 10 + n)
    for trial in range(3):
        g = synth.rng(100 * n + trial).integers(0, 4, size=n)
        u = synth.random_vector(n, 200 * n + trial)
        S = O.sketch_tensor_sym(T, h, g, b)
        want_iuu = O.exact_iuu(T, u)
        want_uuu = O.exact_uuu(T, u)
        for eng in ("direct", "fft"):
            np.testing.assert_allclose(O.contract_iuu(S, u, h, g, b, eng), want_iuu,
                                       rtol=1e-11, atol=1e-11)
            assert abs(O.contract_uuu(S, u, h, g, b, eng) - want_uuu) < 1e-10 * (1 + abs(want_uuu))
        np.testing.assert_allclose(O.contract_iuu_def(S, u, h, g, b), want_iuu, rtol=1e-11, atol=1e-11)
        assert abs(O.contract_uuu_def(S, u, h, g, b) - want_uuu) < 1e-10 * (1 + abs(want_uuu))


def test_printed_tiuu_coefficients_fail_the_collision_free_pin():
    """Eq. (14) as printed weights its four terms (1, 1/6, 1/6, 1); the collision-free pin
    rejects that and accepts the (1/3, 1/6, 1/6, 1/3) reading used by the oracle."""
    n = 4
    h, b = injective_sym_hash(n)
    T = synth.random_symmetric(n, 77)
    u = synth.random_vector(n, 78)
    g = np.array([0, 1, 2, 3])
    S = O.sketch_tensor_sym(T, h, g, b)
    su = O.count_sketch(u, h, g, b, 1)
    s2 = O.count_sketch(u, h, g, b, 2)
    csig = np.conj(O.sigma_of(g))
    t_g0 = C.corr_direct(S, su)[(2 * h) % b] * csig ** 2 * u
    t_g2 = C.corr_direct(S, C.conv_direct(su, su))[h] * csig
    t_g1 = C.corr_direct(S, s2)[h] * csig
    t_s3 = S[(3 * h) % b] * csig ** 3 * u * u
    printed = np.real(t_g0 + t_g2 / 6 + t_g1 / 6 + t_s3)
    assert np.max(np.abs(printed - O.exact_iuu(T, u))) > 1e-3
    np.testing.assert_allclose(O.contract_iuu(S, u, h, g, b), O.exact_iuu(T, u), rtol=1e-11, atol=1e-11)


def test_collision_free_asym_contraction_is_exact():
    n1, n2, n3 = 3, 4, 2
    nmax = 4
    b = 64  # h1(i) = i, h2(j) = 4 j, h3(k) = 16 k: injective on [4]^3 (b = 64)
    h = np.zeros((3, nmax), dtype=np.int64)
    h[0, :] = np.arange(nmax)
    h[1, :] = 4 * np.arange(nmax)
    h[2, :] = 16 * np.arange(nmax)
    g = synth.rng(9).integers(0, 4, size=(3, nmax))
    T = synth.rng(10).standard_normal((n1, n2, n3))
    v = synth.random_vector(n2, 11)
    w = synth.random_vector(n3, 12)
    S = O.sketch_tensor_asym(T, h, g, b)
    for eng in ("direct", "fft"):
        np.testing.assert_allclose(O.contract_ivw_asym(S, v, w, h, g, b, n1, eng),
                                   O.exact_ivw(T, v, w), rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------------ identities with collisions
def test_fast_forms_equal_definition_with_collisions():
    n, b = 6, 32
    h, g = O.cs_hashes(11, 4, 5, [n])
    T = synth.random_symmetric(n, 12)
    u = synth.random_vector(n, 13)
    for m in range(4):
        S = O.sketch_tensor_sym(T, h[m, 0], g[m, 0], b)
        d = O.contract_iuu_def(S, u, h[m, 0], g[m, 0], b)
        for eng in ("direct", "fft"):
            np.testing.assert_allclose(O.contract_iuu(S, u, h[m, 0], g[m, 0], b, eng), d,
                                       rtol=1e-11, atol=1e-11)
            assert abs(O.contract_uuu(S, u, h[m, 0], g[m, 0], b, eng)
                       - O.contract_uuu_def(S, u, h[m, 0], g[m, 0], b)) < 1e-10


def test_invariant_uuu_is_u_dot_iuu():
    """sum_i u_i T^(I,u,u)_i = T^(u,u,u) per sketch: sum_i u_i s~_{Z~_i} = 3 s~_{X~} (App. B)."""
    n, b = 9, 128
    h, g = O.cs_hashes(21, 3, 7, [n])
    T = synth.random_symmetric(n, 22)
    u = synth.random_vector(n, 23)
    for m in range(3):
        S = O.sketch_tensor_sym(T, h[m, 0], g[m, 0], b)
        lhs = float(np.dot(u, O.contract_iuu(S, u, h[m, 0], g[m, 0], b)))
        assert abs(lhs - O.contract_uuu(S, u, h[m, 0], g[m, 0], b)) < 1e-11 * (1 + abs(lhs))


def test_sorted_build_equals_full_build_for_symmetric_tensors():
    """Sec. 3.3: only i <= j <= k need to be read, each weighted by kappa in {1, 3, 6}."""
    n, b = 7, 64
    h, g = O.cs_hashes(31, 2, 6, [n])
    T = synth.random_symmetric(n, 32)
    for m in range(2):
        np.testing.assert_allclose(O.sketch_tensor_sym_sorted(T, h[m, 0], g[m, 0], b),
                                   O.sketch_tensor_sym(T, h[m, 0], g[m, 0], b), atol=1e-12)


def test_integer_sketch_is_exact_and_matches_float():
    n, b = 6, 32
    h, g = O.cs_hashes(41, 1, 5, [n])
    Ti = synth.random_symmetric_int(n, 42)
    si = O.sketch_tensor_sym(Ti, h[0, 0], g[0, 0], b)
    sf = O.sketch_tensor_sym(Ti.astype(np.float64), h[0, 0], g[0, 0], b)
    np.testing.assert_array_equal(si[0].astype(np.float64), sf.real)
    np.testing.assert_array_equal(si[1].astype(np.float64), sf.imag)


def test_rank1_sketch_equals_dense_sketch_and_linearity():
    """Eq. (4) with colliding hashes: s~_{u(x)3} = s~_u * s~_u * s~_u; the sketch is linear (Sec. 3.1)."""
    n, b = 8, 64
    h, g = O.cs_hashes(51, 1, 6, [n])
    h, g = h[0, 0], g[0, 0]
    u = synth.random_vector(n, 52)
    v = synth.random_vector(n, 53)
    U3 = np.einsum("i,j,k->ijk", u, u, u)
    V3 = np.einsum("i,j,k->ijk", v, v, v)
    np.testing.assert_allclose(O.sketch_rank1_sym(u, h, g, b), O.sketch_tensor_sym(U3, h, g, b), atol=1e-12)
    np.testing.assert_allclose(O.sketch_tensor_sym(2.5 * U3 - 0.75 * V3, h, g, b),
                               2.5 * O.sketch_tensor_sym(U3, h, g, b) - 0.75 * O.sketch_tensor_sym(V3, h, g, b),
                               atol=1e-12)
    # deflation of sketches == sketch of the deflated tensor
    T = synth.random_symmetric(n, 54)
    S = O.sketch_tensor_sym(T, h, g, b)[None, :]
    hB, gB = h[None, :], g[None, :]
    np.testing.assert_allclose(O.deflate_sketches(S, 1.7, u, hB, gB, b, "direct")[0],
                               O.sketch_tensor_sym(T - 1.7 * U3, h, g, b), atol=1e-11)
    np.testing.assert_allclose(O.deflate_sketches(S, 1.7, u, hB, gB, b, "fft")[0],
                               O.sketch_tensor_sym(T - 1.7 * U3, h, g, b), atol=1e-11)


def test_rank1_asym_sketch_equals_dense():
    n = 5
    b = 32
    h, g = O.cs_hashes(61, 1, 5, [n, n, n])
    h, g = h[0], g[0]
    u, v, w = (synth.random_vector(n, s) for s in (62, 63, 64))
    np.testing.assert_allclose(O.sketch_rank1_asym(u, v, w, h, g, b),
                               O.sketch_tensor_asym(np.einsum("i,j,k->ijk", u, v, w), h, g, b), atol=1e-12)


def test_entry_recovery_collision_free():
    n = 4
    h, b = injective_sym_hash(n)
    g = np.array([3, 1, 0, 2])
    T = synth.random_symmetric(n, 71)
    S = O.sketch_tensor_sym(T, h, g, b)
    for (i, j, k) in [(0, 0, 0), (0, 1, 1), (2, 0, 2), (3, 1, 2), (1, 2, 3)]:
        assert abs(O.recover_entry_sym(S, h, g, b, i, j, k) - T[i, j, k]) < 1e-12


# ------------------------------------------------------------------ Lemma 1 / Thm. 1 statistics
def test_lemma1_unbiased_and_variance_bound():
    """E <s~_A, s~_{B~}> = <A, B> and Var <= 4^p ||A||^2 ||B||^2 / b (Lemma 1, p = 3)."""
    n, log2b = 5, 4
    b = 1 << log2b
    Bn = 3000
    T = synth.random_symmetric(n, 81)
    u = synth.random_vector(n, 82)
    h, g = O.cs_hashes(83, Bn, log2b, [n])
    est_uuu = np.empty(Bn)
    est_iuu = np.empty((Bn, n))
    for m in range(Bn):
        S = O.sketch_tensor_sym(T, h[m, 0], g[m, 0], b)
        est_iuu[m] = O.contract_iuu(S, u, h[m, 0], g[m, 0], b)
        est_uuu[m] = float(np.dot(u, est_iuu[m]))
    exact = O.exact_uuu(T, u)
    se = est_uuu.std(ddof=1) / np.sqrt(Bn)
    assert abs(est_uuu.mean() - exact) < 4.5 * se
    normX2 = float(np.dot(u, u)) ** 3
    assert est_uuu.var(ddof=1) <= 4 ** 3 * float(np.sum(T * T)) * normX2 / b
    ex_i = O.exact_iuu(T, u)
    se_i = est_iuu.std(axis=0, ddof=1) / np.sqrt(Bn)
    assert np.all(np.abs(est_iuu.mean(axis=0) - ex_i) < 4.5 * se_i)


def test_thm1_error_decays_like_inverse_sqrt_b():
    n = 6
    T = synth.random_symmetric(n, 91)
    u = synth.random_vector(n, 92)
    u /= np.linalg.norm(u)
    exact = O.exact_uuu(T, u)
    rms = []
    for log2b in (6, 8, 10):
        b = 1 << log2b
        h, g = O.cs_hashes(93 + log2b, 400, log2b, [n])
        errs = [O.contract_uuu(O.sketch_tensor_sym(T, h[m, 0], g[m, 0], b), u, h[m, 0], g[m, 0], b) - exact
                for m in range(400)]
        rms.append(np.sqrt(np.mean(np.square(errs))))
    slope = np.polyfit([6, 8, 10], np.log2(rms), 1)[0]
    assert -0.75 < slope < -0.3, (rms, slope)


# ------------------------------------------------------------------ hashing (Sec. 3.3, Prop. 2)
def test_p61_arithmetic_and_prime():
    sympy = pytest.importorskip("sympy")
    assert sympy.isprime(Hh.P61)


def test_hash_polynomial_horner_equals_power_sum():
    coefs = Hh.coefficients(1234, 2, 0, 1, 0, 6)
    for x in (0, 1, 2, 17, 999, 123456):
        direct = sum(c * pow(x, e, Hh.P61) for e, c in enumerate(coefs)) % Hh.P61
        assert Hh.poly_mod_p(coefs, x) == direct


def test_splitmix64_stream_is_the_sequential_generator():
    """Counter form equals stepping the state by the golden gamma and mixing (Steele et al. 2014)."""
    seed = 0x0123456789ABCDEF
    state = seed
    for c in range(8):
        state = (state + Hh.GOLDEN_GAMMA) & Hh.MASK64
        assert Hh.splitmix64_output(seed, c) == Hh.mix64(state)
    assert Hh.mix64(0) == 0


def test_splitmix64_matches_the_published_reference_stream():
    """The first outputs of the reference SplitMix64 generator (Vigna's splitmix64.c, the
    generator of Steele, Lea and Flood, OOPSLA 2014) started from state 0 are the published
    test values 0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4, 0x06c45d188009454f; the hash
    coefficients are this stream's outputs, so a wrong constant or shift fails here."""
    assert [Hh.splitmix64_output(0, c) for c in range(3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_hash_ranges_uniformity_and_sign_moments():
    n, log2b, Bn = 4096, 6, 4
    b = 1 << log2b
    h, g = O.cs_hashes(2024, Bn, log2b, [n])
    assert h.min() >= 0 and h.max() < b and g.min() >= 0 and g.max() <= 3
    for m in range(Bn):
        counts = np.bincount(h[m, 0], minlength=b)
        chi2 = float(np.sum((counts - n / b) ** 2 / (n / b)))
        assert chi2 < b + 6 * np.sqrt(2 * b)          # dof = b - 1
        sig = O.sigma_of(g[m, 0])
        for d in (1, 2, 3):
            assert abs(np.mean(sig ** d)) < 5 / np.sqrt(n)
    # different sketches are independent draws
    assert np.mean(h[0, 0] == h[1, 0]) < 3.0 / b


def test_hash_golden_fixture():
    """Frozen hash values (tests/golden/hashes_seed1.txt, written by tests/golden/make_golden.py
    from the oracle) pin the convention the CUDA path must reproduce bit for bit."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "hashes_seed1.txt")
    rows = [line.split() for line in open(path) if line.strip() and not line.startswith("#")]
    h, g = O.cs_hashes(1, 2, 10, [3, 5, 4])
    for m_s, j_s, i_s, hv, gv in rows:
        m, j, i = int(m_s), int(j_s), int(i_s)
        assert h[m, j, i] == int(hv) and g[m, j, i] == int(gv)


# ------------------------------------------------------------------ median and power method
def test_median_rule():
    assert O.median([3.0, 1.0, 2.0]) == 2.0
    assert O.median([4.0, 1.0, 3.0, 2.0]) == 2.5
    r = synth.rng(5)
    for B in (1, 2, 5, 8, 10, 20):
        x = r.standard_normal(B)
        assert O.median(x) == pytest.approx(float(np.median(x)), abs=0)


def test_exact_rtpm_recovers_planted_components():
    """Sec. 2 / Thm. 2 setting: noise-free orthogonal rank-k tensor is decomposed exactly."""
    n, k = 10, 3
    T, lam, A = synth.planted_symmetric(n, k, 0.0, 101)
    U0 = synth.gaussian_inits(k, 6, n, 102)
    res = O.rtpm_exact(T, U0, 40)
    order = np.argsort(-lam)
    np.testing.assert_allclose(res["lam"], lam[order], rtol=1e-9)
    for r in range(k):
        a = A[:, order[r]]
        assert min(np.linalg.norm(res["V"][r] - a), np.linalg.norm(res["V"][r] + a)) < 1e-8


def test_sketched_rtpm_collision_free_equals_exact():
    """With an injective colliding hash every sketched contraction is exact, so Alg. 1 reduces
    to the plain method step for step (same U0)."""
    n, k = 4, 2
    h1, b = injective_sym_hash(n)
    g1 = np.array([1, 3, 0, 2])
    T, lam, A = synth.planted_symmetric(n, k, 0.05, 111)
    Bn = 3
    h = np.stack([h1] * Bn)
    g = np.stack([(g1 + m) % 4 for m in range(Bn)])
    S = np.stack([O.sketch_tensor_sym(T, h[m], g[m], b) for m in range(Bn)])
    U0 = synth.gaussian_inits(k, 4, n, 112)
    sk = O.rtpm_sketched(S, h, g, b, U0, 15, engine="fft")
    ex = O.rtpm_exact(T, U0, 15)
    # several inits converge to the same component, so tau* is only unique up to such ties
    for r in range(k):
        assert sk["lam_all"][r, sk["tau"][r]] >= sk["lam_all"][r].max() - 1e-12
    np.testing.assert_allclose(sk["lam"], ex["lam"], rtol=1e-9)
    np.testing.assert_allclose(sk["V"], ex["V"], atol=1e-9)


def test_asymmetric_rtpm_with_injective_hashes_is_the_plain_method():
    """Alg. 1 as printed (three hashes, Eq. 1 sketches): with h1(i) = i, h2(j) = n j,
    h3(k) = n^2 k every (i, j, k) has its own bucket, so each T(I,u,u) read-off and each
    deflation is exact and the method reduces to the plain one step for step."""
    n, k = 4, 2
    hrow = np.stack([np.arange(n), n * np.arange(n), n * n * np.arange(n)])
    b = n ** 3
    T, lam, A = synth.planted_symmetric(n, k, 0.05, 211)
    Bn = 3
    h = np.stack([hrow] * Bn)
    g = np.stack([synth.rng(212 + m).integers(0, 4, size=(3, n)) for m in range(Bn)])
    S = np.stack([np.real(O.sketch_tensor_asym(T, h[m], g[m], b)) for m in range(Bn)])
    U0 = synth.gaussian_inits(k, 4, n, 213)
    sk = O.rtpm_sketched_asym(S, h, g, b, U0, 15, engine="fft")
    ex = O.rtpm_exact(T, U0, 15)
    for r in range(k):
        assert sk["lam_all"][r, sk["tau"][r]] >= sk["lam_all"][r].max() - 1e-12
    np.testing.assert_allclose(sk["lam"], ex["lam"], rtol=1e-9)
    np.testing.assert_allclose(sk["V"], ex["V"], atol=1e-9)


# ------------------------------------------------------------------ sketched CP loss, ALS (Alg. 2)
def _injective_asym(n1, n2, n3):
    """h1(i) = i, h2(j) = n1 j, h3(k) = n1 n2 k: H is injective on [n1] x [n2] x [n3]."""
    nmax = max(n1, n2, n3)
    h = np.zeros((3, nmax), dtype=np.int64)
    h[0, :n1] = np.arange(n1)
    h[1, :n2] = n1 * np.arange(n2)
    h[2, :n3] = n1 * n2 * np.arange(n3)
    b = 1 << int(np.ceil(np.log2(n1 * n2 * n3)))
    return h, b


def _cp_problem(seed, dims, R):
    r = synth.rng(seed)
    T = r.standard_normal(dims)
    lam = r.uniform(0.5, 2.0, R)
    A, Bf, C = (r.standard_normal((R, d)) for d in dims)
    return T, lam, A, Bf, C


def test_cp_sketched_loss_is_exact_without_collisions():
    dims = (4, 3, 5)
    h1, b = _injective_asym(*dims)
    T, lam, A, Bf, C = _cp_problem(1, dims, 3)
    g = synth.rng(2).integers(0, 4, size=(2, 3, h1.shape[1]))
    h = np.stack([h1, h1])
    S = np.stack([O.sketch_tensor_asym(T, h[m], g[m], b) for m in range(2)])
    assert abs(O.cp_sketch_loss(S, h, g, b, lam, A, Bf, C) - O.cp_exact_loss(T, lam, A, Bf, C)) < 1e-9


@pytest.mark.parametrize("step", [1e-3, 1e-5])
def test_cp_gradient_matches_central_differences(step):
    dims = (5, 4, 3)
    b = 32
    h, g = O.cs_hashes(3, 2, 5, list(dims))
    T, lam, A, Bf, C = _cp_problem(4, dims, 2)
    S = np.stack([O.sketch_tensor_asym(T, h[m], g[m], b) for m in range(2)])
    grads = O.cp_sketch_grad(S, h, g, b, lam, A, Bf, C)
    params = [lam, A, Bf, C]

    def loss(ps):
        return O.cp_sketch_loss(S, h, g, b, *ps)
    for which in range(4):
        fd = np.zeros_like(params[which])
        for idx in np.ndindex(params[which].shape):
            up = [p.copy() for p in params]
            dn = [p.copy() for p in params]
            up[which][idx] += step
            dn[which][idx] -= step
            fd[idx] = (loss(up) - loss(dn)) / (2 * step)
        np.testing.assert_allclose(fd, grads[which], rtol=1e-4, atol=1e-4 * np.max(np.abs(grads[which])))


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_asymmetric_ivw_is_exact_without_collisions(mode):
    dims = (4, 3, 5)
    h, b = _injective_asym(*dims)
    g = synth.rng(5).integers(0, 4, size=(3, h.shape[1]))
    T = synth.rng(6).standard_normal(dims)
    others = [j for j in range(3) if j != mode]
    V = synth.random_vector(dims[others[0]], 7)
    W = synth.random_vector(dims[others[1]], 8)
    S = O.sketch_tensor_asym(T, h, g, b)
    want = np.einsum("ijk->" + "ijk"[mode] + "".join("ijk"[o] for o in others), T)
    want = np.einsum("xab,a,b->x", want, V, W)
    np.testing.assert_allclose(O.contract_ivw_mode(S, h, g, b, mode, V, W, dims[mode]), want,
                               rtol=1e-12, atol=1e-12)


def test_sketched_als_update_equals_exact_update_without_collisions():
    """With exact T(I, b_r, c_r) columns, Alg. 2 with Eq. 15 is the plain ALS step."""
    dims = (4, 3, 5)
    h1, b = _injective_asym(*dims)
    T, lam, A, Bf, C = _cp_problem(9, dims, 2)
    h = np.stack([h1] * 3)
    g = synth.rng(10).integers(0, 4, size=(3, 3, h1.shape[1]))
    S = np.stack([O.sketch_tensor_asym(T, h[m], g[m], b) for m in range(3)])
    M = O.als_sketched_columns(S, h, g, b, 0, (A, Bf, C))
    T1 = T.reshape(dims[0], -1)                                    # mode-1 unfolding, j-major
    KR = np.stack([np.kron(Bf[r], C[r]) for r in range(2)], axis=1)  # columns b_r (x) c_r
    np.testing.assert_allclose(M.T, T1 @ KR, rtol=1e-10, atol=1e-10)
    out, lam_new = O.als_solve(M, Bf, C)
    ref = (T1 @ KR) @ np.linalg.pinv((Bf @ Bf.T) * (C @ C.T))      # Eq. 15
    np.testing.assert_allclose(out.T * lam_new, ref, rtol=1e-9, atol=1e-9)
