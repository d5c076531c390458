"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on identical seeded inputs.

Tolerances: integer work (hash tables, int64 sketches) bit-exact; FP32 sketches, DFTs and
contraction vectors within 1e-5 relative in the 2-norm per (vector, sketch); recovered
eigenvalues and components within 1e-4.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu

tsk = pytest.importorskip("paper_1506_04448_gb300")


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def t32(x, dev):
    return torch.tensor(np.asarray(x), dtype=torch.float32, device=dev)


# ------------------------------------------------------------------ hashing
@pytest.mark.parametrize("seed,B,log2b,dims", [
    (1, 2, 10, [3, 5, 4]), (7, 5, 10, [50]), (2**63 + 5, 3, 14, [400]), (0, 1, 8, [1]),
    (123, 4, 15, [500, 400, 300]), (99, 64, 12, [33])])
def test_hashes_bit_exact(dev, seed, B, log2b, dims):
    h, g = tsk.cs_hashes(seed, B, log2b, dims, dev)
    ho, go = O.cs_hashes(seed, B, log2b, dims)
    np.testing.assert_array_equal(h.cpu().numpy(), ho)
    np.testing.assert_array_equal(g.cpu().numpy(), go)


# ------------------------------------------------------------------ sketch construction
@pytest.mark.parametrize("n,log2b,B", [(1, 8, 1), (9, 8, 3), (30, 10, 2), (65, 12, 4),
                                       (30, 15, 2), (21, 16, 2)])   # bucket ranges split over blocks
def test_symmetric_int_sketch_bit_exact(dev, n, log2b, B):
    b = 1 << log2b
    Ti = synth.random_symmetric_int(n, 100 + n)
    h, g = tsk.cs_hashes(11 + n, B, log2b, [n], dev)
    S = tsk.sketch_tensor(torch.tensor(Ti, device=dev), h, g, log2b, acc="ci64").cpu().numpy()
    ho, go = O.cs_hashes(11 + n, B, log2b, [n])
    for m in range(B):
        ref = O.sketch_tensor_sym(Ti, ho[m, 0], go[m, 0], b)
        np.testing.assert_array_equal(S[m, :, 0], ref[0])
        np.testing.assert_array_equal(S[m, :, 1], ref[1])


@pytest.mark.parametrize("n,log2b,B", [(5, 8, 2), (37, 10, 3), (100, 14, 2), (40, 15, 2),
                                       (40, 16, 3),
                                       # tile shift (-n) mod 32 of 0, 31 and 15
                                       (32, 10, 2), (33, 11, 2), (97, 12, 3)])
def test_symmetric_float_sketch(dev, n, log2b, B):
    b = 1 << log2b
    T = synth.random_symmetric(n, 200 + n)
    h, g = tsk.cs_hashes(3 + n, B, log2b, [n], dev)
    ho, go = O.cs_hashes(3 + n, B, log2b, [n])
    S32 = tsk.sketch_tensor(t32(T, dev), h, g, log2b).cpu().numpy()
    S64 = tsk.sketch_tensor(torch.tensor(T, device=dev), h, g, log2b, acc="c128").cpu().numpy()
    T32 = T.astype(np.float32).astype(np.float64)
    for m in range(B):
        assert rel(S32[m], O.sketch_tensor_sym(T32, ho[m, 0], go[m, 0], b)) < 1e-5
        assert rel(S64[m], O.sketch_tensor_sym(T, ho[m, 0], go[m, 0], b)) < 1e-12


def test_sketch_accumulate_is_linear(dev):
    n, log2b, B = 20, 10, 2
    A = synth.random_symmetric(n, 1)
    C = synth.random_symmetric(n, 2)
    h, g = tsk.cs_hashes(5, B, log2b, [n], dev)
    S = tsk.sketch_tensor(t32(A, dev), h, g, log2b)
    S = tsk.sketch_tensor(t32(C, dev), h, g, log2b, S=S, accumulate=True)
    R = tsk.sketch_tensor(t32(A + C, dev), h, g, log2b)
    assert rel(S.cpu().numpy(), R.cpu().numpy()) < 1e-5


@pytest.mark.parametrize("n,log2b,B", [(64, 8, 2), (48, 9, 4), (40, 15, 2)])
def test_symmetric_sketch_exact_through_int32_wraps(dev, n, log2b, B):
    """The all-ones tensor quantises every wedge entry to 2^26, so most buckets' int32 sums wrap
    past 2^31 many times: the result is right only if every carry is counted.  Its sketch has
    integer entries below 2^24 (sums of kappa-weighted sigma products), exact in float."""
    b = 1 << log2b
    T = np.ones((n, n, n))
    h, g = tsk.cs_hashes(7 + n, B, log2b, [n], dev)
    ho, go = O.cs_hashes(7 + n, B, log2b, [n])
    S = tsk.sketch_tensor(t32(T, dev), h, g, log2b).cpu().numpy()
    for m in range(B):
        np.testing.assert_array_equal(S[m], O.sketch_tensor_sym(T, ho[m, 0], go[m, 0], b))


def _plant(T, idx, value):
    i, j, k = idx
    for a, b_, c in {(i, j, k), (i, k, j), (j, i, k), (j, k, i), (k, i, j), (k, j, i)}:
        T[a, b_, c] = value


@pytest.mark.parametrize("dtype", ["float32", "float64", "int32"])
def test_symmetric_sketch_max_anywhere_in_a_row(dev, dtype):
    """The fixed-point scale comes from the prepass's max|T| over the wedge rows T[i][j][j..n-1],
    read with 16-byte loads between a scalar head and tail.  One entry 1000 times larger than the
    rest, planted at the start, end or middle of a row (n = 37, so rows start at every offset
    mod 16 bytes), must set the scale: a missed maximum would overflow its quantised value.
    Also over a plane range (the prepass reads only the range's planes)."""
    n, log2b, B = 37, 10, 2
    b = 1 << log2b
    h, g = tsk.cs_hashes(71, B, log2b, [n], dev)
    ho, go = O.cs_hashes(71, B, log2b, [n])
    for t, idx in enumerate([(0, 0, 0), (0, 0, 36), (0, 1, 2), (5, 9, 9), (5, 9, 36), (12, 20, 29),
                             (35, 35, 36), (36, 36, 36)]):
        if dtype == "int32":
            T = synth.random_symmetric_int(n, 500 + t).astype(np.int64)
            big = 1000 * int(np.abs(T).max() + 1)
        else:
            T = synth.random_symmetric(n, 500 + t)
            big = 1000.0
        _plant(T, idx, -big if t % 2 else big)
        Td = torch.tensor(T, device=dev, dtype=getattr(torch, dtype))
        Tref = Td.cpu().numpy().astype(np.float64)
        S = tsk.sketch_tensor(Td, h, g, log2b).cpu().numpy()
        for m in range(B):
            assert rel(S[m], O.sketch_tensor_sym(Tref, ho[m, 0], go[m, 0], b)) < 1e-5, (idx, m)
        p0, p1 = idx[0], min(n, idx[0] + 3)
        Sp = tsk.sketch_tensor_planes(Td[p0:p1].contiguous(), h, g, log2b, p0).cpu().numpy()
        mask = np.minimum(np.minimum(np.arange(n)[:, None, None], np.arange(n)[None, :, None]),
                          np.arange(n)[None, None, :])
        Tm = np.where((mask >= p0) & (mask < p1), Tref, 0.0)
        for m in range(B):
            assert rel(Sp[m], O.sketch_tensor_sym(Tm, ho[m, 0], go[m, 0], b)) < 1e-5, (idx, m)


@pytest.mark.parametrize("scale", [1e-30, 1e-3, 1e6, 1e30])
def test_symmetric_sketch_any_magnitude(dev, scale):
    """The fixed-point step follows max|T| (a power of two), so tiny and huge tensors keep the
    same relative accuracy; two builds of the same tensor are bit-identical."""
    n, log2b, B = 23, 10, 4
    b = 1 << log2b
    T = synth.random_symmetric(n, 31) * scale
    T[3, 5, 7] = T[3, 7, 5] = T[5, 3, 7] = T[5, 7, 3] = T[7, 3, 5] = T[7, 5, 3] = 40 * scale
    h, g = tsk.cs_hashes(9, B, log2b, [n], dev)
    ho, go = O.cs_hashes(9, B, log2b, [n])
    Td = t32(T, dev)
    S = tsk.sketch_tensor(Td, h, g, log2b).cpu().numpy()
    S2 = tsk.sketch_tensor(Td, h, g, log2b).cpu().numpy()
    np.testing.assert_array_equal(S, S2)
    T32 = T.astype(np.float32).astype(np.float64)
    for m in range(B):
        assert rel(S[m], O.sketch_tensor_sym(T32, ho[m, 0], go[m, 0], b)) < 1e-5


def test_symmetric_sketch_into_unaligned_output(dev):
    """S only 8-byte aligned (a complex-float array starting at an odd element): the reduce's
    16-byte stores fall back to scalar stores; write and accumulate both match the aligned
    result bit for bit."""
    n, log2b, B = 40, 10, 3
    b = 1 << log2b
    T = t32(synth.random_symmetric(n, 12), dev)
    h, g = tsk.cs_hashes(21, B, log2b, [n], dev)
    ref = tsk.sketch_tensor(T, h, g, log2b)
    buf = torch.zeros(B * b + 1, dtype=torch.complex64, device=dev)
    S = buf[1:].view(B, b)
    assert S.data_ptr() % 16 == 8
    tsk.sketch_tensor(T, h, g, log2b, S=S)
    assert torch.equal(S, ref)
    tsk.sketch_tensor(T, h, g, log2b, S=S, accumulate=True)
    assert torch.equal(S, ref + ref)


def test_symmetric_sketch_of_zero_and_nonfinite_tensors(dev):
    n, log2b, B = 9, 8, 2
    h, g = tsk.cs_hashes(4, B, log2b, [n], dev)
    Z = torch.zeros((n, n, n), dtype=torch.float32, device=dev)
    assert not tsk.sketch_tensor(Z, h, g, log2b).cpu().numpy().any()
    tsk.check_status(dev)
    Z[1, 2, 3] = float("nan")
    S = tsk.sketch_tensor(Z, h, g, log2b).cpu().numpy()
    assert np.isnan(S.real).all()
    assert tsk.ctx_status(dev) == -5     # TSK_ENONFINITE
    tsk.check_status(dev)


@pytest.mark.parametrize("n,log2b,B", [(50, 12, 4), (33, 13, 6), (61, 12, 8)])
def test_symmetric_float_sketch_several_per_block(dev, n, log2b, B):
    """b <= 2^13 with B divisible by 2 or 4: one block builds two or four sketches from one read
    of its share of the wedge tiles; float and double input."""
    b = 1 << log2b
    T = synth.random_symmetric(n, 300 + n)
    h, g = tsk.cs_hashes(40 + n, B, log2b, [n], dev)
    ho, go = O.cs_hashes(40 + n, B, log2b, [n])
    S32 = tsk.sketch_tensor(t32(T, dev), h, g, log2b).cpu().numpy()
    S64in = tsk.sketch_tensor(torch.tensor(T, device=dev), h, g, log2b).cpu().numpy()
    T32 = T.astype(np.float32).astype(np.float64)
    for m in range(B):
        assert rel(S32[m], O.sketch_tensor_sym(T32, ho[m, 0], go[m, 0], b)) < 1e-5
        assert rel(S64in[m], O.sketch_tensor_sym(T, ho[m, 0], go[m, 0], b)) < 1e-5


@pytest.mark.parametrize("dims,log2b", [((7, 5, 3), 8), ((40, 33, 29), 12), ((50, 40, 30), 15)])
def test_asymmetric_sketch(dev, dims, log2b):
    b = 1 << log2b
    r = synth.rng(sum(dims))
    T = r.standard_normal(dims)
    Ti = r.integers(-500, 500, size=dims).astype(np.int32)
    h, g = tsk.cs_hashes(17, 2, log2b, list(dims), dev)
    ho, go = O.cs_hashes(17, 2, log2b, list(dims))
    S = tsk.sketch_tensor(t32(T, dev), h, g, log2b).cpu().numpy()
    T32 = T.astype(np.float32).astype(np.float64)
    for m in range(2):
        assert rel(S[m], O.sketch_tensor_asym(T32, ho[m], go[m], b)) < 1e-5
    if log2b <= 14:
        Si = tsk.sketch_tensor(torch.tensor(Ti, device=dev), h, g, log2b, acc="ci64").cpu().numpy()
        for m in range(2):
            np.testing.assert_array_equal(Si[m, :, 0], O.sketch_tensor_asym(Ti, ho[m], go[m], b))
            assert not Si[m, :, 1].any()


@pytest.mark.parametrize("scale", [1e-30, 1.0, 1e30])
def test_asymmetric_float_sketch_exact_integer_build(dev, scale):
    """Complex-float asymmetric sketches are summed in exact integers on the grid set by max|T|:
    two builds are bit-identical, tiny and huge tensors keep the relative accuracy, accumulate
    adds the real parts and keeps the imaginary parts, and FP64 and int32 inputs take the same
    path."""
    dims, log2b, B = (31, 26, 45), 11, 3
    b = 1 << log2b
    r = synth.rng(77)
    T = r.standard_normal(dims) * scale
    h, g = tsk.cs_hashes(5, B, log2b, list(dims), dev)
    ho, go = O.cs_hashes(5, B, log2b, list(dims))
    Td = t32(T, dev)
    S = tsk.sketch_tensor(Td, h, g, log2b)
    S2 = tsk.sketch_tensor(Td, h, g, log2b)
    assert torch.equal(S, S2)
    Sn = S.cpu().numpy()
    assert not Sn.imag.any()
    T32 = T.astype(np.float32).astype(np.float64)
    for m in range(B):
        assert rel(Sn[m], O.sketch_tensor_asym(T32, ho[m], go[m], b)) < 1e-5
    acc = torch.full_like(S, complex(1.0, 2.0))
    tsk.sketch_tensor(Td, h, g, log2b, S=acc, accumulate=True)
    an = acc.cpu().numpy()
    np.testing.assert_array_equal(an.imag, 2.0)
    np.testing.assert_allclose(an.real, Sn.real + 1.0, rtol=0, atol=1e-6 * (1 + np.abs(Sn.real).max()))
    S64 = tsk.sketch_tensor(torch.tensor(T, device=dev), h, g, log2b).cpu().numpy()
    for m in range(B):
        assert rel(S64[m], O.sketch_tensor_asym(T, ho[m], go[m], b)) < 1e-5
    if scale == 1.0:
        Ti = r.integers(-1000, 1000, size=dims).astype(np.int32)
        Si = tsk.sketch_tensor(torch.tensor(Ti, device=dev), h, g, log2b).cpu().numpy()
        for m in range(B):
            assert rel(Si[m], O.sketch_tensor_asym(Ti.astype(np.float64), ho[m], go[m], b)) < 1e-6


def test_asymmetric_sketch_with_carries_and_nonfinite(dev):
    """Entries of near-maximal magnitude whose signs cancel sketch 0's signs xi1 xi2 xi3, into
    few buckets (b = 2^6): every add to a bucket of sketch 0 has the same sign, the int32 bucket
    sums pass 2^31 many times, and the exact carries keep the result; then a NaN entry makes the
    sketch NaN and is reported as TSK_ENONFINITE."""
    dims, log2b, B = (64, 64, 64), 6, 2
    b = 1 << log2b
    h, g = tsk.cs_hashes(3, B, log2b, list(dims), dev)
    ho, go = O.cs_hashes(3, B, log2b, list(dims))
    xi = [1.0 - 2.0 * (go[0, j, :dims[j]] & 1) for j in range(3)]
    T = 0.999 * np.einsum("i,j,k->ijk", xi[0], xi[1], xi[2])
    Td = t32(T, dev)
    S = tsk.sketch_tensor(Td, h, g, log2b).cpu().numpy()
    T32 = T.astype(np.float32).astype(np.float64)
    for m in range(B):
        assert rel(S[m], O.sketch_tensor_asym(T32, ho[m], go[m], b)) < 1e-6
    tsk.check_status(dev)
    Td[1, 2, 3] = float("nan")
    S = tsk.sketch_tensor(Td, h, g, log2b).cpu().numpy()
    assert np.isnan(S.real).all()
    assert tsk.ctx_status(dev) == -5     # TSK_ENONFINITE
    tsk.check_status(dev)


# ------------------------------------------------------------------ DFT
@pytest.mark.parametrize("log2b", [8, 9, 10, 11, 12, 13, 14])
def test_sketch_fft(dev, log2b):
    b = 1 << log2b
    r = synth.rng(log2b)
    X = r.standard_normal((3, b)) + 1j * r.standard_normal((3, b))
    Xd = torch.tensor(X, dtype=torch.complex64, device=dev)
    F = tsk.sketch_fft(Xd).cpu().numpy()
    Xi = tsk.sketch_fft(Xd, inverse=True).cpu().numpy()
    X32 = Xd.cpu().numpy().astype(np.complex128)
    for m in range(3):
        assert rel(F[m], O.conv.fft(X32[m])) < 2e-6
        assert rel(Xi[m], O.conv.ifft(X32[m])) < 2e-6


# ------------------------------------------------------------------ rank-1 sketches
@pytest.mark.parametrize("domain", ["time", "freq"])
def test_sketch_rank1_symmetric(dev, domain):
    n, log2b, B, cnt = 30, 10, 3, 4
    b = 1 << log2b
    U = synth.rng(3).standard_normal((cnt, n))
    w = np.array([1.0, -0.5, 2.0, 0.25])
    h, g = tsk.cs_hashes(21, B, log2b, [n], dev)
    ho, go = O.cs_hashes(21, B, log2b, [n])
    S = tsk.sketch_rank1(t32(w, dev), t32(U, dev), h, g, log2b, domain=domain).cpu().numpy()
    U32 = U.astype(np.float32).astype(np.float64)
    for m in range(B):
        ref = sum(w[c] * O.sketch_rank1_sym(U32[c], ho[m, 0], go[m, 0], b) for c in range(cnt))
        if domain == "freq":
            ref = O.conv.fft(ref)
        assert rel(S[m], ref) < 1e-5


def test_sketch_rank1_asymmetric_and_accumulate(dev):
    dims, log2b, B = (9, 7, 5), 9, 2
    b = 1 << log2b
    r = synth.rng(4)
    U, V, W = (r.standard_normal((2, d)) for d in dims)
    w = np.array([0.7, -1.3])
    h, g = tsk.cs_hashes(23, B, log2b, list(dims), dev)
    ho, go = O.cs_hashes(23, B, log2b, list(dims))
    S0 = torch.zeros((B, b), dtype=torch.complex64, device=dev)
    S0[:, 3] = 1.0
    S = tsk.sketch_rank1(t32(w, dev), t32(U, dev), h, g, log2b, V=t32(V, dev), W=t32(W, dev),
                         S=S0, accumulate=True).cpu().numpy()
    f = lambda x: x.astype(np.float32).astype(np.float64)  # noqa: E731
    for m in range(B):
        ref = sum(w[c] * O.sketch_rank1_asym(f(U[c]), f(V[c]), f(W[c]), ho[m], go[m], b) for c in range(2))
        ref[3] += 1.0
        assert rel(S[m], ref) < 1e-5


# ------------------------------------------------------------------ contractions
def _sketches(dev, n, log2b, B, seed, noise=0.1, k=3):
    T, _, _ = synth.planted_symmetric(n, k, noise, seed)
    h, g = tsk.cs_hashes(seed, B, log2b, [n], dev)
    S = tsk.sketch_tensor(t32(T, dev), h, g, log2b)
    FS = tsk.sketch_fft(S)
    ho, go = O.cs_hashes(seed, B, log2b, [n])
    return T, h, g, S, FS, ho, go


@pytest.mark.parametrize("n,log2b,B,L", [(5, 8, 1, 1), (37, 10, 2, 3), (64, 12, 5, 2),
                                         (33, 13, 4, 2), (400, 14, 10, 3),
                                         (20, 9, 40, 2), (12, 8, 64, 2)])   # medians of 40, 64
def test_contract_iuu_and_uuu(dev, n, log2b, B, L):
    b = 1 << log2b
    _, h, g, S, FS, ho, go = _sketches(dev, n, log2b, B, 31 + n)
    U = synth.rng(n).standard_normal((L, n))
    U /= np.linalg.norm(U, axis=1, keepdims=True)
    Ud = t32(U, dev)
    Vmed, Vall = tsk.contract_iuu(FS, S, h, g, Ud, return_all=True)
    lam, lam_all = tsk.contract_uuu(FS, S, h, g, Ud, return_all=True)
    # without per-sketch outputs the call may split each sketch's frequencies over blocks
    Vmed_s = tsk.contract_iuu(FS, S, h, g, Ud).cpu().numpy()
    lam_s = tsk.contract_uuu(FS, S, h, g, Ud).cpu().numpy()
    Sg = S.cpu().numpy().astype(np.complex128)
    Ug = Ud.cpu().numpy().astype(np.float64)
    Vall = Vall.cpu().numpy()
    lam_all = lam_all.cpu().numpy()
    for tau in range(L):
        refs = np.stack([O.contract_iuu(Sg[m], Ug[tau], ho[m, 0], go[m, 0], b, "fft") for m in range(B)])
        lrefs = np.array([O.contract_uuu(Sg[m], Ug[tau], ho[m, 0], go[m, 0], b, "fft") for m in range(B)])
        for m in range(B):
            assert rel(Vall[tau, m], refs[m]) < 1e-5, (tau, m)
            # per entry as well: a single misplaced hashed read would show here at large n
            # (the bound is the 2-norm one shrunk by up to 8 / sqrt(n))
            err = np.max(np.abs(Vall[tau, m] - refs[m]))
            assert err < 1e-5 * min(1.0, 8.0 / np.sqrt(n)) * np.linalg.norm(refs[m]), (tau, m, err)
        assert rel(Vmed[tau].cpu().numpy(), O.median_rows(refs)) < 1e-5
        assert rel(Vmed_s[tau], O.median_rows(refs)) < 1e-5
        scale = np.linalg.norm(refs) / np.sqrt(B)
        assert abs(lam_s[tau] - O.median(lrefs)) < 1e-5 * max(scale, 1e-30)
        assert np.max(np.abs(lam_all[tau] - lrefs)) < 1e-5 * max(scale, 1e-30)
        assert abs(lam[tau].item() - O.median(lrefs)) < 1e-5 * max(scale, 1e-30)
        # per-sketch invariant T^(u,u,u) = <u, T^(I,u,u)> (App. B)
        assert np.max(np.abs(Vall[tau] @ Ug[tau] - lam_all[tau])) < 1e-5 * max(scale, 1e-30)


def test_contract_collision_free_is_exact(dev):
    n = 4
    b = 256
    T = synth.random_symmetric(n, 5)
    hv = np.array([4 ** i for i in range(n)], dtype=np.int32)
    h = torch.tensor(np.stack([hv, hv]), dtype=torch.int32, device=dev)
    gv = np.array([[0, 1, 2, 3], [3, 1, 0, 2]])
    g = torch.tensor(gv, dtype=torch.uint8, device=dev)
    S = tsk.sketch_tensor(t32(T, dev), h, g, 8)
    FS = tsk.sketch_fft(S)
    U = synth.rng(6).standard_normal((2, n))
    Ud = t32(U, dev)
    V = tsk.contract_iuu(FS, S, h, g, Ud).cpu().numpy()
    lam = tsk.contract_uuu(FS, S, h, g, Ud).cpu().numpy()
    T32 = T.astype(np.float32).astype(np.float64)
    Ug = Ud.cpu().numpy().astype(np.float64)
    for tau in range(2):
        assert rel(V[tau], O.exact_iuu(T32, Ug[tau])) < 1e-5
        assert abs(lam[tau] - O.exact_uuu(T32, Ug[tau])) < 1e-5 * np.linalg.norm(T32.ravel())


# ------------------------------------------------------------------ Alg. 1
def _run_rtpm(dev, n, k, L, T_it, B, log2b, seed, noise):
    T, lam_true, A = synth.planted_symmetric(n, k, noise, seed)
    U0 = synth.gaussian_inits(k, L, n, seed + 1)
    h, g = tsk.cs_hashes(seed, B, log2b, [n], dev)
    S = tsk.sketch_tensor(t32(T, dev), h, g, log2b)
    res = tsk.robust_power_method(S, h, g, t32(U0, dev), T_it, return_deflated=True,
                                  return_trace=True)
    tsk.check_status(dev)
    ho, go = O.cs_hashes(seed, B, log2b, [n])
    host = {key: val.cpu().numpy() for key, val in res.items()}
    Sg = S.cpu().numpy().astype(np.complex128)
    U0g = t32(U0, dev).cpu().numpy().astype(np.float64)
    return host, Sg, ho[:, 0], go[:, 0], U0g, lam_true, A


@pytest.mark.parametrize("n,k,L,T_it,B,log2b,noise", [
    (50, 5, 10, 20, 5, 10, 0.01),     # the small planted configuration
    (37, 3, 4, 6, 4, 9, 0.1),         # ragged n, even B
    (16, 2, 3, 5, 1, 8, 0.05),        # a single sketch (median of one)
    (24, 2, 3, 4, 40, 10, 0.01),      # B = 40 as in the paper's largest sketch count
    (30, 2, 3, 4, 4, 13, 0.02),       # b = 2^13: frequencies split over 2 blocks of 2^12
    (20, 2, 3, 4, 3, 15, 0.02),       # b = 2^15: split over 8 blocks of 2^12
    (18, 2, 2, 3, 2, 16, 0.02)])      # b = 2^16: split over 8 blocks of 2^13
def test_rtpm_stepwise_parity(dev, n, k, L, T_it, B, log2b, noise):
    from rtpm_check import check_rtpm_stepwise
    res, Sg, ho, go, U0g, _, _ = _run_rtpm(dev, n, k, L, T_it, B, log2b, 1, noise)
    assert check_rtpm_stepwise(res, Sg, ho, go, 1 << log2b, U0g, T_it) == k * T_it * L


def test_rtpm_recovers_planted_components_at_large_b(dev):
    """Noise-free planted tensor, b = 2^14: the sketched method finds the components (Thm. 2)."""
    n, k = 20, 3
    res, _, _, _, _, lam_true, A = _run_rtpm(dev, n, k, 8, 15, 5, 14, 3, 0.0)
    lam = res["lam"]
    V = res["V"]
    order = np.argsort(-lam_true)
    for r in range(k):
        a = A[:, order[r]]
        assert abs(lam[r] - lam_true[order[r]]) < 0.1
        assert min(np.linalg.norm(V[r] - a), np.linalg.norm(V[r] + a)) < 0.1


def test_rtpm_reports_nonfinite(dev):
    n, B, log2b = 10, 2, 8
    h, g = tsk.cs_hashes(1, B, log2b, [n], dev)
    S = tsk.sketch_tensor(t32(synth.random_symmetric(n, 1), dev), h, g, log2b)
    U0 = torch.zeros((1, 2, n), dtype=torch.float32, device=dev)
    tsk.robust_power_method(S, h, g, U0, 2)
    assert tsk.ctx_status(dev) == -5   # TSK_ENONFINITE
    assert tsk.ctx_status(dev) == 0    # cleared


def test_argument_errors(dev):
    h, g = tsk.cs_hashes(1, 2, 8, [10], dev)
    S = torch.zeros((2, 256), dtype=torch.complex64, device=dev)
    with pytest.raises(tsk.TskError, match="EUNSUPPORTED"):
        tsk.robust_power_method(S, h, g, torch.ones((1, 1, 10), device=dev), 0)
    Sbig = torch.zeros((2, 1 << 15), dtype=torch.complex64, device=dev)
    with pytest.raises(tsk.TskError, match="EUNSUPPORTED"):
        tsk.contract_iuu(Sbig, Sbig, h, g, torch.ones((1, 10), device=dev))
    with pytest.raises(TypeError):
        tsk.contract_iuu(S, S, h, g, torch.ones((1, 10), device=dev, dtype=torch.float64))


def test_rtpm_captured_in_a_cuda_graph(dev):
    """Alg. 1 enqueued once into a CUDA graph (after a warm-up call has grown the workspace and
    created the helper streams) and replayed: every step of the replay passes the step-wise
    oracle check."""
    from rtpm_check import check_rtpm_stepwise
    n, k, L, T_it, B, log2b = 40, 2, 3, 4, 4, 12
    T, _, _ = synth.planted_symmetric(n, k, 0.02, 5)
    U0 = t32(synth.gaussian_inits(k, L, n, 6), dev)
    h, g = tsk.cs_hashes(5, B, log2b, [n], dev)
    S = tsk.sketch_tensor(t32(T, dev), h, g, log2b)
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        tsk.robust_power_method(S, h, g, U0, T_it, return_deflated=True, return_trace=True)
    torch.cuda.current_stream(dev).wait_stream(side)
    torch.cuda.synchronize(dev)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        res = tsk.robust_power_method(S, h, g, U0, T_it, return_deflated=True, return_trace=True)
    graph.replay()
    torch.cuda.synchronize(dev)
    tsk.check_status(dev)
    host = {key: val.cpu().numpy() for key, val in res.items()}
    ho, go = O.cs_hashes(5, B, log2b, [n])
    Sg = S.cpu().numpy().astype(np.complex128)
    U0g = U0.cpu().numpy().astype(np.float64)
    assert check_rtpm_stepwise(host, Sg, ho[:, 0], go[:, 0], 1 << log2b, U0g, T_it) == k * T_it * L
