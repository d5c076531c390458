"""Sketches sharded by planes (Sec. 3.1 linearity): the colliding sketch of the wedge entries
whose first index lies in a plane range, built from that slice of the tensor alone, equals the
oracle's sketch of the tensor masked to those entries, and the partial sketches of a partition
of the planes add up to the sketch of the whole tensor.

Tolerances: int64 sketches bit-exact, FP64 sketches 1e-12 relative, FP32 (complex64) sketches
1e-5 relative in the 2-norm per sketch.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu

tsk = pytest.importorskip("paper_1506_04448_gb300")


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0)


def plane_mask(n, p0, p1):
    """Ordered triples whose smallest index lies in [p0, p1): the wedge entries of planes
    p0 .. p1 - 1 and all their permutations."""
    i = np.arange(n)
    mn = np.minimum(np.minimum(i[:, None, None], i[None, :, None]), i[None, None, :])
    return (mn >= p0) & (mn < p1)


@pytest.mark.parametrize("n,parts,log2b,B", [(37, 3, 10, 2), (64, 4, 12, 3), (9, 12, 8, 1)])
def test_int_planes_bit_exact_and_sum(dev, n, parts, log2b, B):
    b = 1 << log2b
    Ti = synth.random_symmetric_int(n, 300 + n)
    h, g = tsk.cs_hashes(41 + n, B, log2b, [n], dev)
    ho, go = O.cs_hashes(41 + n, B, log2b, [n])
    Td = torch.tensor(Ti, device=dev)
    ranges = tsk.plane_ranges(n, parts)
    assert ranges[0][0] == 0 and ranges[-1][1] == n
    assert all(ranges[r][1] == ranges[r + 1][0] for r in range(parts - 1))
    total = None
    for p0, p1 in ranges:
        Sp = tsk.sketch_tensor_planes(Td[p0:p1].contiguous(), h, g, log2b, p0, acc="ci64")
        Sn = Sp.cpu().numpy()
        Tm = np.where(plane_mask(n, p0, p1), Ti, 0)
        for m in range(B):
            ref = O.sketch_tensor_sym(Tm, ho[m, 0], go[m, 0], b)
            np.testing.assert_array_equal(Sn[m, :, 0], ref[0])
            np.testing.assert_array_equal(Sn[m, :, 1], ref[1])
        total = Sp.clone() if total is None else total + Sp
    full = tsk.sketch_tensor(Td, h, g, log2b, acc="ci64")
    assert torch.equal(total, full)


@pytest.mark.parametrize("acc,dtype,tol", [("c64", np.float32, 1e-5), ("c128", np.float64, 1e-12)])
@pytest.mark.parametrize("n,parts,log2b", [(50, 2, 10), (130, 3, 14)])
def test_float_planes_match_oracle_and_sum(dev, acc, dtype, tol, n, parts, log2b):
    b, B = 1 << log2b, 2
    T = synth.random_symmetric(n, 500 + n).astype(dtype)
    h, g = tsk.cs_hashes(77 + n, B, log2b, [n], dev)
    ho, go = O.cs_hashes(77 + n, B, log2b, [n])
    Td = torch.tensor(T, device=dev)
    Ssum = None
    for p0, p1 in tsk.plane_ranges(n, parts):
        Sp = tsk.sketch_tensor_planes(Td[p0:p1].contiguous(), h, g, log2b, p0, acc=acc)
        Tm = np.where(plane_mask(n, p0, p1), T.astype(np.float64), 0.0)
        for m in range(B):
            ref = O.sketch_tensor_sym(Tm, ho[m, 0], go[m, 0], b)
            assert rel(Sp[m].cpu().numpy(), ref) < tol
        Ssum = Sp.clone() if Ssum is None else Ssum + Sp
    for m in range(B):
        ref = O.sketch_tensor_sym(T.astype(np.float64), ho[m, 0], go[m, 0], b)
        assert rel(Ssum[m].cpu().numpy(), ref) < tol


def test_planes_accumulate_into_one_buffer(dev):
    """accumulate=True adds each range's part into the same S: after all ranges S is the full
    sketch (here bit-equal to sketch_tensor's int64 result)."""
    n, log2b, B = 45, 11, 2
    Ti = synth.random_symmetric_int(n, 9)
    h, g = tsk.cs_hashes(5, B, log2b, [n], dev)
    Td = torch.tensor(Ti, device=dev)
    S = None
    for r, (p0, p1) in enumerate(tsk.plane_ranges(n, 5)):
        S = tsk.sketch_tensor_planes(Td[p0:p1].contiguous(), h, g, log2b, p0, S=S,
                                     accumulate=r > 0, acc="ci64")
    assert torch.equal(S, tsk.sketch_tensor(Td, h, g, log2b, acc="ci64"))


def test_empty_range_and_bad_ranges(dev):
    n, log2b = 12, 8
    T = torch.tensor(synth.random_symmetric(n, 3).astype(np.float32), device=dev)
    h, g = tsk.cs_hashes(1, 1, log2b, [n], dev)
    S = tsk.sketch_tensor_planes(T[4:4].contiguous(), h, g, log2b, 4)
    assert torch.count_nonzero(S).item() == 0
    S1 = tsk.sketch_tensor(T, h, g, log2b)
    S2 = S1.clone()
    tsk.sketch_tensor_planes(T[n:n].contiguous(), h, g, log2b, n, S=S2, accumulate=True)
    assert torch.equal(S1, S2)
    with pytest.raises(ValueError):
        tsk.sketch_tensor_planes(T[0:5].contiguous(), h, g, log2b, 8)
