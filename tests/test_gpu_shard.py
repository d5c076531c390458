"""Sketches sharded by planes (Sec. 3.1 linearity): the colliding sketch of the wedge entries
whose first index lies in a plane range, built from that slice of the tensor alone, equals the
oracle's sketch of the tensor masked to those entries, and the partial sketches of a partition
of the planes add up to the sketch of the whole tensor.  Alg. 1 with the initial vectors split
into shards (robust_power_method_sharded) equals Alg. 1 on all of them.

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


@pytest.mark.parametrize("log2b,B", [(15, 2), (16, 1), (12, 4)])
def test_planes_int32_input_float_sketch_and_bucket_ranges(dev, log2b, B):
    """int32 input into complex-float sketches (the fixed-point path), also where the buckets are
    split into 2 or 4 ranges held by separate blocks (b = 2^15, 2^16) and where one block builds
    several sketches (b = 2^12, B = 4): each plane range against the oracle's masked sketch, and
    the sum of the ranges against the full sketch."""
    n = 40
    b = 1 << log2b
    Ti = synth.random_symmetric_int(n, 60 + log2b)
    h, g = tsk.cs_hashes(3 + log2b, B, log2b, [n], dev)
    ho, go = O.cs_hashes(3 + log2b, B, log2b, [n])
    Td = torch.tensor(Ti, device=dev)
    Ssum = None
    for p0, p1 in tsk.plane_ranges(n, 3):
        Sp = tsk.sketch_tensor_planes(Td[p0:p1].contiguous(), h, g, log2b, p0)
        Tm = np.where(plane_mask(n, p0, p1), Ti, 0).astype(np.float64)
        for m in range(B):
            assert rel(Sp[m].cpu().numpy(), O.sketch_tensor_sym(Tm, ho[m, 0], go[m, 0], b)) < 1e-6
        Ssum = Sp.clone() if Ssum is None else Ssum + Sp
    full = tsk.sketch_tensor(Td, h, g, log2b).cpu().numpy()
    assert rel(Ssum.cpu().numpy(), full) < 1e-6


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


# ------------------------------------------------------------------ Alg. 1 with the initial vectors split
def _planted_problem(dev, n=50, k=4, B=5, log2b=10, L=8, seed=3):
    T, _, _ = synth.planted_symmetric(n, k, 0.001, seed, dtype=np.float32)
    h, g = tsk.cs_hashes(seed, B, log2b, [n], dev)
    S = tsk.sketch_tensor(torch.from_numpy(T).to(dev), h, g, log2b)
    U0 = torch.from_numpy(synth.gaussian_inits(k, L, n, seed + 1).astype(np.float32)).to(dev)
    return S, h, g, U0


def _check_round(ref, r, lam_r, tau_r, v_r):
    lam_ref = float(ref["lam"][r])
    row = ref["lam_all"][r].double().cpu()
    assert abs(lam_r - lam_ref) <= 1e-5 * abs(lam_ref)
    assert float(row[tau_r]) >= float(row.max()) - 1e-5 * abs(float(row.max()))
    assert abs(float(torch.dot(v_r.double(), ref["V"][r].double()))) >= 1 - 1e-6


def test_rounds_over_two_shards_equal_alg1(dev):
    """Every round's L initial vectors split into two shards, each run by one round of the device
    Alg. 1 (robust_power_method with k = 1), the winner chosen by select_first_max and its
    deflated sketches carried on: the same eigenvalues, global taus and components as Alg. 1 on
    all L vectors (the exchange robust_power_method_sharded makes over a process group).  Several
    starts converge to the same component with eigenvalues equal to rounding, and the shared-memory
    float adds of the count sketches make that rounding run-dependent, so the chosen tau is
    checked to attain the round's maximum within 1e-5 rather than to equal the reference's."""
    S, h, g, U0 = _planted_problem(dev)
    T_it = 20
    ref = tsk.robust_power_method(S, h, g, U0, T_it, return_deflated=True, return_trace=True)
    k, L, n = U0.shape
    shards = [(0, 3), (3, L)]                      # uneven on purpose
    Sc = S.clone()
    for r in range(k):
        outs = []
        for lo, hi in shards:
            res = tsk.robust_power_method(Sc, h, g, U0[r:r + 1, lo:hi].contiguous(), T_it,
                                          return_deflated=True)
            outs.append((float(res["lam"][0]), lo + int(res["tau"][0]), res["V"][0],
                         res["S_deflated"]))
        win = tsk.select_first_max([o[0] for o in outs], [o[1] for o in outs])
        lam_r, tau_r, v_r, Sc = outs[win]
        _check_round(ref, r, lam_r, tau_r, v_r)
    assert rel(Sc.cpu().numpy(), ref["S_deflated"].cpu().numpy()) < 1e-4


def test_sharded_alg1_over_an_nccl_group_of_one(dev):
    """robust_power_method_sharded through real NCCL collectives (a process group of one rank on
    this GPU): equal to robust_power_method."""
    import os
    import socket
    import torch.distributed as dist
    os.environ.setdefault("NCCL_NVLS_ENABLE", "0")
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        S, h, g, U0 = _planted_problem(dev, seed=5)
        ref = tsk.robust_power_method(S, h, g, U0, 15, return_deflated=True, return_trace=True)
        res = tsk.robust_power_method_sharded(S, h, g, U0, 15, 0)
        for r in range(U0.shape[0]):
            _check_round(ref, r, float(res["lam"][r]), int(res["tau"][r]), res["V"][r])
        assert rel(res["S_deflated"].cpu().numpy(), ref["S_deflated"].cpu().numpy()) < 1e-4
    finally:
        dist.destroy_process_group()
