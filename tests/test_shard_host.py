"""Host side of sketches sharded by planes (Sec. 3.1 linearity), on CPU.

* plane_ranges partitions the planes 0..n-1 into consecutive ranges of about equal wedge size.
* Two gloo ranks (world_size 2) each sketch the entries of their planes with the oracle and
  add them with allreduce_sketches: both end with the oracle's sketch of the whole tensor
  (int64 bit-exact, complex128 to 1e-12).
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1506_04448_gb300 import allreduce_sketches, plane_ranges


def wedge_size(n, p0, p1):
    return sum((n - i) * (n - i + 1) // 2 for i in range(p0, p1))


@pytest.mark.parametrize("n", [0, 1, 2, 7, 100, 401, 1000])
@pytest.mark.parametrize("parts", [1, 2, 3, 8, 13])
def test_plane_ranges_partition_and_balance(n, parts):
    r = plane_ranges(n, parts)
    assert len(r) == parts
    assert r[0][0] == 0 and r[-1][1] == n
    for a, b in zip(r, r[1:]):
        assert a[1] == b[0]
    assert all(p0 <= p1 for p0, p1 in r)
    total = wedge_size(n, 0, n)
    assert sum(wedge_size(n, p0, p1) for p0, p1 in r) == total
    if n >= 100 and parts <= 13:
        # every range within one plane (at most n(n+1)/2 entries) of an equal share
        for p0, p1 in r:
            assert abs(wedge_size(n, p0, p1) - total / parts) <= n * (n + 1) / 2


def test_plane_ranges_rejects_bad_arguments():
    with pytest.raises(ValueError):
        plane_ranges(10, 0)
    with pytest.raises(ValueError):
        plane_ranges(-1, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _masked(T, p0, p1):
    n = T.shape[0]
    i = np.arange(n)
    mn = np.minimum(np.minimum(i[:, None, None], i[None, :, None]), i[None, None, :])
    return np.where((mn >= p0) & (mn < p1), T, 0)


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    import synth
    n, log2b, seed = 23, 9, 17
    b = 1 << log2b
    ho, go = O.cs_hashes(seed, 1, log2b, [n])
    p0, p1 = plane_ranges(n, world)[rank]
    # exact integer sketches
    Ti = synth.random_symmetric_int(n, 4)
    Si = torch.from_numpy(O.sketch_tensor_sym(_masked(Ti, p0, p1), ho[0, 0], go[0, 0], b))
    allreduce_sketches(Si)
    # complex sketches of a float tensor
    Tf = synth.random_symmetric(n, 5)
    Sf = torch.from_numpy(O.sketch_tensor_sym(_masked(Tf, p0, p1), ho[0, 0], go[0, 0], b))
    allreduce_sketches(Sf)
    full_i = O.sketch_tensor_sym(Ti, ho[0, 0], go[0, 0], b)
    full_f = O.sketch_tensor_sym(Tf, ho[0, 0], go[0, 0], b)
    ok_i = bool(np.array_equal(Si.numpy(), full_i))
    err_f = float(np.linalg.norm(Sf.numpy() - full_f) / np.linalg.norm(full_f))
    out[rank] = (ok_i, err_f, (p0, p1))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_sum_partial_sketches():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][2][1] == res[1][2][0]          # the ranks' planes meet
    for r in range(world):
        ok_i, err_f, _ = res[r]
        assert ok_i
        assert err_f < 1e-12


# ------------------------------------------------------------------ Alg. 1 with the initial vectors split
def test_select_first_max_ties_to_smallest_index():
    from paper_1506_04448_gb300 import select_first_max
    assert select_first_max([1.0, 3.0, 2.0], [0, 4, 8]) == 1
    assert select_first_max([3.0, 3.0, 2.0], [4, 0, 8]) == 1
    assert select_first_max([-1.0], [5]) == 0


def _rtpm_rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    import synth
    from paper_1506_04448_gb300 import robust_power_method_sharded
    n, k, L, T_it, B, log2b = 12, 3, 6, 5, 3, 7
    b = 1 << log2b
    Tn, _, _ = synth.planted_symmetric(n, k, 0.05, 23)
    ho, go = O.cs_hashes(9, B, log2b, [n])
    h, g = ho[:, 0], go[:, 0]
    S = np.stack([O.sketch_tensor_sym(Tn, h[m], g[m], b) for m in range(B)])
    U0 = synth.gaussian_inits(k, L, n, 24)
    per = L // world
    lo = rank * per

    def oracle_round(Sc, U0_round, T):
        res = O.rtpm_sketched(Sc.numpy(), h, g, b, U0_round.numpy()[None], T)
        return (float(res["lam"][0]), int(res["tau"][0]), torch.from_numpy(res["V"][0].copy()),
                torch.from_numpy(res["S_deflated"].copy()))

    res = robust_power_method_sharded(torch.from_numpy(S), None, None,
                                      torch.from_numpy(U0[:, lo:lo + per].copy()), T_it, lo,
                                      run_round=oracle_round)
    ref = O.rtpm_sketched(S, h, g, b, U0, T_it)
    out[rank] = (res["lam"].numpy().tolist(), res["tau"].numpy().tolist(),
                 float(np.abs(res["V"].numpy() - ref["V"]).max()),
                 float(np.abs(res["S_deflated"].numpy() - ref["S_deflated"]).max()),
                 ref["lam"].tolist(), ref["tau"].tolist())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_split_the_initial_vectors():
    """Two ranks each run half of every round's L initial vectors (the oracle's Alg. 1 round as
    the per-rank compute); the all-gather selection and the winner's broadcast reproduce the
    oracle's Alg. 1 on all L vectors: eigenvalues, global tau, components and deflated
    sketches."""
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rtpm_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        lam, tau, dv, ds, lam_ref, tau_ref = res[r]
        np.testing.assert_allclose(lam, lam_ref, rtol=1e-12)
        assert tau == tau_ref
        assert dv < 1e-12 and ds < 1e-10
    assert res[0][1] == res[1][1]
