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
