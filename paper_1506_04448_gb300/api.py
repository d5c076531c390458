"""Python binding of the C ABI in include/tsk.h: argument marshalling only.

Every function takes CUDA torch tensors, checks shapes and dtypes, allocates outputs with torch
(device memory is the only thing torch provides here) and calls the library on the current
torch stream of the tensors' device.  All arithmetic happens in libtsk.so.
"""
from __future__ import annotations

import ctypes
import threading

import torch

from . import _lib

_ctx_lock = threading.Lock()
_ctxs: dict[int, int] = {}


def _ctx(device: torch.device) -> int:
    """Per-device library context bound to the device's current torch stream."""
    lib = _lib.load()
    idx = device.index if device.index is not None else torch.cuda.current_device()
    with _ctx_lock:
        c = _ctxs.get(idx)
        if c is None:
            h = ctypes.c_void_p()
            with torch.cuda.device(idx):
                _lib.check("tsk_ctx_create", lib.tsk_ctx_create(idx, None, ctypes.byref(h)))
            c = h.value
            _ctxs[idx] = c
    stream = torch.cuda.current_stream(idx).cuda_stream
    _lib.check("tsk_ctx_set_stream", lib.tsk_ctx_set_stream(c, ctypes.c_void_p(stream)))
    return c


def _ptr(t: torch.Tensor | None) -> ctypes.c_void_p:
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _need(t: torch.Tensor, name: str, dtype, device: torch.device, shape=None) -> torch.Tensor:
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.device.type != "cuda" or t.device != device:
        raise ValueError(f"{name} must live on {device}, got {t.device}")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _dims(dims) -> ctypes.Array:
    arr = (ctypes.c_int64 * len(dims))(*[int(d) for d in dims])
    return arr


def _hashes_shape(h: torch.Tensor, g: torch.Tensor):
    if h.dim() == 2:
        h = h.unsqueeze(1)
        g = g.unsqueeze(1)
    if h.dim() != 3 or h.shape != g.shape:
        raise ValueError("h and g must have shape [B][M][nmax] (or [B][n] for M = 1)")
    return h, g


def ctx_status(device: torch.device | str | int = "cuda") -> int:
    """Synchronise and return/clear the first device-side status code (0 = ok)."""
    if isinstance(device, int):
        device = torch.device("cuda", device)
    device = torch.device(device) if not isinstance(device, torch.device) else device
    return _lib.load().tsk_ctx_status(_ctx(device))


def check_status(device: torch.device | str = "cuda") -> None:
    rc = ctx_status(device)
    _lib.check("device status", rc)


# ------------------------------------------------------------------ measured roofs
PEAK_FMA, PEAK_SMEM, PEAK_ATOMS = 0, 1, 2


def peak_launch(kind: int, iters: int, sink: torch.Tensor) -> None:
    """Enqueue one roof micro-kernel launch (TSK_PEAK_*) on the current stream of sink's device."""
    rc = _lib.load().tsk_peak_launch(_ctx(sink.device), int(kind), int(iters), _ptr(sink))
    _lib.check("tsk_peak_launch", rc)


def peak_work(kind: int, iters: int, device="cuda") -> float:
    """Work of one peak_launch(kind, iters): flops, bytes or atomic adds."""
    out = ctypes.c_double()
    rc = _lib.load().tsk_peak_work(_ctx(torch.device(device)), int(kind), int(iters), ctypes.byref(out))
    _lib.check("tsk_peak_work", rc)
    return out.value


# ------------------------------------------------------------------ hashing
def cs_hashes(seed: int, B: int, log2b: int, dims, device="cuda"):
    """Hash tables of B sketches: (h int32 [B][M][nmax], g uint8 [B][M][nmax])."""
    device = torch.device(device)
    dims = [int(d) for d in dims]
    M = len(dims)
    nmax = max(dims) if dims else 0
    h = torch.empty((B, M, nmax), dtype=torch.int32, device=device)
    g = torch.empty((B, M, nmax), dtype=torch.uint8, device=device)
    rc = _lib.load().cs_hashes(_ctx(device), ctypes.c_uint64(seed & (2**64 - 1)), B, log2b, M,
                               _dims(dims), _ptr(h), _ptr(g))
    _lib.check("cs_hashes", rc)
    return h, g


# ------------------------------------------------------------------ sketches
_IN_DTYPES = {torch.float32: _lib.TSK_F32, torch.float64: _lib.TSK_F64, torch.int32: _lib.TSK_I32}


def sketch_tensor(T: torch.Tensor, h: torch.Tensor, g: torch.Tensor, log2b: int, *,
                  S: torch.Tensor | None = None, accumulate: bool = False, acc: str = "c64"):
    """Tensor sketches of a dense tensor.  h.shape[1] == 1: colliding sketch of a symmetric
    n^3 tensor (Eq. 7); 3: asymmetric sketch (Eq. 1).  acc: 'c64' (complex64 [B][b]),
    'c128' (complex128 [B][b]) or 'ci64' (int64 [B][b][2], exact)."""
    device = T.device
    if T.dtype not in _IN_DTYPES:
        raise TypeError("T must be float32, float64 or int32")
    _need(T, "T", T.dtype, device)
    h, g = _hashes_shape(h, g)
    _need(h, "h", torch.int32, device)
    _need(g, "g", torch.uint8, device)
    B, M, nmax = h.shape
    if T.dim() != 3:
        raise ValueError("T must be 3-dimensional")
    if M == 1 and not (T.shape[0] == T.shape[1] == T.shape[2] == nmax):
        raise ValueError("symmetric sketch needs an n x n x n tensor with n = h.shape[-1]")
    if M == 3 and max(T.shape) != nmax:
        raise ValueError("asymmetric sketch needs max(T.shape) == h.shape[-1]")
    b = 1 << log2b
    if acc == "c64":
        shape, dt, code = (B, b), torch.complex64, _lib.TSK_C64
    elif acc == "c128":
        shape, dt, code = (B, b), torch.complex128, _lib.TSK_C128
    elif acc == "ci64":
        shape, dt, code = (B, b, 2), torch.int64, _lib.TSK_CI64
    else:
        raise ValueError("acc must be 'c64', 'c128' or 'ci64'")
    if S is None:
        if accumulate:
            raise ValueError("accumulate=True needs S")
        S = torch.empty(shape, dtype=dt, device=device)
    _need(S, "S", dt, device, shape)
    dims = list(T.shape) if M == 3 else [T.shape[0]]
    rc = _lib.load().sketch_tensor(_ctx(device), _ptr(T), _IN_DTYPES[T.dtype], M, _dims(dims),
                                   _ptr(h), _ptr(g), B, log2b, _ptr(S), code, int(accumulate))
    _lib.check("sketch_tensor", rc)
    return S


_ACC_CODES = {"c64": (torch.complex64, _lib.TSK_C64), "c128": (torch.complex128, _lib.TSK_C128),
              "ci64": (torch.int64, _lib.TSK_CI64)}


def sketch_tensor_planes(T_planes: torch.Tensor, h: torch.Tensor, g: torch.Tensor, log2b: int,
                         plane_begin: int, *, S: torch.Tensor | None = None,
                         accumulate: bool = False, acc: str = "c64"):
    """Colliding sketches (Eq. 7) of the wedge entries i <= j <= k whose first index lies in
    [plane_begin, plane_begin + T_planes.shape[0]) of a symmetric n^3 tensor, from the slice
    T_planes = T[plane_begin:plane_end] ([planes][n][n]).  By linearity (Sec. 3.1) the sketches
    of a partition of the planes add up to the sketch of T."""
    device = T_planes.device
    if T_planes.dtype not in _IN_DTYPES:
        raise TypeError("T_planes must be float32, float64 or int32")
    _need(T_planes, "T_planes", T_planes.dtype, device)
    h, g = _hashes_shape(h, g)
    _need(h, "h", torch.int32, device)
    _need(g, "g", torch.uint8, device)
    B, M, n = h.shape
    if M != 1:
        raise ValueError("plane ranges apply to the colliding sketch (h.shape[1] == 1)")
    if T_planes.dim() != 3 or T_planes.shape[1] != n or T_planes.shape[2] != n:
        raise ValueError("T_planes must be [planes][n][n] with n = h.shape[-1]")
    plane_end = plane_begin + T_planes.shape[0]
    if plane_begin < 0 or plane_end > n:
        raise ValueError("planes out of range")
    if acc not in _ACC_CODES:
        raise ValueError("acc must be 'c64', 'c128' or 'ci64'")
    dt, code = _ACC_CODES[acc]
    b = 1 << log2b
    shape = (B, b, 2) if acc == "ci64" else (B, b)
    if S is None:
        if accumulate:
            raise ValueError("accumulate=True needs S")
        S = torch.empty(shape, dtype=dt, device=device)
    _need(S, "S", dt, device, shape)
    rc = _lib.load().sketch_tensor_planes(_ctx(device), _ptr(T_planes), _IN_DTYPES[T_planes.dtype],
                                          n, plane_begin, plane_end, _ptr(h), _ptr(g), B, log2b,
                                          _ptr(S), code, int(accumulate))
    _lib.check("sketch_tensor_planes", rc)
    return S


def plane_ranges(n: int, parts: int) -> list[tuple[int, int]]:
    """Split the planes 0..n-1 of the wedge into `parts` consecutive ranges with about equal
    numbers of wedge entries (plane i holds (n - i)(n - i + 1) / 2 of them).  Host-side only."""
    if parts < 1 or n < 0:
        raise ValueError("need parts >= 1 and n >= 0")
    sizes = [(n - i) * (n - i + 1) // 2 for i in range(n)]
    total = sum(sizes)
    cuts, acc, r = [0], 0, 1
    for i, w in enumerate(sizes):
        acc += w
        while r < parts and acc * parts >= total * r:
            cuts.append(i + 1)
            r += 1
    while len(cuts) < parts:
        cuts.append(n)
    cuts.append(n)
    return [(cuts[r], cuts[r + 1]) for r in range(parts)]


def allreduce_sketches(S: torch.Tensor, group=None) -> torch.Tensor:
    """Sum partial sketches across the ranks of a torch.distributed process group, in place
    (Sec. 3.1: the sketch of a sum of tensors is the sum of their sketches)."""
    import torch.distributed as dist
    buf = torch.view_as_real(S) if S.is_complex() else S
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    return S


def select_first_max(lams, taus) -> int:
    """Index q of the largest lams[q], ties to the smallest global initial-vector index taus[q]:
    Alg. 1's selection (the first maximum over tau) taken over shards of the L initial vectors,
    each of which reports its own first maximum (lam, tau).  Host-side only."""
    best = 0
    for q in range(1, len(lams)):
        if lams[q] > lams[best] or (lams[q] == lams[best] and taus[q] < taus[best]):
            best = q
    return best


def _library_round(S, h, g, U0_round, T):
    res = robust_power_method(S, h, g, U0_round.unsqueeze(0), T, return_deflated=True)
    return float(res["lam"][0].item()), int(res["tau"][0].item()), res["V"][0], res["S_deflated"]


def robust_power_method_sharded(S: torch.Tensor, h: torch.Tensor, g: torch.Tensor,
                                U0_local: torch.Tensor, T: int, tau_offset: int, group=None,
                                run_round=None):
    """Alg. 1 with the L initial vectors of every round split across the ranks of a
    torch.distributed process group.  Every rank holds the same sketches S [B][b] and its slice
    U0_local = U0[:, tau_offset:tau_offset + L_local] [k][L_local][n].  Per round each rank runs
    T power updates of its vectors and selects its first maximum (run_round, by default one round
    of robust_power_method on the device, which also deflates by its own choice in FP64); one
    all-gather of (lambda, global tau) picks the round's winner (select_first_max), and the winner
    broadcasts its component and its deflated sketches, which every rank continues from.  The
    result equals Alg. 1 on all L vectors.  Returns dict(lam [k] float64 and tau [k] int64 (global
    indices) on the host, V [k][n] and S_deflated on S's device).

    run_round(S, U0_round_local [L_local][n], T) -> (lam, tau_local, v [n], S_deflated) may
    replace the device round (the host test of the exchange uses the oracle)."""
    import torch.distributed as dist
    if run_round is None:
        def run_round(S_, U0_round, T_):
            return _library_round(S_, h, g, U0_round, T_)
    world = dist.get_world_size(group)
    ranks = [dist.get_global_rank(group, q) if group is not None else q for q in range(world)]
    k = U0_local.shape[0]
    lam = torch.empty(k, dtype=torch.float64)
    tau = torch.empty(k, dtype=torch.int64)
    Vs = []
    for r in range(k):
        lam_r, tau_r, v, Sd = run_round(S, U0_local[r], T)
        key = torch.tensor([lam_r, float(tau_offset + tau_r)], dtype=torch.float64, device=v.device)
        keys = [torch.empty_like(key) for _ in range(world)]
        dist.all_gather(keys, key, group=group)
        keys = [kk.cpu() for kk in keys]
        win = select_first_max([float(kk[0]) for kk in keys], [float(kk[1]) for kk in keys])
        v = v.clone().contiguous()
        Sd = Sd.clone().contiguous()
        dist.broadcast(v, src=ranks[win], group=group)
        dist.broadcast(torch.view_as_real(Sd) if Sd.is_complex() else Sd, src=ranks[win],
                       group=group)
        lam[r] = float(keys[win][0])
        tau[r] = int(keys[win][1])
        Vs.append(v)
        S = Sd
    V = torch.stack(Vs) if Vs else U0_local.new_empty((0, U0_local.shape[-1]))
    return {"lam": lam, "V": V, "tau": tau, "S_deflated": S}


def sketch_fft(S: torch.Tensor, inverse: bool = False, out: torch.Tensor | None = None):
    """Batched DFT of the rows of a complex64 [B][b] tensor (inverse includes 1/b)."""
    device = S.device
    _need(S, "S", torch.complex64, device)
    B, b = S.shape
    log2b = b.bit_length() - 1
    if 1 << log2b != b:
        raise ValueError("sketch length must be a power of two")
    out = torch.empty_like(S) if out is None else _need(out, "out", torch.complex64, device, S.shape)
    rc = _lib.load().sketch_fft(_ctx(device), _ptr(S), _ptr(out), B, log2b, int(bool(inverse)))
    _lib.check("sketch_fft", rc)
    return out


def sketch_rank1(w: torch.Tensor, U: torch.Tensor, h: torch.Tensor, g: torch.Tensor, log2b: int, *,
                 V: torch.Tensor | None = None, W: torch.Tensor | None = None,
                 domain: str = "time", S: torch.Tensor | None = None, accumulate: bool = False):
    """S (+)= sum_c w[c] sketch(U[c] (x) V[c] (x) W[c]) (Eq. 4); V = W = None with M = 1
    gives the colliding sketch of U[c]^(x)3."""
    device = U.device
    h, g = _hashes_shape(h, g)
    _need(h, "h", torch.int32, device)
    _need(g, "g", torch.uint8, device)
    B, M, nmax = h.shape
    count = U.shape[0]
    _need(w, "w", torch.float32, device, (count,))
    _need(U, "U", torch.float32, device)
    dims = [U.shape[1]]
    if M == 3:
        if V is None or W is None:
            raise ValueError("asymmetric rank-1 sketches need V and W")
        _need(V, "V", torch.float32, device)
        _need(W, "W", torch.float32, device)
        dims = [U.shape[1], V.shape[1], W.shape[1]]
    b = 1 << log2b
    if S is None:
        if accumulate:
            raise ValueError("accumulate=True needs S")
        S = torch.empty((B, b), dtype=torch.complex64, device=device)
    _need(S, "S", torch.complex64, device, (B, b))
    dom = {"time": 0, "freq": 1}[domain]
    rc = _lib.load().sketch_rank1(_ctx(device), count, _ptr(w), _ptr(U), _ptr(V), _ptr(W), M,
                                  _dims(dims), _ptr(h), _ptr(g), B, log2b, dom, _ptr(S),
                                  int(accumulate))
    _lib.check("sketch_rank1", rc)
    return S


# ------------------------------------------------------------------ contractions
def _contract_common(FS, S, h, g, U):
    device = U.device
    _need(FS, "FS", torch.complex64, device)
    B, b = FS.shape
    _need(S, "S", torch.complex64, device, (B, b))
    h, g = _hashes_shape(h, g)
    if h.shape[1] != 1:
        raise ValueError("contractions use the colliding (M = 1) sketch")
    _need(h, "h", torch.int32, device)
    _need(g, "g", torch.uint8, device)
    if U.dim() == 1:
        U = U.unsqueeze(0)
    _need(U, "U", torch.float32, device)
    L, n = U.shape
    if h.shape != (B, 1, n):
        raise ValueError(f"h must have shape [{B}][1][{n}]")
    log2b = b.bit_length() - 1
    return device, B, b, log2b, h, g, U, L, n


def contract_iuu(FS: torch.Tensor, S: torch.Tensor, h: torch.Tensor, g: torch.Tensor,
                 U: torch.Tensor, return_all: bool = False):
    """Sketched T^(I,u,u) of every row of U (App. B, Eq. 14); median over the B sketches.
    Returns Vmed [L][n] (and Vall [L][B][n] with return_all)."""
    device, B, b, log2b, h, g, U, L, n = _contract_common(FS, S, h, g, U)
    Vmed = torch.empty((L, n), dtype=torch.float32, device=device)
    Vall = torch.empty((L, B, n), dtype=torch.float32, device=device) if return_all else None
    rc = _lib.load().contract_iuu(_ctx(device), _ptr(FS), _ptr(S), _ptr(h), _ptr(g), B, log2b,
                                  _ptr(U), L, n, _ptr(Vmed), _ptr(Vall))
    _lib.check("contract_iuu", rc)
    return (Vmed, Vall) if return_all else Vmed


def contract_uuu(FS: torch.Tensor, S: torch.Tensor, h: torch.Tensor, g: torch.Tensor,
                 U: torch.Tensor, return_all: bool = False):
    """Sketched T^(u,u,u) of every row of U (App. B, Eq. 13); median over the B sketches."""
    device, B, b, log2b, h, g, U, L, n = _contract_common(FS, S, h, g, U)
    lam = torch.empty((L,), dtype=torch.float32, device=device)
    lam_all = torch.empty((L, B), dtype=torch.float32, device=device) if return_all else None
    rc = _lib.load().contract_uuu(_ctx(device), _ptr(FS), _ptr(S), _ptr(h), _ptr(g), B, log2b,
                                  _ptr(U), L, n, _ptr(lam), _ptr(lam_all))
    _lib.check("contract_uuu", rc)
    return (lam, lam_all) if return_all else lam


def robust_power_method(S: torch.Tensor, h: torch.Tensor, g: torch.Tensor, U0: torch.Tensor,
                        T: int, return_deflated: bool = False, return_trace: bool = False):
    """Alg. 1 on B colliding sketches S [B][b] (time domain) with initial vectors U0 [k][L][n].
    Returns dict(lam [k] float64, V [k][n], tau [k] int32[, S_deflated [B][b]]
    [, lam_all [k][L], U_iters [k][T][L][n]])."""
    device = S.device
    _need(S, "S", torch.complex64, device)
    B, b = S.shape
    h, g = _hashes_shape(h, g)
    _need(h, "h", torch.int32, device)
    _need(g, "g", torch.uint8, device)
    _need(U0, "U0", torch.float32, device)
    k, L, n = U0.shape
    if h.shape != (B, 1, n):
        raise ValueError(f"h must have shape [{B}][1][{n}]")
    log2b = b.bit_length() - 1
    lam = torch.empty((k,), dtype=torch.float64, device=device)
    V = torch.empty((k, n), dtype=torch.float32, device=device)
    tau = torch.empty((k,), dtype=torch.int32, device=device)
    Sd = torch.empty_like(S) if return_deflated else None
    lam_all = torch.empty((k, L), dtype=torch.float32, device=device) if return_trace else None
    U_iters = (torch.empty((k, max(int(T), 0), L, n), dtype=torch.float32, device=device)
               if return_trace else None)
    rc = _lib.load().robust_power_method(_ctx(device), _ptr(S), _ptr(h), _ptr(g), B, log2b, n, k,
                                         L, int(T), _ptr(U0), _ptr(lam), _ptr(V), _ptr(tau),
                                         _ptr(Sd), _ptr(lam_all), _ptr(U_iters))
    _lib.check("robust_power_method", rc)
    out = {"lam": lam, "V": V, "tau": tau}
    if return_deflated:
        out["S_deflated"] = Sd
    if return_trace:
        out["lam_all"] = lam_all
        out["U_iters"] = U_iters
    return out


def robust_power_method_asym(S: torch.Tensor, h: torch.Tensor, g: torch.Tensor, U0: torch.Tensor,
                             T: int, return_trace: bool = False):
    """Alg. 1 as printed, on B asymmetric sketches S [B][b] (complex64, real parts used) of a
    symmetric tensor with hashes h, g [B][3][n] and initial vectors U0 [k][L][n].
    Returns dict(lam [k] float64, V [k][n], tau [k] int32[, lam_all [k][L], U_iters [k][T][L][n]])."""
    device = S.device
    _need(S, "S", torch.complex64, device)
    B, b = S.shape
    _need(h, "h", torch.int32, device)
    _need(g, "g", torch.uint8, device)
    _need(U0, "U0", torch.float32, device)
    k, L, n = U0.shape
    if tuple(h.shape) != (B, 3, n) or h.shape != g.shape:
        raise ValueError(f"h and g must have shape [{B}][3][{n}]")
    log2b = b.bit_length() - 1
    lam = torch.empty((k,), dtype=torch.float64, device=device)
    V = torch.empty((k, n), dtype=torch.float32, device=device)
    tau = torch.empty((k,), dtype=torch.int32, device=device)
    lam_all = torch.empty((k, L), dtype=torch.float32, device=device) if return_trace else None
    U_iters = (torch.empty((k, int(T), L, n), dtype=torch.float32, device=device)
               if return_trace else None)
    rc = _lib.load().robust_power_method_asym(_ctx(device), _ptr(S), _ptr(h), _ptr(g), B, log2b,
                                              n, k, L, int(T), _ptr(U0), _ptr(lam), _ptr(V),
                                              _ptr(tau), _ptr(lam_all), _ptr(U_iters))
    _lib.check("robust_power_method_asym", rc)
    out = {"lam": lam, "V": V, "tau": tau}
    if return_trace:
        out["lam_all"] = lam_all
        out["U_iters"] = U_iters
    return out


def robust_power_method_launches(B: int, log2b: int, n: int, k: int, L: int, T: int,
                                 device="cuda") -> int:
    """Kernel launches one robust_power_method call makes for these sizes on `device`."""
    device = torch.device(device)
    return int(_lib.load().robust_power_method_launches(_ctx(device), B, log2b, n, k, L, T))


# ------------------------------------------------------------------ end-to-end call
def decompose_symmetric(T, k: int, L: int, T_iters: int, B: int, log2b: int, seed: int,
                        U0, device="cuda"):
    """One call from a host (or device) symmetric tensor to (lambda, V): hashes, colliding
    sketches (Eq. 7) and Alg. 1.  Host inputs are copied to the device and the results are
    copied back to the host when T was given on the host."""
    device = torch.device(device)
    host = T.device.type == "cpu"
    Td = T.to(device, non_blocking=True) if host else T
    U0d = U0.to(device, non_blocking=True) if U0.device.type == "cpu" else U0
    n = Td.shape[0]
    h, g = cs_hashes(seed, B, log2b, [n], device)
    S = sketch_tensor(Td, h, g, log2b)
    res = robust_power_method(S, h, g, U0d, T_iters)
    if host:
        return {key: val.to("cpu") for key, val in res.items()}
    return res


# ------------------------------------------------------------------ asymmetric sketches, CP fitting
def sketch_rfft(S: torch.Tensor) -> torch.Tensor:
    """Half spectra [B][b/2+1] of the real parts of complex64 sketches S [B][b]."""
    device = S.device
    _need(S, "S", torch.complex64, device)
    B, b = S.shape
    log2b = b.bit_length() - 1
    Xh = torch.empty((B, b // 2 + 1), dtype=torch.complex64, device=device)
    rc = _lib.load().sketch_rfft(_ctx(device), _ptr(S), _ptr(Xh), B, log2b)
    _lib.check("sketch_rfft", rc)
    return Xh


def _asym_common(Xh, h, g, dims):
    device = Xh.device
    _need(Xh, "Xh", torch.complex64, device)
    B, nh = Xh.shape
    b = 2 * (nh - 1)
    log2b = b.bit_length() - 1
    if 1 << log2b != b:
        raise ValueError("Xh must hold half spectra of a power-of-two sketch length")
    _need(h, "h", torch.int32, device)
    _need(g, "g", torch.uint8, device)
    if h.dim() != 3 or h.shape[0] != B or h.shape[1] != 3 or h.shape != g.shape:
        raise ValueError("asymmetric hash tables must have shape [B][3][nmax]")
    dims = [int(d) for d in dims]
    if max(dims) != h.shape[2]:
        raise ValueError("max(dims) must equal h.shape[2]")
    return device, B, log2b, dims


def contract_ivw(Xh: torch.Tensor, h: torch.Tensor, g: torch.Tensor, dims, mode: int,
                 V: torch.Tensor, W: torch.Tensor, return_all: bool = False):
    """Sketched T^(I,v,w) with the identity at `mode` and V, W on the other two modes in
    increasing order (Prop. 1; the columns of T_(1)(C (.) B) in Alg. 2); median over sketches."""
    device, B, log2b, dims = _asym_common(Xh, h, g, dims)
    others = [j for j in range(3) if j != mode]
    K = V.shape[0]
    _need(V, "V", torch.float32, device, (K, dims[others[0]]))
    _need(W, "W", torch.float32, device, (K, dims[others[1]]))
    Vmed = torch.empty((K, dims[mode]), dtype=torch.float32, device=device)
    Vall = torch.empty((K, B, dims[mode]), dtype=torch.float32, device=device) if return_all else None
    rc = _lib.load().contract_ivw(_ctx(device), _ptr(Xh), _ptr(h), _ptr(g), B, log2b, _dims(dims),
                                  int(mode), _ptr(V), _ptr(W), K, _ptr(Vmed), _ptr(Vall))
    _lib.check("contract_ivw", rc)
    return (Vmed, Vall) if return_all else Vmed


def cp_sketch_loss(Xh: torch.Tensor, h: torch.Tensor, g: torch.Tensor, dims, lam: torch.Tensor,
                   A: torch.Tensor, Bf: torch.Tensor, C: torch.Tensor, with_grad: bool = True):
    """Sketched CP loss (1/B) sum_m ||s_T^(m) - sum_r lam_r s^(m)_{A[r](x)Bf[r](x)C[r]}||^2 and,
    with_grad, its gradients (lam, A, Bf, C) from the hand-written adjoint kernel."""
    device, B, log2b, dims = _asym_common(Xh, h, g, dims)
    R = lam.shape[0]
    _need(lam, "lam", torch.float32, device, (R,))
    for name, t, d in (("A", A, dims[0]), ("Bf", Bf, dims[1]), ("C", C, dims[2])):
        _need(t, name, torch.float32, device, (R, d))
    loss = torch.empty((), dtype=torch.float32, device=device)
    grads = [torch.empty_like(t) for t in (lam, A, Bf, C)] if with_grad else [None] * 4
    rc = _lib.load().cp_sketch_loss(_ctx(device), _ptr(Xh), _ptr(h), _ptr(g), B, log2b, _dims(dims),
                                    R, _ptr(lam), _ptr(A), _ptr(Bf), _ptr(C), _ptr(loss),
                                    *[_ptr(t) for t in grads])
    _lib.check("cp_sketch_loss", rc)
    return (loss, *grads) if with_grad else loss


class CPSketchLoss(torch.autograd.Function):
    """Differentiable sketched CP loss: forward and the adjoint both run in libtsk (the gradient
    of each factor is a sketched T(I,v,w) contraction of the residual sketch)."""

    @staticmethod
    def forward(ctx, lam, A, Bf, C, Xh, h, g, dims):
        loss, g_lam, g_A, g_B, g_C = cp_sketch_loss(Xh, h, g, dims, lam.detach().contiguous(),
                                                    A.detach().contiguous(), Bf.detach().contiguous(),
                                                    C.detach().contiguous(), with_grad=True)
        ctx.save_for_backward(g_lam, g_A, g_B, g_C)
        return loss

    @staticmethod
    def backward(ctx, grad_out):
        g_lam, g_A, g_B, g_C = ctx.saved_tensors
        return grad_out * g_lam, grad_out * g_A, grad_out * g_B, grad_out * g_C, None, None, None, None


def cp_loss(lam, A, Bf, C, Xh, h, g, dims):
    """Autograd entry point of the sketched CP loss."""
    return CPSketchLoss.apply(lam, A, Bf, C, Xh, h, g, tuple(int(d) for d in dims))


def cp_als_solve(M: torch.Tensor, P: torch.Tensor, Q: torch.Tensor):
    """Eq. 15: out = G^-1 M, G = (P P^T) o (Q Q^T); returns (normalised rows, row norms)."""
    device = M.device
    K, n = M.shape
    _need(M, "M", torch.float32, device)
    _need(P, "P", torch.float32, device)
    _need(Q, "Q", torch.float32, device)
    if P.shape[0] != K or Q.shape[0] != K:
        raise ValueError("P and Q must have K rows")
    out = torch.empty_like(M)
    lam = torch.empty((K,), dtype=torch.float32, device=device)
    rc = _lib.load().cp_als_solve(_ctx(device), _ptr(M), _ptr(P), _ptr(Q), K, n, P.shape[1],
                                  Q.shape[1], _ptr(out), _ptr(lam))
    _lib.check("cp_als_solve", rc)
    return out, lam


def cp_als_step(Xh, h, g, dims, factors):
    """One sweep of the sketched ALS of Alg. 2 with the Gram inverse of Eq. 15: for each mode,
    the sketched T(I, x_r, y_r) columns (median over sketches) and the k x k solve.  Returns
    (lam, [A, Bf, C]) with unit-norm rows."""
    factors = list(factors)
    lam = None
    for mode in range(3):
        p, q = [j for j in range(3) if j != mode]
        M = contract_ivw(Xh, h, g, dims, mode, factors[p], factors[q])
        factors[mode], lam = cp_als_solve(M, factors[p], factors[q])
    return lam, factors


# ------------------------------------------------------------------ many independent problems
class _Problem(ctypes.Structure):
    """Mirror of tsk_problem in include/tsk.h."""
    _fields_ = [("S", ctypes.c_void_p), ("h", ctypes.c_void_p), ("g", ctypes.c_void_p),
                ("U0", ctypes.c_void_p), ("n", ctypes.c_int64), ("k", ctypes.c_int),
                ("log2b", ctypes.c_int), ("lam", ctypes.c_void_p), ("V", ctypes.c_void_p),
                ("tau", ctypes.c_void_p), ("lam_all", ctypes.c_void_p), ("U_iters", ctypes.c_void_p)]


class BatchPlan:
    """Alg. 1 for many independent problems (uneven n, k, b) sharing B, L and T.

    problems: list of dicts with keys S ([B][b] complex64 colliding sketches), h, g ([B][n] or
    [B][1][n]) and U0 ([k][L][n] float32), all on one CUDA device.  run() only enqueues work on
    the current stream (capturable into a CUDA graph); results[i] holds lam, V, tau (and, with
    trace=True, lam_all and U_iters) of problem i after the stream has synchronised."""

    def __init__(self, problems, B: int, L: int, T: int, autotune: bool = True, trace: bool = False):
        self.lib = _lib.load()
        self.device = problems[0]["S"].device
        self.B, self.L, self.T = B, L, T
        self._keep = []
        self.results = []
        arr = (_Problem * len(problems))()
        for i, p in enumerate(problems):
            S = _need(p["S"], "S", torch.complex64, self.device)
            h, g = _hashes_shape(p["h"], p["g"])
            _need(h, "h", torch.int32, self.device)
            _need(g, "g", torch.uint8, self.device)
            U0 = _need(p["U0"], "U0", torch.float32, self.device)
            k, L_, n = U0.shape
            if S.shape[0] != B or L_ != L or h.shape != (B, 1, n):
                raise ValueError(f"problem {i}: shapes do not match B={B}, L={L}")
            b = S.shape[1]
            res = {"lam": torch.empty((k,), dtype=torch.float64, device=self.device),
                   "V": torch.empty((k, n), dtype=torch.float32, device=self.device),
                   "tau": torch.empty((k,), dtype=torch.int32, device=self.device)}
            if trace:
                res["lam_all"] = torch.empty((k, L), dtype=torch.float32, device=self.device)
                res["U_iters"] = torch.empty((k, T, L, n), dtype=torch.float32, device=self.device)
            self.results.append(res)
            self._keep.extend([S, h, g, U0])
            arr[i] = _Problem(S.data_ptr(), h.data_ptr(), g.data_ptr(), U0.data_ptr(), n, k,
                              b.bit_length() - 1, res["lam"].data_ptr(), res["V"].data_ptr(),
                              res["tau"].data_ptr(),
                              res["lam_all"].data_ptr() if trace else 0,
                              res["U_iters"].data_ptr() if trace else 0)
        self._arr = arr
        handle = ctypes.c_void_p()
        rc = self.lib.tsk_batch_create(_ctx(self.device), arr, len(problems), B, L, T,
                                       int(bool(autotune)), ctypes.byref(handle))
        _lib.check("tsk_batch_create", rc)
        self.handle = handle.value

    def block_size(self, log2b: int) -> int:
        return self.lib.tsk_batch_block_size(ctypes.c_void_p(self.handle), log2b)

    def run(self) -> None:
        rc = self.lib.tsk_batch_run(_ctx(self.device), ctypes.c_void_p(self.handle))
        _lib.check("tsk_batch_run", rc)

    def close(self) -> None:
        if getattr(self, "handle", None):
            torch.cuda.synchronize(self.device)
            self.lib.tsk_batch_destroy(ctypes.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ spectral LDA (App. D, Alg. 3)
def _corpus(indptr: torch.Tensor, idx: torch.Tensor, cnt: torch.Tensor, V: int):
    """Check a device CSR corpus; returns (device, D, idx, cnt) with a one-element stand-in for
    empty idx/cnt arrays (the library wants non-null pointers)."""
    device = indptr.device
    _need(indptr, "indptr", torch.int64, device)
    if indptr.dim() != 1 or indptr.numel() < 1:
        raise ValueError("indptr must be a 1-D int64 tensor of D + 1 offsets")
    _need(idx, "idx", torch.int32, device)
    _need(cnt, "cnt", torch.int32, device)
    if idx.shape != cnt.shape or idx.dim() != 1:
        raise ValueError("idx and cnt must be 1-D of equal length")
    if idx.numel() == 0:
        idx = torch.zeros(1, dtype=torch.int32, device=device)
        cnt = torch.ones(1, dtype=torch.int32, device=device)
    if int(V) < 1:
        raise ValueError("V must be >= 1")
    return device, indptr.numel() - 1, idx, cnt


def lda_m2_apply(indptr, idx, cnt, V: int, alpha0: float, X: torch.Tensor) -> torch.Tensor:
    """M2^ X (Eq. moment2) for X [V][c] without forming M2^."""
    device, D, idx, cnt = _corpus(indptr, idx, cnt, V)
    _need(X, "X", torch.float32, device)
    c = X.shape[1]
    if X.shape[0] != V:
        raise ValueError("X must have V rows")
    Y = torch.empty_like(X)
    rc = _lib.load().lda_m2_apply(_ctx(device), _ptr(indptr), _ptr(idx), _ptr(cnt), D, V,
                                  float(alpha0), _ptr(X), c, _ptr(Y))
    _lib.check("lda_m2_apply", rc)
    return Y


def lda_whiten(indptr, idx, cnt, V: int, k: int, alpha0: float, Omega: torch.Tensor,
               power_iters: int = 2):
    """Alg. 3, line 3: W [V][k] with W^T M2^ W = I from the k leading eigenpairs of M2^
    (randomized subspace iteration from Omega [V][c]).  Returns (W, sigma [k] float64, M1 [V])."""
    device, D, idx, cnt = _corpus(indptr, idx, cnt, V)
    _need(Omega, "Omega", torch.float32, device)
    if Omega.dim() != 2 or Omega.shape[0] != V:
        raise ValueError("Omega must be [V][c]")
    c = Omega.shape[1]
    W = torch.empty((V, k), dtype=torch.float32, device=device)
    sigma = torch.empty((k,), dtype=torch.float64, device=device)
    M1 = torch.empty((V,), dtype=torch.float32, device=device)
    rc = _lib.load().lda_whiten(_ctx(device), _ptr(indptr), _ptr(idx), _ptr(cnt), D, V, k,
                                float(alpha0), _ptr(Omega), c, int(power_iters), _ptr(W),
                                _ptr(sigma), _ptr(M1))
    _lib.check("lda_whiten", rc)
    return W, sigma, M1


def lda_whitened_m3(indptr, idx, cnt, V: int, W: torch.Tensor, alpha0: float) -> torch.Tensor:
    """M3^(W, W, W), dense k x k x k (Alg. 3, line 4; Eq. moment3 with Eq. td)."""
    device, D, idx, cnt = _corpus(indptr, idx, cnt, V)
    _need(W, "W", torch.float32, device)
    if W.dim() != 2 or W.shape[0] != V:
        raise ValueError("W must be [V][k]")
    k = W.shape[1]
    M3 = torch.empty((k, k, k), dtype=torch.float32, device=device)
    rc = _lib.load().lda_whitened_m3(_ctx(device), _ptr(indptr), _ptr(idx), _ptr(cnt), D, V,
                                     _ptr(W), k, float(alpha0), _ptr(M3))
    _lib.check("lda_whitened_m3", rc)
    return M3


def lda_sketch_m3(indptr, idx, cnt, V: int, W: torch.Tensor, alpha0: float, h: torch.Tensor,
                  g: torch.Tensor, log2b: int):
    """B colliding sketches of M3^(W, W, W) (Alg. 3, line 4).  Returns (M3, S [B][b])."""
    device, D, idx, cnt = _corpus(indptr, idx, cnt, V)
    _need(W, "W", torch.float32, device)
    k = W.shape[1]
    h, g = _hashes_shape(h, g)
    _need(h, "h", torch.int32, device)
    _need(g, "g", torch.uint8, device)
    B = h.shape[0]
    if h.shape != (B, 1, k):
        raise ValueError(f"h must have shape [B][1][{k}]")
    M3 = torch.empty((k, k, k), dtype=torch.float32, device=device)
    S = torch.empty((B, 1 << log2b), dtype=torch.complex64, device=device)
    rc = _lib.load().lda_sketch_m3(_ctx(device), _ptr(indptr), _ptr(idx), _ptr(cnt), D, V,
                                   _ptr(W), k, float(alpha0), _ptr(h), _ptr(g), B, log2b,
                                   _ptr(M3), _ptr(S))
    _lib.check("lda_sketch_m3", rc)
    return M3, S


def lda_recover(W: torch.Tensor, alpha0: float, lam: torch.Tensor, Vv: torch.Tensor):
    """Alg. 3, line 6: (alpha_hat [k] float64, mu_hat [k][V], row i = topic i)."""
    device = W.device
    _need(W, "W", torch.float32, device)
    V, k = W.shape
    _need(lam, "lam", torch.float64, device, (k,))
    _need(Vv, "Vv", torch.float32, device, (k, k))
    alpha = torch.empty((k,), dtype=torch.float64, device=device)
    mu = torch.empty((k, V), dtype=torch.float32, device=device)
    rc = _lib.load().lda_recover(_ctx(device), _ptr(W), V, k, float(alpha0), _ptr(lam), _ptr(Vv),
                                 _ptr(alpha), _ptr(mu))
    _lib.check("lda_recover", rc)
    return alpha, mu


def spectral_lda(indptr, idx, cnt, V: int, k: int, alpha0: float, Omega: torch.Tensor,
                 U0: torch.Tensor, *, B: int, log2b: int, T: int, seed: int,
                 power_iters: int = 2):
    """Fast spectral LDA (Alg. 3) on the device: whitening, B colliding sketches of
    M3^(W,W,W), Alg. 1 with initial vectors U0 [k][L][k], recovery.
    Returns dict(alpha [k] float64, mu [k][V], lam [k] float64, V [k][k], W, sigma)."""
    W, sigma, _ = lda_whiten(indptr, idx, cnt, V, k, alpha0, Omega, power_iters)
    h, g = cs_hashes(seed, B, log2b, [k], W.device)
    _, S = lda_sketch_m3(indptr, idx, cnt, V, W, alpha0, h, g, log2b)
    res = robust_power_method(S, h, g, U0, T)
    alpha, mu = lda_recover(W, alpha0, res["lam"], res["V"])
    return {"alpha": alpha, "mu": mu, "lam": res["lam"], "V": res["V"], "W": W, "sigma": sigma}


# ------------------------------------------------------------------ order-p symmetric sketches
def cs_hashes_p(seed: int, B: int, log2b: int, p: int, n: int, device="cuda"):
    """Order-p colliding hashes: (h int32 [B][n] in [0, b), g uint8 [B][n] in [0, m)), with h
    (2p)-wise independent and sigma = exp(2 pi i g / m), m = 4 (p = 3) or 8 (p = 4..6)."""
    device = torch.device(device)
    h = torch.empty((B, n), dtype=torch.int32, device=device)
    g = torch.empty((B, n), dtype=torch.uint8, device=device)
    rc = _lib.load().cs_hashes_p(_ctx(device), ctypes.c_uint64(seed & (2**64 - 1)), B, log2b, p, n,
                                 _ptr(h), _ptr(g))
    _lib.check("cs_hashes_p", rc)
    return h, g


def sketch_tensor_p(T: torch.Tensor, h: torch.Tensor, g: torch.Tensor, log2b: int,
                    symmetric: bool = False):
    """Order-p colliding sketches (complex64 [B][b]) of a dense float32 tensor T (p = T.dim()).
    symmetric=True reads only i_1 <= ... <= i_p with multinomial weights (T must be symmetric);
    otherwise every entry is read."""
    device = T.device
    _need(T, "T", torch.float32, device)
    _need(h, "h", torch.int32, device)
    _need(g, "g", torch.uint8, device)
    p, n = T.dim(), T.shape[0]
    B = h.shape[0]
    if h.shape != (B, n) or g.shape != (B, n) or any(d != n for d in T.shape):
        raise ValueError("T must be n^p and h, g [B][n]")
    S = torch.empty((B, 1 << log2b), dtype=torch.complex64, device=device)
    rc = _lib.load().sketch_tensor_p(_ctx(device), _ptr(T.contiguous()), p, n, _ptr(h), _ptr(g), B,
                                     log2b, int(bool(symmetric)), _ptr(S))
    _lib.check("sketch_tensor_p", rc)
    return S


def contract_p(FS: torch.Tensor, S: torch.Tensor, h: torch.Tensor, g: torch.Tensor, U: torch.Tensor,
               p: int, per_sketch: bool = False, medians: bool = True):
    """Sketched T(I,u,...,u) and T(u,...,u) of order p for the rows of U [L][n] against B
    sketches (FS = DFT of S, both complex64 [B][b]).  Returns dict(Vmed [L][n], lam_med [L]
    [, Vall [L][B][n], lam_all [L][B]]); medians=False (with per_sketch) skips the medians."""
    if not medians and not per_sketch:
        raise ValueError("medians=False needs per_sketch=True")
    device = S.device
    for t, nm in ((FS, "FS"), (S, "S")):
        _need(t, nm, torch.complex64, device)
    _need(U, "U", torch.float32, device)
    B, b = S.shape
    L, n = U.shape
    Vmed = torch.empty((L, n), dtype=torch.float32, device=device) if medians else None
    lam_med = torch.empty((L,), dtype=torch.float32, device=device) if medians else None
    Vall = torch.empty((L, B, n), dtype=torch.float32, device=device) if per_sketch else None
    lam_all = torch.empty((L, B), dtype=torch.float32, device=device) if per_sketch else None
    rc = _lib.load().contract_p(_ctx(device), _ptr(FS), _ptr(S), _ptr(h), _ptr(g), B,
                                b.bit_length() - 1, p, _ptr(U), L, n, _ptr(Vmed), _ptr(Vall),
                                _ptr(lam_med), _ptr(lam_all))
    _lib.check("contract_p", rc)
    out = {"Vmed": Vmed, "lam_med": lam_med} if medians else {}
    if per_sketch:
        out["Vall"], out["lam_all"] = Vall, lam_all
    return out


def robust_power_method_p(S: torch.Tensor, h: torch.Tensor, g: torch.Tensor, U0: torch.Tensor,
                          T: int, p: int, return_deflated: bool = False, return_trace: bool = False):
    """Alg. 1 for order p on B colliding sketches S [B][b] with hashes h, g [B][n] and initial
    vectors U0 [k][L][n].  Returns as robust_power_method."""
    device = S.device
    _need(S, "S", torch.complex64, device)
    _need(h, "h", torch.int32, device)
    _need(g, "g", torch.uint8, device)
    _need(U0, "U0", torch.float32, device)
    B, b = S.shape
    k, L, n = U0.shape
    if h.shape != (B, n) or g.shape != (B, n):
        raise ValueError(f"h and g must have shape [{B}][{n}]")
    lam = torch.empty((k,), dtype=torch.float64, device=device)
    V = torch.empty((k, n), dtype=torch.float32, device=device)
    tau = torch.empty((k,), dtype=torch.int32, device=device)
    Sd = torch.empty_like(S) if return_deflated else None
    lam_all = torch.empty((k, L), dtype=torch.float32, device=device) if return_trace else None
    U_iters = (torch.empty((k, int(T), L, n), dtype=torch.float32, device=device)
               if return_trace else None)
    rc = _lib.load().robust_power_method_p(_ctx(device), _ptr(S), _ptr(h), _ptr(g), B,
                                           b.bit_length() - 1, p, n, k, L, int(T), _ptr(U0),
                                           _ptr(lam), _ptr(V), _ptr(tau), _ptr(Sd), _ptr(lam_all),
                                           _ptr(U_iters))
    _lib.check("robust_power_method_p", rc)
    out = {"lam": lam, "V": V, "tau": tau}
    if return_deflated:
        out["S_deflated"] = Sd
    if return_trace:
        out["lam_all"], out["U_iters"] = lam_all, U_iters
    return out


def robust_power_method_p_launches(p: int, k: int, T: int, device="cuda") -> int:
    """Kernel launches robust_power_method_p makes (the figure bench.py reports)."""
    return int(_lib.load().robust_power_method_p_launches(_ctx(torch.device(device)), p, k, T))
