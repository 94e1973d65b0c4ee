"""Torch-facing binding of libmttkrp: argument marshalling only.

Tensors are torch CUDA tensors (device memory); every computation runs in the
library's CUDA kernels on the current torch stream.  Tensors are flat FP32
arrays in the natural linearization (mode 0 fastest, Section 2.1 of the
paper); factor matrices are ``I_k x C`` FP32 row-major; Gram matrices FP64.
"""
from __future__ import annotations

from typing import Optional, Sequence

import torch

from . import _lib as L

ALGOS = {"auto": L.ALGO_AUTO, "fused": L.ALGO_FUSED, "materialized": L.ALGO_MATERIALIZED,
         "two_step": L.ALGO_TWO_STEP}
PRECISIONS = {"auto": L.PREC_AUTO, "fp32": L.PREC_FP32, "bf16x2": L.PREC_BF16X2,
              "bf16x3": L.PREC_BF16X3}


def _stream(dev) -> int:
    return torch.cuda.current_stream(dev).cuda_stream


def _req(t: torch.Tensor, dtype, name: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _req_src(t: torch.Tensor, name: str) -> torch.Tensor:
    """A tensor the library reads in place: a CUDA tensor, or a pinned host tensor (read
    through its mapping into the device address space)."""
    if isinstance(t, torch.Tensor) and not t.is_cuda and t.is_pinned():
        if t.dtype != torch.float32:
            raise TypeError(f"{name} must be {torch.float32}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        return t
    return _req(t, torch.float32, name)


def _opts(algo="auto", precision="auto", splits=0):
    return L.opts(ALGOS[algo] if isinstance(algo, str) else algo,
                  PRECISIONS[precision] if isinstance(precision, str) else precision, splits)


class Workspace:
    """A device byte buffer owned by the caller side (torch), grown on demand.
    The first 256 bytes are the library's status word, zeroed at allocation."""

    def __init__(self, device=None):
        self.device = torch.device(device if device is not None else "cuda")
        self.buf = None

    def get(self, nbytes: int) -> torch.Tensor:
        nbytes = max(int(nbytes), 256)
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = torch.zeros(nbytes, dtype=torch.uint8, device=self.device)
        return self.buf

    def ptr(self, nbytes: int):
        b = self.get(nbytes)
        return b.data_ptr(), b.numel()

    def status(self) -> int:
        """Synchronise the stream and return the device status word (0 = ok)."""
        if self.buf is None:
            return 0
        bits = L.ctypes.c_uint32(0)
        return L.load().mtk_read_status(self.buf.data_ptr(), _stream(self.device), L.ctypes.byref(bits))

    def clear(self):
        if self.buf is not None:
            L.check(L.load().mtk_clear_status(self.buf.data_ptr(), _stream(self.device)), "clear_status")


_default_ws = {}


def default_workspace(device) -> Workspace:
    d = torch.device(device)
    key = d.index if d.index is not None else torch.cuda.current_device()
    if key not in _default_ws:
        _default_ws[key] = Workspace(torch.device("cuda", key))
    return _default_ws[key]


def _factor_ptrs(U, dims, C, skip=None):
    ptrs = []
    for k, u in enumerate(U):
        if k == skip and u is None:
            ptrs.append(None)
            continue
        _req(u, torch.float32, f"U[{k}]")
        if tuple(u.shape) != (int(dims[k]), C):
            raise ValueError(f"U[{k}] must be {int(dims[k])} x {C}, got {tuple(u.shape)}")
        ptrs.append(u.data_ptr())
    return ptrs


def _rank(U, skip=None):
    for k, u in enumerate(U):
        if u is not None and k != skip:
            return int(u.shape[1])
    for u in U:
        if u is not None:
            return int(u.shape[1])
    raise ValueError("no factor matrix given")


def split_tensor(X: torch.Tensor, dims: Sequence[int], *, out: Optional[torch.Tensor] = None,
                 normX2: Optional[torch.Tensor] = None, ws: Optional[Workspace] = None,
                 device=None):
    """Split an FP32 tensor (natural order, dims) into its two BF16 planes (hi, lo) for
    mtk_mttkrp_split, mode 0 padded to a multiple of 8.  Returns (Xs, normX2): Xs an int16
    tensor holding the planes' 16-bit words, normX2 a device FP64 scalar with ||X||^2 from
    the same pass.  X may be a pinned host tensor: the split then reads it in place over the
    host link (one pass, no device copy of X); the planes go to `device` (default: the
    device of `out`, else the current CUDA device)."""
    _req_src(X, "X")
    if X.is_cuda:
        device = X.device
    elif device is None:
        device = out.device if out is not None else torch.device("cuda", torch.cuda.current_device())
    device = torch.device(device)
    lib = L.load()
    dims = [int(d) for d in dims]
    d = L.dims_arr(dims)
    nb = lib.mtk_split_bytes(d, len(dims))
    if nb == 0:
        raise ValueError(f"invalid dims {dims}")
    n = 1
    for v in dims:
        n *= v
    if X.numel() < n:
        raise ValueError("X is smaller than dims")
    nwords = nb // 2
    if out is None:
        out = torch.empty(nwords, dtype=torch.int16, device=device)
    _req(out, torch.int16, "out")
    if out.numel() < nwords:
        raise ValueError(f"split planes need {nwords} 16-bit words")
    if normX2 is None:
        normX2 = torch.empty((), dtype=torch.float64, device=device)
    ws = ws or default_workspace(device)
    wp, wb = ws.ptr(lib.mtk_split_workspace(d, len(dims)))
    L.check(lib.mtk_split_tensor(X.data_ptr(), d, len(dims), out.data_ptr(), normX2.data_ptr(), wp, wb,
                                 _stream(device)), "mtk_split_tensor")
    return out, normX2


def mttkrp(X: Optional[torch.Tensor], dims: Sequence[int], U: Sequence[Optional[torch.Tensor]], n: int, *,
           algo="auto", precision="auto", splits=0, out: Optional[torch.Tensor] = None,
           ws: Optional[Workspace] = None, Xs: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Mode-n MTTKRP M = X_(n) (U_{N-1} kr ... kr U_{n+1} kr U_{n-1} kr ... kr U_0).
    With Xs (the planes from split_tensor) the tensor is read from its BF16 planes
    (mtk_mttkrp_split); X may then be None for shapes the planes kernel takes."""
    if Xs is not None:
        return _mttkrp_split(Xs, X, dims, U, n, algo=algo, precision=precision, splits=splits, out=out, ws=ws)
    _req(X, torch.float32, "X")
    dims = [int(d) for d in dims]
    N = len(dims)
    C = _rank(U, skip=n)
    if X.numel() != int(torch.tensor(dims).prod()):
        raise ValueError("X does not match dims")
    ptrs = _factor_ptrs(U, dims, C, skip=n)
    if out is None:
        out = torch.empty((dims[n], C), dtype=torch.float32, device=X.device)
    _req(out, torch.float32, "out")
    o = _opts(algo, precision, splits)
    lib = L.load()
    d = L.dims_arr(dims)
    need = lib.mtk_mttkrp_workspace(d, N, C, n, L.ctypes.byref(o))
    if need == 0:
        raise ValueError("invalid MTTKRP shape or options")
    ws = ws or default_workspace(X.device)
    wp, wb = ws.ptr(need)
    L.check(lib.mtk_mttkrp(X.data_ptr(), d, N, L.ptr_arr(ptrs), C, n, out.data_ptr(), wp, wb,
                           L.ctypes.byref(o), _stream(X.device)), "mtk_mttkrp")
    return out


def _mttkrp_split(Xs, X, dims, U, n, *, algo, precision, splits, out, ws):
    _req(Xs, torch.int16, "Xs")
    if X is not None:
        _req(X, torch.float32, "X")
    dims = [int(d) for d in dims]
    N = len(dims)
    C = _rank(U, skip=n)
    ptrs = _factor_ptrs(U, dims, C, skip=n)
    lib = L.load()
    if Xs.numel() * 2 < lib.mtk_split_bytes(L.dims_arr(dims), N):
        raise ValueError("Xs is too small for dims")
    if out is None:
        out = torch.empty((dims[n], C), dtype=torch.float32, device=Xs.device)
    _req(out, torch.float32, "out")
    o = _opts(algo, precision, splits)
    d = L.dims_arr(dims)
    need = lib.mtk_mttkrp_split_workspace(d, N, C, n, L.ctypes.byref(o))
    if need == 0:
        raise ValueError("invalid MTTKRP shape or options for the split tensor")
    ws = ws or default_workspace(Xs.device)
    wp, wb = ws.ptr(need)
    L.check(lib.mtk_mttkrp_split(Xs.data_ptr(), X.data_ptr() if X is not None else None, d, N, L.ptr_arr(ptrs), C,
                                 n, out.data_ptr(), wp, wb, L.ctypes.byref(o), _stream(Xs.device)),
            "mtk_mttkrp_split")
    return out


def pack_symmetric(X: torch.Tensor, dims: Sequence[int], *, diag: bool = True,
                   out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """The packed form of a tensor symmetric in modes 0 and 1 (mtk_pack_symmetric): the
    entries with i_0 >= i_1 (diag) or i_0 > i_1 (not diag), flat, Pp * prod(dims[2:]) floats."""
    _req(X, torch.float32, "X")
    dims = [int(d) for d in dims]
    lib = L.load()
    rest = 1
    for d in dims[2:]:
        rest *= d
    n = lib.mtk_sym_packed_rows(dims[0], int(diag)) * rest
    if out is None:
        out = torch.empty(n, dtype=torch.float32, device=X.device)
    _req(out, torch.float32, "out")
    if out.numel() < n:
        raise ValueError(f"the packed tensor needs {n} floats")
    L.check(lib.mtk_pack_symmetric(X.data_ptr(), L.dims_arr(dims), len(dims), int(diag), out.data_ptr(),
                                   _stream(X.device)), "mtk_pack_symmetric")
    return out


def sym_packed_dims(dims: Sequence[int], *, diag: bool = True):
    """Dims of the packed tensor: [Pp] + dims[2:], Pp = mtk_sym_packed_rows(dims[0], diag)
    (what split_tensor takes for pack_symmetric's output)."""
    dims = [int(d) for d in dims]
    return [L.load().mtk_sym_packed_rows(dims[0], int(diag))] + dims[2:]


def mttkrp_sym(Xps: torch.Tensor, dims: Sequence[int], U: Sequence[Optional[torch.Tensor]], n: int, *,
               diag: bool = True, splits=0, out: Optional[torch.Tensor] = None,
               ws: Optional[Workspace] = None) -> torch.Tensor:
    """Mode-n MTTKRP of a tensor symmetric in modes 0 and 1, from the BF16 planes of its
    packed form (split_tensor of pack_symmetric's output with sym_packed_dims, same diag);
    dims are the full
    tensor's.  Without diag the tensor's diagonal i_0 = i_1 counts as zero."""
    _req(Xps, torch.int16, "Xps")
    dims = [int(d) for d in dims]
    N = len(dims)
    C = _rank(U, skip=n)
    ptrs = _factor_ptrs(U, dims, C, skip=n)
    if out is None:
        out = torch.empty((dims[n], C), dtype=torch.float32, device=Xps.device)
    _req(out, torch.float32, "out")
    o = _opts("auto", "auto", splits)
    lib = L.load()
    d = L.dims_arr(dims)
    need = lib.mtk_mttkrp_sym_split_workspace(d, N, int(diag), C, n, L.ctypes.byref(o))
    if need == 0:
        raise L.MtkError(L.MTK_EUNSUPPORTED, "mtk_mttkrp_sym_split_workspace")
    ws = ws or default_workspace(Xps.device)
    wp, wb = ws.ptr(need)
    L.check(lib.mtk_mttkrp_sym_split(Xps.data_ptr(), d, N, int(diag), L.ptr_arr(ptrs), C, n, out.data_ptr(), wp, wb,
                                     L.ctypes.byref(o), _stream(Xps.device)), "mtk_mttkrp_sym_split")
    return out


def ffma_probe(ctas_per_sm: int = 8, iters: int = 4096, *, device=None,
               out: Optional[torch.Tensor] = None) -> float:
    """Launch the FP32 FMA throughput probe (mtk_ffma_probe) on the current stream and
    return the floating-point operations it performs; the caller times it."""
    dev = torch.device(device if device is not None else "cuda")
    lib = L.load()
    n = lib.mtk_ffma_probe_out_floats(ctas_per_sm)
    if out is None:
        out = torch.empty(max(n, 1), dtype=torch.float32, device=dev)
    flops = L.ctypes.c_double(0.0)
    L.check(lib.mtk_ffma_probe(ctas_per_sm, iters, out.data_ptr(), L.ctypes.byref(flops), _stream(dev)),
            "mtk_ffma_probe")
    return flops.value


def khatri_rao(U: Sequence[torch.Tensor], *, reuse: bool = True,
               out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """K = U_0 kr ... kr U_{Z-1}, last operand's row index fastest (Section 4.1)."""
    C = int(U[0].shape[1])
    rows = [int(u.shape[0]) for u in U]
    for k, u in enumerate(U):
        _req(u, torch.float32, f"U[{k}]")
        if int(u.shape[1]) != C:
            raise ValueError("all operands need the same number of columns")
    J = 1
    for r in rows:
        J *= r
    if out is None:
        out = torch.empty((J, C), dtype=torch.float32, device=U[0].device)
    _req(out, torch.float32, "out")
    L.check(L.load().mtk_khatri_rao(L.ptr_arr([u.data_ptr() for u in U]), L.dims_arr(rows), len(U), C,
                                    out.data_ptr(), 1 if reuse else 0, _stream(U[0].device)),
            "mtk_khatri_rao")
    return out


def partial_mttkrp(X, dims, Kp, n, right: bool, *, precision="auto", splits=0, out=None, ws=None):
    """First step of Algorithm 4 (see include/mttkrp.h for the output layout)."""
    _req(X, torch.float32, "X")
    _req(Kp, torch.float32, "Kp")
    dims = [int(d) for d in dims]
    N = len(dims)
    C = int(Kp.shape[1])
    IL = 1
    for d in dims[:n]:
        IL *= d
    IR = 1
    for d in dims[n + 1:]:
        IR *= d
    size = (IL * dims[n] if right else dims[n] * IR) * C
    if out is None:
        out = torch.empty(size, dtype=torch.float32, device=X.device)
    o = _opts("auto", precision, splits)
    lib = L.load()
    d = L.dims_arr(dims)
    need = lib.mtk_partial_mttkrp_workspace(d, N, C, n, 1 if right else 0, L.ctypes.byref(o))
    ws = ws or default_workspace(X.device)
    wp, wb = ws.ptr(need)
    L.check(lib.mtk_partial_mttkrp(X.data_ptr(), d, N, Kp.data_ptr(), C, n, 1 if right else 0,
                                   out.data_ptr(), wp, wb, L.ctypes.byref(o), _stream(X.device)),
            "mtk_partial_mttkrp")
    return out


def partial_mttkrp_split(Xs, dims, U, n, right: bool, *, splits=0, out=None, ws=None):
    """First step of Algorithm 4 on the tensor's BF16 planes (mtk_partial_mttkrp_split).

    U is the list of factors (entries on the side that is not contracted may be None);
    the partial KRP is formed inside the contraction.  Returns T with the layout of
    partial_mttkrp (flat, C slowest)."""
    _req(Xs, torch.int16, "Xs")
    dims = [int(d) for d in dims]
    N = len(dims)
    side = range(n + 1, N) if right else range(0, n)
    if len(side) == 0:
        raise ValueError("no modes to contract on that side of n")
    C = _rank([U[k] for k in side])
    ptrs = [None] * N
    for k in side:
        _req(U[k], torch.float32, f"U[{k}]")
        if tuple(U[k].shape) != (dims[k], C):
            raise ValueError(f"U[{k}] must be {dims[k]} x {C}")
        ptrs[k] = U[k].data_ptr()
    IL = 1
    for d in dims[:n]:
        IL *= d
    IR = 1
    for d in dims[n + 1:]:
        IR *= d
    size = (IL * dims[n] if right else dims[n] * IR) * C
    if out is None:
        out = torch.empty(size, dtype=torch.float32, device=Xs.device)
    _req(out, torch.float32, "out")
    if out.numel() < size:
        raise ValueError("out is too small")
    lib = L.load()
    if Xs.numel() * 2 < lib.mtk_split_bytes(L.dims_arr(dims), N):
        raise ValueError("Xs is too small for dims")
    o = _opts("auto", "auto", splits)
    d = L.dims_arr(dims)
    r = 1 if right else 0
    need = lib.mtk_partial_mttkrp_split_workspace(d, N, C, n, r, L.ctypes.byref(o))
    if need == 0:
        raise L.MtkError(L.MTK_EUNSUPPORTED, "mtk_partial_mttkrp_split_workspace")
    ws = ws or default_workspace(Xs.device)
    wp, wb = ws.ptr(need)
    L.check(lib.mtk_partial_mttkrp_split(Xs.data_ptr(), d, N, L.ptr_arr(ptrs), C, n, r, out.data_ptr(), wp, wb,
                                         L.ctypes.byref(o), _stream(Xs.device)),
            "mtk_partial_mttkrp_split")
    return out


def multi_ttv(T, dims, Ko, n, right: bool, *, out=None):
    """Second step of Algorithm 4."""
    _req(T, torch.float32, "T")
    _req(Ko, torch.float32, "Ko")
    dims = [int(d) for d in dims]
    C = int(Ko.shape[1])
    if out is None:
        out = torch.empty((dims[n], C), dtype=torch.float32, device=T.device)
    L.check(L.load().mtk_multi_ttv(T.data_ptr(), L.dims_arr(dims), len(dims), Ko.data_ptr(), C, n,
                                   1 if right else 0, out.data_ptr(), _stream(T.device)), "mtk_multi_ttv")
    return out


def gram(U: torch.Tensor, *, out=None, ws=None) -> torch.Tensor:
    """G = U^T U in FP64."""
    _req(U, torch.float32, "U")
    I, C = int(U.shape[0]), int(U.shape[1])
    if out is None:
        out = torch.empty((C, C), dtype=torch.float64, device=U.device)
    lib = L.load()
    ws = ws or default_workspace(U.device)
    wp, wb = ws.ptr(lib.mtk_gram_workspace(I, C))
    L.check(lib.mtk_gram(U.data_ptr(), I, C, out.data_ptr(), wp, wb, _stream(U.device)), "mtk_gram")
    return out


def gram_hadamard_solve(G: Sequence[Optional[torch.Tensor]], n: int, M: torch.Tensor, Un: torch.Tensor,
                        *, Gn: Optional[torch.Tensor] = None, ws=None) -> torch.Tensor:
    """U_n = M (Hadamard_{k != n} G_k)^{-1} in place (FP64 Cholesky)."""
    _req(M, torch.float32, "M")
    _req(Un, torch.float32, "Un")
    N = len(G)
    In, C = int(M.shape[0]), int(M.shape[1])
    ptrs = []
    for k, g in enumerate(G):
        if k == n and g is None:
            ptrs.append(None)
        else:
            ptrs.append(_req(g, torch.float64, f"G[{k}]").data_ptr())
    lib = L.load()
    ws = ws or default_workspace(M.device)
    wp, wb = ws.ptr(lib.mtk_solve_workspace(In, C))
    L.check(lib.mtk_gram_hadamard_solve(L.ptr_arr(ptrs), N, C, n, M.data_ptr(), In, Un.data_ptr(),
                                        Gn.data_ptr() if Gn is not None else None, wp, wb,
                                        _stream(M.device)), "mtk_gram_hadamard_solve")
    return Un


def norm2(X: torch.Tensor, *, out=None, ws=None) -> torch.Tensor:
    """||X||^2 in FP64 (device scalar)."""
    _req(X, torch.float32, "X")
    if out is None:
        out = torch.empty((), dtype=torch.float64, device=X.device)
    lib = L.load()
    ws = ws or default_workspace(X.device)
    wp, wb = ws.ptr(lib.mtk_norm2_workspace(X.numel()))
    L.check(lib.mtk_norm2(X.data_ptr(), X.numel(), out.data_ptr(), wp, wb, _stream(X.device)), "mtk_norm2")
    return out


def cp_residual(normX2, M, Um, G, *, r2=None, fit=None):
    """r2 = ||X - [[U]]||^2 via the inner-product identity; fit = 1 - sqrt(r2)/||X||."""
    dev = M.device
    if r2 is None:
        r2 = torch.empty((), dtype=torch.float64, device=dev)
    if fit is None:
        fit = torch.empty((), dtype=torch.float64, device=dev)
    ptrs = [_req(g, torch.float64, "G").data_ptr() for g in G]
    L.check(L.load().mtk_cp_residual(normX2.data_ptr(), _req(M, torch.float32, "M").data_ptr(),
                                     _req(Um, torch.float32, "Um").data_ptr(), int(M.shape[0]),
                                     L.ptr_arr(ptrs), len(G), int(M.shape[1]), r2.data_ptr(),
                                     fit.data_ptr(), _stream(dev)), "mtk_cp_residual")
    return r2, fit


def cp_loss_value(normX2, M, Um, G, *, out=None):
    """f = 0.5 ||X - [[U]]||^2 as an FP32 device scalar (mtk_cp_loss)."""
    dev = M.device
    if out is None:
        out = torch.empty((), dtype=torch.float32, device=dev)
    ptrs = [_req(g, torch.float64, "G").data_ptr() for g in G]
    L.check(L.load().mtk_cp_loss(normX2.data_ptr(), _req(M, torch.float32, "M").data_ptr(),
                                 _req(Um, torch.float32, "Um").data_ptr(), int(M.shape[0]), L.ptr_arr(ptrs),
                                 len(G), int(M.shape[1]), out.data_ptr(), _stream(dev)), "mtk_cp_loss")
    return out


def mttkrp_all(Xs: torch.Tensor, dims: Sequence[int], U: Sequence[torch.Tensor], *, algo="auto",
               out: Optional[Sequence[torch.Tensor]] = None, ws: Optional[Workspace] = None):
    """Every mode's MTTKRP with the same factors, on the tensor's BF16 planes
    (mtk_mttkrp_all_split): the dimension tree for N = 3, 4 unless algo is "fused".
    Returns the list [M_0, ..., M_{N-1}]."""
    _req(Xs, torch.int16, "Xs")
    dims = [int(d) for d in dims]
    N = len(dims)
    C = _rank(U)
    ptrs = _factor_ptrs(U, dims, C)
    if out is None:
        out = [torch.empty((d, C), dtype=torch.float32, device=Xs.device) for d in dims]
    for m in out:
        _req(m, torch.float32, "M")
    o = _opts(algo, "auto", 0)
    lib = L.load()
    d = L.dims_arr(dims)
    need = lib.mtk_mttkrp_all_split_workspace(d, N, C, L.ctypes.byref(o))
    if need == 0:
        raise L.MtkError(L.MTK_EUNSUPPORTED, "mtk_mttkrp_all_split_workspace")
    ws = ws or default_workspace(Xs.device)
    wp, wb = ws.ptr(need)
    L.check(lib.mtk_mttkrp_all_split(Xs.data_ptr(), d, N, L.ptr_arr(ptrs), C, L.ptr_arr([m.data_ptr() for m in out]),
                                     wp, wb, L.ctypes.byref(o), _stream(Xs.device)), "mtk_mttkrp_all_split")
    return list(out)


def cp_gradient(Un, Mn, G, n, *, scale=None, out=None):
    """scale * (U_n Hadamard_{k!=n}(G_k) - M_n)."""
    dev = Un.device
    if out is None:
        out = torch.empty_like(Un)
    ptrs = [None if (k == n and g is None) else _req(g, torch.float64, "G").data_ptr()
            for k, g in enumerate(G)]
    sp = None
    if scale is not None:
        sp = _req(scale, torch.float32, "scale").data_ptr()
    L.check(L.load().mtk_cp_gradient(_req(Un, torch.float32, "Un").data_ptr(),
                                     _req(Mn, torch.float32, "Mn").data_ptr(), L.ptr_arr(ptrs),
                                     len(G), int(Un.shape[1]), n, int(Un.shape[0]), sp, out.data_ptr(),
                                     _stream(dev)), "mtk_cp_gradient")
    return out


def _batch_array(problems):
    """problems: list of (X, dims, U, n, out) with torch CUDA tensors (U[n] may be None)."""
    arr = (L.MtkBatchProblem * len(problems))()
    keep = []
    for p, (X, dims, U, n, out) in enumerate(problems):
        dims = [int(d) for d in dims]
        N = len(dims)
        if N < 2 or N > L.BATCH_MAXN:
            raise ValueError(f"batched problems need 2 <= N <= {L.BATCH_MAXN}")
        C = _rank(U, skip=n)
        _req(X, torch.float32, "X")
        _req(out, torch.float32, "out")
        ptrs = _factor_ptrs(U, dims, C, skip=n)
        arr[p].X = X.data_ptr()
        for k in range(N):
            arr[p].U[k] = ptrs[k]
            arr[p].dims[k] = dims[k]
        arr[p].N, arr[p].n, arr[p].C = N, int(n), C
        arr[p].M = out.data_ptr()
        keep.append((X, U, out))
    return arr, keep


def mttkrp_batched(problems, *, splits=0, ws=None):
    """Every problem (X, dims, U, n, out) of the list in one persistent launch
    (mtk_mttkrp_batched); out is overwritten with the mode-n MTTKRP."""
    arr, _ = _batch_array(problems)
    o = _opts("auto", "auto", splits)
    lib = L.load()
    need = lib.mtk_mttkrp_batched_workspace(arr, len(problems), L.ctypes.byref(o))
    if need == 0:
        raise ValueError("invalid batched MTTKRP problems")
    dev = problems[0][0].device
    ws = ws or default_workspace(dev)
    wp, wb = ws.ptr(need)
    L.check(lib.mtk_mttkrp_batched(arr, len(problems), wp, wb, L.ctypes.byref(o), _stream(dev)),
            "mtk_mttkrp_batched")


class BatchedMTTKRP:
    """A fixed batch of MTTKRP problems (X, dims, U, n, out), run as one persistent launch.

    tune(): the autotuner; it times each candidate number of contraction indices per work
    unit (the k-extent of the tiles) with CUDA events over back-to-back launches and keeps
    the fastest (cached per batch signature for the process).
    capture(): records the launch sequence in a CUDA graph; replay() then runs it."""

    _tuned = {}
    CANDIDATES = (0, 1024, 2048, 4096, 8192, 16384, 32768, 65536)

    def __init__(self, problems, *, splits=0):
        self.problems = list(problems)
        self.parts = [self.problems[i:i + L.BATCH_MAXP] for i in range(0, len(self.problems), L.BATCH_MAXP)]
        self.arrays = [_batch_array(p) for p in self.parts]
        self.device = self.problems[0][0].device
        self.splits = int(splits)
        self.ws = Workspace(self.device)
        self.graph = None
        self.sig = tuple((tuple(int(d) for d in dims), int(n), _rank(U, skip=n)) for _, dims, U, n, _ in self.problems)

    def _need(self, splits):
        lib = L.load()
        o = _opts("auto", "auto", splits)
        need = 0
        for arr, _ in self.arrays:
            w = lib.mtk_mttkrp_batched_workspace(arr, len(arr), L.ctypes.byref(o))
            if w == 0:
                raise ValueError("invalid batched MTTKRP problems")
            need = max(need, w)
        return need

    def run(self, splits=None):
        splits = self.splits if splits is None else int(splits)
        lib = L.load()
        o = _opts("auto", "auto", splits)
        wp, wb = self.ws.ptr(self._need(splits))
        for arr, _ in self.arrays:
            L.check(lib.mtk_mttkrp_batched(arr, len(arr), wp, wb, L.ctypes.byref(o), _stream(self.device)),
                    "mtk_mttkrp_batched")

    def tune(self, reps=5):
        if self.sig in BatchedMTTKRP._tuned:
            self.splits = BatchedMTTKRP._tuned[self.sig]
            return self.splits
        best, best_t = 0, None
        for cand in self.CANDIDATES:
            self.run(cand)
            self.run(cand)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps):
                self.run(cand)
            b.record()
            b.synchronize()
            t = a.elapsed_time(b) / reps
            if best_t is None or t < best_t:
                best, best_t = cand, t
        self.splits = best
        BatchedMTTKRP._tuned[self.sig] = best
        return best

    def capture(self):
        self.ws.get(self._need(self.splits))
        side = torch.cuda.Stream(self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(side):
            self.run()
        torch.cuda.current_stream(self.device).wait_stream(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run()
        self.graph = g
        return g

    def replay(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()


class ALS:
    """CP-ALS driver: holds the workspace, ||X||^2 and the device fit scalar.
    presplit=True splits X into its BF16 planes once (with ||X||^2 in the same pass) and
    runs every MTTKRP on them (mtk_cp_als_sweep_split); precision is then bf16x2.
    normalize=True scales every factor but the last to unit columns after its update (the
    last one carries the weights; the model is the same as without).  capture() records
    one sweep in a CUDA graph, replay() runs it."""

    def __init__(self, X, dims, U, *, algo="auto", precision="auto", splits=0, presplit=False,
                 normalize=False):
        self.presplit = bool(presplit)
        # with presplit, X may be a pinned host tensor: only its planes live on the device
        self.X = _req_src(X, "X") if self.presplit else _req(X, torch.float32, "X")
        self.device = X.device if X.is_cuda else U[0].device
        self.dims = [int(d) for d in dims]
        self.U = list(U)
        self.C = _rank(self.U)
        _factor_ptrs(self.U, self.dims, self.C)
        self.opts = _opts(algo, precision, splits)
        self.opts.normalize = int(bool(normalize))
        self.graph = None
        lib = L.load()
        self._d = L.dims_arr(self.dims)
        need = lib.mtk_cp_als_workspace(self._d, len(self.dims), self.C, L.ctypes.byref(self.opts))
        if need == 0:
            raise ValueError("invalid CP-ALS shape or options")
        self.ws = Workspace(self.device)
        self.ws.get(need)
        self.need = need
        self.Xs = None
        if self.presplit:
            self.Xs, self.normX2 = split_tensor(X, self.dims, ws=Workspace(self.device), device=self.device)
        else:
            self.normX2 = norm2(X, ws=Workspace(self.device))
        self.fit = torch.zeros((), dtype=torch.float64, device=self.device)
        self._uptrs = L.ptr_arr([u.data_ptr() for u in self.U])

    def resplit(self, X: Optional[torch.Tensor] = None) -> None:
        """Re-split the tensor (after its contents changed) and refresh ||X||^2.  With X (a
        tensor of the same dims) the planes are made from X instead, which then becomes the
        tensor of the sweep; X may be a pinned host tensor (read in place over the host link,
        so that a new tensor needs no device copy)."""
        if X is not None:
            if not self.presplit:
                raise ValueError("resplit(X) needs presplit=True")
            _req_src(X, "X")
            if X.numel() < self.X.numel():
                raise ValueError("X is smaller than dims")
            self.X = X
        if self.presplit:
            split_tensor(self.X, self.dims, out=self.Xs, normX2=self.normX2, ws=Workspace(self.device),
                         device=self.device)
        else:
            norm2(self.X, out=self.normX2, ws=Workspace(self.device))

    def sweep(self, with_fit: bool = True) -> None:
        lib = L.load()
        wp, wb = self.ws.ptr(self.need)
        nx = self.normX2.data_ptr() if with_fit else None
        fit = self.fit.data_ptr() if with_fit else None
        st = _stream(self.device)
        if self.presplit:
            L.check(lib.mtk_cp_als_sweep_split(self.Xs.data_ptr(), self.X.data_ptr(), self._d, len(self.dims),
                                               self._uptrs, self.C, nx, fit, wp, wb, L.ctypes.byref(self.opts), st),
                    "mtk_cp_als_sweep_split")
        else:
            L.check(lib.mtk_cp_als_sweep(self.X.data_ptr(), self._d, len(self.dims), self._uptrs, self.C, nx, fit,
                                         wp, wb, L.ctypes.byref(self.opts), st), "mtk_cp_als_sweep")

    def capture(self, with_fit: bool = True):
        """Record one sweep in a CUDA graph: its launches with their arguments (factors,
        planes, workspace and fit stay where they are), the programmatic dependencies
        between them included.  replay() then runs the sweep as one graph launch."""
        self.ws.get(self.need)
        side = torch.cuda.Stream(self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=side, capture_error_mode="thread_local"):
            self.sweep(with_fit)
        torch.cuda.current_stream(self.device).wait_stream(side)
        self.graph = g
        return g

    def replay(self) -> None:
        if self.graph is None:
            self.capture()
        self.graph.replay()

    def status(self) -> int:
        return self.ws.status()


def _per_mode(opts):
    """mttkrp options of one mode: on the planes the algorithm is the fused one (the
    dimension tree, algo "two_step", belongs to mttkrp_all); normX2 is the loss's own."""
    drop = {"normX2"}
    if opts.get("Xs") is not None and opts.get("algo") == "two_step":
        drop.add("algo")
    return {k: v for k, v in opts.items() if k not in drop}


class CPLoss(torch.autograd.Function):
    """f(U_0..U_{N-1}) = 0.5 ||X - [[U_0..U_{N-1}]]||^2 with a hand-written backward:
    df/dU_n = U_n Hadamard_{k!=n}(U_k^T U_k) - MTTKRP(X, n), for every mode n.
    X is treated as a constant.  Usage: CPLoss.apply(X, dims, opts_dict, *U).
    With opts["Xs"] (the planes of X from split_tensor) every MTTKRP runs on the planes;
    when the gradients of several factors are wanted, the forward takes all N MTTKRPs at
    once from mttkrp_all (the dimension tree for N >= 3: two passes over the tensor instead
    of N + 1), the loss from the last one, and the backward reuses them.  opts["normX2"]:
    ||X||^2 as a device FP64 scalar computed once (split_tensor returns it), else the
    forward computes it, one more pass over X."""

    @staticmethod
    def forward(ctx, X, dims, opts, *U):
        dims = [int(d) for d in dims]
        N = len(dims)
        opts = dict(opts or {})
        G = [gram(u) for u in U]
        Xs = opts.get("Xs")
        nx2 = opts.get("normX2")
        if nx2 is None:
            nx2 = norm2(X)
        want = [bool(ctx.needs_input_grad[3 + n]) for n in range(N)]
        Ms = None
        if Xs is not None and sum(want[:N - 1]) > 1:
            Ms = mttkrp_all(Xs, dims, list(U), algo=opts.get("algo", "auto"))
            M = Ms[N - 1]
        else:
            M = mttkrp(None if Xs is not None else X, dims, list(U), N - 1, **_per_mode(opts))
        loss = cp_loss_value(nx2, M, U[N - 1], G)
        ctx.save_for_backward(X, *U)
        ctx.dims = dims
        ctx.opts = opts
        ctx.M_last = M
        ctx.Ms = Ms
        ctx.G = G
        return loss

    @staticmethod
    def backward(ctx, go):
        X, *U = ctx.saved_tensors
        dims, opts, G = ctx.dims, ctx.opts, ctx.G
        N = len(dims)
        scale = go.detach().to(torch.float32).contiguous()
        Xs = opts.get("Xs")
        want = [ctx.needs_input_grad[3 + n] for n in range(N)]
        Ms = ctx.Ms                      # every mode's MTTKRP, from the forward
        grads = []
        for n in range(N):
            if not want[n]:
                grads.append(None)
                continue
            if Ms is not None:
                M = Ms[n]
            else:
                M = ctx.M_last if n == N - 1 else mttkrp(None if Xs is not None else X, dims, list(U), n,
                                                         **_per_mode(opts))
            grads.append(cp_gradient(U[n], M, G, n, scale=scale))
        return (None, None, None, *grads)


def cp_loss(X, dims, U, **opts):
    """0.5 ||X - [[U]]||^2 as an autograd scalar (CPLoss); opts go to mttkrp (Xs: the
    planes, which also route the MTTKRPs through mttkrp_all; normX2: ||X||^2 computed
    once)."""
    return CPLoss.apply(X, list(dims), opts, *U)
