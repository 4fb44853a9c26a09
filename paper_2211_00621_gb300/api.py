"""Thin PyTorch binding of the C ABI (include/accel.h): argument marshalling only.

Each function has the name of the C entry point it calls.  Tensors are CUDA tensors
unless stated; device memory (outputs and workspaces) is allocated with PyTorch, and every
call is issued on ``torch.cuda.current_stream()``.  No computation of the path happens
here: every step runs in the library's kernels.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib as L
from ._lib import (  # noqa: F401  (operator ids, re-exported for callers of this module)
    HMM_BF16_SCALED, HMM_FP32_LOG, LOOP_AXPY, LOOP_SCALE, MAP_ABS, MAP_ADD2, MAP_IDENTITY, MAP_MUL2, MAP_NEG,
    MAP_SCALE, MAP_SQ_PLUS_ONE, PAIR_GRAVITY_SOFTENED, RED_ADD, RED_MAX, RED_MIN, RED_MUL,
)

_DT = {torch.int32: L.I32, torch.int64: L.I64, torch.float32: L.F32, torch.float64: L.F64}
_TORCH = {v: k for k, v in _DT.items()}


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


def _dt(t_or_dtype):
    d = t_or_dtype.dtype if isinstance(t_or_dtype, torch.Tensor) else t_or_dtype
    if d not in _DT:
        raise TypeError(f"unsupported dtype {d}")
    return _DT[d]


def _ws(nbytes: int, device):
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def _need_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("libaccel operates on CUDA tensors")


def set_debug(on: bool):
    """Debug mode: the library validates arguments on host and device and synchronizes."""
    L.load().accel_set_debug(1 if on else 0)


def version() -> str:
    return L.load().accel_version().decode()


# ------------------------------------------------------- device status (accelerate mode)
def set_device_status(word: torch.Tensor | None):
    """Register a device int32 tensor (one element, zero) as the status word of the calls made
    afterwards on this thread (None unregisters): device-side errors of those calls (a bounded
    wait that gave up, a sequence longer than max_T) are recorded there, the first one kept."""
    if word is not None:
        _need_cuda(word)
        if word.dtype != torch.int32 or word.numel() < 1:
            raise TypeError("the status word is a CUDA int32 tensor")
    L.check("accel_set_device_status", L.load().accel_set_device_status(_ptr(word)))


def sync_status(word: torch.Tensor, clear: bool = True):
    """Synchronize the current stream and raise AccelError if the status word records a
    device-side error (clearing it first when `clear`)."""
    _need_cuda(word)
    L.check("accel_sync_status", L.load().accel_sync_status(_ptr(word), 1 if clear else 0, _stream()))


def set_watchdog_ns(budget_ns: int):
    """Run-time budget of a persistent single-CTA BF16 forward launch (0 = no limit)."""
    L.load().accel_set_watchdog_ns(int(budget_ns))


def set_sm_budget(n_sms: int):
    """Most SMs the adjoint's forward recursion may occupy on this host thread (0 = all)."""
    L.load().accel_set_sm_budget(int(n_sms))


def get_sm_budget() -> int:
    return int(L.load().accel_get_sm_budget())


def alu_rate(kind: int, iters: int = 4096, device="cuda") -> float:
    """Measured arithmetic rate of the device (operations per second) for one of
    PROBE_FFMA / PROBE_FFMA2 (FP32 flop), PROBE_RSQRT (MUFU ops), PROBE_DFMA (FP64 flop)."""
    lib = L.load()
    n = 2048 * torch.cuda.get_device_properties(device).multi_processor_count
    scratch = torch.empty(n, dtype=torch.float32, device=device)
    rate = C.c_double(0.0)
    L.check("accel_alu_rate", lib.accel_alu_rate(int(kind), int(iters), _ptr(scratch), C.byref(rate), _stream()))
    return rate.value


def hmm_max_length(offsets: torch.Tensor) -> torch.Tensor:
    """The largest sequence length, max_s offsets[s+1] - offsets[s], as a device int64 [1]
    (computed by the library, asynchronously)."""
    _need_cuda(offsets)
    out = torch.empty(1, dtype=torch.int64, device=offsets.device)
    L.check("hmm_max_length", L.load().hmm_max_length(_ptr(offsets), offsets.numel() - 1, _ptr(out), _stream()))
    return out


# ------------------------------------------------------------------------ marshaling
class RaggedTable:
    """Host-side description of a list of sequences: pinned tables of element pointers and
    lengths (what accel_marshal_ragged reads), built once per list."""

    def __init__(self, seqs, dtype):
        self.seqs = list(seqs)          # keeps the pieces alive
        self.dtype = dtype
        self.S = len(self.seqs)
        for s in self.seqs:
            if s.dtype != dtype:
                raise TypeError("all sequences must have the same dtype")
            if not s.is_cuda and s.numel() and not s.is_pinned():
                raise ValueError("host sequences must be in pinned memory")
        # one page-locked buffer [pointers | lengths], which the library's kernels read in place
        tab = torch.tensor([s.data_ptr() if s.numel() else 0 for s in self.seqs] +
                           [int(s.numel()) for s in self.seqs] or [0, 0], dtype=torch.int64).pin_memory()
        n = max(self.S, 1)
        self.ptrs = tab[:n]
        self.lengths = tab[n:]
        self.total = int(self.lengths[:self.S].sum().item()) if self.S else 0


def ragged_table(seqs, dtype=None):
    dtype = dtype or (seqs[0].dtype if len(seqs) else torch.int32)
    return RaggedTable(seqs, dtype)


def accel_marshal_ragged_table(table: RaggedTable, device="cuda", out=None, ws=None):
    """Flatten the sequences of a RaggedTable into (flat data, int64 offsets) on device."""
    lib = L.load()
    if out is None:
        flat = torch.empty(table.total, dtype=table.dtype, device=device)
        offsets = torch.empty(table.S + 1, dtype=torch.int64, device=device)
    else:
        flat, offsets = out
    need = lib.accel_marshal_ragged_workspace_size(table.S)
    if ws is None or ws.numel() < need:
        ws = _ws(need, flat.device if table.total else offsets.device)
    L.check("accel_marshal_ragged", lib.accel_marshal_ragged(C.c_void_p(table.ptrs.data_ptr()),
                                                             C.c_void_p(table.lengths.data_ptr()), table.S,
                                                             _dt(table.dtype), _ptr(flat), _ptr(offsets), _ptr(ws),
                                                             ws.numel(), _stream()))
    return flat, offsets


def accel_marshal_ragged(seqs, dtype=torch.int32, device="cuda"):
    """Flatten a list of 1-D tensors (CUDA, or pinned CPU readable by the device) into
    (flat data, int64 offsets) on ``device``.  Builds a temporary RaggedTable, so it waits for
    the copy of its tables (keep a RaggedTable and call accel_marshal_ragged_table to stay
    asynchronous)."""
    table = RaggedTable(seqs, dtype)
    out = accel_marshal_ragged_table(table, device)
    torch.cuda.current_stream().synchronize()
    return out


def accel_marshal_nested(groups, dtype=torch.int32, device="cuda"):
    """Flatten [[[T]]] -- a list of groups, each a list of 1-D tensors (CUDA, or pinned CPU) --
    into (flat data, int64 sequence offsets [S+1], int64 group offsets [G+1] into them)."""
    lib = L.load()
    seqs = [t for g in groups for t in g]
    table = RaggedTable(seqs, dtype)
    sizes = torch.tensor([len(g) for g in groups] or [0], dtype=torch.int64).pin_memory()
    G = len(groups)
    flat = torch.empty(table.total, dtype=dtype, device=device)
    offsets = torch.empty(table.S + 1, dtype=torch.int64, device=device)
    goffsets = torch.empty(G + 1, dtype=torch.int64, device=device)
    ws = _ws(lib.accel_marshal_nested_workspace_size(table.S, G), device)
    L.check("accel_marshal_nested", lib.accel_marshal_nested(
        C.c_void_p(table.ptrs.data_ptr()), C.c_void_p(table.lengths.data_ptr()), table.S,
        C.c_void_p(sizes.data_ptr()), G, _dt(dtype), _ptr(flat), _ptr(offsets), _ptr(goffsets), _ptr(ws), ws.numel(),
        _stream()))
    torch.cuda.current_stream().synchronize()        # the temporary pinned tables are read in stream order
    return flat, offsets, goffsets


def accel_unmarshal_ragged(flat, offsets, pinned=True):
    """The inverse of accel_marshal_ragged: a list of S tensors, sequence s = flat[offsets[s]
    : offsets[s+1]], each in its own (pinned host, or device if pinned=False) buffer written
    by the kernel.  Synchronizes the stream."""
    lib = L.load()
    _need_cuda(flat, offsets)
    S = offsets.numel() - 1
    off = offsets.cpu().tolist()
    if pinned:
        outs = [torch.empty(off[s + 1] - off[s], dtype=flat.dtype).pin_memory() for s in range(S)]
    else:
        outs = [torch.empty(off[s + 1] - off[s], dtype=flat.dtype, device=flat.device) for s in range(S)]
    ptrs = torch.tensor([o.data_ptr() if o.numel() else 0 for o in outs] or [0], dtype=torch.int64).pin_memory()
    ws = _ws(lib.accel_unmarshal_ragged_workspace_size(S), flat.device)
    L.check("accel_unmarshal_ragged", lib.accel_unmarshal_ragged(_ptr(flat), flat.numel(), _ptr(offsets), S,
                                                                 _dt(flat.dtype), C.c_void_p(ptrs.data_ptr()),
                                                                 _ptr(ws), ws.numel(), _stream()))
    torch.cuda.current_stream().synchronize()
    return outs


def accel_marshal_records(aos: torch.Tensor, fields, inverse_from=None):
    """Records -> structure of arrays.  ``aos`` is a CUDA tensor whose rows are records
    (any dtype; the record size is its row size in bytes); ``fields`` = [(byte offset,
    torch dtype)].  With ``inverse_from`` (list of per-field tensors), writes them back into
    ``aos`` instead and returns ``aos``."""
    lib = L.load()
    _need_cuda(aos)
    n = aos.shape[0]
    rb = aos[0].numel() * aos.element_size() if n else aos.stride(0) * aos.element_size()
    nf = len(fields)
    offs = (C.c_int32 * nf)(*[int(o) for o, _ in fields])
    dts = (C.c_int32 * nf)(*[_dt(d) for _, d in fields])
    if inverse_from is None:
        cols = [torch.empty(n, dtype=d, device=aos.device) for _, d in fields]
    else:
        cols = list(inverse_from)
    ptrs = (C.c_void_p * nf)(*[c.data_ptr() for c in cols])
    L.check("accel_marshal_records", lib.accel_marshal_records(_ptr(aos), n, rb, nf, offs, dts, ptrs,
                                                               1 if inverse_from is not None else 0, _stream()))
    return aos if inverse_from is not None else cols


# ---------------------------------------------------------------------- map / reduce
def accel_map(op: int, x: torch.Tensor, out_dtype=None, y: torch.Tensor | None = None, scalar: float = 0.0):
    lib = L.load()
    _need_cuda(x, y)
    out_dtype = out_dtype or x.dtype
    out = torch.empty(x.numel(), dtype=out_dtype, device=x.device)
    L.check("accel_map", lib.accel_map(op, _dt(x), _ptr(x), _ptr(y), _dt(out_dtype), _ptr(out), x.numel(),
                                       float(scalar), _stream()))
    return out


def accel_reduce(op: int, x: torch.Tensor, out: torch.Tensor | None = None, ws: torch.Tensor | None = None):
    lib = L.load()
    _need_cuda(x)
    if out is None:
        out = torch.empty(1, dtype=x.dtype, device=x.device)
    need = lib.accel_reduce_workspace_size(x.numel(), _dt(x))
    if ws is None or ws.numel() < need:
        ws = _ws(need, x.device)
    L.check("accel_reduce", lib.accel_reduce(op, _dt(x), _ptr(x), x.numel(), _ptr(out), _ptr(ws), ws.numel(),
                                             _stream()))
    return out


def accel_segreduce(op: int, fused_map: int, data: torch.Tensor, offsets: torch.Tensor, out_dtype=None,
                    scalar: float = 0.0, out: torch.Tensor | None = None, ws: torch.Tensor | None = None):
    lib = L.load()
    _need_cuda(data, offsets)
    S = offsets.numel() - 1
    N = data.numel()
    out_dtype = out_dtype or (torch.int64 if data.dtype in (torch.int32, torch.int64) else data.dtype)
    if out is None:
        out = torch.empty(S, dtype=out_dtype, device=data.device)
    need = lib.accel_segreduce_workspace_size(N, S)
    if ws is None or ws.numel() < need:
        ws = _ws(need, data.device)
    L.check("accel_segreduce", lib.accel_segreduce(op, fused_map, _dt(data), _dt(out), _ptr(data), N,
                                                   _ptr(offsets), S, float(scalar), _ptr(out), _ptr(ws),
                                                   ws.numel(), _stream()))
    return out


def _tensor_desc(t: torch.Tensor):
    d = L.accel_tensor()
    d.data = t.data_ptr()
    d.dtype = _dt(t)
    d.rank = t.dim()
    for i in range(min(t.dim(), L.MAX_RANK)):
        d.dims[i] = t.shape[i]
    return d


def accel_loop(body: int, t0: torch.Tensor, t1: torch.Tensor, scalar: float, n: int | None = None):
    """loop n f with a fixed body, in place on t0 (t0, t1 contiguous)."""
    lib = L.load()
    _need_cuda(t0, t1)
    args = (L.accel_tensor * 2)(_tensor_desc(t0), _tensor_desc(t1))
    n = t0.numel() if n is None else n
    L.check("accel_loop", lib.accel_loop(body, n, args, 2, float(scalar), _stream()))
    return t0


# ------------------------------------------------------------------------------- HMM
def _model(log_A, log_B, log_pi):
    m = L.accel_hmm_model()
    m.K = log_A.shape[0]
    m.M = log_B.shape[1]
    m.log_A = log_A.data_ptr()
    m.log_B = log_B.data_ptr()
    m.log_pi = log_pi.data_ptr()
    return m


def hmm_forward(log_A, log_B, log_pi, obs, offsets, precision=L.HMM_FP32_LOG, total_T: int | None = None,
                out=None, ws=None):
    """Per-sequence log-likelihoods (float64 [S]).  log_A [K,K], log_B [K,M], log_pi [K]
    float32; obs int32 flat; offsets int64 [S+1]."""
    lib = L.load()
    _need_cuda(log_A, log_B, log_pi, obs, offsets)
    for t in (log_A, log_B, log_pi):
        if t.dtype != torch.float32 or not t.is_contiguous():
            raise TypeError("HMM parameters must be contiguous float32")
    m = _model(log_A, log_B, log_pi)
    S = offsets.numel() - 1
    total_T = obs.numel() if total_T is None else total_T
    if out is None:
        out = torch.empty(S, dtype=torch.float64, device=obs.device)
    need = lib.hmm_forward_workspace_size(C.byref(m), S, total_T, precision)
    if ws is None or ws.numel() < need:
        ws = _ws(need, obs.device)
    L.check("hmm_forward", lib.hmm_forward(C.byref(m), precision, _ptr(obs), _ptr(offsets), S, total_T, _ptr(out),
                                           _ptr(ws), ws.numel(), _stream()))
    return out


def hmm_adjoint(log_A, log_B, log_pi, obs, offsets, weights=None, max_T: int | None = None, want_loglik=True,
                ws=None):
    """Gradients of sum_s w_s logL_s w.r.t. (log_A, log_B, log_pi) (float32) and logL
    (float64 [S])."""
    lib = L.load()
    _need_cuda(log_A, log_B, log_pi, obs, offsets, weights)
    m = _model(log_A, log_B, log_pi)
    S = offsets.numel() - 1
    K, M = m.K, m.M
    if max_T is None:
        max_T = int(hmm_max_length(offsets).item()) if S else 0
    gA = torch.empty(K, K, dtype=torch.float32, device=obs.device)
    gB = torch.empty(K, M, dtype=torch.float32, device=obs.device)
    gpi = torch.empty(K, dtype=torch.float32, device=obs.device)
    ll = torch.empty(S, dtype=torch.float64, device=obs.device) if want_loglik else None
    need = lib.hmm_adjoint_workspace_size(C.byref(m), S, obs.numel(), max_T)
    if ws is None or ws.numel() < need:
        ws = _ws(need, obs.device)
    if weights is not None and weights.dtype != torch.float64:
        weights = weights.to(torch.float64)
    L.check("hmm_adjoint", lib.hmm_adjoint(C.byref(m), _ptr(obs), _ptr(offsets), S, obs.numel(), max_T,
                                           _ptr(weights), _ptr(ll), _ptr(gA), _ptr(gB), _ptr(gpi), _ptr(ws),
                                           ws.numel(), _stream()))
    return gA, gB, gpi, ll


class AdjointSaved:
    """The state hmm_adjoint_forward leaves for hmm_adjoint_backward: the workspace (with the
    checkpoints of alpha) and the sizes it was made for."""

    def __init__(self, ws, S, total_T, max_T):
        self.ws, self.S, self.total_T, self.max_T = ws, S, total_T, max_T


def hmm_adjoint_forward(log_A, log_B, log_pi, obs, offsets, max_T: int | None = None, out=None):
    """logL (float64 [S]) by the adjoint's checkpointed FP32 forward, and the saved state for
    hmm_adjoint_backward."""
    lib = L.load()
    _need_cuda(log_A, log_B, log_pi, obs, offsets)
    m = _model(log_A, log_B, log_pi)
    S = offsets.numel() - 1
    if max_T is None:
        max_T = int(hmm_max_length(offsets).item()) if S else 0
    ll = torch.empty(S, dtype=torch.float64, device=obs.device) if out is None else out
    ws = _ws(lib.hmm_adjoint_workspace_size(C.byref(m), S, obs.numel(), max_T), obs.device)
    L.check("hmm_adjoint_forward", lib.hmm_adjoint_forward(C.byref(m), _ptr(obs), _ptr(offsets), S, obs.numel(), max_T,
                                                           _ptr(ll), _ptr(ws), ws.numel(), _stream()))
    return ll, AdjointSaved(ws, S, obs.numel(), max_T)


def hmm_adjoint_backward(log_A, log_B, log_pi, obs, offsets, saved: AdjointSaved, weights=None):
    """Gradients (float32 log_A, log_B, log_pi) of sum_s w_s logL_s from the state a previous
    hmm_adjoint_forward call on the same inputs saved."""
    lib = L.load()
    _need_cuda(log_A, log_B, log_pi, obs, offsets, weights)
    m = _model(log_A, log_B, log_pi)
    K, M = m.K, m.M
    gA = torch.empty(K, K, dtype=torch.float32, device=obs.device)
    gB = torch.empty(K, M, dtype=torch.float32, device=obs.device)
    gpi = torch.empty(K, dtype=torch.float32, device=obs.device)
    if weights is not None and weights.dtype != torch.float64:
        weights = weights.to(torch.float64)
    L.check("hmm_adjoint_backward", lib.hmm_adjoint_backward(
        C.byref(m), _ptr(obs), _ptr(offsets), saved.S, saved.total_T, saved.max_T, _ptr(weights), _ptr(gA), _ptr(gB),
        _ptr(gpi), _ptr(saved.ws), saved.ws.numel(), _stream()))
    return gA, gB, gpi


def accel_pair_histogram(A, edges, B=None):
    """Histogram (int64 [len(edges)+1]) of the angular separations of point pairs: A and B
    are float32 [n, 3] unit vectors (CUDA); edges a strictly decreasing float32 sequence of
    cosines.  B=None counts the pairs i < j of A, else every pair (i in A, j in B)."""
    lib = L.load()
    _need_cuda(A, B)
    cols = [A[:, k].contiguous() for k in range(3)]
    bcols = [B[:, k].contiguous() for k in range(3)] if B is not None else cols
    e = torch.as_tensor(edges, dtype=torch.float32).contiguous().cpu()
    hist = torch.empty(e.numel() + 1, dtype=torch.int64, device=A.device)
    L.check("accel_pair_histogram", lib.accel_pair_histogram(
        _ptr(cols[0]), _ptr(cols[1]), _ptr(cols[2]), A.shape[0], _ptr(bcols[0]), _ptr(bcols[1]), _ptr(bcols[2]),
        B.shape[0] if B is not None else A.shape[0], C.c_void_p(e.data_ptr()), e.numel(), _ptr(hist), _stream()))
    return hist


def hmm_forward_long(log_A, log_B, log_pi, obs, offsets, max_T: int | None = None, out=None, ws=None):
    """logL per sequence (float64 [S]) computed parallel-in-T (chunked products of
    A diag(b(o_t))), for few, very long sequences; K <= 64."""
    lib = L.load()
    _need_cuda(log_A, log_B, log_pi, obs, offsets)
    m = _model(log_A, log_B, log_pi)
    S = offsets.numel() - 1
    if max_T is None:
        max_T = int(hmm_max_length(offsets).item()) if S else 0
    need = lib.hmm_forward_long_workspace_size(C.byref(m), S, obs.numel(), max_T)
    if ws is None or ws.numel() < need:
        ws = _ws(need, obs.device)
    if out is None:
        out = torch.empty(S, dtype=torch.float64, device=obs.device)
    L.check("hmm_forward_long", lib.hmm_forward_long(C.byref(m), _ptr(obs), _ptr(offsets), S, obs.numel(), max_T,
                                                     _ptr(out), _ptr(ws), ws.numel(), _stream()))
    return out


def hmm_mstep(log_A, log_B, log_pi, grad_log_A, grad_log_B, grad_log_pi, want_grad=True, want_new=True):
    """Re-estimation after hmm_adjoint, from its gradients (the expected counts):
    returns (grad_theta, new_log), each a tuple (A, B, pi) of float32 tensors or None --
    the gradient for row-softmax parameters theta (P = softmax(theta) per row) and the
    Baum-Welch M-step log parameters."""
    lib = L.load()
    _need_cuda(log_A, log_B, log_pi, grad_log_A, grad_log_B, grad_log_pi)
    m = _model(log_A, log_B, log_pi)
    gA, gB, gpi = (t.contiguous().to(torch.float32) for t in (grad_log_A, grad_log_B, grad_log_pi))
    th = tuple(torch.empty_like(t) for t in (gA, gB, gpi)) if want_grad else (None, None, None)
    nw = tuple(torch.empty_like(t) for t in (gA, gB, gpi)) if want_new else (None, None, None)
    L.check("hmm_mstep", lib.hmm_mstep(C.byref(m), _ptr(gA), _ptr(gB), _ptr(gpi), _ptr(th[0]), _ptr(th[1]),
                                       _ptr(th[2]), _ptr(nw[0]), _ptr(nw[1]), _ptr(nw[2]), _stream()))
    return (th if want_grad else None), (nw if want_new else None)


def hmm_autotune(log_A, log_B, log_pi, obs, offsets, precision=L.HMM_BF16_SCALED, cache_path=None, ws=None):
    """Times the BF16 forward's launch configurations on these inputs and keeps the fastest
    for later hmm_forward calls (and in `cache_path`, JSON lines, if given).  Returns
    (best ms or 0.0 if cached, (split, rows, pair, units)); pair = 1 (2) when a tile of
    sequences runs on a cluster of two (four) CTAs that split the state columns; units = the
    persistent CTAs or clusters launched (0: all that fit)."""
    lib = L.load()
    m = _model(log_A, log_B, log_pi)
    S = offsets.numel() - 1
    need = lib.hmm_forward_workspace_size(C.byref(m), S, obs.numel(), precision)
    if ws is None or ws.numel() < need:
        ws = _ws(need, obs.device)
    out = torch.empty(S, dtype=torch.float64, device=obs.device)
    best = C.c_float(0.0)
    path = cache_path.encode() if cache_path else None
    L.check("hmm_autotune", lib.hmm_autotune(C.byref(m), precision, _ptr(obs), _ptr(offsets), S, obs.numel(),
                                             _ptr(out), _ptr(ws), ws.numel(), path, C.byref(best), _stream()))
    split, rows, pair, units = C.c_int32(0), C.c_int32(0), C.c_int32(0), C.c_int32(0)
    L.check("hmm_tuned_config", lib.hmm_tuned_config(m.K, m.M, S, C.byref(split), C.byref(rows), C.byref(pair),
                                                     C.byref(units)))
    return best.value, (split.value, rows.value, pair.value, units.value)


class Graph:
    """A captured sequence of library calls on a (non-default) stream, replayed with one
    launch.  Allocate every output and workspace before capturing."""

    def __init__(self):
        self.h = C.c_void_p(0)

    def capture(self, fn, stream=None):
        lib = L.load()
        stream = stream or torch.cuda.current_stream()
        s = C.c_void_p(stream.cuda_stream)
        with torch.cuda.stream(stream):
            L.check("accel_graph_begin", lib.accel_graph_begin(s))
            try:
                result = fn()
            finally:
                h = C.c_void_p(0)
                st = lib.accel_graph_end(s, C.byref(h))
            L.check("accel_graph_end", st)
        self.h = h
        return result

    def launch(self, stream=None):
        lib = L.load()
        stream = stream or torch.cuda.current_stream()
        L.check("accel_graph_launch", lib.accel_graph_launch(self.h, C.c_void_p(stream.cuda_stream)))

    def nodes(self):
        n = C.c_int64(0)
        L.check("accel_graph_node_count", L.load().accel_graph_node_count(self.h, C.byref(n)))
        return n.value

    def __del__(self):
        try:
            if self.h and self.h.value:
                L.load().accel_graph_destroy(self.h)
        except Exception:
            pass


class HMMLogLik(torch.autograd.Function):
    """logL[S] = HMMLogLik.apply(log_A, log_B, log_pi, obs, offsets, precision, max_T=None).

    With FP32 precision and a gradient to take, the forward is the adjoint's checkpointed
    forward (hmm_adjoint_forward), whose saved state the backward uses (hmm_adjoint_backward):
    the forward recursion runs once.  With BF16 precision the forward runs on the tensor cores
    and the backward calls hmm_adjoint.  The incoming gradient enters as per-sequence weights
    (the gradient of sum_s w_s logL_s is linear in w), giving d/d log_A, d/d log_B, d/d log_pi.
    """

    @staticmethod
    def forward(ctx, log_A, log_B, log_pi, obs, offsets, precision=L.HMM_FP32_LOG, max_T=None):
        ctx.saved = None
        ctx.max_T = max_T
        needs = any(ctx.needs_input_grad[:3])
        if precision == L.HMM_FP32_LOG and needs:
            ll, ctx.saved = hmm_adjoint_forward(log_A, log_B, log_pi, obs, offsets, max_T=max_T)
            ctx.save_for_backward(log_A, log_B, log_pi, obs, offsets, None)
            return ll
        # max_T sizes the adjoint's checkpoints: the caller's value, else the library's device
        # reduction over the offsets, launched here and read only in backward
        d_max = hmm_max_length(offsets) if max_T is None and offsets.numel() > 1 else None
        ctx.save_for_backward(log_A, log_B, log_pi, obs, offsets, d_max)
        return hmm_forward(log_A, log_B, log_pi, obs, offsets, precision)

    @staticmethod
    def backward(ctx, grad_out):
        log_A, log_B, log_pi, obs, offsets, d_max = ctx.saved_tensors
        w = grad_out.contiguous().to(torch.float64)
        if ctx.saved is not None:
            gA, gB, gpi = hmm_adjoint_backward(log_A, log_B, log_pi, obs, offsets, ctx.saved, weights=w)
            return gA, gB, gpi, None, None, None, None
        max_T = ctx.max_T if ctx.max_T is not None else (int(d_max.item()) if d_max is not None else 0)
        gA, gB, gpi, _ = hmm_adjoint(log_A, log_B, log_pi, obs, offsets, weights=w, max_T=max_T, want_loglik=False)
        return gA, gB, gpi, None, None, None, None


# ------------------------------------------------------------------------- all-pairs
def pairwise_mapreduce(x, y, z, m, eps: float, op: int = L.PAIR_GRAVITY_SOFTENED, out=None):
    lib = L.load()
    _need_cuda(x, y, z, m)
    n = x.numel()
    if out is None:
        out = tuple(torch.empty(n, dtype=torch.float32, device=x.device) for _ in range(3))
    ax, ay, az = out
    L.check("pairwise_mapreduce", lib.pairwise_mapreduce(op, _ptr(x), _ptr(y), _ptr(z), _ptr(m), n, float(eps),
                                                         _ptr(ax), _ptr(ay), _ptr(az), _stream()))
    return ax, ay, az
