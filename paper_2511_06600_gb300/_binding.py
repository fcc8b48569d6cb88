"""ctypes binding of libhef.so (argument marshalling only).

Every function here forwards device pointers of torch CUDA tensors and the
current CUDA stream to the C ABI declared in include/hef.h; all arithmetic
runs in the library's kernels.  Device memory (outputs and workspaces) is
allocated with torch.  If the library is missing, loading fails loudly: there
is no other implementation.
"""
from __future__ import annotations

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
# HEF_LIBRARY selects another build of the same ABI (the bounds-checked
# libhef_debug.so, see build.py --debug); the default is libhef.so.
LIB_PATH = os.environ.get("HEF_LIBRARY") or os.path.join(HERE, "libhef.so")

HEF_F64, HEF_F32, HEF_BF16 = 0, 1, 2
HEF_REDUCE_MAX, HEF_REDUCE_SUM, HEF_REDUCE_EMBED = 0, 1, 2
HEF_OPS_CLIQUE, HEF_OPS_STAR, HEF_OPS_BOTH = 1, 2, 3
HEF_CLIQUE_HYPEREDGE, HEF_CLIQUE_PAPER = 0, 1
HEF_ERR_INVALID_INPUT = -7

_DTYPES = {HEF_F64: torch.float64, HEF_F32: torch.float32, HEF_BF16: torch.bfloat16}
_CODES = {torch.float64: HEF_F64, torch.float32: HEF_F32, torch.bfloat16: HEF_BF16,
          "f64": HEF_F64, "f32": HEF_F32, "bf16": HEF_BF16}

c_i32, c_i64, c_sz, c_p = ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t, ctypes.c_void_p

_SIGS = {
    "hef_last_error": (ctypes.c_char_p, []),
    "hef_status_string": (ctypes.c_char_p, [c_i32]),
    "hef_abi_version": (c_i32, []),
    "hef_debug_checks": (c_i32, []),
    "hef_debug_set_pin": (c_i32, [c_p, c_i64, c_i32, c_p]),
    "hef_launch_count": (ctypes.c_uint64, []),
    "hef_trace_kernels": (c_i32, [ctypes.c_char_p]),
    "hef_trace_read": (c_i32, [c_i32, ctypes.c_char_p, ctypes.POINTER(c_i64),
                               ctypes.POINTER(ctypes.c_double)]),
    "hef_incidence_workspace_bytes": (c_sz, [c_i64, c_i64, c_i64]),
    "hef_build_incidence": (c_i32, [c_i64, c_i64, c_i64, c_p, c_p, c_p, c_i32, c_p, c_sz, c_p,
                                    ctypes.POINTER(c_p)]),
    "hef_incidence_check": (c_i32, [c_p, c_p, ctypes.POINTER(ctypes.c_uint32),
                                    ctypes.POINTER(c_i64)]),
    "hef_incidence_sizes": (c_i32, [c_p, ctypes.POINTER(c_i64), ctypes.POINTER(c_i64),
                                    ctypes.POINTER(c_i64)]),
    "hef_incidence_export": (c_i32, [c_p, c_p, c_p, c_p, c_p, c_p, c_p]),
    "hef_free_incidence": (None, [c_p]),
    "hef_krylov_workspace_bytes": (c_sz, [c_p, c_i32, c_i32, c_i32]),
    "hef_krylov_basis": (c_i32, [c_p, c_i32, c_i32, c_i32, c_p, c_p, c_p, c_i64, c_p, c_sz, c_p]),
    "hef_krylov_ops_workspace_bytes": (c_sz, [c_p, c_i32, c_i32, c_i32, c_i32]),
    "hef_krylov_basis_ops": (c_i32, [c_p, c_i32, c_i32, c_i32, c_i32, c_p, c_p, c_p, c_i64, c_p,
                                     c_sz, c_p]),
    "hef_orthonormalize_workspace_bytes": (c_sz, [c_i64, c_i32, c_i32]),
    "hef_orthonormalize": (c_i32, [c_i64, c_i32, c_i32, c_p, c_i64, c_p, c_p, c_p, c_sz, c_p]),
    "hef_edge_resistance_workspace_bytes": (c_sz, [c_p, c_i32]),
    "hef_edge_resistance": (c_i32, [c_p, c_p, c_i64, c_i32, c_i32, c_i32, c_p, c_p, c_p, c_p, c_p,
                                    c_p, c_sz, c_p]),
    "hef_edge_resistance_noalloc": (c_i32, [c_p, c_p, c_i64, c_i32, c_i32, c_i32, c_p, c_p, c_p,
                                            c_p, c_p, c_p]),
    "hef_batch_workspace_bytes": (c_sz, [c_p, c_i32, c_i32, c_i32, c_i32]),
    "hef_batch_schedule": (c_i32, [c_p, c_i32, c_i32, c_i32, c_i32, c_p]),
    "hef_resistance_batched": (c_i32, [c_p, c_i32, c_i32, c_i32, c_i32, c_i32, c_p, c_i32, c_p,
                                       c_sz, c_p]),
    "hef_batch_autotune": (c_i32, [c_p, c_i32, c_i32, c_i32, c_i32, c_i32, c_p, c_sz, c_p, c_p,
                                   c_p, c_p]),
    "hef_set_batch_krylov_form": (c_i32, [c_i32]),
    "hef_batch_krylov_form": (c_i32, []),
    "hef_krylov_tape_bytes": (c_sz, [c_p, c_i32, c_i32, c_i32]),
    "hef_set_krylov_persistent": (c_i32, [c_i32]),
    "hef_krylov_basis_tape": (c_i32, [c_p, c_i32, c_i32, c_i32, c_p, c_p, c_p, c_i64, c_p, c_sz,
                                      c_p, c_sz, c_p]),
    "hef_resistance_host_workspace_bytes": (c_sz, [c_i64, c_i64, c_i64, c_i32, c_i32, c_i32]),
    "hef_resistance_host": (c_i32, [c_i64, c_i64, c_i64, c_p, c_p, c_p, c_p, c_p, c_i32, c_i32,
                                    c_i32, c_i32, c_p, c_p, c_sz, c_p]),
    "hef_level_workspace_bytes": (c_sz, [c_i64, c_i64, c_i32]),
    "hef_sort_resistance": (c_i32, [c_i64, c_p, c_p, c_p, c_sz, c_p]),
    "hef_coarsen_level": (c_i32, [c_p, c_p, c_p, c_p, c_p, c_p, c_p, c_i64, c_i32, c_i32, c_p,
                                  ctypes.c_double, ctypes.c_double, c_p, c_p, c_sz, c_p]),
    "hef_edge_resistance_backward_workspace_bytes": (c_sz, [c_p, c_i32, c_i32, c_i32, c_i32]),
    "hef_backward_plan": (c_i32, [c_p, c_i32, c_i32, c_i32, ctypes.c_uint64,
                                  ctypes.POINTER(c_i32), ctypes.POINTER(ctypes.c_uint64)]),
    "hef_edge_resistance_backward": (c_i32, [c_p, c_i32, c_i32, c_i32, c_p, c_p, c_p, c_sz, c_p,
                                             c_i64, c_p, c_p, c_p, c_p, c_p, c_p, c_p, c_p, c_p,
                                             c_sz, c_p]),
}

_lib = None


class HefError(RuntimeError):
    def __init__(self, fn, status, msg):
        super().__init__(f"{fn}: {status_string(status)}: {msg}")
        self.status = status


def lib():
    """Load libhef.so (built in-tree by paper_2511_06600_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                f"{LIB_PATH} is missing: build it with `python -m paper_2511_06600_gb300.build` "
                "(there is no fallback implementation)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def status_string(s):
    return lib().hef_status_string(s).decode()


def launch_count():
    """Kernels launched by the library so far in this process."""
    return int(lib().hef_launch_count())


def trace_kernels(substring):
    """Time every launch of library kernels whose name contains `substring`
    with CUDA events (None stops)."""
    lib().hef_trace_kernels(substring.encode() if substring else None)


def trace_read(cap=64):
    """{kernel name: (launches, total ms)} of the traced launches so far."""
    names = ctypes.create_string_buffer(64 * cap)
    launches = (c_i64 * cap)()
    ms = (ctypes.c_double * cap)()
    k = lib().hef_trace_read(cap, names, launches, ms)
    out = {}
    for i in range(min(k, cap)):
        nm = names.raw[64 * i:64 * (i + 1)].split(b"\0", 1)[0].decode()
        out[nm] = (int(launches[i]), float(ms[i]))
    return out


def _check(fn, status):
    if status != 0:
        raise HefError(fn, status, lib().hef_last_error().decode())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dtype_code(dtype):
    if isinstance(dtype, int):
        return dtype
    return _CODES[dtype]


def _workspace(nbytes, device):
    # 256-byte aligned: the caching allocator returns 512-byte aligned blocks
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def padded_ld(K, dtype):
    """Row stride of an n x K basis: K rounded up to 16 bytes."""
    per = 16 // torch.empty((), dtype=_DTYPES[_dtype_code(dtype)]).element_size()
    return (K + per - 1) // per * per


class Incidence:
    """A built incidence (hef_build_incidence) and the workspace it lives in."""

    def __init__(self, n, eptr, pins, w, clique_mode=HEF_CLIQUE_HYPEREDGE, stream=None):
        L = lib()
        dev = eptr.device
        assert eptr.dtype == torch.int64 and pins.dtype == torch.int32 and w.dtype == torch.float64
        assert eptr.is_cuda and pins.is_cuda and w.is_cuda
        self.n = int(n)
        self.m = int(eptr.numel() - 1)
        self.P = int(pins.numel())
        self.device = dev
        ws = L.hef_incidence_workspace_bytes(self.n, self.m, self.P)
        self.workspace = _workspace(ws, dev)
        # keep the inputs alive until the build has run
        self._inputs = (eptr, pins, w)
        h = c_p()
        _check("hef_build_incidence",
               L.hef_build_incidence(self.n, self.m, self.P, _ptr(eptr), _ptr(pins), _ptr(w),
                                     int(clique_mode), _ptr(self.workspace), ws, _stream(stream),
                                     ctypes.byref(h)))
        self.handle = h

    def check(self, stream=None):
        """Synchronise and raise HefError if device validation failed."""
        detail = ctypes.c_uint32(0)
        where = c_i64(-1)
        st = lib().hef_incidence_check(self.handle, _stream(stream), ctypes.byref(detail),
                                       ctypes.byref(where))
        if st != 0:
            err = HefError("hef_incidence_check", st, lib().hef_last_error().decode())
            err.detail = detail.value
            err.where = where.value
            raise err

    def debug_set_pin(self, slot, value, stream=None):
        """Bounds-checked build only: overwrite pin slot `slot` (internal CSC
        order) with `value`, to plant an index that the checks must catch."""
        _check("hef_debug_set_pin",
               lib().hef_debug_set_pin(self.handle, int(slot), int(value), _stream(stream)))

    def export(self, stream=None):
        dev = self.device
        out = dict(perm=torch.empty(max(self.m, 1), dtype=torch.int32, device=dev)[:self.m],
                   vptr=torch.empty(self.n + 1, dtype=torch.int32, device=dev),
                   vedge=torch.empty(max(self.P, 1), dtype=torch.int32, device=dev)[:self.P],
                   dc=torch.empty(self.n, dtype=torch.float64, device=dev),
                   db=torch.empty(self.n, dtype=torch.float64, device=dev))
        _check("hef_incidence_export",
               lib().hef_incidence_export(self.handle, _ptr(out["perm"]), _ptr(out["vptr"]),
                                          _ptr(out["vedge"]), _ptr(out["dc"]), _ptr(out["db"]),
                                          _stream(stream)))
        return out

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and _lib is not None:
            _lib.hef_free_incidence(h)
            self.handle = None


def build_incidence(n, eptr, pins, w, clique_mode=HEF_CLIQUE_HYPEREDGE, stream=None):
    return Incidence(n, eptr, pins, w, clique_mode, stream)


def krylov_basis(inc, x0_clique, x0_star, k, dtype=torch.float64, V=None, workspace=None,
                 stream=None, ops=HEF_OPS_BOTH):
    """V (n x ldv, dtype): vertex rows of the k Krylov vectors of every chain
    (hef_krylov_basis; hef_krylov_basis_ops for one expansion).  Returns V;
    its first K = 2kS (one expansion: kS) columns are the basis."""
    L = lib()
    code = _dtype_code(dtype)
    S = int(x0_clique.shape[1])
    K = (2 if ops == HEF_OPS_BOTH else 1) * k * S
    if V is None:
        V = torch.empty(inc.n, padded_ld(K, code), dtype=_DTYPES[code], device=inc.device)
    if ops != HEF_OPS_BOTH:
        ws = L.hef_krylov_ops_workspace_bytes(inc.handle, k, S, code, int(ops))
        if ws == 0:
            raise HefError("hef_krylov_ops_workspace_bytes", -6, "unsupported k/S/dtype/ops")
        workspace = _workspace(ws, inc.device) if workspace is None else workspace
        _check("hef_krylov_basis_ops",
               L.hef_krylov_basis_ops(inc.handle, k, S, code, int(ops), _ptr(x0_clique),
                                      _ptr(x0_star), _ptr(V), V.stride(0), _ptr(workspace),
                                      workspace.numel(), _stream(stream)))
        return V
    ws = L.hef_krylov_workspace_bytes(inc.handle, k, S, code)
    if ws == 0:
        raise HefError("hef_krylov_workspace_bytes", -6, "unsupported k/S/dtype")
    if workspace is None:
        workspace = _workspace(ws, inc.device)
    _check("hef_krylov_basis",
           L.hef_krylov_basis(inc.handle, k, S, code, _ptr(x0_clique), _ptr(x0_star), _ptr(V),
                              V.stride(0), _ptr(workspace), workspace.numel(), _stream(stream)))
    return V


def set_krylov_persistent(on):
    """hef_set_krylov_persistent for calls from this thread (0, 1 or 2)."""
    _check("hef_set_krylov_persistent", lib().hef_set_krylov_persistent(int(on)))


def krylov_basis_tape(inc, x0_clique, x0_star, k, dtype=torch.float64, stream=None):
    """hef_krylov_basis_tape: the basis V of krylov_basis plus the tape the
    backward reads.  Returns (V, tape)."""
    L = lib()
    code = _dtype_code(dtype)
    S = int(x0_clique.shape[1])
    K = 2 * k * S
    V = torch.empty(inc.n, padded_ld(K, code), dtype=_DTYPES[code], device=inc.device)
    ws = _workspace(L.hef_krylov_workspace_bytes(inc.handle, k, S, code), inc.device)
    tape = _workspace(L.hef_krylov_tape_bytes(inc.handle, k, S, code), inc.device)
    _check("hef_krylov_basis_tape",
           L.hef_krylov_basis_tape(inc.handle, k, S, code, _ptr(x0_clique), _ptr(x0_star), _ptr(V),
                                   V.stride(0), _ptr(tape), tape.numel(), _ptr(ws), ws.numel(),
                                   _stream(stream)))
    return V, tape


def edge_resistance_backward(inc, k, x0_clique, x0_star, Q, R_fac, scores, dR, tape=None,
                             want_dx0=True, stream=None):
    """hef_edge_resistance_backward: (dw, dx0_clique, dx0_star) from
    dR = dL/dR.  `scores` is the dict of edge_resistance (R, QH, argvec);
    `tape` from krylov_basis_tape, or None to recompute it."""
    L = lib()
    code = _dtype_code(Q.dtype)
    S = int(x0_clique.shape[1])
    dev = Q.device
    ws = _workspace(L.hef_edge_resistance_backward_workspace_bytes(inc.handle, k, S, code,
                                                                   int(tape is None)), dev)
    dw = torch.empty(max(inc.m, 1), dtype=torch.float64, device=dev)[:inc.m]
    dxc = torch.empty_like(x0_clique) if want_dx0 else None
    dxb = torch.empty_like(x0_star) if want_dx0 else None
    dR = dR.to(device=dev, dtype=torch.float64).contiguous()
    _check("hef_edge_resistance_backward",
           L.hef_edge_resistance_backward(
               inc.handle, k, S, code, _ptr(x0_clique), _ptr(x0_star), _ptr(tape),
               0 if tape is None else tape.numel(), _ptr(Q), Q.stride(0), _ptr(R_fac),
               _ptr(scores["QH"]), _ptr(scores["argvec"]), _ptr(scores["R"]), _ptr(dR), _ptr(dw),
               _ptr(dxc), _ptr(dxb), _ptr(ws), ws.numel(), _stream(stream)))
    return dw, dxc, dxb


def backward_plan(inc, k, S, dtype, budget_bytes=0):
    """hef_backward_plan: (keep the tape?, tape bytes) for a budget (0: half
    of the free device memory)."""
    use = c_i32(0)
    tb = ctypes.c_uint64(0)
    _check("hef_backward_plan",
           lib().hef_backward_plan(inc.handle, int(k), int(S), _dtype_code(dtype),
                                   int(budget_bytes), ctypes.byref(use), ctypes.byref(tb)))
    return bool(use.value), int(tb.value)


class HefResistance(torch.autograd.Function):
    """R = HyperEF resistance scores (Algorithm 1, HEF_REDUCE_MAX) as a
    differentiable function of the hyperedge weights w and the random starts
    (x0_clique, x0_star); the structure (n, eptr, pins) and k are fixed.
    Forward keeps the Krylov tape when hef_backward_plan says it fits
    `tape_budget` bytes (0: half of the free device memory), else the
    backward recomputes the chains; backward calls
    hef_edge_resistance_backward."""

    @staticmethod
    def forward(ctx, w, x0_clique, x0_star, n, eptr, pins, k, dtype, clique_mode, tape_budget=0):
        w64 = w.detach().to(torch.float64).contiguous()
        xc = x0_clique.detach().to(torch.float64).contiguous()
        xb = x0_star.detach().to(torch.float64).contiguous()
        inc = build_incidence(n, eptr, pins, w64, clique_mode)
        S = int(xc.shape[1])
        K = 2 * k * S
        keep, _ = backward_plan(inc, k, S, dtype, tape_budget)
        if keep:
            V, tape = krylov_basis_tape(inc, xc, xb, k, dtype)
        else:
            V, tape = krylov_basis(inc, xc, xb, k, dtype), None
        Q, Rf, rank = orthonormalize(V, K, want_R=True)
        scores = edge_resistance(inc, Q, K)
        ctx.state = (inc, k, xc, xb, Q, Rf, scores, tape, w.dtype)
        return scores["R"].clone().to(w.dtype)

    @staticmethod
    def backward(ctx, gR):
        inc, k, xc, xb, Q, Rf, scores, tape, wdt = ctx.state
        dw, dxc, dxb = edge_resistance_backward(inc, k, xc, xb, Q, Rf, scores, gR, tape=tape)
        ctx.state = None
        return dw.to(wdt), dxc, dxb, None, None, None, None, None, None, None


def resistance(w, x0_clique, x0_star, n, eptr, pins, k, dtype=torch.float64,
               clique_mode=HEF_CLIQUE_HYPEREDGE, tape_budget=0):
    """Differentiable scores: HefResistance.apply with keyword defaults."""
    return HefResistance.apply(w, x0_clique, x0_star, n, eptr, pins, k, dtype, clique_mode,
                               tape_budget)


def orthonormalize(V, K, want_R=False, workspace=None, stream=None):
    """In place: the first K columns of V become Q (hef_orthonormalize).
    Returns (V, R or None, rank tensor)."""
    L = lib()
    code = _dtype_code(V.dtype)
    n = V.shape[0]
    ws = L.hef_orthonormalize_workspace_bytes(n, K, code)
    if workspace is None:
        workspace = _workspace(ws, V.device)
    R = torch.empty(K, K, dtype=torch.float64, device=V.device) if want_R else None
    rank = torch.empty(1, dtype=torch.int32, device=V.device)
    _check("hef_orthonormalize",
           L.hef_orthonormalize(n, K, code, _ptr(V), V.stride(0), _ptr(R), _ptr(rank),
                                _ptr(workspace), workspace.numel(), _stream(stream)))
    return V, R, rank


def edge_resistance(inc, Q, K, reduce=HEF_REDUCE_MAX, routing=True, workspace=None, out=None,
                    stream=None):
    """Scores of every hyperedge (hef_edge_resistance); a dict of tensors."""
    L = lib()
    code = _dtype_code(Q.dtype)
    dev = Q.device
    m = inc.m
    if out is None:
        out = dict(R=torch.empty(max(m, 1), dtype=torch.float64, device=dev)[:m],
                   QH=torch.empty(K, dtype=torch.float64, device=dev))
        if routing:
            for key in ("argvec", "pmax", "pmin"):
                out[key] = torch.empty(max(m, 1), dtype=torch.int32, device=dev)[:m]
    ws = L.hef_edge_resistance_workspace_bytes(inc.handle, K)
    if workspace is None:
        workspace = _workspace(ws, dev)
    _check("hef_edge_resistance",
           L.hef_edge_resistance(inc.handle, _ptr(Q), Q.stride(0), K, code, int(reduce),
                                 _ptr(out["R"]), _ptr(out.get("QH")), _ptr(out.get("argvec")),
                                 _ptr(out.get("pmax")), _ptr(out.get("pmin")), _ptr(workspace),
                                 workspace.numel(), _stream(stream)))
    return out


def edge_resistance_noalloc(inc, Q, K, reduce=HEF_REDUCE_MAX, out=None, stream=None):
    """hef_edge_resistance_noalloc: the scores of edge_resistance, with the
    library's fixed scratch instead of a workspace (outputs still needed)."""
    code = _dtype_code(Q.dtype)
    dev = Q.device
    m = inc.m
    if out is None:
        out = dict(R=torch.empty(max(m, 1), dtype=torch.float64, device=dev)[:m],
                   QH=torch.empty(K, dtype=torch.float64, device=dev))
        for key in ("argvec", "pmax", "pmin"):
            out[key] = torch.empty(max(m, 1), dtype=torch.int32, device=dev)[:m]
    _check("hef_edge_resistance_noalloc",
           lib().hef_edge_resistance_noalloc(inc.handle, _ptr(Q), Q.stride(0), K, code, int(reduce),
                                             _ptr(out["R"]), _ptr(out.get("QH")),
                                             _ptr(out.get("argvec")), _ptr(out.get("pmax")),
                                             _ptr(out.get("pmin")), _stream(stream)))
    return out


def hyperedge_resistance(n, eptr, pins, w, x0_clique, x0_star, k, dtype=torch.float64,
                         clique_mode=HEF_CLIQUE_HYPEREDGE, reduce=HEF_REDUCE_MAX, check=True,
                         ops=HEF_OPS_BOTH):
    """Algorithm 1 end to end on the GPU: incidence, Krylov basis, CholQR2,
    scores.  All inputs are CUDA tensors."""
    inc = build_incidence(n, eptr, pins, w, clique_mode)
    S = int(x0_clique.shape[1])
    K = (2 if ops == HEF_OPS_BOTH else 1) * k * S
    V = krylov_basis(inc, x0_clique, x0_star, k, dtype, ops=ops)
    Q, _, rank = orthonormalize(V, K)
    out = edge_resistance(inc, Q, K, reduce)
    if check:
        inc.check()
    out.update(Q=Q[:, :K], rank=rank, incidence=inc)
    return out


class Pipeline:
    """Algorithm 1 on the GPU with every buffer allocated once (the first
    run), so that repeated runs on hypergraphs of one shape allocate nothing:
    hef_build_incidence -> hef_krylov_basis -> hef_orthonormalize ->
    hef_edge_resistance, all on the current stream."""

    def __init__(self, n, m, P, k, S, dtype=torch.float64, clique_mode=HEF_CLIQUE_HYPEREDGE,
                 reduce=HEF_REDUCE_MAX, device=None, routing=True):
        self.n, self.m, self.P, self.k, self.S = int(n), int(m), int(P), int(k), int(S)
        self.K = 2 * self.k * self.S
        self.code = _dtype_code(dtype)
        self.clique_mode = int(clique_mode)
        self.reduce = int(reduce)
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        L = lib()
        dev = self.device
        self.ws_inc = _workspace(L.hef_incidence_workspace_bytes(self.n, self.m, self.P), dev)
        self.V = torch.empty(self.n, padded_ld(self.K, self.code), dtype=_DTYPES[self.code],
                             device=dev)
        self.ws_ortho = _workspace(L.hef_orthonormalize_workspace_bytes(self.n, self.K, self.code),
                                   dev)
        self.rank = torch.empty(1, dtype=torch.int32, device=dev)
        self.out = dict(R=torch.empty(max(self.m, 1), dtype=torch.float64, device=dev)[:self.m],
                        QH=torch.empty(self.K, dtype=torch.float64, device=dev))
        if routing:
            for key in ("argvec", "pmax", "pmin"):
                self.out[key] = torch.empty(max(self.m, 1), dtype=torch.int32, device=dev)[:self.m]
        self.ws_kry = None
        self.ws_score = None
        self.handle = None

    def run(self, eptr, pins, w, x0_clique, x0_star, stream=None):
        L = lib()
        st = _stream(stream)
        h = c_p()
        _check("hef_build_incidence",
               L.hef_build_incidence(self.n, self.m, self.P, _ptr(eptr), _ptr(pins), _ptr(w),
                                     self.clique_mode, _ptr(self.ws_inc), self.ws_inc.numel(), st,
                                     ctypes.byref(h)))
        if self.handle is not None:
            L.hef_free_incidence(self.handle)
        self.handle = h
        if self.ws_kry is None:
            self.ws_kry = _workspace(L.hef_krylov_workspace_bytes(h, self.k, self.S, self.code),
                                     self.device)
            self.ws_score = _workspace(L.hef_edge_resistance_workspace_bytes(h, self.K),
                                       self.device)
        _check("hef_krylov_basis",
               L.hef_krylov_basis(h, self.k, self.S, self.code, _ptr(x0_clique), _ptr(x0_star),
                                  _ptr(self.V), self.V.stride(0), _ptr(self.ws_kry),
                                  self.ws_kry.numel(), st))
        _check("hef_orthonormalize",
               L.hef_orthonormalize(self.n, self.K, self.code, _ptr(self.V), self.V.stride(0),
                                    None, _ptr(self.rank), _ptr(self.ws_ortho),
                                    self.ws_ortho.numel(), st))
        o = self.out
        _check("hef_edge_resistance",
               L.hef_edge_resistance(h, _ptr(self.V), self.V.stride(0), self.K, self.code,
                                     self.reduce, _ptr(o["R"]), _ptr(o["QH"]),
                                     _ptr(o.get("argvec")), _ptr(o.get("pmax")),
                                     _ptr(o.get("pmin")), _ptr(self.ws_score),
                                     self.ws_score.numel(), st))
        return o

    def check(self, stream=None):
        detail = ctypes.c_uint32(0)
        where = c_i64(-1)
        _check("hef_incidence_check",
               lib().hef_incidence_check(self.handle, _stream(stream), ctypes.byref(detail),
                                         ctypes.byref(where)))
        if int(self.rank.item()) < 0:
            raise HefError("hef_orthonormalize", -5, "a tensor-core wait timed out")

    def capture(self, eptr, pins, w, x0_clique, x0_star):
        """Record one run on these input tensors as a CUDA graph; `replay()`
        then reruns the whole path with one launch (inputs may be refilled in
        place between replays)."""
        side = torch.cuda.Stream(device=self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(side):
            self.run(eptr, pins, w, x0_clique, x0_star)
        torch.cuda.current_stream(self.device).wait_stream(side)
        torch.cuda.synchronize(self.device)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.run(eptr, pins, w, x0_clique, x0_star)
        return self.graph

    def replay(self):
        self.graph.replay()
        return self.out

    def __del__(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.hef_free_incidence(self.handle)
            self.handle = None


class _BatchItem(ctypes.Structure):
    """hef_batch_item (include/hef.h)."""
    _fields_ = [("n", c_i64), ("m", c_i64), ("P", c_i64), ("eptr", c_p), ("pins", c_p), ("w", c_p),
                ("x0_clique", c_p), ("x0_star", c_p), ("R_out", c_p), ("QH_out", c_p),
                ("argvec", c_p), ("pmax", c_p), ("pmin", c_p), ("status_out", c_p)]


class Batch:
    """Batched form: Algorithm 1 on G hypergraphs in one call
    (hef_resistance_batched).  `graphs` is a list of dicts of CUDA tensors
    with keys n, eptr, pins, w, x0c, x0b; outputs (R, QH, argvec, pmax, pmin,
    status per item) are allocated once."""

    def __init__(self, graphs, k, S, dtype=torch.float32, clique_mode=HEF_CLIQUE_HYPEREDGE,
                 nstreams=8, device=None):
        self.k, self.S, self.K = int(k), int(S), 2 * int(k) * int(S)
        self.code = _dtype_code(dtype)
        self.clique_mode = int(clique_mode)
        self.device = device or torch.device("cuda", torch.cuda.current_device())
        dev = self.device
        self.graphs = graphs
        self.out = []
        items = (_BatchItem * len(graphs))()
        for g, gr in enumerate(graphs):
            m = int(gr["eptr"].numel() - 1)
            o = dict(R=torch.empty(max(m, 1), dtype=torch.float64, device=dev)[:m],
                     QH=torch.empty(self.K, dtype=torch.float64, device=dev),
                     argvec=torch.empty(max(m, 1), dtype=torch.int32, device=dev)[:m],
                     pmax=torch.empty(max(m, 1), dtype=torch.int32, device=dev)[:m],
                     pmin=torch.empty(max(m, 1), dtype=torch.int32, device=dev)[:m],
                     status=torch.zeros(2, dtype=torch.int32, device=dev))
            self.out.append(o)
            it = items[g]
            it.n, it.m, it.P = int(gr["n"]), m, int(gr["pins"].numel())
            it.eptr, it.pins, it.w = (gr["eptr"].data_ptr(), gr["pins"].data_ptr(),
                                      gr["w"].data_ptr())
            it.x0_clique, it.x0_star = gr["x0c"].data_ptr(), gr["x0b"].data_ptr()
            it.R_out, it.QH_out = o["R"].data_ptr(), o["QH"].data_ptr()
            it.argvec, it.pmax, it.pmin = (o["argvec"].data_ptr(), o["pmax"].data_ptr(),
                                           o["pmin"].data_ptr())
            it.status_out = o["status"].data_ptr()
        self.items = items
        self.G = len(graphs)
        L = lib()
        nb = L.hef_batch_workspace_bytes(items, self.G, self.k, self.S, self.code)
        if nb == 0:
            raise HefError("hef_batch_workspace_bytes", -1, lib().hef_last_error().decode())
        self.workspace = _workspace(nb, dev)
        self.nstreams = int(nstreams)
        self.schedule = None
        self.graph = None

    def run(self, stream=None):
        sched = None if self.schedule is None else self.schedule
        _check("hef_resistance_batched",
               lib().hef_resistance_batched(self.items, self.G, self.k, self.S, self.code,
                                            self.clique_mode, sched, self.nstreams,
                                            _ptr(self.workspace), self.workspace.numel(),
                                            _stream(stream)))
        return self.out

    def autotune(self, stream=None):
        """hef_batch_autotune: keep the fastest stream count and schedule."""
        ns = c_i32(0)
        sched = (c_i32 * self.G)()
        ms = ctypes.c_float(0.0)
        _check("hef_batch_autotune",
               lib().hef_batch_autotune(self.items, self.G, self.k, self.S, self.code,
                                        self.clique_mode, _ptr(self.workspace),
                                        self.workspace.numel(), _stream(stream),
                                        ctypes.byref(ns), sched, ctypes.byref(ms)))
        self.nstreams = ns.value
        self.schedule = sched
        return ns.value, list(sched), ms.value

    def check(self):
        """Raise HefError if any item failed device validation."""
        st = torch.stack([o["status"] for o in self.out]).cpu()
        bad = (st[:, 0] != 0).nonzero().flatten().tolist()
        if bad:
            raise HefError("hef_resistance_batched", HEF_ERR_INVALID_INPUT,
                           f"items {bad} rejected by device validation")

    def capture(self):
        """Record one batched run as a CUDA graph; replay() reruns it."""
        side = torch.cuda.Stream(device=self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(side):
            self.run()
        torch.cuda.current_stream(self.device).wait_stream(side)
        torch.cuda.synchronize(self.device)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.run()
        return self.graph

    def replay(self):
        self.graph.replay()
        return self.out


# ---------------------------------------------------------------- downstream


class _LevelOut(ctypes.Structure):
    """hef_level_out (include/hef.h)."""
    _fields_ = [("R_upd", c_p), ("order", c_p), ("delta", c_p), ("owner", c_p), ("cluster", c_p),
                ("target", c_p), ("dist", c_p), ("final_cluster", c_p), ("eta_out", c_p),
                ("counts", c_p), ("ceptr", c_p), ("cpins", c_p), ("cw", c_p), ("emap", c_p)]


def sort_resistance(R, stream=None):
    """hef_sort_resistance (Algorithm 1 step 6): hyperedge ids by ascending R,
    ties by id."""
    L = lib()
    m = int(R.numel())
    R = R.to(torch.float64).contiguous()
    order = torch.empty(max(m, 1), dtype=torch.int32, device=R.device)[:m]
    ws = _workspace(L.hef_level_workspace_bytes(0, m, 0), R.device)
    _check("hef_sort_resistance",
           L.hef_sort_resistance(m, _ptr(R), _ptr(order), _ptr(ws), ws.numel(), _stream(stream)))
    return order


def coarsen_level(inc, eptr, pins, w, R, eta=None, Q=None, K=None, QH=None, delta=-1.0,
                  quantile=0.5, stream=None):
    """hef_coarsen_level: one coarsening level (Algorithm 2 steps 4-10) from
    the scores R of the incidence `inc` (built from eptr, pins, w).  Returns
    a dict of device tensors; `counts` holds nc, nf, m', P', status (the
    coarse arrays are valid up to m' and P')."""
    L = lib()
    dev = R.device
    n, m, P = inc.n, inc.m, inc.P
    o = dict(R_upd=torch.empty(max(m, 1), dtype=torch.float64, device=dev),
             order=torch.empty(max(m, 1), dtype=torch.int32, device=dev),
             delta=torch.empty(1, dtype=torch.float64, device=dev),
             owner=torch.empty(max(n, 1), dtype=torch.int32, device=dev),
             cluster=torch.empty(max(n, 1), dtype=torch.int32, device=dev),
             target=torch.empty(max(n, 1), dtype=torch.int32, device=dev),
             dist=torch.empty(max(n, 1), dtype=torch.float64, device=dev),
             final_cluster=torch.empty(max(n, 1), dtype=torch.int32, device=dev),
             eta_out=torch.empty(max(n, 1), dtype=torch.float64, device=dev),
             counts=torch.zeros(5, dtype=torch.int32, device=dev),
             ceptr=torch.empty(m + 1, dtype=torch.int64, device=dev),
             cpins=torch.empty(max(P, 1), dtype=torch.int32, device=dev),
             cw=torch.empty(max(m, 1), dtype=torch.float64, device=dev),
             emap=torch.empty(max(m, 1), dtype=torch.int32, device=dev))
    st = _LevelOut(*[_ptr(o[f]) for f, _ in _LevelOut._fields_])
    code = _dtype_code(Q.dtype) if Q is not None else HEF_F64
    Kc = int(K) if Q is not None else 0
    ws = _workspace(L.hef_level_workspace_bytes(n, m, Kc), dev)
    _check("hef_coarsen_level",
           L.hef_coarsen_level(inc.handle, _ptr(eptr), _ptr(pins), _ptr(w), _ptr(R), _ptr(eta),
                               _ptr(Q), Q.stride(0) if Q is not None else 0, Kc, code, _ptr(QH),
                               float(delta), float(quantile), ctypes.byref(st), _ptr(ws),
                               ws.numel(), _stream(stream)))
    o["_keep"] = (ws, R, eta, Q, QH)
    return o


def level_sizes(out):
    """(nc, nf, m', P') of a coarsen_level result (synchronises); raises if
    the contraction's bounded wait ran out."""
    c = out["counts"].cpu().tolist()
    if c[4]:
        raise HefError("hef_coarsen_level", -5, f"contraction wait status {c[4]}")
    return c[0], c[1], c[2], c[3]


def multilevel(n, eptr, pins, w, starts, k, levels, dtype=torch.float32, quantile=0.5,
               min_vertices=2, clique_mode=HEF_CLIQUE_HYPEREDGE):
    """Algorithm 2's level loop (Section III-B): per level, Algorithm 1 on
    the current hypergraph (hef_build_incidence, hef_krylov_basis,
    hef_orthonormalize, hef_edge_resistance), then hef_coarsen_level with the
    previous level's supernode weights, and the coarse hypergraph as the next
    level's input.  `starts(level, n, m)` returns that level's random start
    block (x0_clique n x S, x0_star (n+m) x S, CUDA float64).  Returns the
    per-level records and the cluster of every original vertex."""
    dev = eptr.device
    eta = None
    cur = (int(n), eptr, pins, w)
    of_orig = torch.arange(int(n), dtype=torch.int32, device=dev)
    out = []
    for lv in range(int(levels)):
        nl, ep, pi, wl = cur
        ml = int(ep.numel() - 1)
        if nl < min_vertices or ml < 1:
            break
        x0c, x0b = starts(lv, nl, ml)
        S = int(x0c.shape[1])
        K = 2 * int(k) * S
        inc = build_incidence(nl, ep, pi, wl, clique_mode)
        V = krylov_basis(inc, x0c, x0b, k, dtype)
        Q, _, rank = orthonormalize(V, K)
        sc = edge_resistance(inc, Q, K)
        inc.check()
        lo = coarsen_level(inc, ep, pi, wl, sc["R"], eta, Q, K, sc["QH"], quantile=quantile)
        nc, nf, mc, pc = level_sizes(lo)
        of_orig = lo["final_cluster"][of_orig.long()]
        out.append(dict(n=nl, m=ml, P=int(pi.numel()), R=sc["R"], Q=Q, QH=sc["QH"], K=K,
                        eptr=ep, pins=pi, w=wl, eta=eta, level=lo, nc=nc, nf=nf, m_next=mc,
                        P_next=pc, incidence=inc))
        eta = lo["eta_out"][:nf].clone()
        cur = (nf, lo["ceptr"][:mc + 1].clone(), lo["cpins"][:pc].clone(), lo["cw"][:mc].clone())
    return out, of_orig


def resistance_host_workspace(n, m, P, k, S, dtype=torch.float32, device=None):
    """Device workspace of hef_resistance_host."""
    nb = lib().hef_resistance_host_workspace_bytes(int(n), int(m), int(P), int(k), int(S),
                                                   _dtype_code(dtype))
    if nb == 0:
        raise HefError("hef_resistance_host_workspace_bytes", -1, "bad sizes")
    return _workspace(nb, device or torch.device("cuda", torch.cuda.current_device()))


def resistance_host(n, eptr, pins, w, x0_clique, x0_star, k, dtype=torch.float32, R_out=None,
                    workspace=None, clique_mode=HEF_CLIQUE_HYPEREDGE, stream=None):
    """hef_resistance_host: Algorithm 1 from HOST (CPU) tensors; returns R as
    a host tensor (synchronises the stream)."""
    m = int(eptr.numel() - 1)
    P = int(pins.numel())
    S = int(x0_clique.shape[1])
    for t in (eptr, pins, w, x0_clique, x0_star):
        assert not t.is_cuda and t.is_contiguous()
    if R_out is None:
        R_out = torch.empty(m, dtype=torch.float64)
    if workspace is None:
        workspace = resistance_host_workspace(n, m, P, k, S, dtype)
    _check("hef_resistance_host",
           lib().hef_resistance_host(int(n), m, P, _ptr(eptr), _ptr(pins), _ptr(w),
                                     _ptr(x0_clique), _ptr(x0_star), int(k), S,
                                     _dtype_code(dtype), int(clique_mode), _ptr(R_out),
                                     _ptr(workspace), workspace.numel(), _stream(stream)))
    return R_out


def set_batch_krylov_form(form):
    """hef_set_batch_krylov_form for batched calls from this thread: 1 = one
    cooperative Krylov launch for all items, 0 = per-step launches per item."""
    _check("hef_set_batch_krylov_form", lib().hef_set_batch_krylov_form(int(form)))


def batch_krylov_form():
    return int(lib().hef_batch_krylov_form())
