"""ctypes binding of libkb (include/kb.h): argument marshalling only.

Every numerical step runs inside the CUDA library; this module converts Python/numpy/torch
arguments to the C types of the ABI, calls the entry point of the same name and turns
negative status codes into :class:`KbError`.  It refuses to run without the compiled
library (there is no Python or CPU fallback).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkb.so")

METHODS = {"cbl": 0, "gbl": 1, "sbl": 2, "cheb": 3, "cheb2": 4}
PHIS = {"exp": 0, "spline": 1}
DTYPES = {"f32": 0, "bf16": 1, "f64": 2}
KB_GRAPH_SKIP_SYMMETRY_CHECK = 1
KB_GRAPH_NORMALIZED = 2
STATUS = {0: "KB_OK", -1: "KB_ERR_ARG", -2: "KB_ERR_CSR", -3: "KB_ERR_NODES", -4: "KB_ERR_CUDA",
          -5: "KB_ERR_NOMEM", -6: "KB_ERR_BREAKDOWN", -7: "KB_ERR_UNSUPPORTED", -8: "KB_ERR_BUSY",
          -9: "KB_ERR_ORTHOGONALITY", 1: "KB_PENDING"}
KB_PENDING = 1


class KbError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class kb_params(ctypes.Structure):
    _fields_ = [("t", ctypes.c_double), ("eps", ctypes.c_double), ("s", ctypes.c_double),
                ("lambda_max", ctypes.c_double), ("reorth", ctypes.c_int32),
                ("basis", ctypes.c_int32), ("no_frontier", ctypes.c_int32),
                ("two_pass", ctypes.c_int32), ("tol", ctypes.c_double)]


class kb_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("steps_done", ctypes.c_int32),
                ("breakdown_step", ctypes.c_int32), ("spmm_launches", ctypes.c_int32),
                ("lambda_used", ctypes.c_double), ("est_change", ctypes.c_double)]


class kb_server_config(ctypes.Structure):
    _fields_ = [("streams", ctypes.c_int32), ("queue_capacity", ctypes.c_int32),
                ("memory_budget", ctypes.c_int64), ("fallback_sbl", ctypes.c_int32)]


class kb_kernel_stats(ctypes.Structure):
    _fields_ = [("kernel_class", ctypes.c_int32), ("launches", ctypes.c_int32),
                ("total_ms", ctypes.c_double), ("alg_bytes", ctypes.c_double),
                ("alg_flops", ctypes.c_double)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libkb.so (raises if it was not built: no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing; build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    L.kb_graph_create.argtypes = [i64, vp, vp, vp, i32, vp, P(vp)]
    L.kb_graph_create.restype = ctypes.c_int
    L.kb_graph_destroy.argtypes = [vp]
    L.kb_graph_destroy.restype = None
    L.kb_graph_info.argtypes = [vp, P(i64), P(i64), P(dbl), P(i32)]
    L.kb_graph_info.restype = ctypes.c_int
    L.kb_graph_lambda_bounds.argtypes = [vp, P(dbl), P(dbl)]
    L.kb_graph_lambda_bounds.restype = ctypes.c_int
    for name in ("kb_krylov_apply", "kb_krylov_apply_host"):
        f = getattr(L, name)
        f.argtypes = [vp, ctypes.c_int, ctypes.c_int, P(kb_params), vp, i32, i32, vp, vp, P(kb_info)]
        f.restype = ctypes.c_int
    L.kb_status_string.argtypes = [ctypes.c_int]
    L.kb_status_string.restype = ctypes.c_char_p
    L.kb_last_error.argtypes = []
    L.kb_last_error.restype = ctypes.c_char_p
    L.kb_version.restype = ctypes.c_int
    L.kb_cheb_lobatto_coeffs.argtypes = [ctypes.c_int, P(kb_params), i32, dbl, i32, vp]
    L.kb_cheb_lobatto_coeffs.restype = ctypes.c_int
    L.kb_exp_series_coeffs.argtypes = [dbl, dbl, dbl, vp, i32, P(i32)]
    L.kb_exp_series_coeffs.restype = ctypes.c_int
    L.kb_spline_quadrature.argtypes = [dbl, dbl, dbl, dbl, vp, vp, i32, P(i32), P(i32)]
    L.kb_spline_quadrature.restype = ctypes.c_int
    L.kb_profile_enable.argtypes = [i32]
    L.kb_profile_enable.restype = ctypes.c_int
    L.kb_profile_read.argtypes = [P(kb_kernel_stats), i32, P(i32)]
    L.kb_profile_read.restype = ctypes.c_int
    L.kb_launch_counter.argtypes = []
    L.kb_launch_counter.restype = ctypes.c_int64
    L.kb_kernel_class_name.argtypes = [i32]
    L.kb_kernel_class_name.restype = ctypes.c_char_p
    L.kb_workspace_bytes.argtypes = [vp, ctypes.c_int, ctypes.c_int, P(kb_params), i32, i32,
                                     P(ctypes.c_uint64)]
    L.kb_workspace_bytes.restype = ctypes.c_int
    L.kb_rls_predict.argtypes = [vp, ctypes.c_int, ctypes.c_int, P(kb_params), vp, i32, i32, vp,
                                 dbl, vp, vp, vp, P(kb_info)]
    L.kb_rls_predict.restype = ctypes.c_int
    L.kb_server_create.argtypes = [i32, P(kb_server_config), P(vp)]
    L.kb_server_create.restype = ctypes.c_int
    L.kb_server_submit.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, P(kb_params), vp, i32, i32,
                                   vp, P(i64)]
    L.kb_server_submit.restype = ctypes.c_int
    L.kb_server_poll.argtypes = [vp, i64, i32, P(kb_info), P(dbl)]
    L.kb_server_poll.restype = ctypes.c_int
    L.kb_server_destroy.argtypes = [vp]
    L.kb_server_destroy.restype = ctypes.c_int
    _lib = L
    return L


def _check(rc: int):
    if rc != 0:
        raise KbError(rc, lib().kb_last_error().decode())


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(a) -> int:
    """Address of a numpy array or torch tensor (host or device)."""
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def make_params(t=1.0, eps=0.01, s=1.0, lambda_max=0.0, reorth=0, basis="f32",
                no_frontier=0, two_pass=0, tol=0.0) -> kb_params:
    """kb_params with the C defaults (fields as documented in include/kb.h): reorth 0/1/2
    (none / full / local, cbl), basis "f32" / "bf16" / "f64", two_pass 1 keeps three blocks
    and runs the recurrence twice, tol > 0 (cbl) stops at the first check step whose projected
    result changed by at most tol (m is then the largest number of steps)."""
    return kb_params(float(t), float(eps), float(s), float(lambda_max), int(reorth),
                     DTYPES[basis] if isinstance(basis, str) else int(basis), int(no_frontier),
                     int(two_pass), float(tol))


class Graph:
    """Device copy of a CSR graph Laplacian (kb_graph_create / kb_graph_destroy)."""

    def __init__(self, rowptr, col, val=None, flags=0, stream=None):
        self._keep = [np.ascontiguousarray(rowptr, dtype=np.int32),
                      np.ascontiguousarray(col, dtype=np.int32)]
        if val is not None:
            self._keep.append(np.ascontiguousarray(val, dtype=np.float32))
        n = self._keep[0].size - 1
        h = ctypes.c_void_p()
        rc = lib().kb_graph_create(n, self._keep[0].ctypes.data, self._keep[1].ctypes.data,
                                   self._keep[2].ctypes.data if val is not None else None,
                                   int(flags), _stream_ptr(stream), ctypes.byref(h))
        self._keep = None
        _check(rc)
        self.handle = h

    @classmethod
    def from_csr(cls, g, **kw):
        return cls(g.rowptr, g.col, g.val, **kw)

    def info(self):
        n, nnz, lam, su = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double(), ctypes.c_int32()
        _check(lib().kb_graph_info(self.handle, ctypes.byref(n), ctypes.byref(nnz),
                                   ctypes.byref(lam), ctypes.byref(su)))
        gb, pb = ctypes.c_double(), ctypes.c_double()
        _check(lib().kb_graph_lambda_bounds(self.handle, ctypes.byref(gb), ctypes.byref(pb)))
        return {"n": n.value, "nnz_offdiag": nnz.value, "lambda_max": lam.value,
                "standard_unit": bool(su.value), "lambda_projected": pb.value}

    @property
    def n(self):
        return self.info()["n"]

    @property
    def lambda_max(self):
        return self.info()["lambda_max"]

    def destroy(self):
        if getattr(self, "handle", None):
            lib().kb_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.destroy()


def kb_graph_create(rowptr, col, val=None, flags=0, stream=None) -> Graph:
    return Graph(rowptr, col, val, flags, stream)


def kb_krylov_apply(graph: Graph, method: str, phi: str, params: kb_params, nodes, M: int, m: int,
                    Y, stream=None, info: bool = False):
    """Y (device, n x M float32, row-major) <- approximation of phi(L) E_W."""
    nodes = np.ascontiguousarray(nodes, dtype=np.int32)
    inf = kb_info() if info else None
    rc = lib().kb_krylov_apply(graph.handle, METHODS[method], PHIS[phi], ctypes.byref(params),
                               nodes.ctypes.data, int(M), int(m), ctypes.c_void_p(_ptr(Y)),
                               _stream_ptr(stream), ctypes.byref(inf) if info else None)
    _check(rc)
    if info:
        return {"status": inf.status, "steps_done": inf.steps_done,
                "breakdown_step": inf.breakdown_step, "spmm_launches": inf.spmm_launches,
                "lambda_used": inf.lambda_used, "est_change": inf.est_change}
    return None


def kb_krylov_apply_host(graph: Graph, method: str, phi: str, params: kb_params, nodes, M: int,
                         m: int, Y_host, stream=None, info: bool = False):
    """Same as kb_krylov_apply with Y in host memory (numpy array or pinned tensor)."""
    nodes = np.ascontiguousarray(nodes, dtype=np.int32)
    inf = kb_info() if info else None
    rc = lib().kb_krylov_apply_host(graph.handle, METHODS[method], PHIS[phi], ctypes.byref(params),
                                    nodes.ctypes.data, int(M), int(m), ctypes.c_void_p(_ptr(Y_host)),
                                    _stream_ptr(stream), ctypes.byref(inf) if info else None)
    _check(rc)
    if info:
        return {"status": inf.status, "steps_done": inf.steps_done,
                "breakdown_step": inf.breakdown_step, "spmm_launches": inf.spmm_launches,
                "lambda_used": inf.lambda_used, "est_change": inf.est_change}
    return None


def kb_cheb_lobatto_coeffs(phi: str, params: kb_params, m: int, lam: float, sqrt_phi=False):
    c = np.zeros(m + 1, dtype=np.float64)
    _check(lib().kb_cheb_lobatto_coeffs(PHIS[phi], ctypes.byref(params), int(m), float(lam),
                                        int(bool(sqrt_phi)), c.ctypes.data))
    return c


def kb_exp_series_coeffs(t: float, lam: float, tol: float = 1e-17, cap: int = 100000):
    d = np.zeros(cap, dtype=np.float64)
    cnt = ctypes.c_int32()
    _check(lib().kb_exp_series_coeffs(float(t), float(lam), float(tol), d.ctypes.data, int(cap),
                                      ctypes.byref(cnt)))
    return d[:cnt.value].copy()


def kb_spline_quadrature(eps: float, s: float, lam: float, tol: float = 1e-14, cap: int = 4096):
    """(shift, weight, s_int) of the quadrature form of (eps + lambda)^{-s} on [0, lam]."""
    sh = np.zeros(cap, dtype=np.float64)
    w = np.zeros(cap, dtype=np.float64)
    cnt = ctypes.c_int32()
    si = ctypes.c_int32()
    _check(lib().kb_spline_quadrature(float(eps), float(s), float(lam), float(tol), sh.ctypes.data,
                                      w.ctypes.data, int(cap), ctypes.byref(cnt), ctypes.byref(si)))
    return sh[:cnt.value].copy(), w[:cnt.value].copy(), si.value


def kb_profile_enable(on: bool = True):
    _check(lib().kb_profile_enable(int(bool(on))))


def kb_profile_read():
    arr = (kb_kernel_stats * 16)()
    cnt = ctypes.c_int32()
    _check(lib().kb_profile_read(arr, 16, ctypes.byref(cnt)))
    out = {}
    for i in range(cnt.value):
        s = arr[i]
        out[lib().kb_kernel_class_name(s.kernel_class).decode()] = {
            "launches": s.launches, "total_ms": s.total_ms, "alg_bytes": s.alg_bytes,
            "alg_flops": s.alg_flops}
    return out


def kb_launch_counter() -> int:
    return int(lib().kb_launch_counter())


def kernel_columns(graph: Graph, method: str, phi: str, nodes, m: int, stream=None, info=False,
                   **params):
    """Allocate Y on the current CUDA device (torch) and run kb_krylov_apply."""
    import torch
    nodes = np.ascontiguousarray(nodes, dtype=np.int32)
    Y = torch.empty((graph.n, nodes.size), dtype=torch.float32, device="cuda")
    r = kb_krylov_apply(graph, method, phi, make_params(**params), nodes, nodes.size, m, Y,
                        stream=stream, info=info)
    return (Y, r) if info else Y


def kb_cheb_apply_fixed_scratch(graph: Graph, phi: str, params: kb_params, nodes, M: int, m: int,
                                Y, stream=None):
    """KB_CHEB into device Y using the library's fixed scratch array (no allocation)."""
    L = lib()
    if not hasattr(L, "_fixed_scratch_typed"):
        L.kb_cheb_apply_fixed_scratch.argtypes = [ctypes.c_void_p, ctypes.c_int,
                                                  ctypes.POINTER(kb_params), ctypes.c_void_p,
                                                  ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                                  ctypes.c_void_p]
        L.kb_cheb_apply_fixed_scratch.restype = ctypes.c_int
        L._fixed_scratch_typed = True
    nodes = np.ascontiguousarray(nodes, dtype=np.int32)
    _check(L.kb_cheb_apply_fixed_scratch(graph.handle, PHIS[phi], ctypes.byref(params),
                                         nodes.ctypes.data, int(M), int(m),
                                         ctypes.c_void_p(_ptr(Y)), _stream_ptr(stream)))


def kb_workspace_bytes(graph: Graph, method: str, phi: str, params: kb_params, M: int, m: int) -> int:
    """Device scratch bytes one kb_krylov_apply call takes (kb_workspace_bytes)."""
    b = ctypes.c_uint64()
    _check(lib().kb_workspace_bytes(graph.handle, METHODS[method], PHIS[phi], ctypes.byref(params),
                                    int(M), int(m), ctypes.byref(b)))
    return int(b.value)


class Server:
    """Request queue over kb_krylov_apply (kb_server_create / submit / poll / destroy).

    fallback_sbl: rerun a cbl / gbl request that ends in a rank-deficient block
    (KB_ERR_BREAKDOWN) as sbl; its info then carries the block breakdown step."""

    def __init__(self, streams: int = 4, queue_capacity: int = 4096, memory_budget: int = 0,
                 device: int = 0, fallback_sbl: bool = False):
        cfg = kb_server_config(int(streams), int(queue_capacity), int(memory_budget),
                               int(bool(fallback_sbl)))
        h = ctypes.c_void_p()
        _check(lib().kb_server_create(int(device), ctypes.byref(cfg), ctypes.byref(h)))
        self.handle = h
        self._keep = {}   # ticket -> (graph, Y) kept alive until the request is polled

    def submit(self, graph: Graph, method: str, phi: str, params: kb_params, nodes, m: int, Y) -> int:
        nodes = np.ascontiguousarray(nodes, dtype=np.int32)
        t = ctypes.c_int64()
        _check(lib().kb_server_submit(self.handle, graph.handle, METHODS[method], PHIS[phi],
                                      ctypes.byref(params), nodes.ctypes.data, int(nodes.size), int(m),
                                      ctypes.c_void_p(_ptr(Y)), ctypes.byref(t)))
        self._keep[t.value] = (graph, Y)
        return t.value

    def poll(self, ticket: int, wait_ms: int = 0):
        """None while pending; else (info dict, latency in ms).  Raises KbError on failure."""
        inf = kb_info()
        lat = ctypes.c_double()
        rc = lib().kb_server_poll(self.handle, int(ticket), int(wait_ms), ctypes.byref(inf),
                                  ctypes.byref(lat))
        if rc == KB_PENDING:
            return None
        self._keep.pop(ticket, None)
        _check(rc)
        return ({"status": inf.status, "steps_done": inf.steps_done,
                 "breakdown_step": inf.breakdown_step, "spmm_launches": inf.spmm_launches,
                 "lambda_used": inf.lambda_used, "est_change": inf.est_change}, lat.value)

    def close(self):
        if self.handle:
            _check(lib().kb_server_destroy(self.handle))
            self.handle = None
            self._keep.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def kb_rls_predict(graph: Graph, method: str, phi: str, params: kb_params, nodes, m: int, labels,
                   gamma: float, y_pred, stream=None):
    """RLS predictor (kb_rls_predict): fills device y_pred (n float32), returns c (numpy)."""
    nodes = np.ascontiguousarray(nodes, dtype=np.int32)
    lab = np.ascontiguousarray(labels, dtype=np.float64)
    c = np.zeros(nodes.size, dtype=np.float64)
    _check(lib().kb_rls_predict(graph.handle, METHODS[method], PHIS[phi], ctypes.byref(params),
                                nodes.ctypes.data, int(nodes.size), int(m), lab.ctypes.data,
                                float(gamma), ctypes.c_void_p(_ptr(y_pred)), c.ctypes.data,
                                _stream_ptr(stream), None))
    return c
