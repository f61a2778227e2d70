"""ctypes binding of the dcflow C ABI (include/dcflow.h).

Argument marshalling only: every step of the loadflow runs inside
libdcflow.so.  PyTorch supplies device memory and streams.  Loading fails
loudly when the library has not been built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_char_p, c_double, c_int32, c_int64, c_void_p

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdcflow.so")

DCFLOW_OK = 0
FP64, FP32 = 0, 1
PRECISIONS = {"fp64": FP64, "fp32": FP32}


class Options(ctypes.Structure):
    _fields_ = [("precision", c_int32), ("device", c_int32), ("chunk_topo", c_int32),
                ("island_tol", c_double)]


class Study(ctypes.Structure):
    _fields_ = [("mon", POINTER(c_int32)), ("n_mon", c_int32),
                ("cont", POINTER(c_int32)), ("n_cont", c_int32),
                ("limit", POINTER(c_double)),
                ("split_bus", POINTER(c_int32)), ("n_split_bus", c_int32),
                ("outage_cand", POINTER(c_int32)), ("n_outage_cand", c_int32)]


class Batch(ctypes.Structure):
    _fields_ = [("n_topo", c_int32), ("split_ptr", c_void_p), ("split_sub", c_void_p),
                ("split_mask", c_void_p), ("out_ptr", c_void_p), ("out_branch", c_void_p),
                ("n_time", c_int32), ("inj", c_void_p), ("n_var", c_int32),
                ("var_ptr", c_void_p), ("var_bus", c_void_p), ("var_delta", c_void_p)]


class Results(ctypes.Structure):
    _fields_ = [("n0_flow", c_void_p), ("n0_max_loading", c_void_p), ("n1_max_loading", c_void_p),
                ("overload_sum", c_void_p), ("worst_cont", c_void_p), ("worst_mon", c_void_p),
                ("best_var", c_void_p), ("island_flag", c_void_p), ("n_island_cont", c_void_p),
                ("n1_cont_max", c_void_p)]


EXPORTED = ["dcflow_default_options", "dcflow_setup", "dcflow_base_ptdf", "dcflow_base_ptdf_noalloc",
            "dcflow_set_study",
            "dcflow_solve_batch", "dcflow_last_launch_count", "dcflow_profile", "dcflow_profile_read",
            "dcflow_gemm_bf16", "dcflow_destroy", "dcflow_strerror", "dcflow_last_error"]

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libdcflow.so (build it with paper_2501_17529_b300.csrc.build first)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libdcflow.so not built at {path}; run python -m paper_2501_17529_b300.csrc.build")
    lib = ctypes.CDLL(path)
    lib.dcflow_default_options.argtypes = [POINTER(Options)]
    lib.dcflow_default_options.restype = None
    lib.dcflow_setup.argtypes = [POINTER(c_void_p), c_int32, c_int32, POINTER(c_int32), POINTER(c_int32),
                                 POINTER(c_double), c_int32, POINTER(Options)]
    lib.dcflow_setup.restype = c_int32
    lib.dcflow_base_ptdf.argtypes = [c_void_p, POINTER(c_int32), c_int32, c_void_p, c_void_p]
    lib.dcflow_base_ptdf.restype = c_int32
    lib.dcflow_base_ptdf_noalloc.argtypes = [c_void_p, POINTER(c_int32), c_int32, c_void_p, c_void_p]
    lib.dcflow_base_ptdf_noalloc.restype = c_int32
    lib.dcflow_set_study.argtypes = [c_void_p, POINTER(Study)]
    lib.dcflow_set_study.restype = c_int32
    lib.dcflow_solve_batch.argtypes = [c_void_p, POINTER(Batch), POINTER(Results), c_void_p]
    lib.dcflow_solve_batch.restype = c_int32
    lib.dcflow_last_launch_count.argtypes = [c_void_p]
    lib.dcflow_last_launch_count.restype = c_int64
    lib.dcflow_profile.argtypes = [c_void_p, c_int32]
    lib.dcflow_profile.restype = c_int32
    lib.dcflow_profile_read.argtypes = [c_void_p, POINTER(c_double), POINTER(c_int64)]
    lib.dcflow_profile_read.restype = c_int32
    lib.dcflow_gemm_bf16.argtypes = [c_int32, c_int32, c_int32, c_void_p, c_int32, c_void_p, c_int32, c_void_p,
                                     c_int32, c_void_p, c_int32, c_int32, c_void_p]
    lib.dcflow_gemm_bf16.restype = c_int32
    lib.dcflow_destroy.argtypes = [c_void_p]
    lib.dcflow_destroy.restype = None
    lib.dcflow_strerror.argtypes = [c_int32]
    lib.dcflow_strerror.restype = c_char_p
    lib.dcflow_last_error.argtypes = []
    lib.dcflow_last_error.restype = c_char_p
    _lib = lib
    return lib


class DCFlowError(RuntimeError):
    def __init__(self, code: int, where: str):
        lib = load_library()
        super().__init__(f"{where}: {lib.dcflow_strerror(code).decode()} ({code}): "
                         f"{lib.dcflow_last_error().decode()}")
        self.code = code


def _check(rc: int, where: str):
    if rc != DCFLOW_OK:
        raise DCFlowError(rc, where)


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(POINTER(c_int32))


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(POINTER(c_double))


def _ptr(t):
    return None if t is None else c_void_p(t.data_ptr())


def _stream_ptr(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return c_void_p(s.cuda_stream)


# ---------------------------------------------------------------------------
# entry points (same names as the C ABI)
# ---------------------------------------------------------------------------

def dcflow_default_options() -> Options:
    o = Options()
    load_library().dcflow_default_options(byref(o))
    return o


def dcflow_setup(n_bus, f, t, b, slack, precision="fp32", device=-1, chunk_topo=0, island_tol=0.0):
    lib = load_library()
    o = dcflow_default_options()
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.device = int(device)
    o.chunk_topo = int(chunk_topo)
    if island_tol:
        o.island_tol = float(island_tol)
    fa, fp = _i32(f)
    ta, tp = _i32(t)
    ba, bp = _f64(b)
    ctx = c_void_p()
    _check(lib.dcflow_setup(byref(ctx), int(n_bus), int(fa.size), fp, tp, bp, int(slack), byref(o)),
           "dcflow_setup")
    return ctx


def dcflow_base_ptdf(ctx, rows, out, stream=None):
    ra, rp = _i32(rows)
    _check(load_library().dcflow_base_ptdf(ctx, rp, int(ra.size), _ptr(out), _stream_ptr(stream)),
           "dcflow_base_ptdf")


def dcflow_base_ptdf_noalloc(ctx, rows, out, stream=None):
    """Rows of the base PTDF without any device allocation (fixed 8 MiB workspace
    inside the library); for callers that cannot allocate device memory."""
    ra, rp = _i32(rows)
    _check(load_library().dcflow_base_ptdf_noalloc(ctx, rp, int(ra.size), _ptr(out), _stream_ptr(stream)),
           "dcflow_base_ptdf_noalloc")


def dcflow_set_study(ctx, mon, cont, limit, split_bus=None, outage_cand=None):
    ma, mp = _i32(mon)
    ca, cp = _i32(cont)
    la, lp = _f64(limit)
    s = Study(mp, int(ma.size), cp, int(ca.size), lp, None, 0, None, 0)
    keep = [ma, ca, la]
    if split_bus is not None:
        sa, spp = _i32(split_bus)
        keep.append(sa)
        s.split_bus, s.n_split_bus = spp, int(sa.size)
    if outage_cand is not None:
        oa, op = _i32(outage_cand)
        keep.append(oa)
        s.outage_cand, s.n_outage_cand = op, int(oa.size)
    _check(load_library().dcflow_set_study(ctx, byref(s)), "dcflow_set_study")


def dcflow_solve_batch(ctx, batch: Batch, results: Results, stream=None):
    _check(load_library().dcflow_solve_batch(ctx, byref(batch), byref(results), _stream_ptr(stream)),
           "dcflow_solve_batch")


def dcflow_last_launch_count(ctx) -> int:
    return int(load_library().dcflow_last_launch_count(ctx))


def dcflow_profile(ctx, enable: bool):
    _check(load_library().dcflow_profile(ctx, 1 if enable else 0), "dcflow_profile")


def dcflow_profile_read(ctx):
    ms, n = c_double(), c_int64()
    _check(load_library().dcflow_profile_read(ctx, byref(ms), byref(n)), "dcflow_profile_read")
    return {"n1_ms": ms.value, "n1_launches": n.value}


def dcflow_gemm_bf16(A, B, bias=None, relu=False, out=None, out_bf16=False, stream=None):
    """D = A @ B^T (+ bias) (ReLU) on the tensor cores; A [M, K], B [N, K] bf16 torch tensors."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    if out is None:
        out = torch.empty((M, N), dtype=torch.bfloat16 if out_bf16 else torch.float32, device=A.device)
    _check(load_library().dcflow_gemm_bf16(M, N, K, _ptr(A), A.stride(0), _ptr(B), B.stride(0), _ptr(bias),
                                           1 if relu else 0, _ptr(out), out.stride(0), 1 if out_bf16 else 0,
                                           _stream_ptr(stream)), "dcflow_gemm_bf16")
    return out


def dcflow_destroy(ctx):
    if ctx is not None and ctx.value:
        load_library().dcflow_destroy(ctx)


def dcflow_strerror(code: int) -> str:
    return load_library().dcflow_strerror(int(code)).decode()


# ---------------------------------------------------------------------------
# torch-side convenience (device memory only; no arithmetic)
# ---------------------------------------------------------------------------

class DeviceBatch:
    """Device copies of the topology CSR, injections and optional candidates."""

    def __init__(self, topo, inj, var=None, device="cuda"):
        import torch
        self.n_topo = int(topo.n_topo)
        self.n_time = int(np.atleast_2d(inj).shape[0])
        self.split_ptr = torch.as_tensor(np.asarray(topo.split_ptr, np.int32), device=device)
        self.split_sub = torch.as_tensor(np.asarray(topo.split_sub, np.int32), device=device)
        self.split_mask = torch.as_tensor(np.asarray(topo.split_mask, np.uint64).view(np.int64), device=device)
        self.out_ptr = torch.as_tensor(np.asarray(topo.out_ptr, np.int32), device=device)
        self.out_branch = torch.as_tensor(np.asarray(topo.out_branch, np.int32), device=device)
        self.inj = torch.as_tensor(np.ascontiguousarray(np.atleast_2d(inj), np.float64), device=device)
        self.n_var = 0 if var is None else int(var.n_var)
        if self.n_var:
            self.var_ptr = torch.as_tensor(np.asarray(var.var_ptr, np.int32), device=device)
            self.var_bus = torch.as_tensor(np.asarray(var.var_bus, np.int32), device=device)
            self.var_delta = torch.as_tensor(np.asarray(var.var_delta, np.float64), device=device)
        else:
            self.var_ptr = self.var_bus = self.var_delta = None

    def cstruct(self) -> Batch:
        return Batch(self.n_topo, _ptr(self.split_ptr), _ptr(self.split_sub), _ptr(self.split_mask),
                     _ptr(self.out_ptr), _ptr(self.out_branch), self.n_time, _ptr(self.inj), self.n_var,
                     _ptr(self.var_ptr), _ptr(self.var_bus), _ptr(self.var_delta))


class DeviceResults:
    """Caller-owned device outputs of one batch."""

    def __init__(self, n_topo, n_time, n_mon, want_flows=False, want_var=False, device="cuda", n_cont=0,
                 want_cont_max=False):
        import torch
        nt = max(1, n_topo * n_time)
        self.n0_flow = torch.empty(max(1, n_topo * n_time * n_mon), dtype=torch.float64, device=device) if want_flows else None
        self.n0_max_loading = torch.empty(nt, dtype=torch.float64, device=device)
        self.n1_max_loading = torch.empty(nt, dtype=torch.float64, device=device)
        self.overload_sum = torch.empty(nt, dtype=torch.float64, device=device)
        self.worst_cont = torch.empty(nt, dtype=torch.int32, device=device)
        self.worst_mon = torch.empty(nt, dtype=torch.int32, device=device)
        self.best_var = torch.empty(nt, dtype=torch.int32, device=device) if want_var else None
        self.island_flag = torch.empty(max(1, n_topo), dtype=torch.uint8, device=device)
        self.n_island_cont = torch.empty(max(1, n_topo), dtype=torch.int32, device=device)
        self.n1_cont_max = (torch.empty(max(1, n_topo * n_time * n_cont), dtype=torch.float32, device=device)
                            if want_cont_max else None)
        self.shape = (n_topo, n_time, n_mon)
        self.n_cont = n_cont

    def cstruct(self) -> Results:
        return Results(_ptr(self.n0_flow), _ptr(self.n0_max_loading), _ptr(self.n1_max_loading),
                       _ptr(self.overload_sum), _ptr(self.worst_cont), _ptr(self.worst_mon),
                       _ptr(self.best_var), _ptr(self.island_flag), _ptr(self.n_island_cont),
                       _ptr(self.n1_cont_max))

    def to_host(self) -> dict:
        N, T, M = self.shape
        out = {
            "n0_max": self.n0_max_loading[:N * T].cpu().numpy().reshape(N, T),
            "n1_max": self.n1_max_loading[:N * T].cpu().numpy().reshape(N, T),
            "ovl": self.overload_sum[:N * T].cpu().numpy().reshape(N, T),
            "worst_cont": self.worst_cont[:N * T].cpu().numpy().reshape(N, T).astype(np.int64),
            "worst_mon": self.worst_mon[:N * T].cpu().numpy().reshape(N, T).astype(np.int64),
            "status": self.island_flag[:N].cpu().numpy().astype(np.int64),
            "n_island_cont": self.n_island_cont[:N].cpu().numpy().astype(np.int64),
        }
        if self.best_var is not None:
            out["best_var"] = self.best_var[:N * T].cpu().numpy().reshape(N, T).astype(np.int64)
        if self.n0_flow is not None:
            out["n0_flow"] = self.n0_flow[:N * T * M].cpu().numpy().reshape(N, T, M)
        if self.n1_cont_max is not None:
            out["cont_max"] = self.n1_cont_max[:N * T * self.n_cont].cpu().numpy().reshape(N, T, self.n_cont)
        return out


class Solver:
    """One grid + study on the current CUDA device."""

    def __init__(self, grid, precision="fp32", chunk_topo=0, island_tol=0.0, device=-1):
        self.grid = grid
        self.ctx = dcflow_setup(grid.n_bus, grid.f, grid.t, grid.b, grid.slack, precision=precision,
                                device=device, chunk_topo=chunk_topo, island_tol=island_tol)
        self.n_mon = 0
        self.n_cont = 0

    def set_study(self, mon, cont, limit, split_bus=None, outage_cand=None):
        dcflow_set_study(self.ctx, mon, cont, limit, split_bus, outage_cand)
        self.n_mon = int(np.asarray(mon).size)
        self.n_cont = int(np.asarray(cont).size)

    def base_ptdf(self, rows, stream=None):
        import torch
        rows = np.asarray(rows, np.int32)
        out = torch.empty((rows.size, self.grid.n_bus), dtype=torch.float64, device="cuda")
        dcflow_base_ptdf(self.ctx, rows, out, stream)
        return out

    def solve(self, dbatch: DeviceBatch, want_flows=False, results: DeviceResults | None = None, stream=None,
              want_cont_max=False):
        res = results or DeviceResults(dbatch.n_topo, dbatch.n_time, self.n_mon, want_flows, dbatch.n_var > 0,
                                       n_cont=self.n_cont, want_cont_max=want_cont_max)
        dcflow_solve_batch(self.ctx, dbatch.cstruct(), res.cstruct(), stream)
        return res

    def last_launch_count(self) -> int:
        return dcflow_last_launch_count(self.ctx)

    def close(self):
        dcflow_destroy(self.ctx)
        self.ctx = None

    def __del__(self):
        try:
            if getattr(self, "ctx", None) is not None:
                self.close()
        except Exception:
            pass
