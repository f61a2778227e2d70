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
FP64, FP32, BF16X3 = 0, 1, 2
PRECISIONS = {"fp64": FP64, "fp32": FP32, "bf16x3": BF16X3}


class Options(ctypes.Structure):
    _fields_ = [("precision", c_int32), ("device", c_int32), ("chunk_topo", c_int32),
                ("island_tol", c_double), ("compact_n1", c_int32), ("autotune", c_int32),
                ("autotune_sample", c_int32), ("tie_band", c_double), ("output_first", c_int32)]


class Schedule(ctypes.Structure):
    """dcflow_schedule: chunk budget, rank classes, compacted N-1, remainder, measured ms."""
    _fields_ = [("budget_mb", c_int32), ("rank_bounds", c_int32 * 3), ("compact_n1", c_int32),
                ("remainder", c_int32), ("ms", ctypes.c_float)]

    def as_dict(self):
        return {"budget_mb": int(self.budget_mb), "rank_bounds": [int(x) for x in self.rank_bounds],
                "compact_n1": int(self.compact_n1), "remainder": int(self.remainder), "ms": float(self.ms)}


class Study(ctypes.Structure):
    _fields_ = [("mon", POINTER(c_int32)), ("n_mon", c_int32),
                ("cont", POINTER(c_int32)), ("n_cont", c_int32),
                ("limit", POINTER(c_double)),
                ("split_bus", POINTER(c_int32)), ("n_split_bus", c_int32),
                ("outage_cand", POINTER(c_int32)), ("n_outage_cand", c_int32),
                ("n_multi", c_int32), ("multi_ptr", POINTER(c_int32)), ("multi_branch", POINTER(c_int32))]


class Batch(ctypes.Structure):
    _fields_ = [("n_topo", c_int32), ("split_ptr", c_void_p), ("split_sub", c_void_p),
                ("split_mask", c_void_p), ("out_ptr", c_void_p), ("out_branch", c_void_p),
                ("n_time", c_int32), ("inj", c_void_p), ("n_var", c_int32),
                ("var_ptr", c_void_p), ("var_bus", c_void_p), ("var_delta", c_void_p),
                ("n_gen", c_int32), ("gen_bus", c_void_p), ("gen_p", c_void_p),
                ("n_inj", c_int32), ("inj_bus", c_void_p), ("inj_p", c_void_p), ("ti_ptr", c_void_p),
                ("ti_mask", c_void_p)]


class Results(ctypes.Structure):
    _fields_ = [("n0_flow", c_void_p), ("n0_max_loading", c_void_p), ("n1_max_loading", c_void_p),
                ("overload_sum", c_void_p), ("worst_cont", c_void_p), ("worst_mon", c_void_p),
                ("best_var", c_void_p), ("island_flag", c_void_p), ("n_island_cont", c_void_p),
                ("n1_cont_max", c_void_p), ("top_k", c_int32), ("top_cont", c_void_p), ("top_mon", c_void_p),
                ("top_loading", c_void_p), ("gen_max_loading", c_void_p), ("worst_gen", c_void_p),
                ("gen_overload_sum", c_void_p), ("multi_max_loading", c_void_p), ("worst_multi", c_void_p),
                ("multi_overload_sum", c_void_p), ("n_island_multi", c_void_p)]


class ScreenOptions(ctypes.Structure):
    _fields_ = [("top_k", c_int32), ("fallback_logit", ctypes.c_float), ("min_prob", ctypes.c_float)]


class ScreenReport(ctypes.Structure):
    _fields_ = [("n_eval", c_void_p), ("fallback", c_void_p), ("pred", c_void_p), ("evaluated", c_void_p)]


EXPORTED = ["dcflow_default_options", "dcflow_setup", "dcflow_base_ptdf", "dcflow_base_ptdf_noalloc",
            "dcflow_set_study",
            "dcflow_solve_batch", "dcflow_last_launch_count", "dcflow_autotune", "dcflow_set_schedule",
            "dcflow_last_schedule", "dcflow_profile", "dcflow_profile_read",
            "dcflow_profile_read_kind",
            "dcflow_gemm_bf16",
            "dcflow_screen_create", "dcflow_screen_destroy", "dcflow_screen_dims", "dcflow_screen_features",
            "dcflow_screen_labels", "dcflow_screen_backward", "dcflow_screen_adam", "dcflow_screen_train_step",
            "dcflow_screen_check", "dcflow_screen_logits", "dcflow_screen_get", "dcflow_screen_set",
            "dcflow_screen_adam_step", "dcflow_solve_batch_screened", "dcflow_selftest_bounded_wait",
            "dcflow_destroy", "dcflow_strerror", "dcflow_last_error"]

SCREEN_TENSORS = ("W1", "b1", "W2", "b2", "W3", "b3")
SCREEN_KINDS = ("param", "grad", "m", "v")

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
    lib.dcflow_autotune.argtypes = [c_void_p, POINTER(Batch), POINTER(Results), c_void_p, POINTER(Schedule), c_int32,
                                    POINTER(c_int32), POINTER(Schedule)]
    lib.dcflow_autotune.restype = c_int32
    lib.dcflow_set_schedule.argtypes = [c_void_p, POINTER(Schedule)]
    lib.dcflow_set_schedule.restype = c_int32
    lib.dcflow_last_schedule.argtypes = [c_void_p, POINTER(Schedule)]
    lib.dcflow_last_schedule.restype = c_int32
    lib.dcflow_profile.argtypes = [c_void_p, c_int32]
    lib.dcflow_profile.restype = c_int32
    lib.dcflow_profile_read.argtypes = [c_void_p, POINTER(c_double), POINTER(c_int64)]
    lib.dcflow_profile_read.restype = c_int32
    lib.dcflow_profile_read_kind.argtypes = [c_void_p, c_int32, POINTER(c_double), POINTER(c_int64)]
    lib.dcflow_profile_read_kind.restype = c_int32
    lib.dcflow_gemm_bf16.argtypes = [c_int32, c_int32, c_int32, c_void_p, c_int32, c_void_p, c_int32, c_void_p,
                                     c_int32, c_void_p, c_int32, c_int32, c_void_p]
    lib.dcflow_gemm_bf16.restype = c_int32
    f = ctypes.c_float
    sigs = {
        "dcflow_screen_create": ([c_void_p, c_int32, ctypes.c_uint64, POINTER(c_void_p)], c_int32),
        "dcflow_screen_destroy": ([c_void_p], None),
        "dcflow_screen_dims": ([c_void_p] + [POINTER(c_int32)] * 5, c_int32),
        "dcflow_screen_features": ([c_void_p, c_void_p, POINTER(Batch), c_void_p, c_int64, c_void_p, c_void_p],
                                   c_int32),
        "dcflow_screen_labels": ([c_void_p, c_void_p, c_int64, c_int32, c_void_p, c_int64, c_void_p], c_int32),
        "dcflow_screen_backward": ([c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_void_p, c_int32, c_void_p,
                                    c_void_p], c_int32),
        "dcflow_screen_adam": ([c_void_p, f, c_void_p], c_int32),
        "dcflow_screen_train_step": ([c_void_p, c_void_p, c_int64, c_void_p, c_int64, c_void_p, c_int32, f,
                                      c_void_p, c_void_p], c_int32),
        "dcflow_screen_check": ([c_void_p, c_void_p], c_int32),
        "dcflow_screen_logits": ([c_void_p, c_void_p, c_int64, c_int64, c_void_p, c_int64, c_void_p], c_int32),
        "dcflow_screen_get": ([c_void_p, c_int32, c_int32, c_void_p], c_int32),
        "dcflow_screen_set": ([c_void_p, c_int32, c_int32, c_void_p], c_int32),
        "dcflow_screen_adam_step": ([c_void_p, POINTER(c_int64), c_int32], c_int32),
        "dcflow_solve_batch_screened": ([c_void_p, POINTER(Batch), POINTER(Results), c_void_p,
                                         POINTER(ScreenOptions), POINTER(ScreenReport), c_void_p], c_int32),
        "dcflow_selftest_bounded_wait": ([c_void_p, c_void_p], c_int32),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
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


def dcflow_setup(n_bus, f, t, b, slack, precision="fp32", device=-1, chunk_topo=0, island_tol=0.0, compact_n1=False,
                 autotune=False, autotune_sample=0, output_first=False):
    lib = load_library()
    o = dcflow_default_options()
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.device = int(device)
    o.chunk_topo = int(chunk_topo)
    o.compact_n1 = int(bool(compact_n1))
    o.autotune = int(bool(autotune))
    o.output_first = int(bool(output_first))
    o.autotune_sample = int(autotune_sample)
    if island_tol:
        o.island_tol = float(island_tol)
    fa, fp = _i32(f)
    ta, tp = _i32(t)
    ba, bp = _f64(b)
    ctx = c_void_p()
    _check(lib.dcflow_setup(byref(ctx), int(n_bus), int(fa.size), fp, tp, bp, int(slack), byref(o)),
           "dcflow_setup")
    return ctx


def dcflow_autotune(ctx, batch, results, stream=None, max_tried=32):
    """Tune the schedule on `batch` (a Batch / Results pair of ctypes structs); returns (pick, tried) as dicts."""
    tried = (Schedule * max_tried)()
    n = c_int32(0)
    pick = Schedule()
    _check(load_library().dcflow_autotune(ctx, byref(batch), byref(results), _stream_ptr(stream), tried,
                                          int(max_tried), byref(n), byref(pick)), "dcflow_autotune")
    return pick.as_dict(), [tried[i].as_dict() for i in range(min(n.value, max_tried))]


def dcflow_set_schedule(ctx, sched=None):
    """Fix the schedule (a dict with budget_mb, rank_bounds, compact_n1, remainder) or, with None, release it."""
    if sched is None:
        _check(load_library().dcflow_set_schedule(ctx, None), "dcflow_set_schedule")
        return
    s = Schedule()
    s.budget_mb = int(sched.get("budget_mb", 8192))
    rb = list(sched.get("rank_bounds", [4, 8, 16])) + [0, 0, 0]
    for i in range(3):
        s.rank_bounds[i] = int(rb[i])
    s.compact_n1 = int(sched.get("compact_n1", 0))
    s.remainder = int(sched.get("remainder", 1))
    _check(load_library().dcflow_set_schedule(ctx, byref(s)), "dcflow_set_schedule")


def dcflow_last_schedule(ctx):
    s = Schedule()
    _check(load_library().dcflow_last_schedule(ctx, byref(s)), "dcflow_last_schedule")
    return s.as_dict()


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


def dcflow_set_study(ctx, mon, cont, limit, split_bus=None, outage_cand=None, multi=None):
    """multi: optional list of branch sets (1-4 branches each) that fail together."""
    ma, mp = _i32(mon)
    ca, cp = _i32(cont)
    la, lp = _f64(limit)
    s = Study(mp, int(ma.size), cp, int(ca.size), lp, None, 0, None, 0, 0, None, None)
    keep = [ma, ca, la]
    if split_bus is not None:
        sa, spp = _i32(split_bus)
        keep.append(sa)
        s.split_bus, s.n_split_bus = spp, int(sa.size)
    if outage_cand is not None:
        oa, op = _i32(outage_cand)
        keep.append(oa)
        s.outage_cand, s.n_outage_cand = op, int(oa.size)
    if multi is not None and len(multi):
        ptr = np.zeros(len(multi) + 1, np.int64)
        ptr[1:] = np.cumsum([len(m) for m in multi])
        pa, pp = _i32(ptr)
        ba, bp = _i32(np.concatenate([np.asarray(m, np.int64).ravel() for m in multi]))
        keep += [pa, ba]
        s.n_multi, s.multi_ptr, s.multi_branch = len(multi), pp, bp
    _check(load_library().dcflow_set_study(ctx, byref(s)), "dcflow_set_study")


def dcflow_solve_batch(ctx, batch: Batch, results: Results, stream=None):
    _check(load_library().dcflow_solve_batch(ctx, byref(batch), byref(results), _stream_ptr(stream)),
           "dcflow_solve_batch")


def dcflow_last_launch_count(ctx) -> int:
    return int(load_library().dcflow_last_launch_count(ctx))


def dcflow_profile(ctx, enable: bool):
    _check(load_library().dcflow_profile(ctx, 1 if enable else 0), "dcflow_profile")


PROFILE_KINDS = {"n1": 0, "multi": 1, "multi_prep": 2, "gen": 3, "topcases": 4, "expand": 5}


def dcflow_profile_read_kind(ctx, kind):
    ms, n = c_double(), c_int64()
    k = PROFILE_KINDS[kind] if isinstance(kind, str) else int(kind)
    _check(load_library().dcflow_profile_read_kind(ctx, k, byref(ms), byref(n)), "dcflow_profile_read_kind")
    return ms.value, n.value


def dcflow_profile_read(ctx):
    """Timed kernel milliseconds and launches since dcflow_profile(ctx, True), per kind."""
    out = {}
    for name in PROFILE_KINDS:
        ms, n = dcflow_profile_read_kind(ctx, name)
        out[f"{name}_ms"], out[f"{name}_launches"] = ms, n
    return out


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


def dcflow_screen_create(ctx, max_rows, seed=0):
    out = c_void_p()
    _check(load_library().dcflow_screen_create(ctx, int(max_rows), int(seed), byref(out)), "dcflow_screen_create")
    return out


def dcflow_screen_destroy(scr):
    load_library().dcflow_screen_destroy(scr)


def dcflow_screen_dims(scr):
    v = [c_int32() for _ in range(5)]
    _check(load_library().dcflow_screen_dims(scr, *[byref(x) for x in v]), "dcflow_screen_dims")
    return dict(zip(("F", "F_pad", "H", "C", "C_pad"), (x.value for x in v)))


def dcflow_screen_features(ctx, scr, batch: Batch, X, ldx, status=None, stream=None):
    _check(load_library().dcflow_screen_features(ctx, scr, byref(batch), _ptr(X), int(ldx), _ptr(status),
                                                 _stream_ptr(stream)), "dcflow_screen_features")


def dcflow_screen_labels(scr, cont_max, n_rows, k, Y, ldy, stream=None):
    _check(load_library().dcflow_screen_labels(scr, _ptr(cont_max), int(n_rows), int(k), _ptr(Y), int(ldy),
                                               _stream_ptr(stream)), "dcflow_screen_labels")


def dcflow_screen_backward(scr, X, ldx, Y, ldy, rows, n, loss, stream=None):
    _check(load_library().dcflow_screen_backward(scr, _ptr(X), int(ldx), _ptr(Y), int(ldy), _ptr(rows), int(n),
                                                 _ptr(loss), _stream_ptr(stream)), "dcflow_screen_backward")


def dcflow_screen_adam(scr, lr, stream=None):
    _check(load_library().dcflow_screen_adam(scr, float(lr), _stream_ptr(stream)), "dcflow_screen_adam")


def dcflow_screen_train_step(scr, X, ldx, Y, ldy, rows, n, lr, loss, stream=None):
    _check(load_library().dcflow_screen_train_step(scr, _ptr(X), int(ldx), _ptr(Y), int(ldy), _ptr(rows), int(n),
                                                   float(lr), _ptr(loss), _stream_ptr(stream)),
           "dcflow_screen_train_step")


def dcflow_screen_check(scr, stream=None):
    _check(load_library().dcflow_screen_check(scr, _stream_ptr(stream)), "dcflow_screen_check")


def dcflow_screen_logits(scr, X, ldx, n_rows, Z, ldz, stream=None):
    _check(load_library().dcflow_screen_logits(scr, _ptr(X), int(ldx), int(n_rows), _ptr(Z), int(ldz),
                                               _stream_ptr(stream)), "dcflow_screen_logits")


def dcflow_screen_get(scr, tensor, kind, out: np.ndarray):
    assert out.dtype == np.float32 and out.flags.c_contiguous
    _check(load_library().dcflow_screen_get(scr, int(tensor), int(kind), out.ctypes.data_as(c_void_p)),
           "dcflow_screen_get")
    return out


def dcflow_screen_set(scr, tensor, kind, values: np.ndarray):
    v = np.ascontiguousarray(values, np.float32)
    _check(load_library().dcflow_screen_set(scr, int(tensor), int(kind), v.ctypes.data_as(c_void_p)),
           "dcflow_screen_set")


def dcflow_screen_adam_step(scr, t=None):
    v = c_int64(0 if t is None else int(t))
    _check(load_library().dcflow_screen_adam_step(scr, byref(v), 0 if t is None else 1), "dcflow_screen_adam_step")
    return v.value


def dcflow_solve_batch_screened(ctx, batch: Batch, results: Results, scr, opt: ScreenOptions,
                                report: ScreenReport, stream=None):
    _check(load_library().dcflow_solve_batch_screened(ctx, byref(batch), byref(results), scr, byref(opt),
                                                      byref(report), _stream_ptr(stream)),
           "dcflow_solve_batch_screened")


def dcflow_selftest_bounded_wait(ctx, stream=None) -> int:
    """Return code of the bounded-wait self-test (DCFLOW_ERR_TIMEOUT = -5 is the designed outcome)."""
    return int(load_library().dcflow_selftest_bounded_wait(ctx, _stream_ptr(stream)))


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

    def __init__(self, topo, inj, var=None, device="cuda", gen_bus=None, gen_p=None, ti=None):
        """ti: injection topologies (inj_bus, inj_p [T, n_inj], ti_ptr, ti_mask), e.g.
        synth.InjectionTopologies."""
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
        self.n_gen = 0 if gen_bus is None else int(np.asarray(gen_bus).size)
        if self.n_gen:
            self.gen_bus = torch.as_tensor(np.asarray(gen_bus, np.int32), device=device)
            self.gen_p = torch.as_tensor(np.ascontiguousarray(np.atleast_2d(gen_p), np.float64), device=device)
        else:
            self.gen_bus = self.gen_p = None
        self.has_ti = ti is not None
        self.n_inj = 0
        self.inj_bus = self.inj_p = self.ti_ptr = self.ti_mask = None
        if self.has_ti:
            self.n_inj = int(np.asarray(ti.inj_bus).size)
            self.inj_bus = torch.as_tensor(np.asarray(ti.inj_bus, np.int32), device=device)
            self.inj_p = torch.as_tensor(np.ascontiguousarray(np.atleast_2d(ti.inj_p), np.float64), device=device)
            self.ti_ptr = torch.as_tensor(np.asarray(ti.ti_ptr, np.int32), device=device)
            self.ti_mask = torch.as_tensor(np.asarray(ti.ti_mask, np.uint64).view(np.int64), device=device)

    def cstruct(self) -> Batch:
        return Batch(self.n_topo, _ptr(self.split_ptr), _ptr(self.split_sub), _ptr(self.split_mask),
                     _ptr(self.out_ptr), _ptr(self.out_branch), self.n_time, _ptr(self.inj), self.n_var,
                     _ptr(self.var_ptr), _ptr(self.var_bus), _ptr(self.var_delta), self.n_gen,
                     _ptr(self.gen_bus), _ptr(self.gen_p), self.n_inj, _ptr(self.inj_bus), _ptr(self.inj_p),
                     _ptr(self.ti_ptr), _ptr(self.ti_mask))


class DeviceResults:
    """Caller-owned device outputs of one batch."""

    def __init__(self, n_topo, n_time, n_mon, want_flows=False, want_var=False, device="cuda", n_cont=0,
                 want_cont_max=False, top_k=0, want_gen=False, want_multi=False):
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
        self.top_k = int(top_k)
        nk = max(1, n_topo * n_time * self.top_k)
        self.top_cont = torch.empty(nk, dtype=torch.int32, device=device) if top_k else None
        self.top_mon = torch.empty(nk, dtype=torch.int32, device=device) if top_k else None
        self.top_loading = torch.empty(nk, dtype=torch.float32, device=device) if top_k else None
        self.gen_max_loading = torch.empty(nt, dtype=torch.float64, device=device) if want_gen else None
        self.worst_gen = torch.empty(nt, dtype=torch.int32, device=device) if want_gen else None
        self.gen_overload_sum = torch.empty(nt, dtype=torch.float64, device=device) if want_gen else None
        self.multi_max_loading = torch.empty(nt, dtype=torch.float64, device=device) if want_multi else None
        self.worst_multi = torch.empty(nt, dtype=torch.int32, device=device) if want_multi else None
        self.multi_overload_sum = torch.empty(nt, dtype=torch.float64, device=device) if want_multi else None
        self.n_island_multi = torch.empty(max(1, n_topo), dtype=torch.int32, device=device) if want_multi else None
        self.shape = (n_topo, n_time, n_mon)
        self.n_cont = n_cont

    def cstruct(self) -> Results:
        return Results(_ptr(self.n0_flow), _ptr(self.n0_max_loading), _ptr(self.n1_max_loading),
                       _ptr(self.overload_sum), _ptr(self.worst_cont), _ptr(self.worst_mon),
                       _ptr(self.best_var), _ptr(self.island_flag), _ptr(self.n_island_cont),
                       _ptr(self.n1_cont_max), self.top_k, _ptr(self.top_cont), _ptr(self.top_mon),
                       _ptr(self.top_loading), _ptr(self.gen_max_loading), _ptr(self.worst_gen),
                       _ptr(self.gen_overload_sum), _ptr(self.multi_max_loading), _ptr(self.worst_multi),
                       _ptr(self.multi_overload_sum), _ptr(self.n_island_multi))

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
        if self.gen_max_loading is not None:
            out["gen_max"] = self.gen_max_loading[:N * T].cpu().numpy().reshape(N, T)
            out["worst_gen"] = self.worst_gen[:N * T].cpu().numpy().reshape(N, T).astype(np.int64)
            out["gen_ovl"] = self.gen_overload_sum[:N * T].cpu().numpy().reshape(N, T)
        if self.multi_max_loading is not None:
            out["multi_max"] = self.multi_max_loading[:N * T].cpu().numpy().reshape(N, T)
            out["worst_multi"] = self.worst_multi[:N * T].cpu().numpy().reshape(N, T).astype(np.int64)
            out["multi_ovl"] = self.multi_overload_sum[:N * T].cpu().numpy().reshape(N, T)
            out["n_island_multi"] = self.n_island_multi[:N].cpu().numpy().astype(np.int64)
        if self.top_k:
            k = self.top_k
            out["top_cont"] = self.top_cont[:N * T * k].cpu().numpy().reshape(N, T, k).astype(np.int64)
            out["top_mon"] = self.top_mon[:N * T * k].cpu().numpy().reshape(N, T, k).astype(np.int64)
            out["top_loading"] = self.top_loading[:N * T * k].cpu().numpy().reshape(N, T, k).astype(np.float64)
        return out


class Solver:
    """One grid + study on the current CUDA device."""

    def __init__(self, grid, precision="fp32", chunk_topo=0, island_tol=0.0, device=-1, compact_n1=False,
                 autotune=False, autotune_sample=0, output_first=False):
        self.grid = grid
        self.ctx = dcflow_setup(grid.n_bus, grid.f, grid.t, grid.b, grid.slack, precision=precision,
                                device=device, chunk_topo=chunk_topo, island_tol=island_tol, compact_n1=compact_n1,
                                autotune=autotune, autotune_sample=autotune_sample, output_first=output_first)
        self.n_mon = 0
        self.n_cont = 0
        self.n_multi = 0

    def set_study(self, mon, cont, limit, split_bus=None, outage_cand=None, multi=None):
        dcflow_set_study(self.ctx, mon, cont, limit, split_bus, outage_cand, multi)
        self.n_mon = int(np.asarray(mon).size)
        self.n_cont = int(np.asarray(cont).size)
        self.n_multi = 0 if multi is None else len(multi)

    def base_ptdf(self, rows, stream=None):
        import torch
        rows = np.asarray(rows, np.int32)
        out = torch.empty((rows.size, self.grid.n_bus), dtype=torch.float64, device="cuda")
        dcflow_base_ptdf(self.ctx, rows, out, stream)
        return out

    def solve(self, dbatch: DeviceBatch, want_flows=False, results: DeviceResults | None = None, stream=None,
              want_cont_max=False, top_k=0, want_multi=None):
        """want_multi: evaluate the study's multi-outage sets (default: whenever it has some and the batch
        has no injection candidates)."""
        if want_multi is None:
            want_multi = self.n_multi > 0 and dbatch.n_var == 0 and not dbatch.has_ti
        res = results or DeviceResults(dbatch.n_topo, dbatch.n_time, self.n_mon, want_flows,
                                       dbatch.n_var > 0 or dbatch.has_ti,
                                       n_cont=self.n_cont, want_cont_max=want_cont_max, top_k=top_k,
                                       want_gen=dbatch.n_gen > 0, want_multi=want_multi)
        dcflow_solve_batch(self.ctx, dbatch.cstruct(), res.cstruct(), stream)
        return res

    def autotune(self, dbatch: DeviceBatch, results: DeviceResults | None = None, stream=None):
        """Tune the schedule on `dbatch` (kept for batches of its shape); returns (pick, tried)."""
        res = results or DeviceResults(dbatch.n_topo, dbatch.n_time, self.n_mon, False,
                                       dbatch.n_var > 0 or dbatch.has_ti, n_cont=self.n_cont)
        return dcflow_autotune(self.ctx, dbatch.cstruct(), res.cstruct(), stream)

    def set_schedule(self, sched=None):
        dcflow_set_schedule(self.ctx, sched)

    def last_schedule(self):
        return dcflow_last_schedule(self.ctx)

    def solve_screened(self, dbatch: DeviceBatch, screener: "Screener", top_k=64, fallback_logit=float("inf"),
                       results: DeviceResults | None = None, want_pred=False, stream=None, min_prob=0.0,
                       want_evaluated=False):
        """Screened N-1 (the union of each topology's top_k scored contingencies, plus every contingency
        predicted with a probability above min_prob); returns (results, report)."""
        import torch
        res = results or DeviceResults(dbatch.n_topo, dbatch.n_time, self.n_mon, n_cont=self.n_cont)
        N, T = dbatch.n_topo, dbatch.n_time
        W = (self.n_cont + 31) // 32
        rep = {"n_eval": torch.empty(max(1, N), dtype=torch.int32, device="cuda"),
               "fallback": torch.empty(max(1, N), dtype=torch.uint8, device="cuda"),
               "pred": (torch.empty(max(1, N * T * top_k), dtype=torch.int32, device="cuda") if want_pred else None),
               "evaluated": (torch.empty(max(1, N * W), dtype=torch.int32, device="cuda") if want_evaluated
                             else None)}
        dcflow_solve_batch_screened(self.ctx, dbatch.cstruct(), res.cstruct(), screener.scr,
                                    ScreenOptions(int(top_k), float(fallback_logit), float(min_prob)),
                                    ScreenReport(_ptr(rep["n_eval"]), _ptr(rep["fallback"]), _ptr(rep["pred"]),
                                                 _ptr(rep["evaluated"])),
                                    stream)
        return res, rep

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


class Screener:
    """The learned contingency screener of one Solver's study (device state in libdcflow)."""

    def __init__(self, solver: Solver, max_rows=8192, seed=0):
        self.solver = solver
        self.scr = dcflow_screen_create(solver.ctx, max_rows, seed)
        self.max_rows = int(max_rows)
        d = dcflow_screen_dims(self.scr)
        self.F, self.F_pad, self.H, self.C, self.C_pad = d["F"], d["F_pad"], d["H"], d["C"], d["C_pad"]

    def features(self, dbatch: DeviceBatch, stream=None):
        """Feature rows [n_topo * n_time, F_pad] (bf16) and the topology status [n_topo] (uint8)."""
        import torch
        X = torch.empty((dbatch.n_topo * dbatch.n_time, self.F_pad), dtype=torch.bfloat16, device="cuda")
        st = torch.empty(max(1, dbatch.n_topo), dtype=torch.uint8, device="cuda")
        dcflow_screen_features(self.solver.ctx, self.scr, dbatch.cstruct(), X, self.F_pad, st, stream)
        return X, st[:dbatch.n_topo]

    def labels(self, cont_max, k=64, stream=None):
        """uint8 labels [rows, C_pad] from per-contingency maximum loadings [rows * C] (float32)."""
        import torch
        rows = cont_max.numel() // self.C
        Y = torch.empty((rows, self.C_pad), dtype=torch.uint8, device="cuda")
        dcflow_screen_labels(self.scr, cont_max, rows, k, Y, self.C_pad, stream)
        return Y

    def backward(self, X, Y, rows=None, n=None, stream=None):
        import torch
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        n = int(rows.numel() if rows is not None else (n or X.shape[0]))
        dcflow_screen_backward(self.scr, X, X.stride(0), Y, Y.stride(0), rows, n, loss, stream)
        return loss

    def adam(self, lr, stream=None):
        dcflow_screen_adam(self.scr, lr, stream)

    def train_step(self, X, Y, rows, lr, loss, stream=None):
        dcflow_screen_train_step(self.scr, X, X.stride(0), Y, Y.stride(0), rows, int(rows.numel()), lr, loss,
                                 stream)

    def check(self, stream=None):
        dcflow_screen_check(self.scr, stream)

    def logits(self, X, n_rows=None, stream=None):
        import torch
        n = int(X.shape[0] if n_rows is None else n_rows)
        Z = torch.empty((max(1, n), self.C), dtype=torch.float32, device="cuda")
        dcflow_screen_logits(self.scr, X, X.stride(0), n, Z, self.C, stream)
        return Z[:n]

    def shape(self, name):
        return {"W1": (self.H, self.F), "b1": (self.H,), "W2": (self.H, self.H), "b2": (self.H,),
                "W3": (self.C, self.H), "b3": (self.C,)}[name]

    def get(self, name, kind="param"):
        out = np.empty(self.shape(name), np.float32)
        return dcflow_screen_get(self.scr, SCREEN_TENSORS.index(name), SCREEN_KINDS.index(kind), out)

    def set(self, name, values, kind="param"):
        v = np.asarray(values, np.float32)
        assert v.shape == self.shape(name), (name, v.shape)
        dcflow_screen_set(self.scr, SCREEN_TENSORS.index(name), SCREEN_KINDS.index(kind), v)

    def state(self) -> dict:
        """Parameters, Adam moments and step counter (a checkpoint)."""
        st = {f"{k}.{n}": self.get(n, k) for n in SCREEN_TENSORS for k in ("param", "m", "v")}
        st["adam_t"] = np.array(dcflow_screen_adam_step(self.scr), np.int64)
        return st

    def load_state(self, st: dict):
        for n in SCREEN_TENSORS:
            for k in ("param", "m", "v"):
                self.set(n, st[f"{k}.{n}"], k)
        dcflow_screen_adam_step(self.scr, int(st["adam_t"]))

    def save(self, path):
        np.savez(path, **self.state())

    def load(self, path):
        with np.load(path) as z:
            self.load_state({k: z[k] for k in z.files})

    def close(self):
        if self.scr is not None:
            dcflow_screen_destroy(self.scr)
            self.scr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
