"""Python binding of the GB300 level-blocked matrix-power kernel (MPK) library.

Thin ctypes layer over the C ABI declared in ``include/mpk.h``: every function
here has the name of the C entry point it calls and only marshals arguments
(torch CUDA tensors -> device pointers, the current torch stream -> the
plan's cudaStream_t).  All computation runs in the CUDA kernels of
``csrc/``; there is no CPU fallback.  If the shared library has not been
built, every call raises ``RuntimeError``.

Build it in-tree with :func:`build` (nvcc, sm_103a).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_CSRC = os.path.join(_HERE, "csrc")
_BUILD = os.path.join(_HERE, "_build")
LIB_PATH = os.path.join(_BUILD, "libmpk.so")
HEADER = os.path.join(_ROOT, "include", "mpk.h")
SOURCES = ["mpk_plan.cu", "mpk_exec.cu", "mpk_batch.cu", "mpk_tune.cu", "mpk_mlp.cu", "mpk_inspect.cu", "mpk_poly.cu",
           "mpk_host.cu", "mpk_calib.cu", "mpk_krylov.cu"]
NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-I" + os.path.join(_ROOT, "include")]

MPK_OK, MPK_ERR_INVALID, MPK_ERR_CUDA, MPK_ERR_OOM, MPK_ERR_TIMEOUT, MPK_ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5
MPK_F64, MPK_F32, MPK_F32_BF16VAL, MPK_F64_DF = 0, 1, 2, 3
MPK_IO_PERMUTED, MPK_ASYNC, MPK_SWEEP_ONE = 1, 2, 4
MPK_TUNE_STAGE, MPK_TUNE_EVICT_LAST, MPK_TUNE_NO_SORT, MPK_TUNE_RESIDENT = 1, 2, 4, 8
PLAN_PHASES = ("attributes+validation", "bfs_levels", "renumber+permute", "level_sizes+precision",
               "groups+recursion", "tiles+pack+deps", "grid+issue_order", "flags+release")

PRECISIONS = {"f64": MPK_F64, "f32": MPK_F32, "bf16val": MPK_F32_BF16VAL, "f64df": MPK_F64_DF}


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile csrc/*.cu for sm_103a into _build/libmpk.so (in parallel)."""
    os.makedirs(_BUILD, exist_ok=True)
    deps = [os.path.join(_CSRC, s) for s in SOURCES] + [os.path.join(_CSRC, "mpk_internal.cuh"), HEADER]
    newest = max(os.path.getmtime(d) for d in deps)
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= newest:
        return LIB_PATH
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(_BUILD, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc] + NVCC_FLAGS + ["-c", os.path.join(_CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd))
        subprocess.check_call(cmd)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc, "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-o", tmp] + objs)
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class mpk_csr(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int64), ("rowptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p), ("assume_symmetric", C.c_int32)]


class mpk_opts(C.Structure):
    _fields_ = [("root", C.c_int32), ("cache_bytes", C.c_double), ("safety_f", C.c_double),
                ("prec", C.c_int32), ("nrhs", C.c_int32), ("tile_rows", C.c_int32),
                ("ctas_per_sm", C.c_int32), ("timeout_s", C.c_double), ("stream", C.c_void_p),
                ("lag", C.c_double), ("tune", C.c_uint32), ("recursion", C.c_int32),
                ("sweep", C.c_int32)]


class mpk_tune_candidate(C.Structure):
    _fields_ = [("tile_rows", C.c_int32), ("safety_f", C.c_double), ("tune", C.c_uint32), ("p_sweep", C.c_int32),
                ("ms", C.c_double), ("status", C.c_int32)]


class mpk_plan_stats(C.Structure):
    _fields_ = [("n", C.c_int32), ("p", C.c_int32), ("nrhs", C.c_int32), ("prec", C.c_int32),
                ("nnz", C.c_int64), ("n_levels", C.c_int32), ("n_groups", C.c_int32),
                ("n_tiles", C.c_int32), ("max_level_rows", C.c_int32), ("tile_rows", C.c_int32),
                ("grid_ctas", C.c_int32), ("val_bytes", C.c_int32), ("packed_entries", C.c_int64),
                ("matrix_bytes", C.c_int64), ("device_bytes", C.c_int64), ("plan_ms", C.c_double),
                ("cache_bytes", C.c_double), ("slope", C.c_double), ("staged", C.c_int32),
                ("smem_bytes", C.c_int32), ("sorted", C.c_int32), ("resident", C.c_int32),
                ("dep_span", C.c_int32), ("rec_stages", C.c_int32),
                ("sweep", C.c_int32), ("phase_ms", C.c_double * 8)]


_lib = None
_lock = threading.Lock()


def load(path: str | None = None):
    """Load the shared library (no CUDA call is made by loading it)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = path or LIB_PATH
        if not os.path.exists(path):
            raise RuntimeError(f"the MPK CUDA library is not built ({path}); run "
                               "paper_2205_01598_gb300.build() first")
        lib = C.CDLL(path)
        vp, i32, i64, u32, f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint32, C.c_double
        sig = {
            "mpk_opts_default": ([C.POINTER(mpk_opts)], C.c_int),
            "mpk_plan": ([C.POINTER(mpk_csr), i32, C.POINTER(mpk_opts), C.POINTER(vp)], C.c_int),
            "mpk_plan_info": ([vp, C.POINTER(mpk_plan_stats)], C.c_int),
            "mpk_plan_perm": ([vp, vp, vp, vp, vp], C.c_int),
            "mpk_plan_schedule": ([vp, vp, vp, vp], C.c_int),
            "mpk_run": ([vp, vp, vp, u32], C.c_int),
            "mpk_run_host": ([vp, vp, vp, u32], C.c_int),
            "mpk_baseline_run": ([vp, vp, vp, u32], C.c_int),
            "mpk_gershgorin": ([vp, C.POINTER(f64), C.POINTER(f64)], C.c_int),
            "mpk_cheb_coeffs_schroedinger": ([i32, f64, f64, f64, vp], C.c_int),
            "mpk_cheb": ([vp, vp, i32, f64, f64, vp, vp, u32], C.c_int),
            "mpk_cheb_host": ([vp, vp, i32, f64, f64, vp, vp, u32], C.c_int),
            "mpk_cheb_real": ([vp, vp, i32, f64, f64, vp, vp, u32], C.c_int),
            "mpk_cheb_steps": ([vp, vp, i32, f64, f64, i32, vp, vp, u32], C.c_int),
            "mpk_cheb_real_host": ([vp, vp, i32, f64, f64, vp, vp, u32], C.c_int),
            "mpk_cheb_coeffs_heat": ([i32, f64, f64, f64, vp], C.c_int),
            "mpk_cheb_coeffs_inverse": ([i32, f64, f64, vp], C.c_int),
            "mpk_permute_vectors": ([vp, vp, vp, i32, i32, i32], C.c_int),
            "mpk_plan_destroy": ([vp], C.c_int),
            "mpk_strerror": ([C.c_int], C.c_char_p),
            "mpk_plan_last_error": ([vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)], C.c_int),
            "mpk_plan_debug_drop_flag": ([vp, i32, i32], C.c_int),
            "mpk_levels_noalloc": ([i32, i64, vp, vp, i32, vp, C.POINTER(i32), vp, f64], C.c_int),
            "mpk_plan_features": ([vp, vp, i32], C.c_int),
            "mpk_probe_fma": ([i32, i32, i64, vp, vp, C.POINTER(f64)], C.c_int),
            "mpk_cg": ([vp, vp, vp, f64, i32, C.POINTER(i32), C.POINTER(f64), u32], C.c_int),
            "mpk_sstep_cg": ([vp, vp, vp, f64, i32, f64, C.POINTER(i32), C.POINTER(f64), u32], C.c_int),
            "mpk_mlp_create": ([i32, i32, i32, C.c_uint64, vp, C.POINTER(vp)], C.c_int),
            "mpk_mlp_num_params": ([vp], C.c_int32),
            "mpk_mlp_get_params": ([vp, vp, i32], C.c_int),
            "mpk_mlp_set_params": ([vp, vp, i32], C.c_int),
            "mpk_mlp_forward": ([vp, vp, i32, vp], C.c_int),
            "mpk_mlp_loss_grad": ([vp, vp, vp, vp, i32, C.POINTER(f64), vp], C.c_int),
            "mpk_mlp_adam_step": ([vp, C.c_float, C.c_float, C.c_float, C.c_float], C.c_int),
            "mpk_mlp_destroy": ([vp], C.c_int),
            "mpk_tune_default_grid": ([i32, C.POINTER(mpk_tune_candidate), i32, C.POINTER(i32)], C.c_int),
            "mpk_autotune": ([C.POINTER(mpk_csr), i32, C.POINTER(mpk_opts), f64, C.POINTER(mpk_tune_candidate), i32,
                              C.POINTER(i32)], C.c_int),
            "mpk_batch_create": ([C.POINTER(vp), i32, C.POINTER(vp)], C.c_int),
            "mpk_batch_info": ([vp, C.POINTER(i32), C.POINTER(i32)], C.c_int),
            "mpk_batch_run": ([vp, C.POINTER(vp), C.POINTER(vp), u32], C.c_int),
            "mpk_batch_graph_capture": ([vp, C.POINTER(vp), C.POINTER(vp)], C.c_int),
            "mpk_batch_graph_launch": ([vp, u32], C.c_int),
            "mpk_batch_destroy": ([vp], C.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
        return lib


class MpkError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        msg = load().mpk_strerror(code).decode() if _lib is not None else str(code)
        super().__init__(f"{where}: {msg} ({code})")


def _check(code, where):
    if code != MPK_OK:
        raise MpkError(code, where)


def _ptr(t):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _want(t, numel, dtype, name):
    """Checks a tensor that an entry point reads or writes as `numel`
    elements of `dtype`: the C ABI cannot see sizes, so a mismatch is
    rejected here, before anything is launched."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch.Tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name}: expected dtype {dtype}, got {t.dtype}")
    if t.numel() != numel:
        raise ValueError(f"{name}: expected {numel} elements, got {t.numel()}")


def _ptrs(*specs):
    """Device pointers of (tensor, numel, dtype, name) specs, all checked first."""
    for spec in specs:
        _want(*spec)
    return [_ptr(spec[0]) for spec in specs]


def _csr(rowptr, col, val, assume_symmetric):
    import torch
    for t, dt, name in ((rowptr, torch.int32, "rowptr"), (col, torch.int32, "col"), (val, torch.float64, "val")):
        if not isinstance(t, torch.Tensor) or t.dtype != dt:
            raise TypeError(f"{name}: expected a {dt} tensor")
    if rowptr.numel() < 1 or col.numel() != val.numel():
        raise ValueError("rowptr needs n + 1 entries and col / val the same length nnz")
    return mpk_csr(n=rowptr.numel() - 1, nnz=col.numel(), rowptr=_ptr(rowptr), col=_ptr(col), val=_ptr(val),
                   assume_symmetric=int(bool(assume_symmetric)))


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


class Plan:
    """Owner of an ``mpk_plan_t``; released by :func:`mpk_plan_destroy` or GC."""

    def __init__(self, handle, p, nrhs, prec, n, stream):
        self.handle = handle
        self.p, self.nrhs, self.prec, self.n = p, nrhs, prec, n
        self.stream = stream

    @property
    def vec_dtype(self):
        import torch
        return torch.float64 if self.prec in (MPK_F64, MPK_F64_DF) else torch.float32

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.mpk_plan_destroy(self.handle)
            self.handle = None


def mpk_opts_default():
    o = mpk_opts()
    _check(load().mpk_opts_default(C.byref(o)), "mpk_opts_default")
    return o


def mpk_plan(rowptr, col, val, p, *, assume_symmetric=True, root=0, cache_bytes=0.0, safety_f=0.5,
             prec="f64", nrhs=1, tile_rows=0, ctas_per_sm=0, timeout_s=2.0, lag=-1.0, tune=0,
             recursion=0, sweep=0, stream=None) -> Plan:
    """Level-blocked plan of the CRS matrix (rowptr, col: int32 CUDA tensors,
    val: float64 CUDA tensor) for powers 1..p (mpk_plan); sweep = q < p runs
    the powers in sweeps of q inside the one launch."""
    A = _csr(rowptr, col, val, assume_symmetric)
    lib = load()
    o = mpk_opts_default()
    o.root, o.cache_bytes, o.safety_f = int(root), float(cache_bytes), float(safety_f)
    o.prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    o.nrhs, o.tile_rows, o.ctas_per_sm, o.timeout_s = int(nrhs), int(tile_rows), int(ctas_per_sm), float(timeout_s)
    o.stream = _stream(stream)
    o.lag = float(lag)
    o.tune = int(tune)
    o.recursion = int(recursion)
    o.sweep = int(sweep)
    h = C.c_void_p()
    _check(lib.mpk_plan(C.byref(A), int(p), C.byref(o), C.byref(h)), "mpk_plan")
    return Plan(h, int(p), int(nrhs), o.prec, A.n, stream)


def mpk_tune_default_grid(k):
    """Default search grid of mpk_autotune for k powers: list of dicts."""
    arr = (mpk_tune_candidate * 64)()
    n = C.c_int32()
    _check(load().mpk_tune_default_grid(int(k), arr, 64, C.byref(n)), "mpk_tune_default_grid")
    return [{"tile_rows": arr[i].tile_rows, "safety_f": arr[i].safety_f, "tune": arr[i].tune,
             "p_sweep": arr[i].p_sweep} for i in range(n.value)]


def mpk_autotune(rowptr, col, val, k, candidates, *, prec="f64", nrhs=1, min_time_s=0.05, assume_symmetric=True,
                 stream=None):
    """Times each candidate (dicts with tile_rows, safety_f, tune, p_sweep) for
    the MPK with k powers (mpk_autotune); returns (best index, list of ms
    (-1 for failures))."""
    A = _csr(rowptr, col, val, assume_symmetric)
    lib = load()
    o = mpk_opts_default()
    o.prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    o.nrhs = int(nrhs)
    o.stream = _stream(stream)
    arr = (mpk_tune_candidate * len(candidates))()
    for i, c in enumerate(candidates):
        arr[i].tile_rows, arr[i].safety_f = int(c["tile_rows"]), float(c["safety_f"])
        arr[i].tune, arr[i].p_sweep = int(c.get("tune", 0)), int(c["p_sweep"])
    best = C.c_int32()
    _check(lib.mpk_autotune(C.byref(A), int(k), C.byref(o), float(min_time_s), arr, len(candidates),
                            C.byref(best)), "mpk_autotune")
    return best.value, [arr[i].ms for i in range(len(candidates))]


def mpk_plan_info(plan: Plan) -> dict:
    s = mpk_plan_stats()
    _check(load().mpk_plan_info(plan.handle, C.byref(s)), "mpk_plan_info")
    out = {name: getattr(s, name) for name, _ in mpk_plan_stats._fields_}
    out["phase_ms"] = list(out["phase_ms"])
    return out


def mpk_plan_features(plan: Plan) -> np.ndarray:
    """The 25 planner features of the plan's matrix (mpk_plan_features)."""
    out = np.zeros(32, dtype=np.float32)
    n = load().mpk_plan_features(plan.handle, out.ctypes.data_as(C.c_void_p), 32)
    if n < 0:
        _check(n, "mpk_plan_features")
    return out[:n].copy()


def mpk_plan_perm(plan: Plan):
    """(perm, level_ptr, group_ptr, level) as int32 CUDA tensors."""
    import torch
    info = mpk_plan_info(plan)
    dev = torch.device("cuda", torch.cuda.current_device())
    perm = torch.empty(plan.n, dtype=torch.int32, device=dev)
    lp = torch.empty(info["n_levels"] + 1, dtype=torch.int32, device=dev)
    gp = torch.empty(info["n_groups"] + 1, dtype=torch.int32, device=dev)
    lev = torch.empty(plan.n, dtype=torch.int32, device=dev)
    _check(load().mpk_plan_perm(plan.handle, _ptr(perm), _ptr(lp), _ptr(gp), _ptr(lev)), "mpk_plan_perm")
    return perm, lp, gp, lev


def mpk_plan_schedule(plan: Plan):
    """(work, dep_lo, dep_hi) as host int32 arrays (mpk_plan_schedule)."""
    info = mpk_plan_info(plan)
    work = np.empty(info["n_tiles"] * plan.p, dtype=np.int32)
    lo = np.empty(info["n_tiles"], dtype=np.int32)
    hi = np.empty(info["n_tiles"], dtype=np.int32)
    _check(load().mpk_plan_schedule(plan.handle, work.ctypes.data_as(C.c_void_p), lo.ctypes.data_as(C.c_void_p),
                                    hi.ctypes.data_as(C.c_void_p)), "mpk_plan_schedule")
    return work, lo, hi


def _flags(permuted, asynchronous):
    return (MPK_IO_PERMUTED if permuted else 0) | (MPK_ASYNC if asynchronous else 0)


def _mpk_io(plan, x, Y):
    blk = plan.n * plan.nrhs
    return _ptrs((x, blk, plan.vec_dtype, "x"), (Y, plan.p * blk, plan.vec_dtype, "Y"))


def mpk_run(plan: Plan, x, Y, permuted=False, asynchronous=False):
    """Y[k-1] = A^k x, k = 1..p, level-blocked (mpk_run); x: n x nrhs, Y:
    p x n x nrhs, both in the plan's vector precision."""
    xp, yp = _mpk_io(plan, x, Y)
    _check(load().mpk_run(plan.handle, xp, yp, _flags(permuted, asynchronous)), "mpk_run")


def mpk_run_host(plan: Plan, x, Y, permuted=False, asynchronous=False):
    """mpk_run with x (n x nrhs) and Y (p x n x nrhs) in HOST memory
    (mpk_run_host): the library copies x in and every power out, overlapping
    the copies with the reordering.  Pinned CPU tensors give full-speed,
    overlapped copies; with asynchronous=True synchronise the plan's stream
    before reading Y."""
    blk = plan.n * plan.nrhs
    _want(Y, plan.p * blk, plan.vec_dtype, "Y")
    xp = _host_vec(x, blk, plan.vec_dtype, "x")
    yp = _host_vec(Y, plan.p * blk, plan.vec_dtype, "Y")
    _check(load().mpk_run_host(plan.handle, xp, yp, _flags(permuted, asynchronous)), "mpk_run_host")


def mpk_baseline_run(plan: Plan, x, Y, permuted=False, asynchronous=False):
    """Y[k-1] = A^k x by p back-to-back SpMV launches (mpk_baseline_run)."""
    xp, yp = _mpk_io(plan, x, Y)
    _check(load().mpk_baseline_run(plan.handle, xp, yp, _flags(permuted, asynchronous)), "mpk_baseline_run")


def mpk_gershgorin(plan: Plan):
    lo, hi = C.c_double(), C.c_double()
    _check(load().mpk_gershgorin(plan.handle, C.byref(lo), C.byref(hi)), "mpk_gershgorin")
    return lo.value, hi.value


def mpk_cheb_coeffs_schroedinger(M, c, r, dt) -> np.ndarray:
    out = np.empty(2 * (M + 1), dtype=np.float64)
    _check(load().mpk_cheb_coeffs_schroedinger(int(M), float(c), float(r), float(dt),
                                               out.ctypes.data_as(C.c_void_p)), "mpk_cheb_coeffs_schroedinger")
    return out[0::2] + 1j * out[1::2]


def mpk_cheb_coeffs_heat(M, c, r, tau) -> np.ndarray:
    """Real coefficients (M+1,) of exp(-tau A) in T_k((A - c)/r) (mpk_cheb_coeffs_heat)."""
    out = np.empty(M + 1, dtype=np.float64)
    _check(load().mpk_cheb_coeffs_heat(int(M), float(c), float(r), float(tau), out.ctypes.data_as(C.c_void_p)),
           "mpk_cheb_coeffs_heat")
    return out


def mpk_cheb_coeffs_inverse(M, c, r) -> np.ndarray:
    """Real coefficients (M+1,) of A^{-1} in T_k((A - c)/r) for a spectrum in
    [c - r, c + r], c > r >= 0 (mpk_cheb_coeffs_inverse)."""
    out = np.empty(M + 1, dtype=np.float64)
    _check(load().mpk_cheb_coeffs_inverse(int(M), float(c), float(r), out.ctypes.data_as(C.c_void_p)),
           "mpk_cheb_coeffs_inverse")
    return out


def mpk_cheb_real(plan: Plan, coef, c, r, x, y, permuted=False, asynchronous=False, one_power_per_launch=False):
    """y = sum_k coef_k T_k((A - c)/r) x for real x (n,) in the plan precision
    and y (n,) float64 CUDA tensors; coef: real host array of length M+1
    (mpk_cheb_real)."""
    import torch
    ci = np.ascontiguousarray(coef, dtype=np.float64)
    xp, yp = _ptrs((x, plan.n * plan.nrhs, plan.vec_dtype, "x"), (y, plan.n * plan.nrhs, torch.float64, "y"))
    _check(load().mpk_cheb_real(plan.handle, ci.ctypes.data_as(C.c_void_p), ci.shape[0] - 1, float(c), float(r),
                                xp, yp,
                                _flags(permuted, asynchronous) | (MPK_SWEEP_ONE if one_power_per_launch else 0)),
           "mpk_cheb_real")


def mpk_cheb(plan: Plan, coef, c, r, x, y, permuted=False, asynchronous=False, one_power_per_launch=False):
    """y = sum_k coef_k T_k((A - c)/r) x (mpk_cheb); x: (n, 2) plan precision,
    y: (n, 2) float64 CUDA tensors; coef: complex host array of length M+1."""
    import torch
    coef = np.asarray(coef, dtype=np.complex128)
    ci = np.empty(2 * coef.shape[0], dtype=np.float64)
    ci[0::2], ci[1::2] = coef.real, coef.imag
    xp, yp = _ptrs((x, plan.n * plan.nrhs, plan.vec_dtype, "x"), (y, plan.n * plan.nrhs, torch.float64, "y"))
    _check(load().mpk_cheb(plan.handle, ci.ctypes.data_as(C.c_void_p), coef.shape[0] - 1, float(c), float(r),
                           xp, yp,
                           _flags(permuted, asynchronous) | (MPK_SWEEP_ONE if one_power_per_launch else 0)), "mpk_cheb")


def mpk_cheb_steps(plan: Plan, coef, c, r, nsteps, x, y, permuted=False, asynchronous=False,
                   one_power_per_launch=False):
    """nsteps time steps of the Chebyshev propagation in sweeps that run
    across the steps (mpk_cheb_steps): complex coef (plan nrhs = 2, x and y
    of shape (n, 2)) or real coef (nrhs = 1, shape (n,)); y float64."""
    import torch
    coef = np.asarray(coef)
    if plan.nrhs == 2:
        cz = np.asarray(coef, dtype=np.complex128)
        ci = np.empty(2 * cz.shape[0], dtype=np.float64)
        ci[0::2], ci[1::2] = cz.real, cz.imag
        M = cz.shape[0] - 1
    else:
        ci = np.ascontiguousarray(coef, dtype=np.float64)
        M = ci.shape[0] - 1
    xp, yp = _ptrs((x, plan.n * plan.nrhs, plan.vec_dtype, "x"), (y, plan.n * plan.nrhs, torch.float64, "y"))
    _check(load().mpk_cheb_steps(plan.handle, ci.ctypes.data_as(C.c_void_p), M, float(c), float(r), int(nsteps), xp,
                                 yp, _flags(permuted, asynchronous) | (MPK_SWEEP_ONE if one_power_per_launch else 0)),
           "mpk_cheb_steps")


def _host_vec(t, numel, dtype, name):
    _want(t, numel, dtype, name)
    if t.is_cuda or not t.is_contiguous():
        raise TypeError(f"{name}: expected a contiguous CPU tensor")
    return C.c_void_p(t.data_ptr())


def mpk_cheb_host(plan: Plan, coef, c, r, x, y, permuted=False, asynchronous=False):
    """mpk_cheb with x (n, 2) and y (n, 2) float64 in HOST memory (mpk_cheb_host)."""
    import torch
    coef = np.asarray(coef, dtype=np.complex128)
    ci = np.empty(2 * coef.shape[0], dtype=np.float64)
    ci[0::2], ci[1::2] = coef.real, coef.imag
    xp = _host_vec(x, plan.n * plan.nrhs, plan.vec_dtype, "x")
    yp = _host_vec(y, plan.n * plan.nrhs, torch.float64, "y")
    _check(load().mpk_cheb_host(plan.handle, ci.ctypes.data_as(C.c_void_p), coef.shape[0] - 1, float(c), float(r),
                                xp, yp, _flags(permuted, asynchronous)), "mpk_cheb_host")


def mpk_cheb_real_host(plan: Plan, coef, c, r, x, y, permuted=False, asynchronous=False):
    """mpk_cheb_real with x (n,) and y (n,) float64 in HOST memory (mpk_cheb_real_host)."""
    import torch
    ci = np.ascontiguousarray(coef, dtype=np.float64)
    xp = _host_vec(x, plan.n * plan.nrhs, plan.vec_dtype, "x")
    yp = _host_vec(y, plan.n * plan.nrhs, torch.float64, "y")
    _check(load().mpk_cheb_real_host(plan.handle, ci.ctypes.data_as(C.c_void_p), ci.shape[0] - 1, float(c),
                                     float(r), xp, yp, _flags(permuted, asynchronous)), "mpk_cheb_real_host")


def mpk_permute_vectors(plan: Plan, src, dst, count, to_level):
    """count blocks of n x nrhs elements (4- or 8-byte) between the caller's
    numbering and the plan's level order (mpk_permute_vectors)."""
    numel = int(count) * plan.n * plan.nrhs
    sp, dp = _ptrs((src, numel, getattr(src, "dtype", None), "src"), (dst, numel, getattr(src, "dtype", None), "dst"))
    _check(load().mpk_permute_vectors(plan.handle, sp, dp, int(count), src.element_size(), int(bool(to_level))),
           "mpk_permute_vectors")


def mpk_plan_last_error(plan: Plan):
    code, k, t = C.c_int32(), C.c_int32(), C.c_int32()
    _check(load().mpk_plan_last_error(plan.handle, C.byref(code), C.byref(k), C.byref(t)), "mpk_plan_last_error")
    return code.value, k.value, t.value


def mpk_plan_debug_drop_flag(plan: Plan, tile, power):
    """Test hook: the next wavefront launch does not publish item (tile, power)."""
    _check(load().mpk_plan_debug_drop_flag(plan.handle, int(tile), int(power)), "mpk_plan_debug_drop_flag")


def mpk_levels_noalloc(rowptr, col, root=0, level=None, stream=None, timeout_s=2.0):
    """Eq. 3 levels computed without any device allocation by the library
    (mpk_levels_noalloc); returns (level tensor, number of levels).  Pass a
    pre-allocated int32 `level` of length n so that nothing is allocated."""
    import torch
    n = rowptr.numel() - 1
    if level is None:
        level = torch.empty(n, dtype=torch.int32, device=rowptr.device)
    rp, cp, lp = _ptrs((rowptr, n + 1, torch.int32, "rowptr"), (col, col.numel(), torch.int32, "col"),
                       (level, n, torch.int32, "level"))
    nl = C.c_int32()
    _check(load().mpk_levels_noalloc(n, col.numel(), rp, cp, int(root), lp,
                                     C.byref(nl), _stream(stream), float(timeout_s)), "mpk_levels_noalloc")
    return level, nl.value


def mpk_probe_fma(prec, sink, blocks_per_sm=8, iters=1 << 14, stream=None):
    """Launches the FMA-chain probe (mpk_probe_fma) on the stream without
    waiting; returns its flop count.  prec "f64" or "f32"; sink: a CUDA
    tensor of at least 8 bytes.  The caller times the launch."""
    if not hasattr(sink, "is_cuda") or not sink.is_cuda or sink.numel() * sink.element_size() < 8:
        raise TypeError("sink: expected a CUDA tensor of at least 8 bytes")
    fl = C.c_double()
    _check(load().mpk_probe_fma(PRECISIONS[prec], int(blocks_per_sm), int(iters), _ptr(sink), _stream(stream),
                                C.byref(fl)), "mpk_probe_fma")
    return fl.value


def mpk_cg(plan: Plan, b, x, tol=1e-10, max_steps=10000, permuted=False):
    """Conjugate gradients with the plan's SpMV (mpk_cg); b, x: n float64
    CUDA tensors, x the initial guess, overwritten.  Returns (steps, relres)."""
    import torch
    bp, xp = _ptrs((b, plan.n, torch.float64, "b"), (x, plan.n, torch.float64, "x"))
    st, rel = C.c_int32(), C.c_double()
    _check(load().mpk_cg(plan.handle, bp, xp, float(tol), int(max_steps), C.byref(st), C.byref(rel),
                         MPK_IO_PERMUTED if permuted else 0), "mpk_cg")
    return st.value, rel.value


def mpk_sstep_cg(plan: Plan, b, x, tol=1e-10, max_steps=10000, rho=0.0, permuted=False):
    """s-step CG with one MPK of [p r] per s = plan.p steps (mpk_sstep_cg);
    the plan has nrhs = 2.  Returns (steps, relres)."""
    import torch
    bp, xp = _ptrs((b, plan.n, torch.float64, "b"), (x, plan.n, torch.float64, "x"))
    st, rel = C.c_int32(), C.c_double()
    _check(load().mpk_sstep_cg(plan.handle, bp, xp, float(tol), int(max_steps), float(rho), C.byref(st),
                               C.byref(rel), MPK_IO_PERMUTED if permuted else 0), "mpk_sstep_cg")
    return st.value, rel.value


class Batch:
    """Owner of an ``mpk_batch_t`` (keeps its plans alive)."""

    def __init__(self, handle, plans):
        self.handle, self.plans = handle, list(plans)

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.mpk_batch_destroy(self.handle)
            self.handle = None


def _batch_io(batch, xs, Ys):
    """Per-plan input and output pointers, each checked against its plan."""
    if len(xs) != len(batch.plans) or len(Ys) != len(batch.plans):
        raise ValueError(f"expected {len(batch.plans)} inputs and outputs, one per plan")
    specs = []
    for pl, x, Y in zip(batch.plans, xs, Ys):
        blk = pl.n * pl.nrhs
        specs += [(x, blk, pl.vec_dtype, "x"), (Y, pl.p * blk, pl.vec_dtype, "Y")]
    ps = [q.value for q in _ptrs(*specs)]
    return (C.c_void_p * len(xs))(*ps[0::2]), (C.c_void_p * len(Ys))(*ps[1::2])


def mpk_batch_create(plans) -> Batch:
    """One persistent launch for several plans (mpk_batch_create)."""
    hs = (C.c_void_p * len(plans))(*[p.handle.value if isinstance(p.handle, C.c_void_p) else p.handle
                                     for p in plans])
    h = C.c_void_p()
    _check(load().mpk_batch_create(hs, len(plans), C.byref(h)), "mpk_batch_create")
    return Batch(h, plans)


def mpk_batch_info(batch: Batch):
    n, g = C.c_int32(), C.c_int32()
    _check(load().mpk_batch_info(batch.handle, C.byref(n), C.byref(g)), "mpk_batch_info")
    return {"n_items": n.value, "grid_ctas": g.value}


def mpk_batch_run(batch: Batch, xs, Ys, asynchronous=False):
    px, py = _batch_io(batch, xs, Ys)
    _check(load().mpk_batch_run(batch.handle, px, py, MPK_ASYNC if asynchronous else 0), "mpk_batch_run")


def mpk_batch_graph_capture(batch: Batch, xs, Ys):
    px, py = _batch_io(batch, xs, Ys)
    _check(load().mpk_batch_graph_capture(batch.handle, px, py), "mpk_batch_graph_capture")


def mpk_batch_graph_launch(batch: Batch, asynchronous=False):
    _check(load().mpk_batch_graph_launch(batch.handle, MPK_ASYNC if asynchronous else 0), "mpk_batch_graph_launch")


def mpk_batch_destroy(batch: Batch):
    if batch.handle:
        _check(load().mpk_batch_destroy(batch.handle), "mpk_batch_destroy")
        batch.handle = None


class Mlp:
    """The planner's network (mpk_mlp_*): parameters and training on the GPU."""

    def __init__(self, n_in, n_hidden, n_out, seed=7, stream=None):
        self.shape = (int(n_in), int(n_hidden), int(n_out))
        self.handle = C.c_void_p()
        _check(load().mpk_mlp_create(self.shape[0], self.shape[1], self.shape[2], int(seed), _stream(stream),
                                     C.byref(self.handle)), "mpk_mlp_create")
        self.num_params = load().mpk_mlp_num_params(self.handle)

    def get_params(self) -> np.ndarray:
        out = np.empty(self.num_params, dtype=np.float32)
        _check(load().mpk_mlp_get_params(self.handle, out.ctypes.data_as(C.c_void_p), self.num_params),
               "mpk_mlp_get_params")
        return out

    def set_params(self, params):
        p = np.ascontiguousarray(params, dtype=np.float32)
        _check(load().mpk_mlp_set_params(self.handle, p.ctypes.data_as(C.c_void_p), p.size), "mpk_mlp_set_params")

    def _batch(self, X):
        import torch
        if not isinstance(X, torch.Tensor) or X.dim() != 2:
            raise TypeError("X: expected a 2-D torch.Tensor (batch x inputs)")
        _want(X, X.shape[0] * self.shape[0], torch.float32, "X")
        return X.shape[0]

    def forward(self, X):
        import torch
        b = self._batch(X)
        Y = torch.empty(b, self.shape[2], dtype=torch.float32, device=X.device)
        _check(load().mpk_mlp_forward(self.handle, _ptr(X), b, _ptr(Y)), "mpk_mlp_forward")
        return Y

    def loss_grad(self, X, T, M, want_grad=False):
        import torch
        b = self._batch(X)
        xp, tp, mp = _ptrs((X, b * self.shape[0], torch.float32, "X"), (T, b * self.shape[2], torch.float32, "T"),
                           (M, b * self.shape[2], torch.float32, "M"))
        loss = C.c_double()
        g = np.empty(self.num_params, dtype=np.float32) if want_grad else None
        _check(load().mpk_mlp_loss_grad(self.handle, xp, tp, mp, b, C.byref(loss),
                                        g.ctypes.data_as(C.c_void_p) if want_grad else None), "mpk_mlp_loss_grad")
        return (loss.value, g) if want_grad else loss.value

    def adam_step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(load().mpk_mlp_adam_step(self.handle, lr, beta1, beta2, eps), "mpk_mlp_adam_step")

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.mpk_mlp_destroy(self.handle)
            self.handle = None


def mpk_plan_destroy(plan: Plan):
    if plan.handle:
        _check(load().mpk_plan_destroy(plan.handle), "mpk_plan_destroy")
        plan.handle = None


def mpk_strerror(code: int) -> str:
    return load().mpk_strerror(int(code)).decode()


def csr_to_device(A, device="cuda"):
    """Copies a host CRS (objects with rowptr/col/val numpy arrays) to CUDA tensors."""
    import torch
    return (torch.from_numpy(np.ascontiguousarray(A.rowptr, dtype=np.int32)).to(device),
            torch.from_numpy(np.ascontiguousarray(A.col, dtype=np.int32)).to(device),
            torch.from_numpy(np.ascontiguousarray(A.val, dtype=np.float64)).to(device))
