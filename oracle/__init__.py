"""FP64 CPU oracle for the level-blocked matrix-power kernel.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; never by the library.  It shares
no code with the CUDA path.  The arithmetic lives in ``mpk_oracle.c`` (plain
sequential C, FP64, compiled with ``-ffp-contract=off``); this module builds it
with gcc and wraps it with ctypes, converting numpy arrays only.

Functions and the passages of the paper they restate:
  spmv, mpk            Sec. 3.1, Fig. 1 (baseline MPK: pm back-to-back SpMVs)
  bfs_levels           Sec. 4.1, Eq. 3 (+ restart rule for disconnected graphs)
  level_perm           Sec. 4.1 (level-consecutive renumbering), Fig. 3e level_ptr
  permute_csr          Sec. 4.1 footnote (symmetric permutation P A P^T)
  level_groups         Sec. 4.2.1, Eq. 5 (greedy level groups)
  lp_order             Sec. 4.2, Fig. 5 (diagonal traversal of the Lp diagram)
  lb_mpk               Sec. 4.2, Fig. 5 run sequentially (levels or level groups)
  gershgorin           spectral interval used for the Chebyshev scaling (Sec. 7)
  cheb_coeffs_schroedinger, cheb   Sec. 7, Eq. 7-9
  omp_pxspmv           the multicore comparator (Sec. 6): Fig. 1 with rows split
                       statically over OpenMP threads (mpk_omp.c, built apart)

Every function here is pinned by ``tests/test_oracle_*.py`` against closed
forms, dense brute force, the paper's worked examples and invariants.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mpk_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile mpk_oracle.c into oracle/_build/liboracle.so (gcc, FP64, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_OMP_SRC = os.path.join(_HERE, "mpk_omp.c")
_OMP_PATH = os.path.join(_BUILD, "libomp_pxspmv.so")
_omp_lib = None


def build_omp(force: bool = False):
    """Compile mpk_omp.c (gcc -fopenmp) into oracle/_build/libomp_pxspmv.so;
    returns its path, or None when the compiler has no OpenMP."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_OMP_PATH) or os.path.getmtime(_OMP_PATH) < os.path.getmtime(_OMP_SRC):
        tmp = _OMP_PATH + f".tmp{os.getpid()}"
        r = subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", tmp,
                            _OMP_SRC], capture_output=True)
        if r.returncode != 0:
            return None
        os.replace(tmp, _OMP_PATH)
    return _OMP_PATH


def omp_pxspmv(A, x, p):
    """p back-to-back FP64 SpMVs on all OpenMP threads of the host; returns
    (Y, threads).  Raises RuntimeError when OpenMP is not available."""
    global _omp_lib
    with _lock:
        if _omp_lib is None:
            path = build_omp()
            if path is None:
                raise RuntimeError("gcc without OpenMP: the multicore comparator is unavailable")
            lib = C.CDLL(path)
            i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
            f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
            lib.omp_pxspmv.argtypes = [C.c_int, i32p, i32p, f64p, C.c_int, f64p, f64p]
            lib.omp_pxspmv.restype = None
            lib.omp_pxspmv_threads.restype = C.c_int
            _omp_lib = lib
    x = np.ascontiguousarray(x, dtype=np.float64)
    Y = np.empty((p, A.n), dtype=np.float64)
    _omp_lib.omp_pxspmv(A.n, np.ascontiguousarray(A.rowptr, dtype=np.int32), np.ascontiguousarray(A.col, dtype=np.int32),
                        np.ascontiguousarray(A.val, dtype=np.float64), int(p), x, Y)
    return Y, int(_omp_lib.omp_pxspmv_threads())


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
            f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
            i32, f64 = C.c_int32, C.c_double
            lib.oracle_spmv_rows.argtypes = [i32p, i32p, f64p, i32, f64p, f64p, i32, i32]
            lib.oracle_mpk.argtypes = [i32, i32p, i32p, f64p, i32, i32, f64p, f64p]
            lib.oracle_bfs_levels.argtypes = [i32, i32p, i32p, i32, i32, i32p]
            lib.oracle_bfs_levels.restype = i32
            lib.oracle_level_perm.argtypes = [i32, i32p, i32, i32p, i32p, i32p]
            lib.oracle_permute_csr.argtypes = [i32, i32p, i32p, f64p, i32p, i32p, i32p, i32p, f64p]
            lib.oracle_level_groups.argtypes = [i32, f64p, i32, f64, f64, i32p]
            lib.oracle_level_groups.restype = i32
            lib.oracle_recursive_levels.argtypes = [i32, i32p, i32p, i32, f64p, i32, f64, f64, i32, i32p, i32p,
                                                    C.POINTER(i32), i32p, C.POINTER(i32), i32p]
            lib.oracle_recursive_levels.restype = i32
            lib.oracle_cg.argtypes = [i32, i32p, i32p, f64p, f64p, f64p, f64, i32, C.POINTER(f64)]
            lib.oracle_cg.restype = i32
            lib.oracle_sstep_cg.argtypes = [i32, i32p, i32p, f64p, f64p, f64p, i32, f64, f64, i32, C.POINTER(f64)]
            lib.oracle_sstep_cg.restype = i32
            lib.oracle_lp_order.argtypes = [i32, i32, i32p, i32p]
            lib.oracle_lp_order.restype = C.c_int64
            lib.oracle_lb_mpk.argtypes = [i32, i32p, i32p, f64p, i32, i32p, i32, i32, f64p, f64p]
            lib.oracle_gershgorin.argtypes = [i32, i32p, i32p, f64p, C.POINTER(f64), C.POINTER(f64)]
            lib.oracle_cheb_coeffs_schroedinger.argtypes = [i32, f64, f64, f64, f64p]
            lib.oracle_cheb.argtypes = [i32, i32p, i32p, f64p, f64, f64, i32, f64p, f64p, f64p]
            lib.oracle_cheb_coeffs_heat.argtypes = [i32, f64, f64, f64, f64p]
            lib.oracle_cheb_real.argtypes = [i32, i32p, i32p, f64p, f64, f64, i32, f64p, f64p, f64p]
            _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def spmv(A, x):
    """y = A x (Fig. 1); x shape (n,) or (n, nrhs)."""
    return mpk(A, x, 1)[0]


def mpk(A, x, pm):
    """Baseline MPK (Sec. 3.1): returns Y with Y[k-1] = A^k x, k = 1..pm."""
    lib = _load()
    x = _f64(x)
    nrhs = 1 if x.ndim == 1 else x.shape[1]
    Y = np.empty((pm,) + x.shape, dtype=np.float64)
    lib.oracle_mpk(A.n, _i32(A.rowptr), _i32(A.col), _f64(A.val), pm, nrhs, x, Y)
    return Y


def bfs_levels(A, root=0, symmetrize=False):
    """Eq. 3 levels: returns (level[n] int32, nlevels)."""
    lib = _load()
    level = np.empty(A.n, dtype=np.int32)
    L = lib.oracle_bfs_levels(A.n, _i32(A.rowptr), _i32(A.col), int(root), int(bool(symmetrize)), level)
    return level, int(L)


def level_perm(level, nlevels):
    """Level-consecutive renumbering: returns (perm, iperm, level_ptr)."""
    lib = _load()
    n = level.shape[0]
    perm = np.empty(n, dtype=np.int32)
    iperm = np.empty(n, dtype=np.int32)
    level_ptr = np.empty(nlevels + 1, dtype=np.int32)
    lib.oracle_level_perm(n, _i32(level), nlevels, perm, iperm, level_ptr)
    return perm, iperm, level_ptr


def permute_csr(A, perm, iperm):
    """P A P^T with each row's columns ascending; returns a CSR of the same class."""
    lib = _load()
    prow = np.empty(A.n + 1, dtype=np.int32)
    pcol = np.empty(A.nnz, dtype=np.int32)
    pval = np.empty(A.nnz, dtype=np.float64)
    lib.oracle_permute_csr(A.n, _i32(A.rowptr), _i32(A.col), _f64(A.val), _i32(perm), _i32(iperm),
                           prow, pcol, pval)
    return type(A)(A.n, prow, pcol, pval, name=A.name + "-perm")


def level_groups(level_weight, pm, f, C_bytes):
    """Eq. 5 greedy groups: returns group_ptr (level indices), length G+1."""
    lib = _load()
    w = _f64(level_weight)
    gp = np.empty(w.shape[0] + 1, dtype=np.int32)
    G = lib.oracle_level_groups(w.shape[0], w, int(pm), float(f), float(C_bytes), gp)
    return gp[:G + 1].copy()


def recursive_levels(A, weights, pm, f, C_bytes, s_max, root=0):
    """Sec. 4.4 recursion: returns (perm, level_ptr, group_ptr, group_stage,
    stages) with the finest levels, the groups as ranges of them, the stage
    that made each group, and the number of stages that refined something."""
    lib = _load()
    n = A.n
    perm = np.empty(n, dtype=np.int32)
    lp = np.empty(n + 1, dtype=np.int32)
    gp = np.empty(n + 1, dtype=np.int32)
    gs = np.empty(n + 1, dtype=np.int32)
    nl, ng = C.c_int32(), C.c_int32()
    st = lib.oracle_recursive_levels(n, _i32(A.rowptr), _i32(A.col), int(root), _f64(weights), int(pm), float(f),
                                     float(C_bytes), int(s_max), perm, lp, C.byref(nl), gp, C.byref(ng), gs)
    return perm, lp[:nl.value + 1].copy(), gp[:ng.value + 1].copy(), gs[:ng.value].copy(), int(st)


def cg(A, b, x0=None, tol=1e-10, max_iter=10000):
    """Conjugate gradients (FP64): returns (x, steps, relres)."""
    lib = _load()
    x = np.zeros(A.n) if x0 is None else _f64(x0).copy()
    rel = C.c_double()
    it = lib.oracle_cg(A.n, _i32(A.rowptr), _i32(A.col), _f64(A.val), _f64(b), x, float(tol), int(max_iter),
                       C.byref(rel))
    return x, int(it), rel.value


def sstep_cg(A, b, s, rho, x0=None, tol=1e-10, max_steps=10000):
    """s-step CG with the monomial basis scaled by rho^-k (FP64): returns
    (x, steps, relres of the recurred residual)."""
    lib = _load()
    x = np.zeros(A.n) if x0 is None else _f64(x0).copy()
    rel = C.c_double()
    st = lib.oracle_sstep_cg(A.n, _i32(A.rowptr), _i32(A.col), _f64(A.val), _f64(b), x, int(s), float(rho),
                             float(tol), int(max_steps), C.byref(rel))
    return x, int(st), rel.value


def lp_order(nlevels, pm):
    """Fig. 5 execution order: arrays (i, p) of the L_m * pm nodes, step 0 first."""
    lib = _load()
    cap = max(1, nlevels * pm)
    ni = np.empty(cap, dtype=np.int32)
    npw = np.empty(cap, dtype=np.int32)
    s = lib.oracle_lp_order(int(nlevels), int(pm), ni, npw)
    return ni[:s].copy(), npw[:s].copy()


def lb_mpk(Aperm, unit_ptr, x, pm, fill=np.nan):
    """Fig. 5 run sequentially over units (levels or level groups) of an
    already permuted matrix; Y starts filled with `fill` so that a read of a
    not-yet-computed entry shows up in the result."""
    lib = _load()
    x = _f64(x)
    nrhs = 1 if x.ndim == 1 else x.shape[1]
    Y = np.full((pm,) + x.shape, fill, dtype=np.float64)
    up = _i32(unit_ptr)
    lib.oracle_lb_mpk(Aperm.n, _i32(Aperm.rowptr), _i32(Aperm.col), _f64(Aperm.val),
                      up.shape[0] - 1, up, pm, nrhs, x, Y)
    return Y


def gershgorin(A):
    lib = _load()
    lo, hi = C.c_double(), C.c_double()
    lib.oracle_gershgorin(A.n, _i32(A.rowptr), _i32(A.col), _f64(A.val), C.byref(lo), C.byref(hi))
    return lo.value, hi.value


def cheb_coeffs_schroedinger(M, c, r, dt):
    """Complex coefficients (M+1,) of exp(-i H dt) in T_k((H-c)/r)."""
    lib = _load()
    out = np.empty(2 * (M + 1), dtype=np.float64)
    lib.oracle_cheb_coeffs_schroedinger(int(M), float(c), float(r), float(dt), out)
    return out[0::2] + 1j * out[1::2]


def cheb(A, coef, c, r, x):
    """y = sum_k coef_k T_k((A-c)/r) x for complex x (Eq. 7-9), FP64."""
    lib = _load()
    coef = np.asarray(coef, dtype=np.complex128)
    M = coef.shape[0] - 1
    xi = np.empty((A.n, 2), dtype=np.float64)
    xi[:, 0] = np.real(x)
    xi[:, 1] = np.imag(x)
    ci = np.empty(2 * (M + 1), dtype=np.float64)
    ci[0::2] = coef.real
    ci[1::2] = coef.imag
    y = np.empty((A.n, 2), dtype=np.float64)
    lib.oracle_cheb(A.n, _i32(A.rowptr), _i32(A.col), _f64(A.val), float(c), float(r), int(M), ci, xi, y)
    return y[:, 0] + 1j * y[:, 1]


def cheb_coeffs_heat(M, c, r, tau):
    """Real coefficients (M+1,) of exp(-tau A) in T_k((A-c)/r) (modified Bessel)."""
    lib = _load()
    out = np.empty(M + 1, dtype=np.float64)
    lib.oracle_cheb_coeffs_heat(int(M), float(c), float(r), float(tau), out)
    return out


def cheb_coeffs_inverse(M, c, r, nodes=4096):
    """Coefficients (M+1,) of 1/lambda on [c-r, c+r] in T_k((lambda-c)/r), the
    approximate inverse that a polynomial preconditioner applies through the
    MPK (Sec. 1 and Sec. 8 name polynomial preconditioning as an MPK
    consumer; the expansion itself is the textbook Chebyshev series of 1/x),
    by Chebyshev-Gauss quadrature of f(t) = 1/(c + r t):
    c_k = (2 - delta_k0)/N sum_j f(cos th_j) cos(k th_j), th_j = pi (j+1/2)/N."""
    th = np.pi * (np.arange(nodes) + 0.5) / nodes
    f = 1.0 / (c + r * np.cos(th))
    k = np.arange(M + 1)
    out = (np.cos(np.outer(k, th)) * f[None, :]).sum(1) / nodes
    out[1:] *= 2.0
    return out


def cheb_real(A, coef, c, r, x):
    """y = sum_k coef_k T_k((A-c)/r) x for real x and coef (Eq. 7-9), FP64."""
    lib = _load()
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    M = coef.shape[0] - 1
    y = np.empty(A.n, dtype=np.float64)
    lib.oracle_cheb_real(A.n, _i32(A.rowptr), _i32(A.col), _f64(A.val), float(c), float(r), int(M), coef,
                         _f64(x), y)
    return y
