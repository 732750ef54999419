"""The allocation-free levels entry point (mpk_levels_noalloc), for callers
that may not allocate device memory after start-up (a host that sizes all
device memory once, under a fixed budget or a hard GPU quota).  It keeps its
scratch in a static device array of the library; its output must equal the
levels of the normal entry point (mpk_plan, read back with mpk_plan_perm)
exactly, on two calls in a row (the second call reuses the array the first
one left behind), and a call after a warm-up call must not change the
device's free memory or the default memory pool's usage.

This file is collected last on purpose."""
import ctypes as C
import gc

import numpy as np
import pytest
import torch

import mpk_inputs as mi
import paper_2205_01598_gb300 as mpk

pytestmark = pytest.mark.gpu


def _cudart():
    for name in ("libcudart.so.13", "libcudart.so", "/usr/local/cuda/lib64/libcudart.so"):
        try:
            return C.CDLL(name)
        except OSError:
            continue
    return None


def _device_memory_state():
    """(free device bytes, default pool's reserved bytes, default pool's used
    bytes, torch's allocated bytes) on the current device, after a garbage
    collection (so that tensors of earlier tests are released first)."""
    gc.collect()
    torch.cuda.synchronize()
    free, _ = torch.cuda.mem_get_info()
    reserved = used = None
    rt = _cudart()
    if rt is not None:
        dev = C.c_int()
        pool = C.c_void_p()
        if rt.cudaGetDevice(C.byref(dev)) == 0 and rt.cudaDeviceGetDefaultMemPool(C.byref(pool), dev) == 0:
            r, u = C.c_uint64(), C.c_uint64()
            if rt.cudaMemPoolGetAttribute(pool, 0x5, C.byref(r)) == 0:   # cudaMemPoolAttrReservedMemCurrent
                reserved = r.value
            if rt.cudaMemPoolGetAttribute(pool, 0x7, C.byref(u)) == 0:   # cudaMemPoolAttrUsedMemCurrent
                used = u.value
    return free, reserved, used, torch.cuda.memory_allocated()


def _levels_noalloc(lib, rp, cl, root, out):
    nl = C.c_int32()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = lib.mpk_levels_noalloc(rp.numel() - 1, cl.numel(), C.c_void_p(rp.data_ptr()), C.c_void_p(cl.data_ptr()),
                                root, C.c_void_p(out.data_ptr()), C.byref(nl), stream, 2.0)
    return rc, nl.value


@pytest.mark.parametrize("make,root", [
    (lambda: mi.stencil2d_7pt(8), 0),
    (lambda: mi.laplace3d(40), 0),
    (lambda: mi.random_sparse(2500, 1.3 / 2500, 17), 5),      # many components: restart rule
    (lambda: mi.anderson3d(20), 123),
])
def test_noalloc_levels_equal_plan_levels_twice(make, root):
    mpk.build()
    lib = mpk.load()
    A = make()
    rp, cl, va = mpk.csr_to_device(A)
    plan = mpk.mpk_plan(rp, cl, va, 2, root=root, assume_symmetric=True)
    ref_levels = mpk.mpk_plan_perm(plan)[3].cpu()
    ref_n = mpk.mpk_plan_info(plan)["n_levels"]
    for _ in range(2):
        out = torch.full((A.n,), -7, dtype=torch.int32, device="cuda")
        rc, nl = _levels_noalloc(lib, rp, cl, root, out)
        assert rc == mpk.MPK_OK, mpk.mpk_strerror(rc)
        assert nl == ref_n
        assert torch.equal(out.cpu(), ref_levels)


def test_noalloc_call_allocates_no_device_memory():
    mpk.build()
    lib = mpk.load()
    A = mi.laplace3d(60)
    rp, cl, _ = mpk.csr_to_device(A)
    out = torch.empty(A.n, dtype=torch.int32, device="cuda")
    rc, nl = _levels_noalloc(lib, rp, cl, 0, out)          # warm-up: loads the kernels
    assert rc == mpk.MPK_OK and nl == 3 * 59 + 1
    before = _device_memory_state()
    for _ in range(2):
        rc, nl = _levels_noalloc(lib, rp, cl, 0, out)
        assert rc == mpk.MPK_OK and nl == 3 * 59 + 1
    after = _device_memory_state()
    # the driver's free bytes and the default pool are unchanged; torch's
    # own count can only have shrunk (it tracks torch tensors, none made here)
    assert after[:3] == before[:3] and after[3] <= before[3]
    # the binding's wrapper passes the caller's output through unchanged
    lev, nl2 = mpk.mpk_levels_noalloc(rp, cl, 0, out)
    assert lev.data_ptr() == out.data_ptr() and nl2 == nl
    again = _device_memory_state()
    assert again[:3] == before[:3] and again[3] <= before[3]


def test_noalloc_rejects_sizes_beyond_the_scratch():
    lib = mpk.load()
    n = (1 << 20) + 1
    rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    cl = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    rc, _ = _levels_noalloc(lib, rp, cl, 0, out)
    assert rc == mpk.MPK_ERR_UNSUPPORTED
    # and a malformed matrix inside the limit is refused, not read out of bounds
    A = mi.laplace2d(10)
    rp, cl, _ = mpk.csr_to_device(A)
    bad = cl.clone()
    bad[3] = A.n + 5
    out = torch.empty(A.n, dtype=torch.int32, device="cuda")
    rc, _ = _levels_noalloc(lib, rp, bad, 0, out)
    assert rc == mpk.MPK_ERR_INVALID
    # the entry point still works after the refusals
    rc, nl = _levels_noalloc(lib, rp, cl, 0, out)
    assert rc == mpk.MPK_OK and nl == 19
