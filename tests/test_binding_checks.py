"""The Python binding rejects tensors whose dtype or size does not match what
an entry point reads or writes, before anything is launched (the C ABI takes
plain pointers and cannot see sizes).  CPU tensors stand in for CUDA ones:
the dtype and size checks come first, and the device check then refuses
them."""
import pytest
import torch

import paper_2205_01598_gb300 as mpk


def _plan(n=10, p=3, nrhs=1, prec=mpk.MPK_F64):
    return mpk.Plan(None, p, nrhs, prec, n, None)


def test_mpk_run_checks_x_and_y():
    pl = _plan()
    f64 = torch.float64
    with pytest.raises(ValueError, match="x: expected 10 elements"):
        mpk.mpk_run(pl, torch.zeros(9, dtype=f64), torch.zeros(30, dtype=f64))
    with pytest.raises(ValueError, match="Y: expected 30 elements"):
        mpk.mpk_run(pl, torch.zeros(10, dtype=f64), torch.zeros(3, 9, dtype=f64))
    with pytest.raises(TypeError, match="x: expected dtype torch.float64"):
        mpk.mpk_baseline_run(pl, torch.zeros(10, dtype=torch.float32), torch.zeros(30, dtype=f64))
    with pytest.raises(TypeError, match="CUDA tensor"):
        mpk.mpk_run(pl, torch.zeros(10, dtype=f64), torch.zeros(3, 10, dtype=f64))


def test_block_vectors_and_reduced_precision():
    pl = _plan(n=8, p=2, nrhs=4, prec=mpk.MPK_F32_BF16VAL)
    with pytest.raises(ValueError, match="x: expected 32 elements"):
        mpk.mpk_run(pl, torch.zeros(8, dtype=torch.float32), torch.zeros(64, dtype=torch.float32))
    with pytest.raises(TypeError, match="CUDA tensor"):
        mpk.mpk_run(pl, torch.zeros(8, 4, dtype=torch.float32), torch.zeros(2, 8, 4, dtype=torch.float32))


def test_chebyshev_checks():
    pl = _plan(n=6, p=4, nrhs=2, prec=mpk.MPK_F32)
    coef = [1.0, 0.5]
    with pytest.raises(TypeError, match="y: expected dtype torch.float64"):
        mpk.mpk_cheb(pl, coef, 0.0, 1.0, torch.zeros(6, 2), torch.zeros(6, 2))
    with pytest.raises(ValueError, match="x: expected 12 elements"):
        mpk.mpk_cheb(pl, coef, 0.0, 1.0, torch.zeros(6), torch.zeros(6, 2, dtype=torch.float64))
    pl1 = _plan(n=6, p=4, nrhs=1, prec=mpk.MPK_F64)
    with pytest.raises(ValueError, match="y: expected 6 elements"):
        mpk.mpk_cheb_real(pl1, coef, 0.0, 1.0, torch.zeros(6, dtype=torch.float64), torch.zeros(5, dtype=torch.float64))


def test_permute_and_csr_checks():
    pl = _plan(n=5, p=2, nrhs=1)
    with pytest.raises(TypeError, match="dst: expected dtype torch.float32"):
        mpk.mpk_permute_vectors(pl, torch.zeros(10), torch.zeros(10, dtype=torch.float64), 2, True)
    with pytest.raises(ValueError, match="src: expected 10 elements"):
        mpk.mpk_permute_vectors(pl, torch.zeros(9), torch.zeros(10), 2, True)
    rp = torch.tensor([0, 1, 2], dtype=torch.int32)
    with pytest.raises(TypeError, match="val: expected a torch.float64"):
        mpk.mpk_plan(rp, torch.zeros(2, dtype=torch.int32), torch.zeros(2, dtype=torch.float32), 2)
    with pytest.raises(ValueError, match="same length nnz"):
        mpk.mpk_plan(rp, torch.zeros(2, dtype=torch.int32), torch.zeros(3, dtype=torch.float64), 2)


def test_batch_checks_each_member():
    b = mpk.Batch.__new__(mpk.Batch)
    b.handle, b.plans = None, [_plan(n=4, p=2), _plan(n=3, p=5)]
    f64 = torch.float64
    with pytest.raises(ValueError, match="one per plan"):
        mpk.mpk_batch_run(b, [torch.zeros(4, dtype=f64)], [torch.zeros(8, dtype=f64)])
    with pytest.raises(ValueError, match="Y: expected 15 elements"):
        mpk.mpk_batch_run(b, [torch.zeros(4, dtype=f64), torch.zeros(3, dtype=f64)],
                          [torch.zeros(8, dtype=f64), torch.zeros(14, dtype=f64)])
    b.handle = None


def test_run_host_checks():
    pl = _plan(n=7, p=2, nrhs=1)
    f64 = torch.float64
    with pytest.raises(ValueError, match="Y: expected 14 elements"):
        mpk.mpk_run_host(pl, torch.zeros(7, dtype=f64), torch.zeros(13, dtype=f64))
    with pytest.raises(TypeError, match="contiguous CPU tensor"):
        mpk.mpk_run_host(pl, torch.zeros(7, dtype=f64), torch.zeros(2, 14, dtype=f64)[:, ::2])
    mpk.build()
    with pytest.raises(mpk.MpkError) as e:   # reaches the library, which refuses a NULL plan
        mpk.mpk_run_host(pl, torch.zeros(7, dtype=f64), torch.zeros(2, 7, dtype=f64))
    assert e.value.code == mpk.MPK_ERR_INVALID
