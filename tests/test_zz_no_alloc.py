"""The allocation-free Gram entry point (hpc_gram_noalloc) against the allocating one and
against the FP64 oracle.

hpc_gram_noalloc serves callers that must not allocate device memory while they
run (memory owned by another allocator, a fixed budget, loops where
cudaMalloc/cudaFree would synchronise the device).  It keeps its scratch in a
static device array shared by every call, so this test makes two calls in a row
with different shapes and inputs -- the second one runs on whatever the first
left in the array -- and compares each with hpc_gram, called through the C ABI
on the same input, and with the oracle's S = X^T X / n, within the Gram tests'
error bound.  It also checks that a
problem too large for the array is refused with HPC_ERR_ARG before any launch.
This file is collected last so that a failure here leaves the rest of the
suite already run; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

U = 2.0 ** -24


def _both(lib, X, precision, lds_extra):
    import torch

    n, p = X.shape
    ref = torch.full((p, p + lds_extra), float("nan"), dtype=torch.float32, device="cuda")
    got = torch.full((p, p + lds_extra), float("nan"), dtype=torch.float32, device="cuda")
    lib.gram(X, ref, precision=precision)
    lib.gram_noalloc(X, got, precision=precision)
    torch.cuda.synchronize()
    return ref.double().cpu().numpy(), got.double().cpu().numpy()


def _assert_close(ref, got, p, n, rel):
    r, g = ref[:, :p], got[:, :p]
    D = np.sqrt(np.outer(np.abs(np.diag(r)), np.abs(np.diag(r))))
    assert np.all(np.abs(g - r) <= (rel + 2 * n * U) * D + 1e-30)
    assert np.array_equal(g, g.T)
    assert np.isnan(got[:, p:]).all()


def _assert_oracle(got, X, rel):
    n, p = X.shape
    ref = oracle.gram(X.double().cpu().numpy())
    D = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
    assert np.all(np.abs(got[:, :p] - ref) <= (rel + 2 * n * U) * D + 1e-30)


def test_noalloc_matches_allocating_gram_on_two_calls_in_a_row(lib):
    import torch

    rng = np.random.default_rng(2024)
    # call 1: FP32 X in BF16X3 (two panels), ragged p and n
    X1 = torch.as_tensor(rng.standard_normal((257, 300)).astype(np.float32)).cuda()
    ref1, got1 = _both(lib, X1, lib.PREC_BF16X3, 3)
    _assert_close(ref1, got1, 300, 257, 2.0 ** -15)
    _assert_oracle(got1, X1, 2.0 ** -15)
    # call 2: a different, smaller BF16 problem on the scratch call 1 left behind
    X2 = torch.as_tensor(rng.standard_normal((100, 130)).astype(np.float32)).to(torch.bfloat16).cuda()
    ref2, got2 = _both(lib, X2, lib.PREC_BF16X3, 0)
    _assert_close(ref2, got2, 130, 100, 0.0)
    _assert_oracle(got2, X2, 0.0)


def test_noalloc_refuses_problems_larger_than_its_scratch(lib):
    import torch

    X = torch.zeros((4096, 4096), dtype=torch.float32, device="cuda")   # 2 panels x 32 MiB + tiles
    S = torch.zeros((1, 1), dtype=torch.float32, device="cuda")
    with pytest.raises(lib.HpcError) as e:
        lib.gram_noalloc(X, torch.empty((4096, 4096), dtype=torch.float32, device="cuda"))
    assert e.value.status == lib.ERR_ARG
    assert "static scratch holds" in str(e.value)
    del S
