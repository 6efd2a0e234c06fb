"""Tensor-core Gram (tcgen05 + TMA) against the FP64 oracle's S = X^T X / n.

Error bounds per entry, with D_ij = sqrt(S_ii S_jj) >= sum_k |x_ki x_kj| / n:
  BF16 X   : products exact, FP32 accumulation       |dS| <= 2 n u D
  BF16X3   : x = hi + lo (+ r), per product <= 2^-15  |dS| <= (2^-15 + 2 n u) D
  TF32     : inputs rounded to 10-bit mantissas       |dS| <= (2^-10 + 2 n u) D
with u = 2^-24.  Shapes cover ragged p (not a multiple of the 128 x 256 tile),
ragged n (not a multiple of the 64-element K slab), n = 1 and p = 1.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

U = 2.0 ** -24


def _gram(lib, X, precision, lds_extra=5):
    import torch

    n, p = X.shape
    S = torch.full((p, p + lds_extra), float("nan"), dtype=torch.float32, device="cuda")
    lib.gram(X, S, precision=precision)
    torch.cuda.synchronize()
    return S


def _check(got, Xd, rel):
    n = Xd.shape[0]
    ref = oracle.gram(Xd)
    D = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
    err = np.abs(got - ref)
    bound = (rel + 2 * n * U) * D + 1e-30
    assert np.all(err <= bound), float(np.max(err / bound))
    assert np.array_equal(got, got.T)


@pytest.mark.parametrize("n,p", [(257, 300), (64, 256), (1, 40), (700, 513), (96, 1)])
def test_bf16x3_on_fp32_x(lib, n, p):
    import torch

    rng = np.random.default_rng(n + 3 * p)
    X = rng.standard_normal((n, p)).astype(np.float32)
    S = _gram(lib, torch.as_tensor(X).cuda(), lib.PREC_BF16X3)
    got = S[:, :p].double().cpu().numpy()
    _check(got, X.astype(np.float64), 2.0 ** -15)
    assert torch.isnan(S[:, p:]).all()


@pytest.mark.parametrize("n,p", [(300, 700), (33, 257), (130, 1024), (65, 520)])
def test_single_product_on_bf16_x(lib, n, p):
    """p % 8 == 0 takes the 16-byte transpose of X into the panel; the others the
    element-wise edges; n not a multiple of 64 leaves a zero-padded K tail."""
    import torch

    rng = np.random.default_rng(p)
    Xb = torch.as_tensor(rng.standard_normal((n, p)).astype(np.float32)).to(torch.bfloat16)
    S = _gram(lib, Xb.cuda(), lib.PREC_BF16X3)
    got = S[:, :p].double().cpu().numpy()
    _check(got, Xb.float().numpy().astype(np.float64), 0.0)


def test_tf32(lib):
    import torch

    rng = np.random.default_rng(9)
    X = rng.standard_normal((200, 330)).astype(np.float32)
    S = _gram(lib, torch.as_tensor(X).cuda(), lib.PREC_TF32)
    got = S[:, :330].double().cpu().numpy()
    _check(got, X.astype(np.float64), 2.0 ** -10)


def test_bf16x3_at_several_bands(lib):
    """p = 4200 spans more than one band of 16 row blocks and 17 column blocks (ragged)."""
    import torch

    rng = np.random.default_rng(17)
    X = rng.standard_normal((640, 4200)).astype(np.float32)
    S = _gram(lib, torch.as_tensor(X).cuda(), lib.PREC_BF16X3, lds_extra=0)
    got = S.double().cpu().numpy()
    _check(got, X.astype(np.float64), 2.0 ** -15)


def test_solver_with_tensor_core_gram_matches_oracle(lib):
    """A whole solve on the BF16X3 Gram reaches the oracle's estimate to the FP32 tolerance."""
    import torch

    from workloads import small_problem

    X = small_problem(900, 600, 5.0, 12).astype(np.float32)
    S = oracle.gram(X)
    ref = oracle.solve(S, 0.15, 0.1, eps=1e-9, max_iter=20000)
    with lib.Solver(torch.as_tensor(X).cuda(), 0.15, 0.1, precision=lib.PREC_BF16X3, eps=1e-7) as s:
        assert s.precision_name() == "bf16x3"
        s.solve()
        om = s.omega_dense()
    assert np.linalg.norm(om - ref.omega) / np.linalg.norm(ref.omega) < 1e-5


@pytest.mark.parametrize("bf16", [True, False])
def test_host_x_pinned_or_pageable_gives_the_device_result(lib, bf16):
    """X from device memory, from pinned host memory (read in place through its device
    mapping) and from pageable host memory (staged): the same S, maxima and estimate."""
    import torch

    from workloads import small_problem

    n, p = 500, 700
    X = torch.as_tensor(small_problem(p, n, 5.0, 21).astype(np.float32))
    if bf16:
        X = X.to(torch.bfloat16)
    rng = np.random.default_rng(3)
    r, c = rng.integers(0, p, 200), rng.integers(0, p, 200)
    out = []
    for src in (X.cuda(), X.pin_memory(), X.clone()):
        with lib.Solver(None, 0.15, 0.1, n=n, p=p, xdtype=lib.BF16 if bf16 else lib.F32,
                        precision=lib.PREC_BF16X3, eps=1e-7) as s:
            s.load_x(src)
            m = s.block_maxima()
            e = s.s_entries(r, c)
            st = s.solve().as_dict()
            out.append((m, e, s.get_omega(np.float64), st["iterations"]))
    m0, e0, om0, it0 = out[0]
    for m, e, om, it in out[1:]:
        assert np.array_equal(m, m0)
        assert np.array_equal(e, e0)
        assert it == it0
        assert np.array_equal(om.col, om0.col) and np.array_equal(om.val, om0.val)


@pytest.mark.parametrize("src,dt", [("device", "bf16"), ("pinned", "bf16"), ("pageable", "bf16"),
                                    ("pinned", "f32"), ("device", "f32")])
def test_prefetch_gives_the_load_result(lib, src, dt):
    """hpc_prefetch_x stages the next X's panels while the current data solves; the next
    load_x of that X gives the same S, maxima and estimate as a plain load.  A prefetch
    of one X followed by the load of another is discarded."""
    import torch

    from workloads import small_problem

    n, p = 400, 1024
    tdt = torch.bfloat16 if dt == "bf16" else torch.float32
    mk = lambda seed: torch.as_tensor(small_problem(p, n, 5.0, seed).astype(np.float32)).to(tdt)
    X1, X2 = mk(31), mk(32)
    if src == "device":
        X1, X2 = X1.cuda(), X2.cuda()
    elif src == "pinned":
        X1, X2 = X1.pin_memory(), X2.pin_memory()
    rng = np.random.default_rng(5)
    r, c = rng.integers(0, p, 300), rng.integers(0, p, 300)

    def run(steps):
        with lib.Solver(None, 0.1, 0.1, n=n, p=p, xdtype=lib.BF16 if dt == "bf16" else lib.F32,
                        precision=lib.PREC_BF16X3, eps=1e-7) as s:
            for act, X in steps:
                if act == "load":
                    s.load_x(X)
                elif act == "prefetch":
                    s.prefetch_x(X)
                else:
                    s.solve()
            return s.block_maxima(), s.s_entries(r, c), s.solve().as_dict()["iterations"], s.omega_dense()

    ref2 = run([("load", X2)])
    # staged, then loaded directly (the staged copy)
    got2 = run([("load", X1), ("prefetch", X2), ("solve", None), ("load", X2)])
    # pipelined: staged before the current load, prepared after its Gram, loaded next
    pip2 = run([("load", X1), ("solve", None), ("prefetch", X2), ("load", X1), ("solve", None), ("load", X2)])
    ref1 = run([("load", X1)])
    # a staged X that is not loaded next: the load of another X is not affected
    got1 = run([("load", X2), ("prefetch", X2), ("solve", None), ("load", X1)])
    pip1 = run([("prefetch", X2), ("load", X2), ("prefetch", X2), ("load", X1)])
    for got, ref in ((got2, ref2), (pip2, ref2), (got1, ref1), (pip1, ref1)):
        assert np.array_equal(got[0], ref[0])
        assert np.array_equal(got[1], ref[1])
        assert got[2] == ref[2]
        assert np.array_equal(got[3], ref[3])


@pytest.mark.parametrize("xdt", ["bf16", "f32"])
def test_chunked_accumulation_removes_the_truncation_bias(lib, xdt):
    """The tensor core adds each MMA into the FP32 accumulator with truncation, which biases
    a long sum towards zero (about 0.6 ulp of the partial sum per MMA).  With the K loop cut
    into chunks summed in FP32 round-to-nearest (gram_chunk, default 512 K for BF16 X and
    256 K for BF16X3) the diagonal's mean relative error against the FP64 Gram stays within
    0.6 * 2^-23 per MMA of a chunk (32 or 48 MMAs); one chunk over all n = 8192 (a
    gram_chunk >= n) shows the bias the chunking removes.  Both stay within the per-entry
    bound, and the chunked S is exactly symmetric."""
    import torch

    n, p = 8192, 384
    rng = np.random.default_rng(23)
    X = rng.standard_normal((n, p)).astype(np.float32)
    Xt = torch.as_tensor(X).cuda()
    if xdt == "bf16":
        Xt = Xt.to(torch.bfloat16)
        Xd = Xt.float().cpu().numpy().astype(np.float64)
        per_chunk = 32
    else:
        Xd = X.astype(np.float64)
        per_chunk = 48
    ref = np.diag(oracle.gram(Xd))
    bias = {}
    for chunk in (0, n):
        with lib.Solver(Xt, 0.5, 0.1, precision=lib.PREC_BF16X3) as s:
            s.set_tuning(gram_chunk=chunk)
            s.load_x(Xt)
            d = s.s_entries(np.arange(p), np.arange(p))
        bias[chunk] = float(np.mean((d - ref) / ref))
    assert abs(bias[0]) <= 0.6 * 2.0 ** -23 * per_chunk * 1.5, bias
    assert bias[n] < -4 * abs(bias[0]), bias
