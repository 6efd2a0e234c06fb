"""Block maxima of the bound screening: max |S_ij| per (row i, column block), j != i,
rounded up to BF16.  The tensor-core Gram writes them from its epilogue; the FP32
and FP64 modes by a pass over S.  Both must equal the BF16 round-up of the exact
maximum of the S the library itself computed (an upper bound that is as tight as
BF16 allows), including ragged p and n and the diagonal blocks."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _bf16_up(a32):
    """Non-negative float32 values rounded up to BF16, returned as float32."""
    u = np.ascontiguousarray(a32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = np.where(u & 0xFFFF, u + 0x10000, u) >> 16
    return (u.astype(np.uint32) << 16).view(np.float32)


def _f32_up(a64):
    """float64 -> float32 rounded towards +inf."""
    f = a64.astype(np.float32)
    lo = f.astype(np.float64) < a64
    f[lo] = np.nextafter(f[lo], np.float32(np.inf))
    return f


def _expected(S, block):
    p = S.shape[0]
    nb = -(-p // block)
    A = np.abs(S.copy())
    np.fill_diagonal(A, 0)
    pad = nb * block - p
    A = np.pad(A, ((0, 0), (0, pad)))
    return A.reshape(p, nb, block).max(axis=2)


@pytest.mark.parametrize("case", ["bf16x3_700", "bf16x3_1300", "tf32_520", "bf16x_600", "fp32_600", "fp64_300"])
def test_block_maxima_equal_the_rounded_up_exact_maxima(lib, case):
    import torch

    kind, p = case.split("_")
    p = int(p)
    n = {700: 300, 1300: 257, 520: 130, 600: 200, 300: 150}[p]
    rng = np.random.default_rng(p)
    X = rng.standard_normal((n, p)).astype(np.float32) * rng.uniform(0.5, 2.0, size=p).astype(np.float32)
    opt = {}
    if kind == "bf16x3":
        Xt, prec = torch.as_tensor(X), lib.PREC_BF16X3
    elif kind == "tf32":
        Xt, prec = torch.as_tensor(X), lib.PREC_TF32
    elif kind == "bf16x":
        Xt, prec = torch.as_tensor(X).to(torch.bfloat16), lib.PREC_BF16X3
    elif kind == "fp32":
        Xt, prec = torch.as_tensor(X), lib.PREC_FP32
    else:
        Xt, prec = torch.as_tensor(X.astype(np.float64)), lib.PREC_FP64
        opt = dict(value_dtype=lib.F64)
    Xd = Xt.cuda()
    with lib.Solver(Xd, 0.1, 0.1, precision=prec, **opt) as s:
        got = s.block_maxima()
    # the same product through the stateless entry point (same kernels, same bits)
    sdt = torch.float64 if kind == "fp64" else torch.float32
    S = torch.empty((p, p), dtype=sdt, device="cuda")
    lib.gram(Xd, S, precision=prec)
    torch.cuda.synchronize()
    S = S.cpu().numpy()
    block = 64 if kind == "fp64" else 128
    m = _expected(S, block)
    want = _bf16_up(_f32_up(m) if kind == "fp64" else m.astype(np.float32))
    assert got.shape == want.shape
    assert np.array_equal(got, want)


@pytest.mark.parametrize("p,n,f64,lam1", [
    (1024, 500, False, 0.08),     # 8 blocks: group maxima, two-level item selection, vector row masks
    (1100, 600, False, 0.06),     # 9 blocks: the per-block selection and row masks
    (512, 300, True, 0.08),       # FP64 (blocks of 64 columns)
    (2048, 700, False, 0.03),     # rows with many neighbours (the row kernel covers more blocks)
])
def test_bound_screening_changes_no_bit(lib, p, n, f64, lam1):
    """The bounds only decide which segments of S are read: a solve with them equals,
    bit for bit, the solve that streams the whole upper triangle and every block of
    the rows with neighbours."""
    import torch

    from workloads import small_problem

    X = small_problem(p, n, 5.0, p + 3).astype(np.float64 if f64 else np.float32)
    opt = dict(value_dtype=lib.F64, precision=lib.PREC_FP64, eps=1e-9) if f64 else \
        dict(precision=lib.PREC_FP32, eps=1e-7)
    out = []
    for bounds in (1, 0):
        with lib.Solver(torch.as_tensor(X).cuda(), lam1, 0.1, max_iter=20000, **opt) as s:
            s.set_tuning(screen_bounds=bounds)
            st = s.solve().as_dict()
            out.append((s.get_omega(np.float64), st))
    (a, sa), (b, sb) = out
    assert sa["status"] == 0 and sb["status"] == 0
    for key in ("iterations", "ls_trials", "nnz", "F", "rel_change"):
        assert sa[key] == sb[key], key
    assert np.array_equal(a.row_ptr, b.row_ptr)
    assert np.array_equal(a.col, b.col)
    assert np.array_equal(a.val, b.val)
    assert sa["nnz"] > p                  # off-diagonal entries survive
