"""hpc_autotune / hpc_set_tuning: launch shapes are chosen by timing, leave the
iterates unchanged, and the autotuner leaves the iterate as it found it."""
import numpy as np
import pytest

from workloads import small_problem

pytestmark = pytest.mark.gpu


def _torch():
    import torch

    assert torch.cuda.is_available()
    return torch


def test_autotune_picks_valid_shapes_and_keeps_results(lib):
    torch = _torch()
    X = torch.as_tensor(small_problem(600, 300, 5.0, seed=41).astype(np.float32)).cuda()
    with lib.Solver(X, 0.12, 0.1, precision=lib.PREC_BF16X3, eps=1e-7) as ref:
        ref.solve()
        om_ref = ref.omega_dense()
        st_ref = ref.stats.as_dict()
    with lib.Solver(X, 0.12, 0.1, precision=lib.PREC_BF16X3, eps=1e-7) as s:
        best, trials = s.autotune(X, iters=2)
        knobs = {t["knob"] for t in trials}
        assert {"gram_band", "gram_maxima", "gram_schedule", "ls_window", "rows_ctas_per_sm",
                "ls_blocks_per_sm"} <= knobs
        assert all(t["ms"] > 0 for t in trials)
        assert s.get_tuning() == best
        assert best["ls_window"] in (2, 4, 8, 16) and 1 <= best["rows_ctas_per_sm"] <= 4
        assert best["fused_tail"] == 0          # the tail's form is not tuned
        st = s.solve().as_dict()
        om = s.omega_dense()
    assert np.array_equal(om, om_ref)
    assert st["iterations"] == st_ref["iterations"] and st["ls_trials"] == st_ref["ls_trials"]


@pytest.mark.parametrize("shape", [
    dict(rows_ctas_per_sm=3, ls_blocks_per_sm=3, ls_window=4),     # the 3-CTA forms
    dict(rows_ctas_per_sm=1, ls_blocks_per_sm=1, ls_window=2),
    dict(rows_ctas_per_sm=4, ls_blocks_per_sm=0, ls_window=16, gram_band=2, gram_maxima=0),
    dict(gram_schedule=0, gram_band=16),                           # static tile order
    dict(gram_schedule=1, gram_band=4),
    dict(fused_tail=1, ls_window=4),                               # the one-launch tail
    dict(fused_tail=1, ls_blocks_per_sm=1, ls_window=16),
])
def test_launch_shapes_give_the_default_iterates(lib, shape):
    """Every form the knobs select reaches the default shapes' estimate, iteration for
    iteration, including the row kernel's and line-search kernel's 3-CTA forms."""
    torch = _torch()
    X = torch.as_tensor(small_problem(1024, 400, 5.0, seed=17).astype(np.float32)).cuda()
    out = []
    for kw in ({}, shape):
        with lib.Solver(X, 0.08, 0.1, precision=lib.PREC_BF16X3, eps=1e-7) as s:
            if kw:
                s.set_tuning(**kw)
                s.load_x(X)
            st = s.solve().as_dict()
            out.append((s.omega_dense(), st))
    (a, sa), (b, sb) = out
    assert np.array_equal(a, b)
    assert sa["iterations"] == sb["iterations"] and sa["ls_trials"] == sb["ls_trials"]


def test_autotune_restores_the_iterate(lib):
    torch = _torch()
    X = torch.as_tensor(small_problem(300, 200, 4.0, seed=43).astype(np.float32)).cuda()
    with lib.Solver(X, 0.1, 0.1, precision=lib.PREC_FP32) as s:
        s.iterate(3)
        before = s.omega_dense()
        s.autotune(None, iters=2)
        assert np.array_equal(s.omega_dense(), before)
        s.iterate(2)
        after_tuned = s.omega_dense()
    with lib.Solver(X, 0.1, 0.1, precision=lib.PREC_FP32) as s:
        s.iterate(5)
        assert np.array_equal(s.omega_dense(), after_tuned)


@pytest.mark.parametrize("bad", [dict(gram_band=0), dict(ls_window=3), dict(rows_ctas_per_sm=5),
                                 dict(ls_blocks_per_sm=-1), dict(gram_maxima=2), dict(screen_bounds=2),
                                 dict(fused_tail=2),
                                 dict(gram_schedule=3)])
def test_set_tuning_rejects_out_of_range(lib, bad):
    torch = _torch()
    X = torch.as_tensor(small_problem(64, 40, 3.0, seed=1).astype(np.float32)).cuda()
    with lib.Solver(X, 0.1, 0.1) as s:
        with pytest.raises(lib.HpcError):
            s.set_tuning(**bad)
        s.set_tuning(gram_band=4, ls_window=2, rows_ctas_per_sm=1, ls_blocks_per_sm=1)
        t = s.get_tuning()
        assert {k: t[k] for k in ("gram_band", "ls_window", "ls_blocks_per_sm", "rows_ctas_per_sm")} == \
            dict(gram_band=4, ls_window=2, ls_blocks_per_sm=1, rows_ctas_per_sm=1)
