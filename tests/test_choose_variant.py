"""Lemma 3.1's choice between Cov and Obs (hpc_choose_variant; host code, no GPU):
- with gamma_sparse = gamma_dense its two costs are the lemma's flop counts, recomputed here
  from the lemma's formulas;
- for many s its decision is the lemma's condition d/p < n / ((p - n) t);
- p <= n always chooses Cov; the default constants and the argument checks."""
import numpy as np
import pytest


def _choose(lib, *a):
    return lib.choose_variant(*a)


@pytest.mark.parametrize("n,p,s,t,d", [(100, 40000, 28, 3, 2), (12800, 40000, 15, 4, 2), (5000, 8000, 40, 2, 9),
                                       (32768, 65536, 56, 3, 1)])
def test_costs_are_the_lemmas_flop_counts(lib, n, p, s, t, d):
    v, cov, obs = _choose(lib, n, p, s, t, d, 1.0)
    assert cov == pytest.approx(2.0 * n * p * p + 2.0 * d * p * p * (s * t + 1), rel=1e-14)
    assert obs == pytest.approx(2.0 * n * p * p * s + 2.0 * d * n * p * (s * t + 1), rel=1e-14)
    assert v == (lib.COV if cov < obs else lib.OBS)


def test_large_s_decision_is_the_lemmas_condition(lib):
    rng = np.random.default_rng(0)
    agree = 0
    for _ in range(400):
        p = int(rng.integers(1000, 100000))
        n = int(rng.integers(10, p))
        t = float(rng.integers(1, 8))
        d = float(rng.uniform(1, 60))
        v, _, _ = _choose(lib, n, p, 1e7, t, d, 1.0)
        cond = d / p < n / ((p - n) * t)
        agree += (v == lib.COV) == cond
    assert agree >= 398          # ties of the limit aside


def test_defaults_and_arguments(lib):
    v, cov, obs = _choose(lib, 200, 100, 0, 0, 0, 0)
    assert v == lib.COV                       # p <= n: S is no larger than X
    v0, c0, o0 = _choose(lib, 100, 40000)
    v1, c1, o1 = _choose(lib, 100, 40000, 40, 3, 2, 26.0)
    assert (v0, c0, o0) == (v1, c1, o1)
    with pytest.raises(lib.HpcError):
        _choose(lib, 0, 10)
