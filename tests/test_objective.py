"""The sparsity bound (Sec. 2.2) and the augmented objective (Sec. 2.4,
Eq. eq:augmented) through the C ABI against the oracle.  Host-side calls: no
GPU needed."""

import numpy as np
import pytest

from oracle import gp_oracle as O
from paper_2205_09070_gb300 import gpsparse as G
from paper_2205_09070_gb300 import workloads as W


@pytest.mark.parametrize("dim,n1,n2", [(1, 1, 1), (2, 2, 3), (3, 4, 8), (3, 8, 16)])
def test_sparsity_estimate_and_gradient_match_the_oracle(dim, n1, n2):
    rng = np.random.default_rng(dim * 100 + n1 * 10 + n2)
    h = W.pack_h(rng.uniform(0, 1, (n1, n2, dim)), rng.uniform(0.01, 0.3, (n1, n2)), rng.normal(0, 1, (n1, n2)),
                 0.05, 1.0, 1e-4)
    for vol in (1.0, 0.37):
        s, g = G.sparsity_estimate(dim, n1, n2, h, vol)
        assert s == pytest.approx(O.sparsity_upper_bound(h, dim, n1, n2, vol), rel=1e-13)
        assert np.allclose(g, O.sparsity_upper_bound_grad(h, dim, n1, n2, vol), rtol=1e-13, atol=0)


def test_augmented_objective_matches_the_oracle_and_rejects_bad_input():
    p = W.grad_3d(seed=3, n=10)
    rng = np.random.default_rng(7)
    lml, lg = -1234.5, rng.normal(0, 10, len(p.h))
    val, g, s = G.augmented_objective(p.dim, p.n1, p.n2, p.h, 1.0, lml, lg)
    ov, og, os_ = O.augmented_objective(lml, lg, p.h, p.dim, p.n1, p.n2, 1.0)
    assert s == pytest.approx(os_, rel=1e-13)
    assert val == pytest.approx(ov, rel=1e-13)
    assert np.allclose(g, og, rtol=1e-12, atol=1e-12 * np.abs(og).max())
    bad = p.h.copy()
    bad[p.dim] = -0.1  # a negative radius
    with pytest.raises(G.GPError) as e:
        G.sparsity_estimate(p.dim, p.n1, p.n2, bad, 1.0)
    assert e.value.status == G.GP_ERR_INVALID_ARG
    with pytest.raises(G.GPError) as e:
        G.augmented_objective(p.dim, p.n1, p.n2, p.h, 0.0, lml, lg)
    assert e.value.status == G.GP_ERR_INVALID_ARG


def test_augmented_objective_sign_and_the_s_above_one_regime():
    # the printed objective (2 - s) lnL: its derivative in s is -lnL, so with
    # lnL < 0 a larger s (denser K) raises it, with lnL > 0 a smaller s does;
    # s is the uncapped bound, here above 1 and above 2 for large bumps in a
    # small domain, where the weight on lnL turns negative
    dim, n1, n2 = 3, 2, 3
    rng = np.random.default_rng(11)
    base = W.pack_h(rng.uniform(0, 1, (n1, n2, dim)), np.full((n1, n2), 0.2), rng.normal(0, 1, (n1, n2)),
                    0.05, 1.0, 1e-4)
    for lml in (-250.0, 40.0):
        vals = []
        for vol in (1.0, 0.2, 0.12, 0.1, 0.05):
            v, _, s = G.augmented_objective(dim, n1, n2, base, vol, lml, None)
            assert v == pytest.approx((2.0 - s) * lml, rel=1e-14)
            vals.append((s, v))
        ss = [s for s, _ in vals]
        assert ss == sorted(ss) and ss[0] < 1.0 < ss[2] and ss[-1] > 2.0   # s grows as the domain shrinks
        # finite differences in s have the sign of -lnL
        for (s_a, v_a), (s_b, v_b) in zip(vals, vals[1:]):
            assert np.sign(v_b - v_a) == np.sign(-lml)
        # above s = 2 the value and lnL have opposite signs
        assert np.sign(vals[-1][1]) == -np.sign(lml)
