"""GPU tests of gp_train (Sec. 2.4 objectives ascended by Adam, the reading of
Sec. 4's gradient-based training) through the C ABI: the iterates and the
trace against the oracle's training loop on the same-probe estimator (FP64),
ascent of each objective on the FP32 path, feasibility under Eq.
eq:constrained, and the argument checks."""

import numpy as np
import pytest

from oracle import gp_oracle as O
from paper_2205_09070_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NV, M, SEED = 8, 20, 7


@pytest.fixture(scope="module")
def G():
    import __graft_entry__ as g
    g.build()
    from paper_2205_09070_gb300 import gpsparse
    assert torch.cuda.is_available()
    return gpsparse


def theta_eps(p, objective):
    """Adam's eps at 1e-4 of the largest starting gradient in theta, so that a
    component far below the solver's error bound moves by a negligible step
    instead of a sign step (both sides take the same eps)."""
    lml, g, _ = O.lml_grad_same_probes(p.x, p.y, p.h, p.dim, p.n1, p.n2, NV, M, SEED)
    if objective == "augmented":
        _, g, _ = O.augmented_objective(lml, g, p.h, p.dim, p.n1, p.n2)
    pos = O.positive_entries(len(p.h), p.dim, p.n1, p.n2)
    return 1e-4 * float(np.max(np.abs(np.where(pos, p.h * g, g))))


@pytest.mark.parametrize("objective", ["lml", "augmented", "constrained"])
def test_train_matches_the_oracle(G, objective):
    p = W.small_2d(seed=1, n=500)
    n_steps, lr = 3, 0.05
    eps = theta_eps(p, objective)
    s0 = O.sparsity_upper_bound(p.h, p.dim, p.n1, p.n2)
    s_max = 1.02 * s0 if objective == "constrained" else 0.0
    ref_h, ref_tr = O.train_same_probes(p.x, p.y, p.h, p.dim, p.n1, p.n2, NV, M, SEED, objective, n_steps, lr,
                                        eps=eps, s_max=s_max)
    gp = G.GP(p.dim, p.n1, p.n2)
    o = G.default_opts(precision="fp64", n_probes=NV, lanczos_steps=M, cg_rtol=1e-11, seed=SEED)
    h, tr, info = gp.train(torch.as_tensor(p.x, device="cuda"), torch.as_tensor(p.y, device="cuda"), p.h, o,
                           objective=objective, n_steps=n_steps, lr=lr, eps=eps, s_max=s_max)
    print(objective, "objective", tr[:, 0], "oracle", ref_tr[:, 0])
    # ln L within the FP64 same-probe estimator's agreement (its SLQ term to
    # 1e-7); the iterates follow the gradients, which agree far more closely
    assert np.allclose(tr, ref_tr, rtol=1e-6, atol=0.0)
    assert np.allclose(h, ref_h, rtol=1e-7, atol=1e-9 * np.max(np.abs(ref_h)))
    assert not np.allclose(h, p.h)                      # the steps moved h
    if objective == "constrained":
        assert np.all(tr[:, 2] < s_max)
    gp.close()


@pytest.mark.parametrize("objective", ["lml", "augmented", "constrained"])
def test_train_ascends_on_the_fp32_path(G, objective):
    p = W.small_2d(seed=3, n=2000)
    s0 = O.sparsity_upper_bound(p.h, p.dim, p.n1, p.n2)
    s_max = 1.01 * s0
    gp = G.GP(p.dim, p.n1, p.n2)
    o = G.default_opts(precision="fp32", n_probes=16, lanczos_steps=30, seed=SEED)
    h, tr, _ = gp.train(torch.as_tensor(p.x, device="cuda"), torch.as_tensor(p.y, device="cuda"), p.h, o,
                        objective=objective, n_steps=6, lr=0.01, s_max=s_max)
    print(objective, tr[:, 0])
    assert tr[-1, 0] > tr[0, 0]
    assert np.all(np.isfinite(tr)) and np.all(np.isfinite(h))
    if objective == "augmented":
        assert np.allclose(tr[:, 0], (2.0 - tr[:, 2]) * tr[:, 1], rtol=1e-14)
    else:
        assert np.array_equal(tr[:, 0], tr[:, 1])
    if objective == "constrained":
        assert np.all(tr[:, 2] < s_max)
    # s in the trace is the host sparsity bound at each iterate
    s_end, _ = G.sparsity_estimate(p.dim, p.n1, p.n2, h, 1.0)
    assert tr[-1, 2] == s_end
    gp.close()


def test_train_argument_checks(G):
    p = W.small_2d(seed=1, n=300)
    gp = G.GP(p.dim, p.n1, p.n2)
    x, y = torch.as_tensor(p.x, device="cuda"), torch.as_tensor(p.y, device="cuda")
    s0 = O.sparsity_upper_bound(p.h, p.dim, p.n1, p.n2)
    bad = [dict(objective=3), dict(lr=0.0), dict(lr=np.nan), dict(n_steps=-1), dict(domain_volume=0.0),
           dict(beta1=1.0), dict(eps=-1.0), dict(objective="constrained", s_max=0.5 * s0),
           dict(objective="constrained", s_max=0.0)]
    for kw in bad:
        with pytest.raises(G.GPError) as e:
            gp.train(x, y, p.h, G.default_opts(), **kw)
        assert e.value.status == G.GP_ERR_INVALID_ARG, kw
    h0 = p.h.copy()
    h0[-2] = 0.0                                          # A = 0 cannot be stepped in ln A
    with pytest.raises(G.GPError) as e:
        gp.train(x, y, h0, G.default_opts())
    assert e.value.status == G.GP_ERR_INVALID_ARG
    # zero steps: one evaluation, h unchanged
    h, tr, _ = gp.train(x, y, p.h, G.default_opts(), n_steps=0)
    assert np.array_equal(h, p.h) and tr.shape == (1, 3) and np.isfinite(tr[0, 0])
    gp.close()
