"""GPU parity of the posterior mean (Sec. 2.1: kappa^T (K + V)^-1 y) through
the C ABI against the FP64 oracle: the cross-covariance sums checked against
the oracle's dense kappa applied to the GPU's own alpha (independent of the
solver's accuracy), the full prediction against the oracle's dense solve, exact
zeros off the supports, and the argument and edge cases."""

import ctypes

import numpy as np
import pytest

from oracle import gp_oracle as O
from paper_2205_09070_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import __graft_entry__ as g
    g.build()
    from paper_2205_09070_gb300 import gpsparse
    assert torch.cuda.is_available()
    return gpsparse


def mixture_small(n=6000, seed=41):
    return W.mixture_3d(seed=seed, n=n, r_s=0.005 * (5e6 / n) ** (1.0 / 3.0))


CASES = {
    "small_2d": lambda: W.small_2d(seed=1),
    "grad_3d": lambda: W.grad_3d(seed=3, n=3000),
    "mixture": lambda: mixture_small(),
}


_KAPPA = {}


def _cross_K_hp(case, p, xs):
    if case not in _KAPPA:
        _KAPPA[case] = O.cross_K_hp(xs, p.x, p.h, p.dim, p.n1, p.n2, p.beta)
    return _KAPPA[case]


def query_points(p, n_new=700, seed=5):
    # fresh points over a box a little larger than the data, some training
    # points, and two points far outside everything
    rng = np.random.default_rng(seed)
    lo, hi = p.x.min(axis=0) - 0.1, p.x.max(axis=0) + 0.1
    fresh = rng.uniform(lo, hi, (n_new, p.dim))
    train = p.x[rng.choice(p.n, 200, replace=False)]
    far = np.full((2, p.dim), 7.0)
    far[1] = -5.0
    return np.ascontiguousarray(np.vstack([fresh, train, far]))


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_predict_matches_oracle(G, case, prec):
    p = CASES[case]()
    xs = query_points(p)
    gp = G.GP(p.dim, p.n1, p.n2, p.beta)
    x = torch.as_tensor(p.x, device="cuda")
    y = torch.as_tensor(p.y, device="cuda")
    gp.assemble(x, p.h, precision=prec)
    rtol = 1e-10 if prec == "fp64" else 1e-6
    o = G.default_opts(precision=prec, cg_rtol=rtol)
    mean, info = gp.predict(y, torch.as_tensor(xs, device="cuda"), opts=o)
    m = mean.cpu().numpy()
    # the kernel's sums: oracle kappa times the GPU's own alpha
    alpha, _ = gp.solve(y, torch.zeros_like(y), o)
    a = alpha.cpu().numpy()
    # kappa with every pair evaluated to full accuracy (oracle.cross_K_hp)
    kappa = _cross_K_hp(case, p, xs)
    ref_sum = kappa @ a
    scale = np.abs(kappa) @ np.abs(a)
    # a sum of n_q FP64 products is within ~n_q 1e-16 of sum |kappa||alpha|
    worst = float(np.max(np.abs(m - ref_sum) / np.where(scale > 0, scale, 1.0)))
    print(case, prec, "worst kernel-sum error / sum|kappa||alpha|", worst)
    assert np.all(np.abs(m - ref_sum) <= 1e-11 * scale)
    # the whole prediction against the oracle's dense solve
    ref = O.predict_mean(p.x, p.y, p.h, xs, p.dim, p.n1, p.n2, p.beta)
    err = np.max(np.abs(m - ref)) / np.max(np.abs(ref))
    print(case, prec, "iters", info["iters"], "max rel error of the mean", err)
    assert err < (1e-6 if prec == "fp64" else 5e-3), err
    # outside everything: exactly zero
    assert m[-1] == 0.0 and m[-2] == 0.0
    _, mask_s = O.bump_table(xs, p.h, p.dim, p.n1, p.n2, p.beta)
    assert np.all(m[mask_s == 0] == 0.0)
    gp.close()


def test_predict_host_arrays_and_edge_cases(G):
    p = W.small_2d(seed=1)
    xs = query_points(p, n_new=100)
    gp = G.GP(p.dim, p.n1, p.n2, p.beta)
    lib = G.load()
    mean = np.zeros(len(xs))
    o = G.default_opts(precision="fp64", cg_rtol=1e-10)
    info = G.Info()
    # before any assembly
    st = lib.gp_predict(gp._h, p.y.ctypes.data, xs.ctypes.data, len(xs), mean.ctypes.data, ctypes.byref(o),
                        ctypes.byref(info))
    assert st == G.GP_ERR_NOT_ASSEMBLED
    gp.assemble(torch.as_tensor(p.x, device="cuda"), p.h, precision="fp64")
    # host arrays in and out, against device arrays in and out
    m_host, _ = gp.predict(p.y, xs, opts=o)
    m_dev, _ = gp.predict(torch.as_tensor(p.y, device="cuda"), torch.as_tensor(xs, device="cuda"), opts=o)
    assert np.array_equal(m_host, m_dev.cpu().numpy())
    # no test points
    st = lib.gp_predict(gp._h, p.y.ctypes.data, None, 0, None, ctypes.byref(o), ctypes.byref(info))
    assert st == G.GP_OK
    # missing outputs
    st = lib.gp_predict(gp._h, p.y.ctypes.data, xs.ctypes.data, len(xs), None, ctypes.byref(o), ctypes.byref(info))
    assert st == G.GP_ERR_INVALID_ARG
    gp.close()


def test_predict_when_no_training_point_is_active(G):
    # every training point outside every bump: K = sigma^2 I, kappa = 0
    p = W.small_2d(seed=1, n=300)
    h = p.h.copy()
    per = p.dim + 2
    for b in range(p.n1 * p.n2):
        h[b * per: b * per + p.dim] = 50.0   # centres far away
    gp = G.GP(p.dim, p.n1, p.n2, p.beta)
    gp.assemble(torch.as_tensor(p.x, device="cuda"), h, precision="fp32")
    mean, info = gp.predict(torch.as_tensor(p.y, device="cuda"),
                            torch.as_tensor(query_points(p, n_new=50), device="cuda"))
    assert info["n_active"] == 0
    assert torch.count_nonzero(mean).item() == 0
    gp.close()


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_predict_var_matches_oracle(G, case, prec):
    """Posterior variance k(x*, x*) - kappa^T K^-1 kappa (Sec. 2.1,
    Eq. eq:pred_distr) at 902 test points (15 blocks of 64 right-hand sides,
    the last ragged) against the oracle's dense solve with full-accuracy K,
    kappa and prior: within the first-order effect of stopping the block's CG
    at rtol, rtol |khat| |Khat^-1 khat| (times 4: the recursive residual the
    CG stops on is not the true one), plus the stored entries' rounding
    (relative 1e-12 FP64, 1e-5 FP32 of |khat|^T |Khat^-1 khat|) and 1e-12 of
    the prior variance (an FP64 sum of squared bump values, whose rounding
    near a bump's edge reaches ~1e-14 relative)."""
    p = CASES[case]()
    xs = query_points(p)
    gp = G.GP(p.dim, p.n1, p.n2, p.beta)
    gp.assemble(torch.as_tensor(p.x, device="cuda"), p.h, precision=prec)
    rtol = 1e-10 if prec == "fp64" else 1e-6
    var, info = gp.predict_var(torch.as_tensor(xs, device="cuda"), opts=G.default_opts(precision=prec, cg_rtol=rtol))
    v = var.cpu().numpy()
    kappa = _cross_K_hp(case, p, xs)
    prior = O.prior_var_hp(xs, p.h, p.dim, p.n1, p.n2, p.beta)
    Khp = O.dense_K_hp(p.x, p.h, p.dim, p.n1, p.n2, p.beta)
    ref = O.predict_var(p.x, p.h, xs, p.dim, p.n1, p.n2, p.beta, kappa=kappa, prior=prior, K=Khp)
    sens, absum = O.predict_var_sensitivity(p.x, p.h, xs, p.dim, p.n1, p.n2, p.beta, kappa=kappa)
    tol = 4.0 * rtol * sens + (1e-12 if prec == "fp64" else 1e-5) * absum + 1e-12 * prior
    worst = float(np.max(np.abs(v - ref) / np.where(tol > 0, tol, 1.0)))
    print(case, prec, "iters", info["iters"], "worst |var - ref| / tol", worst)
    assert np.all(np.abs(v - ref) <= tol)
    assert np.all(v[prior == 0.0] == 0.0)       # outside every bump
    gp.close()


def test_predict_var_without_active_training_points_is_the_prior(G):
    # no training point (N = 0): kappa = 0 and the variance is k(x*, x*)
    p = W.small_2d(seed=1, n=300)
    xs = query_points(p, n_new=100)
    gp = G.GP(p.dim, p.n1, p.n2, p.beta)
    gp.assemble(torch.zeros((0, p.dim), dtype=torch.float64, device="cuda"), p.h, precision="fp32")
    var, _ = gp.predict_var(xs)
    assert np.allclose(var, O.prior_var_hp(xs, p.h, p.dim, p.n1, p.n2, p.beta), rtol=1e-12, atol=0)
    assert np.any(var > 0)
    gp.close()
