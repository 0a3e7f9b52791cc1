"""GPU parity of the core-kernel product k_c * k_s (Sec. 2.2: kernels can be
multiplied, so the sparsity-discovering kernel k_s multiplies a core kernel,
here the squared exponential exp(-|x1 - x2|^2 / (2 l^2)) with the length scale
l one more hyperparameter) through the C ABI against the oracle: every stored
entry against the full-accuracy evaluation, LML and gradient (including
d/dl) against the same-probe estimator, the posterior mean's sums against
the oracle's cross-covariance, and the argument checks."""

import ctypes

import numpy as np
import pytest

from oracle import gp_oracle as O
from paper_2205_09070_gb300 import workloads as W

from helpers import canonical_gpu_csr, canonical_oracle_csr, grad_ok, value_tol_ok

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

RTOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module")
def G():
    import __graft_entry__ as g
    g.build()
    from paper_2205_09070_gb300 import gpsparse
    assert torch.cuda.is_available()
    return gpsparse


def with_core(p, ell):
    """The workload's hyperparameters with the core length scale appended."""
    return np.append(p.h, ell)


CASES = {
    # l below r_s so the core shapes every entry: k_c at the support edge is
    # exp(-0.05^2 / (2 0.03^2)) = 0.25 (2-D) and exp(-0.09^2 / (2 0.05^2)) = 0.2 (3-D)
    "small_2d": (lambda: W.small_2d(seed=1), 0.03),
    "grad_3d": (lambda: W.grad_3d(seed=3, n=3000), 0.05),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_core_assembly_pattern_and_every_value(G, case, prec):
    make, ell = CASES[case]
    p = make()
    h = with_core(p, ell)
    gp = G.GP(p.dim, p.n1, p.n2, p.beta, core=G.GP_CORE_SQEXP)
    assert gp.n_params == len(p.h) + 1
    info = gp.assemble(torch.as_tensor(p.x, device="cuda"), h, precision=prec)
    r, c, v = canonical_gpu_csr(gp.get_csr())
    ro, co, vo, mask = canonical_oracle_csr(p.x, h, p.dim, p.n1, p.n2, p.beta, key=("core", case))
    assert info["nnz"] == len(ro)
    assert np.array_equal(r, ro) and np.array_equal(c, co)   # the core does not change the pattern
    diag = np.zeros(p.n)
    dm = ro == co
    diag[ro[dm]] = vo[dm]
    ok, worst = value_tol_ok(v, vo, diag, ro, co, RTOL[prec], prec)
    print(case, prec, "nnz", len(ro), "worst relative error", worst)
    assert ok, worst
    gp.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_core_lml_and_gradient_same_probes(G, prec):
    p = W.small_2d(seed=1)
    h = with_core(p, 0.03)
    nv, m, seed = 16, 40, 1234
    rtol = 1e-10 if prec == "fp64" else 1e-6
    gp = G.GP(p.dim, p.n1, p.n2, p.beta, core=G.GP_CORE_SQEXP)
    opts = G.default_opts(precision=prec, n_probes=nv, lanczos_steps=m, cg_rtol=rtol, seed=seed)
    lml, grad, info = gp.lml_grad(torch.as_tensor(p.x, device="cuda"), torch.as_tensor(p.y, device="cuda"), h, opts)
    ref, gref, rinfo = O.lml_grad_same_probes(p.x, p.y, h, p.dim, p.n1, p.n2, nv, m, seed, with_bounds=True)
    assert len(grad) == len(h)
    assert info["quad_form"] == pytest.approx(rinfo["quad_form"], rel=1e-9 if prec == "fp64" else 1e-5)
    assert info["logdet"] == pytest.approx(rinfo["logdet"], rel=1e-7 if prec == "fp64" else 1e-5)
    ok, worst = grad_ok(grad, gref, rinfo, rtol, 2.0)
    print(prec, "core grad |dg| / (rtol (sens_quad + sens_trace / 2))", worst, "d/dl", grad[-1], gref[-1])
    assert ok, worst
    assert gref[-1] != 0.0
    gp.close()


def test_core_posterior_mean_kernel_sums(G):
    p = W.grad_3d(seed=3, n=3000)
    h = with_core(p, 0.05)
    rng = np.random.default_rng(5)
    xs = np.ascontiguousarray(np.vstack([rng.uniform(0, 1, (300, p.dim)), p.x[:100]]))
    gp = G.GP(p.dim, p.n1, p.n2, p.beta, core=G.GP_CORE_SQEXP)
    x, y = torch.as_tensor(p.x, device="cuda"), torch.as_tensor(p.y, device="cuda")
    gp.assemble(x, h, precision="fp64")
    o = G.default_opts(precision="fp64", cg_rtol=1e-10)
    mean, _ = gp.predict(y, torch.as_tensor(xs, device="cuda"), opts=o)
    alpha, _ = gp.solve(y, torch.zeros_like(y), o)
    kappa = O.cross_K_hp(xs, p.x, h, p.dim, p.n1, p.n2, p.beta)
    a = alpha.cpu().numpy()
    m = mean.cpu().numpy()
    assert np.all(np.abs(m - kappa @ a) <= 1e-11 * (np.abs(kappa) @ np.abs(a)))
    gp.close()


def test_core_argument_checks(G):
    p = W.small_2d(seed=1, n=200)
    lib = G.load()
    bad = G.KernelDesc(p.dim, p.n1, p.n2, p.beta, 7)
    h = ctypes.c_void_p()
    assert lib.gp_create(ctypes.byref(h), ctypes.byref(bad), 0, None) == G.GP_ERR_INVALID_ARG
    gp = G.GP(p.dim, p.n1, p.n2, p.beta, core=G.GP_CORE_SQEXP)
    for ell in (0.0, -1.0, np.inf, np.nan):
        with pytest.raises(G.GPError) as e:
            gp.assemble(torch.as_tensor(p.x, device="cuda"), with_core(p, ell))
        assert e.value.status == G.GP_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        gp.assemble(torch.as_tensor(p.x, device="cuda"), p.h)   # l missing
    gp.close()
