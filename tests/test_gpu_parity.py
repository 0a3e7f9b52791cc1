"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle on
the same seeded inputs (sizes the oracle finishes in seconds, spanning many
cells, warps and blocks with ragged tails)."""

import math

import numpy as np
import pytest

from oracle import gp_oracle as O
from paper_2205_09070_gb300 import workloads as W

from helpers import canonical_gpu_csr, canonical_oracle_csr, grad_ok, value_tol_ok

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# relative tolerance of every stored entry against the oracle's full-accuracy
# value (helpers.value_tol_ok): the FP32 bound is the one the method's FP32
# path is held to; FP64 leaves three decades over its rounding (~1e-15)
RTOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2205_09070_gb300 import gpsparse as G
    assert torch.cuda.is_available()
    return G


def mixture_small(n=8000, seed=15):
    # the clustered 3-D mixture at a size the brute-force oracle handles; the
    # stationary radius grows as N^(-1/3) so neighbours per row stay alike
    return W.mixture_3d(seed=seed, n=n, r_s=0.005 * (5e6 / n) ** (1.0 / 3.0))


CASES = {
    "small_2d": lambda: W.small_2d(seed=1),
    "grad_3d": lambda: W.grad_3d(seed=3, n=3000),
    "mixture": lambda: mixture_small(),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_assembly_pattern_bit_exact_and_values(lib, case, prec):
    p = CASES[case]()
    gp = lib.GP(p.dim, p.n1, p.n2, p.beta)
    x = torch.as_tensor(p.x, device="cuda")
    info = gp.assemble(x, p.h, precision=prec)
    csr = gp.get_csr()
    r, c, v = canonical_gpu_csr(csr)
    ro, co, vo, mask = canonical_oracle_csr(p.x, p.h, p.dim, p.n1, p.n2, p.beta, key=case)
    assert info["n_active"] == int(np.sum(mask != 0))
    assert info["nnz"] == len(ro)
    assert np.array_equal(r, ro) and np.array_equal(c, co)          # bit-exact pattern
    # each internal row's columns are ascending
    for q in range(len(csr.perm)):
        seg = csr.col[csr.row_ptr[q]:csr.row_ptr[q + 1]]
        assert np.all(np.diff(seg) > 0)
    diag = np.zeros(p.n)
    dm = ro == co
    diag[ro[dm]] = vo[dm]
    ok, worst = value_tol_ok(v, vo, diag, ro, co, RTOL[prec], prec)
    print(case, prec, "nnz", len(ro), "worst relative error", worst)
    assert ok, worst
    gp.close()


@pytest.mark.parametrize("prec,B", [("fp64", 0), ("fp32", 0), ("fp32", 8), ("fp32", 16), ("fp32", 32), ("fp32", 64),
                                    ("fp32", 128)])
def test_solve_matches_dense(lib, prec, B):
    p = W.small_2d(seed=1)
    gp = lib.GP(p.dim, p.n1, p.n2, p.beta)
    x = torch.as_tensor(p.x, device="cuda")
    y = torch.as_tensor(p.y, device="cuda")
    gp.assemble(x, p.h, precision=prec)
    rtol = 1e-10 if prec == "fp64" else 1e-6
    alpha, info = gp.solve(y, torch.zeros_like(y), lib.default_opts(precision=prec, cg_rtol=rtol, precond_block=B))
    assert info["precond_block"] == (B if prec == "fp32" else 0)
    print(prec, B, "iters", info["iters"], "max_rel", info["max_rel_resid"])
    K = O.dense_K(p.x, p.h, p.dim, p.n1, p.n2)
    ref = np.linalg.solve(K, p.y)
    a = alpha.cpu().numpy()
    # relative error in the K-norm is bounded by sqrt(cond(Khat)) * rtol
    err = np.linalg.norm(a - ref) / np.linalg.norm(ref)
    assert err < (1e-7 if prec == "fp64" else 2e-3), err
    gp.close()


@pytest.mark.parametrize("prec,B", [("fp64", 0), ("fp32", 0), ("fp32", 8), ("fp32", 16), ("fp32", 32), ("fp32", 64),
                                    ("fp32", 128)])
def test_lml_and_grad_same_probes(lib, prec, B):
    """Same probes: the GPU's SLQ log-determinant and Hutchinson gradient
    against the oracle's dense evaluation of the same estimator.  The
    estimator does not depend on the solver: B = 0 runs one plain CG, B > 0 a
    short Lanczos run for SLQ plus block-Jacobi preconditioned CG."""
    p = W.small_2d(seed=1)
    nv, m, seed = 16, 40, 1234
    gp = lib.GP(p.dim, p.n1, p.n2, p.beta)
    x = torch.as_tensor(p.x, device="cuda")
    y = torch.as_tensor(p.y, device="cuda")
    rtol = 1e-10 if prec == "fp64" else 1e-6
    opts = lib.default_opts(precision=prec, n_probes=nv, lanczos_steps=m, cg_rtol=rtol, seed=seed,
                            precond_block=B)
    lml, grad, info = gp.lml_grad(x, y, p.h, opts)
    ref, gref, rinfo = same_probe_reference(p, nv, m, seed)
    print(prec, B, "lml", lml, ref, "logdet", info["logdet"], rinfo["logdet"], "quad", info["quad_form"],
          rinfo["quad_form"], "iters", info["iters"])
    assert info["quad_form"] == pytest.approx(rinfo["quad_form"], rel=1e-9 if prec == "fp64" else 1e-5)
    assert info["logdet"] == pytest.approx(rinfo["logdet"], rel=1e-7 if prec == "fp64" else 1e-5)
    # every component within the first-order effect of stopping the solves at
    # rtol (helpers.grad_solver_bound)
    ok, worst = grad_ok(grad, gref, rinfo, rtol, GRAD_SAFETY[prec])
    print(prec, B, "grad |dg| / (rtol (sens_quad + sens_trace / 2))", worst)
    assert ok, worst
    gp.close()


# safety factor over the first-order solver bound (helpers.grad_solver_bound):
# the bound itself held with ratios <= 0.15 on GB300 for every block size and
# both precisions; 2 leaves room for the rounding the first-order model omits
GRAD_SAFETY = {"fp64": 2.0, "fp32": 2.0}
_REF = {}


def same_probe_reference(p, nv, m, seed):
    key = (p.name, p.n, nv, m, seed)
    if key not in _REF:
        _REF[key] = O.lml_grad_same_probes(p.x, p.y, p.h, p.dim, p.n1, p.n2, nv, m, seed, with_bounds=True)
    return _REF[key]


def test_gradient_identities_hold_on_gpu(lib):
    # the estimator is linear in dK/dtheta with one weight matrix W, so the
    # Euler identities of K = A k~ o FF^T + s2 I hold exactly for any probes:
    #   A g_A + s2 g_s2 = 1/2 y^T alpha - N/2,  sum_b a_b g_ab = 2 A g_A
    p = W.grad_3d(seed=3, n=3000)
    gp = lib.GP(p.dim, p.n1, p.n2, p.beta)
    x = torch.as_tensor(p.x, device="cuda")
    y = torch.as_tensor(p.y, device="cuda")
    opts = lib.default_opts(precision="fp32", n_probes=16, lanczos_steps=32, cg_rtol=1e-6, seed=5)
    lml, g, info = gp.lml_grad(x, y, p.h, opts)
    P = O.unpack_h(p.h, p.dim, p.n1, p.n2)
    lhs = P["A"] * g[-2] + P["sigma2"] * g[-1]
    assert lhs == pytest.approx(0.5 * info["quad_form"] - 0.5 * p.n, rel=1e-4)
    amp = [(b * (p.dim + 2)) + p.dim + 1 for b in range(p.n1 * p.n2)]
    assert sum(p.h[i] * g[i] for i in amp) == pytest.approx(2 * P["A"] * g[-2], rel=1e-4, abs=1e-6 * abs(g).max())
    gp.close()


def test_preconditioning_cuts_iterations_not_the_estimate(lib):
    """Block-Jacobi PCG changes the solver only: the estimate moves by no more
    than the solver tolerance allows, the SLQ terms come from the same
    lanczos_steps Lanczos iterations, and the solve needs fewer iterations."""
    p = W.grad_3d(seed=3, n=4000)
    gp = lib.GP(p.dim, p.n1, p.n2, p.beta)
    x = torch.as_tensor(p.x, device="cuda")
    y = torch.as_tensor(p.y, device="cuda")
    res = {}
    for B in (0, 8, 16, 32, 64, 128):
        o = lib.default_opts(precision="fp32", n_probes=16, lanczos_steps=30, cg_rtol=1e-6, seed=17,
                             precond_block=B)
        res[B] = gp.lml_grad(x, y, p.h, o)
    l0, g0, i0 = res[0]
    assert i0["lanczos_iters"] == 0 and i0["precond_block"] == 0
    scale = np.abs(g0) + 1e-3 * np.abs(g0).max()
    for B in (8, 16, 32, 64, 128):
        l, g, info = res[B]
        print(B, "iters", info["iters"], "vs", i0["iters"], "lanczos", info["lanczos_iters"])
        assert info["precond_block"] == B
        assert info["lanczos_iters"] == min(30, i0["iters"])
        assert info["iters"] < i0["iters"]
        assert info["logdet"] == pytest.approx(i0["logdet"], rel=1e-5)
        assert info["quad_form"] == pytest.approx(i0["quad_form"], rel=1e-5)
        assert np.max(np.abs(g - g0) / scale) < 2e-3
    gp.close()
