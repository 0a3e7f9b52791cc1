"""GPU parity of the truncated-Taylor randomized log-determinant (the estimator
Sec. 2.5 cites; GP_FLAG_LOGDET_TAYLOR) through the C ABI against the oracle's
dense evaluation of the same estimator on the same probes, plus its edge
cases.  The solves, and so the quadratic form, are those of the SLQ path."""

import math

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


CASES = {
    "small_2d": lambda: W.small_2d(seed=1),
    "grad_3d": lambda: W.grad_3d(seed=3, n=3000),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("B", [0, 128])
def test_taylor_logdet_matches_same_probe_oracle(G, case, B):
    p = CASES[case]()
    nv, m, seed = 16, 30, 2024
    gp = G.GP(p.dim, p.n1, p.n2, p.beta)
    x = torch.as_tensor(p.x, device="cuda")
    y = torch.as_tensor(p.y, device="cuda")
    o = G.default_opts(precision="fp32", n_probes=nv, lanczos_steps=m, cg_rtol=1e-6, seed=seed, precond_block=B,
                       flags=G.GP_FLAG_LOGDET_TAYLOR)
    lml, info = gp.lml(x, y, p.h, o)
    ref, gam, a = O.logdet_taylor_same_probes(p.x, p.h, p.dim, p.n1, p.n2, nv, m, seed, p.beta)
    print(case, B, "logdet", info["logdet"], ref, "a", a, "stderr", info["logdet_stderr"])
    assert info["logdet"] == pytest.approx(ref, rel=1e-5)
    se = np.std(gam, ddof=1) / math.sqrt(nv)
    assert info["logdet_stderr"] == pytest.approx(se, rel=1e-2, abs=1e-6 * abs(ref))
    # the solves are the SLQ path's: same quadratic form
    o2 = G.default_opts(precision="fp32", n_probes=nv, lanczos_steps=m, cg_rtol=1e-6, seed=seed, precond_block=B)
    lml2, info2 = gp.lml(x, y, p.h, o2)
    assert info["quad_form"] == pytest.approx(info2["quad_form"], rel=1e-6)
    assert lml == pytest.approx(-0.5 * info["quad_form"] - 0.5 * info["logdet"], rel=1e-12)
    gp.close()


def test_taylor_logdet_gradient_and_edge_cases(G):
    p = W.small_2d(seed=1, n=400)
    gp = G.GP(p.dim, p.n1, p.n2, p.beta)
    x = torch.as_tensor(p.x, device="cuda")
    y = torch.as_tensor(p.y, device="cuda")
    flags = G.GP_FLAG_LOGDET_TAYLOR
    # the gradient's trace term does not depend on the log-determinant estimator
    o = G.default_opts(precision="fp32", n_probes=8, lanczos_steps=20, cg_rtol=1e-6, seed=9, flags=flags)
    o_slq = G.default_opts(precision="fp32", n_probes=8, lanczos_steps=20, cg_rtol=1e-6, seed=9)
    _, g_t, _ = gp.lml_grad(x, y, p.h, o)
    _, g_s, _ = gp.lml_grad(x, y, p.h, o_slq)
    assert np.allclose(g_t, g_s, rtol=1e-6, atol=1e-9 * np.abs(g_s).max())
    # FP64 path: not offered
    with pytest.raises(G.GPError) as e:
        gp.lml(x, y, p.h, G.default_opts(precision="fp64", n_probes=8, lanczos_steps=20, flags=flags))
    assert e.value.status == G.GP_ERR_UNSUPPORTED
    # every point outside every bump: exact noise model
    h = p.h.copy()
    per = p.dim + 2
    for b in range(p.n1 * p.n2):
        h[b * per: b * per + p.dim] = 50.0
    lml, info = gp.lml(x, y, h, o)
    s2 = h[-1]
    assert info["n_active"] == 0
    assert info["logdet"] == pytest.approx(p.n * math.log(s2), rel=1e-12)
    gp.close()
