"""The torch.autograd.Function over gp_lml_grad: its forward value is the
library's ln L, its backward returns the adjoint kernels' gradient (times the
upstream gradient), which matches the oracle's same-probe gradient."""

import numpy as np
import pytest

from oracle import gp_oracle as O
from paper_2205_09070_gb300 import workloads as W

from helpers import grad_ok

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import __graft_entry__ as g
    g.build()
    from paper_2205_09070_gb300 import gpsparse
    assert torch.cuda.is_available()
    return gpsparse


def test_autograd_backward_is_the_adjoint_gradient(G):
    from paper_2205_09070_gb300.autograd import log_marginal_likelihood
    p = W.small_2d(seed=1)
    nv, m, seed = 16, 40, 1234
    gp = G.GP(p.dim, p.n1, p.n2, p.beta)
    x = torch.as_tensor(p.x, device="cuda")
    y = torch.as_tensor(p.y, device="cuda")
    o = G.default_opts(precision="fp32", n_probes=nv, lanczos_steps=m, cg_rtol=1e-6, seed=seed)
    h = torch.tensor(p.h, dtype=torch.float64, requires_grad=True)
    lml_t = log_marginal_likelihood(h, x, y, gp, o)
    (-2.0 * lml_t).backward()
    lml, grad, _ = gp.lml_grad(x, y, p.h, o)
    assert lml_t.item() == lml
    assert np.array_equal(h.grad.numpy(), -2.0 * grad)
    ref, gref, rinfo = O.lml_grad_same_probes(p.x, p.y, p.h, p.dim, p.n1, p.n2, nv, m, seed,
                                              with_bounds=True)
    ok, worst = grad_ok(grad, gref, rinfo, 1e-6, 2.0)  # first-order solver bound at rtol 1e-6
    print("grad |dg| / (rtol (sens_quad + sens_trace / 2))", worst)
    assert ok, worst
    gp.close()
