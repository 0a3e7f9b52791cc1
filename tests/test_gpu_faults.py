"""Error paths through the C ABI, every failure made on the host (no device
fault, trap or hang): an allocation that fails as an out-of-memory would, a
matrix that is not positive definite, a non-finite CG scalar, non-finite
targets, the iteration cap.  After each, the same context evaluates normally
and gives bitwise what a fresh context gives."""

import numpy as np
import pytest

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


def run(G, gp, p, prec, flags=0, y=None, **kw):
    o = G.default_opts(precision=prec, n_probes=8, lanczos_steps=20, cg_rtol=1e-6 if prec == "fp32" else 1e-10,
                       seed=3, flags=flags, **kw)
    yy = torch.as_tensor(p.y if y is None else y, device="cuda")
    return gp.lml_grad(torch.as_tensor(p.x, device="cuda"), yy, p.h, o)


def expect_status(G, status, fn):
    with pytest.raises(G.GPError) as e:
        fn()
    assert e.value.status == status, G.status_string(e.value.status)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_injected_faults_report_and_leave_the_context_usable(G, prec):
    p = W.small_2d(seed=1, n=800)
    ref_gp = G.GP(p.dim, p.n1, p.n2, p.beta)
    lml_ref, g_ref, _ = run(G, ref_gp, p, prec)
    ref_gp.close()
    # a fresh context whose first allocations fail
    gp = G.GP(p.dim, p.n1, p.n2, p.beta)
    expect_status(G, G.GP_ERR_OOM, lambda: run(G, gp, p, prec, G.GP_FLAG_FAULT_OOM))
    lml, g, _ = run(G, gp, p, prec)
    assert lml == lml_ref and np.array_equal(g, g_ref)
    # the matrix negated: CG meets p^T K p < 0
    expect_status(G, G.GP_ERR_NOT_SPD, lambda: run(G, gp, p, prec, G.GP_FLAG_FAULT_NOT_SPD))
    lml, g, _ = run(G, gp, p, prec)
    assert lml == lml_ref and np.array_equal(g, g_ref)
    # a NaN in a stored entry: the CG scalars turn non-finite
    expect_status(G, G.GP_ERR_NOT_SPD, lambda: run(G, gp, p, prec, G.GP_FLAG_FAULT_NAN))
    lml, g, _ = run(G, gp, p, prec)
    assert lml == lml_ref and np.array_equal(g, g_ref)
    # non-finite targets are an argument error, not a NaN likelihood
    ybad = p.y.copy()
    ybad[int(np.argmax(np.abs(p.y)))] = np.nan
    expect_status(G, G.GP_ERR_INVALID_ARG, lambda: run(G, gp, p, prec, y=ybad))
    lml, g, _ = run(G, gp, p, prec)
    assert lml == lml_ref and np.array_equal(g, g_ref)
    # the iteration cap: status NOT_CONVERGED
    expect_status(G, G.GP_ERR_NOT_CONVERGED, lambda: run(G, gp, p, prec, max_iter=3))
    lml, g, _ = run(G, gp, p, prec)
    assert lml == lml_ref and np.array_equal(g, g_ref)
    gp.close()

