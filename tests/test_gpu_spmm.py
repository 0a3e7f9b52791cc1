"""GPU parity of the four forms of the FP32 sparse product Q = Khat P (per-lane
cp.async stage, TMA gather4 stage, and either stage with several float4
columns per lane) and of the autotuner that picks one.  Each form is forced through
gp_opts.flags and checked through the C ABI against the oracle's dense
evaluation of the same estimator (same probes, Sec. 2.5 solves), over column
counts kp = 4 .. 68 that select every lane layout; on a clustered matrix the
forms are checked against each other and against the plain FP64 path."""

import numpy as np
import pytest

from oracle import gp_oracle as O
from paper_2205_09070_gb300 import workloads as W

from helpers import grad_ok

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FORMS = ["cpasync", "tma", "tma_wide", "cpasync_wide", "window"]


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2205_09070_gb300 import gpsparse as G
    assert torch.cuda.is_available()
    return G


def wide_lw(kq):
    # float4 columns per lane of the wide form (1: the wide form is the plain TMA form)
    return 3 if kq % 3 == 0 and kq >= 6 else 2 if kq % 2 == 0 and kq >= 4 else 1


def expected_variant(G, form, kp):
    if form == "window":
        return G.GP_SPMM_WINDOW
    wide = wide_lw(kp // 4) > 1
    if form == "cpasync" or (form == "cpasync_wide" and not wide):
        return G.GP_SPMM_CPASYNC
    if form == "cpasync_wide":
        return G.GP_SPMM_CPASYNC_WIDE
    if form == "tma" or not wide:
        return G.GP_SPMM_TMA
    return G.GP_SPMM_TMA_WIDE


_ORACLE = {}


def oracle_pieces(p, key, nv, m, seed):
    if (key, nv) not in _ORACLE:
        _ORACLE[(key, nv)] = O.lml_grad_same_probes(p.x, p.y, p.h, p.dim, p.n1, p.n2, nv, m, seed,
                                                    with_grad=False)[2]
    return _ORACLE[(key, nv)]


# kp = 4, 16, 36, 48, 68: float4 columns KQ = 1, 4, 9, 12, 17; wide lanes hold 1, 2, 3, 3, 1
@pytest.mark.parametrize("nv", [3, 12, 35, 47, 64])
@pytest.mark.parametrize("form", FORMS)
def test_form_matches_same_probe_estimator(lib, form, nv):
    p = W.grad_3d(seed=3, n=3000)
    m, seed = 30, 77
    gp = lib.GP(p.dim, p.n1, p.n2, p.beta)
    x = torch.as_tensor(p.x, device="cuda")
    y = torch.as_tensor(p.y, device="cuda")
    opts = lib.default_opts(precision="fp32", n_probes=nv, lanczos_steps=m, cg_rtol=1e-6, seed=seed,
                            precond_block=32, flags=lib.SPMM_FLAGS[form])
    lml, info = gp.lml(x, y, p.h, opts)
    ref = oracle_pieces(p, "grad_3d", nv, m, seed)
    kp = (nv + 1 + 3) // 4 * 4
    assert info["kp"] == kp
    assert info["spmm_variant"] == expected_variant(lib, form, kp)
    print(form, nv, "quad", info["quad_form"], ref["quad_form"], "logdet", info["logdet"], ref["logdet"],
          "iters", info["iters"])
    assert info["quad_form"] == pytest.approx(ref["quad_form"], rel=1e-5)
    assert info["logdet"] == pytest.approx(ref["logdet"], rel=1e-5)
    gp.close()


@pytest.mark.parametrize("form", FORMS)
def test_form_gradient_matches_same_probe_estimator(lib, form):
    p = W.small_2d(seed=1)
    nv, m, seed = 35, 40, 1234  # kp = 36: the wide form holds three float4 per lane
    gp = lib.GP(p.dim, p.n1, p.n2, p.beta)
    x = torch.as_tensor(p.x, device="cuda")
    y = torch.as_tensor(p.y, device="cuda")
    opts = lib.default_opts(precision="fp32", n_probes=nv, lanczos_steps=m, cg_rtol=1e-6, seed=seed,
                            flags=lib.SPMM_FLAGS[form])
    lml, grad, info = gp.lml_grad(x, y, p.h, opts)
    ref, gref, rinfo = O.lml_grad_same_probes(p.x, p.y, p.h, p.dim, p.n1, p.n2, nv, m, seed,
                                              with_bounds=True)
    assert info["spmm_variant"] == expected_variant(lib, form, 36)
    assert info["quad_form"] == pytest.approx(rinfo["quad_form"], rel=1e-5)
    assert info["logdet"] == pytest.approx(rinfo["logdet"], rel=1e-5)
    ok, worst = grad_ok(grad, gref, rinfo, 1e-6, 2.0)  # first-order solver bound at rtol 1e-6
    print("grad |dg| / (rtol (sens_quad + sens_trace / 2))", worst)
    assert ok, worst
    gp.close()


@pytest.mark.parametrize("form", FORMS)
def test_form_solve_matches_dense(lib, form):
    # gp_solve runs one column (kp = 4): every lane of the wide form holds one float4
    p = W.small_2d(seed=1)
    gp = lib.GP(p.dim, p.n1, p.n2, p.beta)
    x = torch.as_tensor(p.x, device="cuda")
    y = torch.as_tensor(p.y, device="cuda")
    gp.assemble(x, p.h, precision="fp32")
    alpha, info = gp.solve(y, torch.zeros_like(y), lib.default_opts(precision="fp32", cg_rtol=1e-6,
                                                                     flags=lib.SPMM_FLAGS[form]))
    assert info["spmm_variant"] == expected_variant(lib, form, 4)
    ref = np.linalg.solve(O.dense_K(p.x, p.h, p.dim, p.n1, p.n2), p.y)
    err = np.linalg.norm(alpha.cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err < 2e-3, err
    gp.close()


def clustered(n=60_000, seed=21):
    # the clustered 3-D mixture: dense cluster cores with hundreds of blocks
    # per block row next to sparse background rows
    return W.mixture_3d(seed=seed, n=n, r_s=0.005 * (5e6 / n) ** (1.0 / 3.0))


def test_forms_agree_on_clustered_matrix_and_with_fp64_path(lib):
    p = clustered()
    nv, m, seed = 32, 30, 99
    gp = lib.GP(p.dim, p.n1, p.n2, p.beta)
    x = torch.as_tensor(p.x, device="cuda")
    y = torch.as_tensor(p.y, device="cuda")
    res = {}
    for form in FORMS:
        o = lib.default_opts(precision="fp32", n_probes=nv, lanczos_steps=m, cg_rtol=1e-6, seed=seed,
                             flags=lib.SPMM_FLAGS[form])
        res[form] = gp.lml_grad(x, y, p.h, o)
        assert res[form][2]["spmm_variant"] == expected_variant(lib, form, 36)
    o64 = lib.default_opts(precision="fp64", n_probes=nv, lanczos_steps=m, cg_rtol=1e-6, seed=seed)
    l64, g64, i64 = gp.lml_grad(x, y, p.h, o64)
    print("n_active", i64["n_active"], "nnz", i64["nnz"])
    assert i64["n_active"] > 5000  # thousands of block rows, dense and sparse
    scale = np.abs(g64) + 1e-3 * np.abs(g64).max()
    for form, (l, g, info) in res.items():
        print(form, "quad", info["quad_form"], i64["quad_form"], "logdet", info["logdet"], i64["logdet"])
        assert info["quad_form"] == pytest.approx(i64["quad_form"], rel=1e-5)
        assert info["logdet"] == pytest.approx(i64["logdet"], rel=1e-5)
        assert np.max(np.abs(g - g64) / scale) < 2e-3
    gp.close()


def test_autotuner_choice_is_stable_and_shared(lib):
    p = clustered(n=40_000, seed=23)
    o = lib.default_opts(precision="fp32", n_probes=16, lanczos_steps=20, cg_rtol=1e-6, seed=5)
    x = torch.as_tensor(p.x, device="cuda")
    y = torch.as_tensor(p.y, device="cuda")
    a = lib.GP(p.dim, p.n1, p.n2, p.beta)
    l1, g1, i1 = a.lml_grad(x, y, p.h, o)
    l2, g2, i2 = a.lml_grad(x, y, p.h, o)
    b = lib.GP(p.dim, p.n1, p.n2, p.beta)
    l3, g3, i3 = b.lml_grad(x, y, p.h, o)
    assert i1["spmm_variant"] in (lib.GP_SPMM_CPASYNC, lib.GP_SPMM_TMA, lib.GP_SPMM_TMA_WIDE,
                                  lib.GP_SPMM_CPASYNC_WIDE, lib.GP_SPMM_WINDOW)
    assert i1["spmm_variant"] == i2["spmm_variant"] == i3["spmm_variant"]
    assert l1 == l2 == l3
    assert np.array_equal(g1, g2) and np.array_equal(g1, g3)
    a.close()
    b.close()
