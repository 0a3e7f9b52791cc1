"""GPU parity on the named workloads: the 163-hyperparameter gradient case,
the 20,000-point subset of the 200,000-point precision case, and sampled rows
of the full 1,000,000-point measurement workload in the launch configuration
bench.py times (FP32_MIXED, 32 probes, 50 Lanczos steps, rtol 1e-6)."""

import numpy as np
import pytest

from oracle import gp_oracle as O
from paper_2205_09070_gb300 import workloads as W

from helpers import grad_ok, grad_solver_bound

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import __graft_entry__ as g
    g.build()
    from paper_2205_09070_gb300 import gpsparse
    return gpsparse


def dev(a):
    return torch.as_tensor(a, device="cuda")


def test_gradient_163_parameters(G):
    """163 hyperparameters (4 x 8 bumps in 3-D), N = 5,000: GPU gradient vs the
    oracle's same-probe estimator (tight) and its exact gradient (within the
    Hutchinson estimator's spread)."""
    p = W.grad_3d(seed=3, n=5000)
    assert len(p.h) == 163
    nv, m, seed = 16, 40, 77
    gp = G.GP(p.dim, p.n1, p.n2)
    res = {}
    for prec, rtol in (("fp64", 1e-10), ("fp32", 1e-6)):
        o = G.default_opts(precision=prec, n_probes=nv, lanczos_steps=m, cg_rtol=rtol, seed=seed, precond_block=0)
        res[prec] = gp.lml_grad(dev(p.x), dev(p.y), p.h, o)
    ref, gref, rinfo = O.lml_grad_same_probes(p.x, p.y, p.h, p.dim, p.n1, p.n2, nv, m, seed, with_bounds=True)
    for prec, rtol, safety in (("fp64", 1e-10, 2.0), ("fp32", 1e-6, 2.0)):
        lml, g, info = res[prec]
        assert info["quad_form"] == pytest.approx(rinfo["quad_form"], rel=1e-8 if prec == "fp64" else 1e-5)
        assert info["logdet"] == pytest.approx(rinfo["logdet"], rel=1e-7 if prec == "fp64" else 1e-5)
        # every component within the first-order solver bound (helpers.grad_solver_bound)
        ok, worst = grad_ok(g, gref, rinfo, rtol, safety)
        print(prec, "grad |dg| / (rtol (sens_quad + sens_trace / 2))", worst)
        assert ok, (prec, worst)
    # exact gradient: the quadratic part is shared, the trace part is a
    # 16-probe Hutchinson estimate whose trace enters with weight 1/2: every
    # component within 6 of its standard errors (plus the solver bound)
    _, gx = O.lml_grad_exact(p.x, p.y, p.h, p.dim, p.n1, p.n2)
    g = res["fp64"][1]
    tol = 6.0 * 0.5 * rinfo["grad_trace_se"] + grad_solver_bound(rinfo, 1e-10, 2.0)
    z = np.abs(g - gx) / np.where(tol > 0, tol, 1.0)
    print("exact gradient: worst |g - g_exact| / (6 SE / 2 + solver bound)", float(z.max()))
    assert np.all((np.abs(g - gx) <= tol) | ((tol == 0) & (np.abs(g - gx) <= 1e-12 * np.abs(gx).max())))
    gp.close()


def test_precision_subset_20k(G):
    """The first 20,000 points of the 200,000-point uniform 3-D workload (4 x 8
    bumps, radii U(0.02, 0.05), r_s = 0.02): pattern, nnz, LML of both
    precisions against the oracle's same-probe estimator."""
    full = W.uniform_3d(seed=2, n=200_000)
    n = 20_000
    x, y = full.x[:n], full.y[:n]
    nv, m, seed = 32, 32, 5
    gp = G.GP(full.dim, full.n1, full.n2)
    ref, _, rinfo = O.lml_grad_same_probes(x, y, full.h, full.dim, full.n1, full.n2, nv, m, seed,
                                           with_grad=False)
    rp, col, _ = O.assemble_csr(x, full.h, full.dim, full.n1, full.n2)
    _, mask = O.bump_table(x, full.h, full.dim, full.n1, full.n2)
    nnz_active = int(np.sum(np.diff(rp)[mask != 0]))
    for prec, tol in (("fp64", 1e-9), ("fp32", 1e-6)):
        o = G.default_opts(precision=prec, n_probes=nv, lanczos_steps=m,
                           cg_rtol=1e-10 if prec == "fp64" else 1e-6, seed=seed)
        lml, info = gp.lml(dev(x), dev(y), full.h, o)
        assert info["n_active"] == int(np.sum(mask != 0))
        assert info["nnz"] == nnz_active
        assert lml == pytest.approx(ref, rel=tol), prec
    gp.close()


def test_bench_workload_sampled_rows(G):
    """The full 1,000,000-point mixture in the bench configuration: sampled
    rows of K against brute force over all N points (pattern bit-exact,
    values within the FP32 tolerance), and identities that hold at any size."""
    p = W.mixture_1m()
    gp = G.GP(p.dim, p.n1, p.n2)
    o = G.default_opts(precision="fp32", n_probes=32, lanczos_steps=50, cg_rtol=1e-6, seed=2022, max_iter=20000)
    x, y = dev(p.x), dev(p.y)
    lml, g, info = gp.lml_grad(x, y, p.h, o)
    csr = gp.get_csr()
    table = O.bump_table(p.x, p.h, p.dim, p.n1, p.n2)
    P = O.unpack_h(p.h, p.dim, p.n1, p.n2)
    assert info["n_active"] == int(np.sum(table[1] != 0))
    rng = np.random.default_rng(0)
    rows = np.sort(rng.choice(len(csr.perm), 48, replace=False))
    # rows with the most entries (cluster cores) as well
    heavy = np.argsort(np.diff(csr.row_ptr))[-16:]
    for r in np.concatenate([rows, heavy]):
        i = int(csr.perm[r])
        cols = csr.perm[csr.col[csr.row_ptr[r]:csr.row_ptr[r + 1]]].astype(np.int64)
        vals = csr.val[csr.row_ptr[r]:csr.row_ptr[r + 1]]
        order = np.argsort(cols)
        pat, v = O.pair_rows(p.x, p.h, p.dim, p.n1, p.n2, [i], table=table)
        ref_cols = np.nonzero(pat[0])[0]
        assert np.array_equal(cols[order], ref_cols), r
        # values: every entry of the row within 1e-5 relative of the oracle's
        # full-accuracy value (floor: one FP32 denormal step of Khat)
        ref_v = O.entries_hp(p.x, p.h, p.dim, p.n1, p.n2, np.full(len(ref_cols), i), ref_cols)
        kdiag = O.entries_hp(p.x, p.h, p.dim, p.n1, p.n2, ref_cols, ref_cols)
        kii = kdiag[ref_cols == i][0]
        err = np.abs(vals[order] - ref_v)
        floor = 2.0 ** -149 * np.sqrt(kii * kdiag)
        assert np.all(err <= 1e-5 * np.abs(ref_v) + floor), (r, float(np.max(err / np.abs(ref_v))))
    # Euler identities of the estimator (exact for any probes, see the oracle pins)
    assert P["A"] * g[-2] + P["sigma2"] * g[-1] == pytest.approx(0.5 * info["quad_form"] - 0.5 * p.n, rel=1e-4)
    amp = [b * (p.dim + 2) + p.dim + 1 for b in range(p.n1 * p.n2)]
    assert sum(p.h[i] * g[i] for i in amp) == pytest.approx(2 * P["A"] * g[-2], rel=1e-3, abs=1e-6 * abs(g).max())
    # the solve on the same assembly: residual of sampled rows with the oracle's rows
    alpha, sinfo = gp.solve(y, torch.zeros_like(y), G.default_opts(precision="fp32", cg_rtol=1e-6, max_iter=20000))
    a = alpha.cpu().numpy()
    num = den = 0.0
    for r in rows:
        i = int(csr.perm[r])
        _, v = O.pair_rows(p.x, p.h, p.dim, p.n1, p.n2, [i], table=table)
        num += (float(v[0] @ a) - p.y[i]) ** 2
        den += p.y[i] ** 2
    assert np.sqrt(num / den) < 1e-3
    gp.close()


def test_5m_workload_sampled_rows(G):
    """The literal 5,000,000-point configuration (mixture, r_s = 0.005, 8 x 16
    bumps) in the bench's FP32 launch configuration: sampled rows of K against
    brute force over all N points (pattern bit-exact, every value within
    1e-5 of the full-accuracy oracle) and the Euler identities of the
    gradient estimator at that size."""
    p = W.mixture_3d(seed=5, n=5_000_000)
    gp = G.GP(p.dim, p.n1, p.n2)
    o = G.default_opts(precision="fp32", n_probes=32, lanczos_steps=50, cg_rtol=1e-6, seed=2022, max_iter=20000)
    lml, g, info = gp.lml_grad(dev(p.x), dev(p.y), p.h, o)
    assert np.isfinite(lml) and np.all(np.isfinite(g))
    csr = gp.get_csr()
    table = O.bump_table(p.x, p.h, p.dim, p.n1, p.n2)
    assert info["n_active"] == int(np.sum(table[1] != 0))
    rng = np.random.default_rng(1)
    rows = np.sort(rng.choice(len(csr.perm), 24, replace=False))
    heavy = np.argsort(np.diff(csr.row_ptr))[-8:]
    for r in np.concatenate([rows, heavy]):
        i = int(csr.perm[r])
        cols = csr.perm[csr.col[csr.row_ptr[r]:csr.row_ptr[r + 1]]].astype(np.int64)
        vals = csr.val[csr.row_ptr[r]:csr.row_ptr[r + 1]]
        order = np.argsort(cols)
        pat, _ = O.pair_rows(p.x, p.h, p.dim, p.n1, p.n2, [i], table=table)
        ref_cols = np.nonzero(pat[0])[0]
        assert np.array_equal(cols[order], ref_cols), r
        ref_v = O.entries_hp(p.x, p.h, p.dim, p.n1, p.n2, np.full(len(ref_cols), i), ref_cols)
        kdiag = O.entries_hp(p.x, p.h, p.dim, p.n1, p.n2, ref_cols, ref_cols)
        kii = kdiag[ref_cols == i][0]
        err = np.abs(vals[order] - ref_v)
        assert np.all(err <= 1e-5 * np.abs(ref_v) + 2.0 ** -149 * np.sqrt(kii * kdiag)), r
    P = O.unpack_h(p.h, p.dim, p.n1, p.n2)
    assert P["A"] * g[-2] + P["sigma2"] * g[-1] == pytest.approx(0.5 * info["quad_form"] - 0.5 * p.n, rel=1e-4)
    amp = [b * (p.dim + 2) + p.dim + 1 for b in range(p.n1 * p.n2)]
    assert sum(p.h[i] * g[i] for i in amp) == pytest.approx(2 * P["A"] * g[-2], rel=1e-3, abs=1e-6 * abs(g).max())
    gp.close()
