"""GPU edge cases and error paths through the C ABI: empty and single-point
inputs, all points outside every bump, host vs device pointers, invalid
arguments, the iteration cap, ragged batches."""

import ctypes
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


def opts(G, prec="fp32", **kw):
    base = dict(precision=prec, n_probes=8, lanczos_steps=20, cg_rtol=1e-8 if prec == "fp64" else 1e-6, seed=3)
    base.update(kw)
    return G.default_opts(**base)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_empty_input(G, prec):
    p = W.small_2d(seed=1, n=10)
    gp = G.GP(p.dim, p.n1, p.n2)
    x = torch.zeros((0, 2), dtype=torch.float64, device="cuda")
    y = torch.zeros(0, dtype=torch.float64, device="cuda")
    lml, grad, info = gp.lml_grad(x, y, p.h, opts(G, prec))
    assert lml == 0.0 and info["n"] == 0 and info["nnz"] == 0
    assert np.all(grad == 0.0)
    gp.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_single_point(G, prec):
    # N = 1 inside a bump: K = A C f^2 + s2, exact LML = -y^2/(2K) - ln(K)/2;
    # SLQ is exact for a 1x1 matrix (Khat = 1)
    c = np.array([[[0.5, 0.5]]])
    h = W.pack_h(c, np.array([[0.3]]), np.array([[1.7]]), 0.1, 1.3, 0.01)
    x = np.array([[0.52, 0.47]])
    y = np.array([0.8])
    K = O.dense_K(x, h, 2, 1, 1)[0, 0]
    expect = -0.5 * y[0] ** 2 / K - 0.5 * math.log(K)
    gp = G.GP(2, 1, 1)
    lml, grad, info = gp.lml_grad(torch.as_tensor(x, device="cuda"), torch.as_tensor(y, device="cuda"), h,
                                  opts(G, prec))
    assert info["n_active"] == 1 and info["nnz"] == 1
    assert lml == pytest.approx(expect, rel=1e-12 if prec == "fp64" else 1e-6)
    lx, gx = O.lml_grad_exact(x, y, h, 2, 1, 1)
    assert np.allclose(grad, gx, rtol=1e-8 if prec == "fp64" else 1e-4, atol=1e-10 * np.abs(gx).max())
    gp.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_all_points_inactive(G, prec):
    p = W.small_2d(seed=2, n=3000)
    P = O.unpack_h(p.h, p.dim, p.n1, p.n2)
    h = W.pack_h(np.full((p.n1, p.n2, 2), 7.0), P["radii"], P["amps"], P["r_s"], P["A"], P["sigma2"])
    gp = G.GP(p.dim, p.n1, p.n2)
    lml, grad, info = gp.lml_grad(torch.as_tensor(p.x, device="cuda"), torch.as_tensor(p.y, device="cuda"), h,
                                  opts(G, prec))
    s2 = P["sigma2"]
    expect = -0.5 * float(p.y @ p.y) / s2 - 0.5 * p.n * math.log(s2)
    assert info["n_active"] == 0 and info["nnz"] == 0
    assert lml == pytest.approx(expect, rel=1e-13)
    assert grad[-1] == pytest.approx(0.5 * float(p.y @ p.y) / s2 ** 2 - 0.5 * p.n / s2, rel=1e-12)
    assert np.all(grad[:-1] == 0.0)
    gp.close()


def test_host_and_device_pointers_agree(G):
    p = W.grad_3d(seed=3, n=2000)
    o = opts(G, "fp32")
    gp = G.GP(p.dim, p.n1, p.n2)
    l_dev, g_dev, _ = gp.lml_grad(torch.as_tensor(p.x, device="cuda"), torch.as_tensor(p.y, device="cuda"), p.h, o)
    l_host, g_host, _ = gp.lml_grad(p.x, p.y, p.h, o)                 # numpy (pageable host)
    gpin = torch.zeros(gp.n_params, dtype=torch.float64, device="cuda")
    l_pin, _, _ = gp.lml_grad(torch.as_tensor(p.x).pin_memory(), torch.as_tensor(p.y).pin_memory(), p.h, o,
                              grad=gpin)
    assert l_dev == l_host == l_pin                                    # deterministic reductions
    assert np.array_equal(g_dev, g_host)
    assert np.array_equal(gpin.cpu().numpy(), g_dev)
    gp.close()


def test_repeat_calls_bitwise_identical(G):
    p = W.mixture_3d(seed=9, n=30000, r_s=0.005 * (5e6 / 30000) ** (1 / 3))
    x = torch.as_tensor(p.x, device="cuda")
    y = torch.as_tensor(p.y, device="cuda")
    gp = G.GP(p.dim, p.n1, p.n2)
    o = opts(G, "fp32", n_probes=32, lanczos_steps=50)
    a = gp.lml_grad(x, y, p.h, o)
    b = gp.lml_grad(x, y, p.h, o)
    assert a[0] == b[0] and np.array_equal(a[1], b[1])
    gp.close()


def test_invalid_arguments_are_rejected(G):
    p = W.small_2d(seed=1, n=200)
    gp = G.GP(p.dim, p.n1, p.n2)
    x = torch.as_tensor(p.x, device="cuda")
    y = torch.as_tensor(p.y, device="cuda")
    bad = []
    h = p.h.copy(); h[0] = np.nan; bad.append(h)                        # non-finite centre
    h = p.h.copy(); h[2] = -0.1; bad.append(h)                          # negative bump radius
    h = p.h.copy(); h[-3] = 0.0; bad.append(h)                          # zero stationary radius
    h = p.h.copy(); h[-1] = 0.0; bad.append(h)                          # zero noise
    h = p.h.copy(); h[-2] = -1.0; bad.append(h)                         # negative amplitude A
    for hb in bad:
        with pytest.raises(G.GPError) as e:
            gp.lml(x, y, hb, opts(G))
        assert e.value.status == G.GP_ERR_INVALID_ARG
    for o in (opts(G, n_probes=0), opts(G, n_probes=65), opts(G, lanczos_steps=0), opts(G, max_iter=0),
              opts(G, cg_rtol=0.0), opts(G, precision=7), opts(G, precond_block=5), opts(G, precond_block=256),
              opts(G, batch_workers=-1), opts(G, batch_workers=17)):
        with pytest.raises(G.GPError) as e:
            gp.lml(x, y, p.h, o)
        assert e.value.status == G.GP_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        gp.lml(x, y, p.h[:-1], opts(G))                                 # checked by the binding
    gp.close()
    fresh = G.GP(p.dim, p.n1, p.n2)
    with pytest.raises(G.GPError) as e:
        fresh.get_csr()
    assert e.value.status == G.GP_ERR_NOT_ASSEMBLED
    with pytest.raises(G.GPError) as e:
        fresh.solve(y)
    assert e.value.status == G.GP_ERR_NOT_ASSEMBLED
    fresh.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_iteration_cap_reports_not_converged(G, prec):
    p = W.small_2d(seed=1)
    gp = G.GP(p.dim, p.n1, p.n2)
    x = torch.as_tensor(p.x, device="cuda")
    y = torch.as_tensor(p.y, device="cuda")
    with pytest.raises(G.GPError) as e:
        gp.lml_grad(x, y, p.h, opts(G, prec, max_iter=3, check_every=1))
    assert e.value.status == G.GP_ERR_NOT_CONVERGED
    lml, grad, info = gp.lml_grad(x, y, p.h, opts(G, prec, max_iter=3, check_every=1), allow_not_converged=True)
    assert info["iters"] == 3 and np.isfinite(lml) and np.all(np.isfinite(grad))
    gp.close()


def _batch(G, seeds=(4, 5), n_inst=6, n_range=(1, 4000)):
    probs = W.batch_2d(seed=seeds[0], n_inst=n_inst, n_range=n_range)
    probs[1] = W.batch_2d(seed=seeds[1], n_inst=1, n_range=(1, 1))[0]          # an instance with N = 1
    offsets = np.concatenate([[0], np.cumsum([q.n for q in probs])])
    x = torch.as_tensor(np.concatenate([q.x for q in probs]), device="cuda")
    y = torch.as_tensor(np.concatenate([q.y for q in probs]), device="cuda")
    h = np.stack([q.h for q in probs])
    return probs, offsets, x, y, h


def _singles(G, gp, probs, o):
    out = []
    for q in probs:
        out.append(gp.lml_grad(torch.as_tensor(q.x, device="cuda"), torch.as_tensor(q.y, device="cuda"), q.h, o))
    return out


@pytest.mark.parametrize("precond_block", [128, 64, 16, 0])
def test_grouped_batch_matches_single_calls(G, precond_block):
    """The grouped CG launches (the batched default for FP32): every
    instance's ln L and gradient bitwise equal to its own call with the wide
    cp.async product, for each form of the block-Jacobi apply (128-, 64- and
    16-row blocks) and without the preconditioner."""
    probs, offsets, x, y, h = _batch(G)
    gp = G.GP(2, 2, 4)
    o = opts(G, "fp32", precond_block=precond_block)
    lml_b, grad_b, info = gp.lml_grad_batched(offsets, x, y, h, o)
    one = opts(G, "fp32", precond_block=precond_block, flags=G.GP_FLAG_SPMM_CPASYNC_WIDE)
    singles = _singles(G, gp, probs, one)
    for k, (l1, g1, _) in enumerate(singles):
        assert lml_b[k] == l1, (k, probs[k].n)
        assert np.array_equal(grad_b[k], g1), (k, probs[k].n)
    assert info["iters"] == max(i["iters"] for _, _, i in singles)
    gp.close()


def test_grouped_batch_from_host_inputs(G):
    """Host arrays for x, y, lml and grad: each instance is staged in on its
    own worker stream before the grouped launches, with the device-input
    results bit for bit."""
    probs, offsets, x, y, h = _batch(G)
    gp = G.GP(2, 2, 4)
    o = opts(G, "fp32")
    lml_d, grad_d, _ = gp.lml_grad_batched(offsets, x, y, h, o)
    lml_h, grad_h, _ = gp.lml_grad_batched(offsets, x.cpu().numpy(), y.cpu().numpy(), h, o)
    assert np.array_equal(lml_d, lml_h) and np.array_equal(grad_d, grad_h)
    gp.close()


def test_worker_stream_batch_matches_single_calls(G):
    """GP_FLAG_BATCH_STREAMS: whole instances on the worker streams, each
    bitwise equal to its own call with the same options."""
    probs, offsets, x, y, h = _batch(G)
    gp = G.GP(2, 2, 4)
    o = opts(G, "fp32", flags=G.GP_FLAG_BATCH_STREAMS)
    lml_b, grad_b, _ = gp.lml_grad_batched(offsets, x, y, h, o)
    for k, (l1, g1, _) in enumerate(_singles(G, gp, probs, opts(G, "fp32"))):
        assert lml_b[k] == l1
        assert np.array_equal(grad_b[k], g1)
    gp.close()


def test_grouped_batch_retires_instances_at_their_own_counts(G):
    """Instances whose runs need very different iteration counts (sizes 200 to
    12,000 points, r_s from 0.02 to 0.08) in one group: each leaves the
    grouped launches when its own run finishes, so its count and result equal
    its own call's."""
    probs, offsets, x, y, h = _batch(G, seeds=(9, 10), n_inst=24, n_range=(200, 12000))
    gp = G.GP(2, 2, 4)
    o = opts(G, "fp32", check_every=4)
    lml_b, grad_b, info = gp.lml_grad_batched(offsets, x, y, h, o)
    one = opts(G, "fp32", check_every=4, flags=G.GP_FLAG_SPMM_CPASYNC_WIDE)
    singles = _singles(G, gp, probs, one)
    counts = [i["iters"] for _, _, i in singles]
    assert max(counts) > 2 * min(c for c in counts if c > 0)
    for k, (l1, g1, _) in enumerate(singles):
        assert lml_b[k] == l1 and np.array_equal(grad_b[k], g1), k
    # a second call on the same context reuses the workspaces and gives the same
    lml_c, grad_c, _ = gp.lml_grad_batched(offsets, x, y, h, o)
    assert np.array_equal(lml_b, lml_c) and np.array_equal(grad_b, grad_c)
    gp.close()


def test_grouped_batch_in_two_waves(G):
    """260 small instances: two waves of grouped launches (256, then 4) on
    the same worker workspaces, every instance bitwise equal to its own call."""
    probs = W.batch_2d(seed=13, n_inst=260, n_range=(1, 300))
    offsets = np.concatenate([[0], np.cumsum([q.n for q in probs])])
    x = torch.as_tensor(np.concatenate([q.x for q in probs]), device="cuda")
    y = torch.as_tensor(np.concatenate([q.y for q in probs]), device="cuda")
    h = np.stack([q.h for q in probs])
    gp = G.GP(2, 2, 4)
    lml_b, grad_b, _ = gp.lml_grad_batched(offsets, x, y, h, opts(G, "fp32"))
    one = opts(G, "fp32", flags=G.GP_FLAG_SPMM_CPASYNC_WIDE)
    for k, (l1, g1, _) in enumerate(_singles(G, gp, probs, one)):
        assert lml_b[k] == l1 and np.array_equal(grad_b[k], g1), (k, probs[k].n)
    gp.close()


def test_grouped_batch_reports_the_iteration_cap(G):
    probs, offsets, x, y, h = _batch(G)
    gp = G.GP(2, 2, 4)
    for flags in (0, G.GP_FLAG_BATCH_STREAMS):
        with pytest.raises(G.GPError) as e:
            gp.lml_grad_batched(offsets, x, y, h, opts(G, "fp32", max_iter=3, check_every=1, flags=flags))
        assert e.value.status == G.GP_ERR_NOT_CONVERGED
    # the context stays usable
    lml_b, _, _ = gp.lml_grad_batched(offsets, x, y, h, opts(G, "fp32"))
    assert np.all(np.isfinite(lml_b))
    gp.close()


def test_block_jacobi_128_with_the_most_probes(G):
    # 64 probes (kp = 68) with 128-row blocks: the largest panels of R, Q and
    # M^-1 the streamed update handles
    p = W.grad_3d(seed=3, n=2000)
    gp = G.GP(p.dim, p.n1, p.n2)
    x = torch.as_tensor(p.x, device="cuda")
    y = torch.as_tensor(p.y, device="cuda")
    l128, i128 = gp.lml(x, y, p.h, opts(G, n_probes=64, precond_block=128))
    l32, i32 = gp.lml(x, y, p.h, opts(G, n_probes=64, precond_block=32))
    assert i128["precond_block"] == 128 and i128["kp"] == 68
    assert i128["iters"] <= i32["iters"]
    assert i128["quad_form"] == pytest.approx(i32["quad_form"], rel=1e-5)
    assert i128["logdet"] == pytest.approx(i32["logdet"], rel=1e-5)
    gp.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batched_instances_match_the_oracle(G, prec):
    """Independent GPs of the many-instance configuration (2-D, 2 x 4 bumps
    each with its own hyperparameters, r_s U(0.02, 0.08), y plus 16 probes),
    sizes from 1 to 1,500 points, through gp_lml_grad_batched: every instance's
    LML pieces against the oracle's same-probe estimator, and its gradient
    within the first-order solver bound."""
    from oracle import gp_oracle as O
    from helpers import grad_ok
    probs = W.batch_2d(seed=41, n_inst=5, n_range=(200, 1500))
    probs[2] = W.batch_2d(seed=42, n_inst=1, n_range=(1, 1))[0]          # N = 1
    offsets = np.concatenate([[0], np.cumsum([q.n for q in probs])])
    x = np.concatenate([q.x for q in probs])
    y = np.concatenate([q.y for q in probs])
    h = np.stack([q.h for q in probs])
    nv, m, seed = 16, 32, 7
    rtol = 1e-10 if prec == "fp64" else 1e-6
    o = G.default_opts(precision=prec, n_probes=nv, lanczos_steps=m, cg_rtol=rtol, seed=seed)
    gp = G.GP(2, 2, 4)
    lml_b, grad_b, info = gp.lml_grad_batched(offsets, torch.as_tensor(x, device="cuda"),
                                              torch.as_tensor(y, device="cuda"), h, o)
    for k, q in enumerate(probs):
        ref, gref, rinfo = O.lml_grad_same_probes(q.x, q.y, q.h, 2, 2, 4, nv, m, seed, with_bounds=True)
        # the estimator's pieces enter ln L; with N = 1 the log-determinant is exact
        assert lml_b[k] == pytest.approx(ref, rel=1e-9 if prec == "fp64" else 1e-5, abs=1e-9), (k, q.n)
        ok, worst = grad_ok(grad_b[k], gref, rinfo, rtol, 2.0)
        print(prec, "instance", k, "N", q.n, "grad worst / bound", worst)
        assert ok, (k, q.n, worst)
    gp.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_most_bumps_pattern_and_every_value(G, prec):
    """The largest bump count the library takes (16 functions x 32 bumps, the
    bump table's parameters then fill 40 KB of shared memory beside the
    per-warp queues of its FP64 work), against the oracle: the pattern bit-exact,
    every stored value within the format's tolerance."""
    from helpers import canonical_gpu_csr, canonical_oracle_csr, value_tol_ok
    rng = np.random.default_rng(12)
    n, n1, n2 = 600, 16, 32
    x = rng.uniform(0.0, 1.0, (n, 2))
    centres = rng.uniform(0.0, 1.0, (n1, n2, 2))
    radii = rng.uniform(0.05, 0.12, (n1, n2))
    amps = rng.normal(0.0, 1.0, (n1, n2))
    h = W.pack_h(centres, radii, amps, 0.08, 1.0, 1e-4)
    gp = G.GP(2, n1, n2)
    info = gp.assemble(torch.as_tensor(x, device="cuda"), h, precision=prec)
    r, c, v = canonical_gpu_csr(gp.get_csr())
    ro, co, vo, mask = canonical_oracle_csr(x, h, 2, n1, n2, key=("most_bumps",))
    assert info["n_active"] == int(np.sum(mask != 0))
    assert np.array_equal(r, ro) and np.array_equal(c, co)
    diag = np.zeros(n)
    dm = ro == co
    diag[ro[dm]] = vo[dm]
    ok, worst = value_tol_ok(v, vo, diag, ro, co, 1e-12 if prec == "fp64" else 1e-5, prec)
    print(prec, "nnz", len(ro), "worst relative error", worst)
    assert ok, worst
    gp.close()


def _pattern_and_values(G, x, h, dim, n1, n2, prec, key):
    from helpers import canonical_gpu_csr, canonical_oracle_csr, value_tol_ok
    gp = G.GP(dim, n1, n2)
    info = gp.assemble(torch.as_tensor(x, device="cuda"), h, precision=prec)
    r, c, v = canonical_gpu_csr(gp.get_csr())
    ro, co, vo, mask = canonical_oracle_csr(x, h, dim, n1, n2, key=key)
    assert info["n_active"] == int(np.sum(mask != 0))
    assert np.array_equal(r, ro) and np.array_equal(c, co)
    diag = np.zeros(x.shape[0])
    dm = ro == co
    diag[ro[dm]] = vo[dm]
    ok, worst = value_tol_ok(v, vo, diag, ro, co, 1e-12 if prec == "fp64" else 1e-5, prec)
    gp.close()
    return ok, worst, len(ro)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_elongated_domain_uses_the_morton_order(G, prec):
    """Clusters along a strip 40,000 r_s long: the cell grid padded to a
    power-of-two square needs 2 x 16 bits plus a sub-cell bit, more than the
    32-bit sort key holds, so the points follow the Morton order instead of
    the Hilbert curve; the pattern and every value still match the oracle."""
    rng = np.random.default_rng(21)
    r_s, n1, n2 = 0.05, 2, 6
    # 12 clusters of 150 points, 3 r_s across, spread along the strip (the
    # first and last at its ends, so the active points span 40,000 cells);
    # one bump per cluster and function
    cx = np.sort(rng.uniform(0.0, 40000 * r_s, n1 * n2))
    cx[0], cx[-1] = 2 * r_s, 39998 * r_s
    x = np.concatenate([np.column_stack([c + rng.uniform(-1.5 * r_s, 1.5 * r_s, 150),
                                         rng.uniform(0.0, r_s, 150)]) for c in cx])
    centres = np.column_stack([cx, np.full(n1 * n2, 0.5 * r_s)])
    centres = centres[rng.permutation(n1 * n2)].reshape(n1, n2, 2)
    radii = rng.uniform(2.5 * r_s, 4.0 * r_s, (n1, n2))
    amps = rng.normal(0.0, 1.0, (n1, n2))
    h = W.pack_h(centres, radii, amps, r_s, 1.0, 1e-4)
    ok, worst, nnz = _pattern_and_values(G, x, h, 2, n1, n2, prec, ("strip",))
    print(prec, "nnz", nnz, "worst relative error", worst)
    assert ok, worst


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_coordinates_far_from_the_origin(G, prec):
    """The small 2-D workload moved by 1000 along each axis (20,000 r_s): the
    double-float coordinates of the FP32 fill then carry an absolute error of
    about 2^-45 x 1000, so more entries near the support edge take the FP64
    route; pattern and values still match the oracle on the moved points."""
    p = W.small_2d(seed=5, n=1500)
    x = p.x + 1000.0
    h = p.h.copy()
    np_ = p.dim + 2
    for b in range(p.n1 * p.n2):
        h[b * np_: b * np_ + p.dim] += 1000.0  # bump centres move with the points
    ok, worst, nnz = _pattern_and_values(G, x, h, p.dim, p.n1, p.n2, prec, ("moved", 5))
    print(prec, "nnz", nnz, "worst relative error", worst)
    assert ok, worst
