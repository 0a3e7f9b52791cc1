"""Pins for the FP64 CPU oracle: each check ties an oracle function to
something other than itself (an independently derived formula, a closed-form
special case, a library routine on a special case, a brute-force loop, an
exact identity, finite differences, or a published test vector)."""

import math
import os

import numpy as np
import pytest

from oracle import gp_oracle as O
from paper_2205_09070_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.txt")


def golden():
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()[:2]
                out[k] = float(v)
    return out


def series_kstat(rho, terms=2000):
    """k~/C as the positive power series in s = sqrt(1 - rho^2), derived by
    expanding atanh: sum_{n>=2} 6 s^(2n+1) / ((2n-1)(2n+1))."""
    s = np.sqrt(1.0 - rho * rho)
    n = np.arange(2, terms)[:, None]
    return O.KSTAT_PREFACTOR * np.sum(6.0 * s ** (2 * n + 1) / ((2 * n - 1) * (2 * n + 1)), axis=0)


def small_problem(seed=11, n=150, dim=2, n1=2, n2=2, r_s=0.35, radii=(0.3, 0.5), sigma2=1e-2):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, (n, dim))
    y = np.sin(3 * x[:, 0]) + rng.normal(0, 0.1, n)
    c = rng.uniform(0.2, 0.8, (n1, n2, dim))
    r = rng.uniform(radii[0], radii[1], (n1, n2))
    a = rng.normal(0, 1, (n1, n2))
    h = W.pack_h(c, r, a, r_s, 1.3, sigma2)
    return x, y, h, dim, n1, n2


# --------------------------------------------------------------------- k~

def test_kstat_value_at_zero_matches_paper_prefactor():
    g = golden()
    assert O.kstat(np.array([0.0]))[0] == pytest.approx(g["kstat_at_zero"], rel=1e-15)


def test_kstat_matches_independent_series():
    rho = np.linspace(0.45, 0.999999, 4001)
    ref = series_kstat(rho)
    got = O.kstat(rho)
    # the closed form loses digits to cancellation near rho -> 1: compare on
    # the kernel's own scale k~(0)
    assert np.max(np.abs(got - ref)) < 1e-14 * O.KSTAT_PREFACTOR
    mid = rho < 0.95
    assert np.max(np.abs(got[mid] / ref[mid] - 1.0)) < 1e-12


def decimal_series_kstat(s2, digits=50):
    """k~/C as the positive series in s (Decimal, `digits` digits):
    sum_{n>=2} 6 s^(2n+1) / ((2n-1)(2n+1)), summed until the terms vanish."""
    from decimal import Decimal, localcontext
    with localcontext() as ctx:
        ctx.prec = digits
        s2 = Decimal(s2)
        s = s2.sqrt()
        total, n, power = Decimal(0), 2, s ** 5
        while True:
            term = 6 * power / ((2 * n - 1) * (2 * n + 1))
            if term < total * Decimal(10) ** (-digits - 2) or term == 0:
                break
            total += term
            power *= s2
            n += 1
        return total


def test_kstat_hp_matches_series_up_to_the_support_edge():
    # the printed form evaluated with 60 digits against the independently
    # derived positive series (no cancellation) for rho in [0.5, 1), down to
    # s^2 = 1 - rho^2 = 1e-14 where the float64 printed form has no digit left
    from decimal import Decimal, localcontext
    C = O.KSTAT_PREFACTOR
    for s2 in [0.75, 0.5, 0.1, 1e-2, 1.99e-2, 1e-3, 1e-4, 1e-6, 1e-8, 1e-10, 1e-12, 1e-14]:
        with localcontext() as ctx:
            ctx.prec = O.HP_DIGITS
            got = O.kstat_hp(1 - Decimal(s2))
        ref = float(decimal_series_kstat(s2)) * C
        assert float(got) == pytest.approx(ref, rel=1e-14), s2
    # where the float64 printed form does not cancel, it agrees to rounding
    rho = np.linspace(0.0, 0.5, 51)
    with localcontext() as ctx:
        ctx.prec = O.HP_DIGITS
        hp = np.array([float(O.kstat_hp(Decimal(float(r)) ** 2)) for r in rho])
    assert np.allclose(hp, O.kstat(rho), rtol=1e-14, atol=0)
    assert hp[0] == pytest.approx(golden()["kstat_at_zero"], rel=1e-15)


def test_entries_hp_match_float64_where_well_conditioned():
    # full-accuracy entries against the float64 brute force: equal to a few
    # ulps away from the support edges; everywhere within the float64 form's
    # absolute cancellation error (a few ulps of its O(1) terms, times A C
    # sum_m |f_m f_m|) plus the float64 bump's relative error near its own
    # edge (beta ulp / u^2, below 1e-10 while the bump is a normal number, u > 1/708);
    # diagonal A C sum F^2 + s2
    x, y, h, dim, n1, n2 = small_problem(seed=61, n=120, dim=3, n1=2, n2=3, r_s=0.45, radii=(0.3, 0.6))
    p = O.unpack_h(h, dim, n1, n2)
    rp, col, val = O.assemble_csr(x, h, dim, n1, n2)
    rows = np.repeat(np.arange(len(x)), np.diff(rp))
    hp = O.entries_hp(x, h, dim, n1, n2, rows, col)
    d2 = np.sum((x[rows] - x[col]) ** 2, axis=1)
    F, mask = O.bump_table(x, h, dim, n1, n2)
    S_abs = np.sum(np.abs(F[rows] * F[col]), axis=1)
    assert np.all(np.abs(hp - val) <= 1e-14 * p["A"] * O.KSTAT_PREFACTOR * S_abs + 1e-10 * np.abs(val))
    # away from every edge (rho < 0.9, each point well inside its bumps or
    # outside all) the float64 form is accurate to rounding
    def deep(i):
        ok = True
        for m in range(n1):
            for b in range(n2):
                q = np.sum((x[i] - p["centres"][m, b]) ** 2) / p["radii"][m, b] ** 2
                ok = ok and (q < 0.8 or q > 1.0)
        return ok
    good = (d2 < (0.9 * p["r_s"]) ** 2) & np.array([deep(i) and deep(j) for i, j in zip(rows, col)]) \
        & (S_abs > 0) & (np.abs(val) > 1e-3 * p["A"] * O.KSTAT_PREFACTOR * S_abs)
    assert good.sum() > 50
    assert np.allclose(hp[good], val[good], rtol=1e-13, atol=0)
    # symmetric and the diagonal closed form
    hp_t = O.entries_hp(x, h, dim, n1, n2, col, rows)
    assert np.array_equal(hp, hp_t)
    dg = rows == col
    assert np.allclose(hp[dg], p["A"] * O.KSTAT_PREFACTOR * np.sum(F ** 2, axis=1)[rows[dg]] + p["sigma2"],
                       rtol=1e-14)


def test_bump_sums_hp_match_float64_inside_and_the_edge_series():
    # f_m in decimal against the float64 bump table well inside the support,
    # and against exp(beta - beta/u) with u from an exact rational near the edge
    from decimal import Decimal, localcontext
    x, y, h, dim, n1, n2 = small_problem(seed=62, n=200, dim=2, n1=2, n2=2)
    F, mask = O.bump_table(x, h, dim, n1, n2)
    p, cand = O._hp_candidate_bumps(x, h, dim, n1, n2)
    with localcontext() as ctx:
        ctx.prec = O.HP_DIGITS
        for i in range(len(x)):
            f = O.bump_sums_hp(x[i], p, dim, n1, n2, 1.0, cand[i])
            for m in range(n1):
                assert float(f[m]) == pytest.approx(F[i, m], rel=1e-12, abs=1e-300)
        # a point at distance r (1 - 2^-30) from a unit bump: u = 2^-29 - 2^-60
        pt = np.array([1.0 - 2.0 ** -30, 0.0])
        hh = W.pack_h(np.zeros((1, 1, 2)), np.array([[1.0]]), np.array([[1.0]]), 0.1, 1.0, 1e-2)
        pp, cc = O._hp_candidate_bumps(pt[None, :], hh, 2, 1, 1)
        val = O.bump_sums_hp(pt, pp, 2, 1, 1, 1.0, cc[0])[0]
        u = 1 - (Decimal(1) - Decimal(2) ** -30) ** 2
        assert val == (1 - 1 / u).exp()


def test_kstat_support_and_monotone():
    rho = np.linspace(0.0, 1.5, 3001)
    k = O.kstat(rho)
    assert np.all(k[rho >= 1.0] == 0.0)
    assert np.all(k[rho < 1.0] > 0.0)
    assert np.all(np.diff(k[rho <= 1.0]) <= 0.0)


def test_kstat_derivative_fd_and_series():
    rho = np.linspace(0.01, 0.99, 99)
    eps = 1e-6
    fd = (O.kstat(rho + eps) - O.kstat(rho - eps)) / (2 * eps)
    d = O.kstat_drho(rho)
    assert np.max(np.abs(fd - d)) < 1e-8
    # the series converges slowly as s -> 1; check it where 4000 terms suffice
    r2 = rho[rho >= 0.3]
    s = np.sqrt(1 - r2 ** 2)
    n = np.arange(1, 4000)[:, None]
    ser = -6 * O.KSTAT_PREFACTOR * r2 * np.sum(s ** (2 * n + 1) / (2 * n + 1), axis=0)
    assert np.max(np.abs(ser - O.kstat_drho(r2))) < 1e-12
    assert np.all(O.kstat_drho(np.array([1.0, 1.2])) == 0.0)


# --------------------------------------------------------------------- bumps

def test_bump_special_values():
    c = np.array([0.3, 0.4])
    r, a = 0.2, -1.7
    for beta in (0.5, 1.0, 3.0):
        x = np.array([c, c + [r * math.sqrt(0.5), 0.0], c + [r, 0.0], c + [0.0, 1.01 * r]])
        phi, inside = O.bump_phi(x, c, r, a, beta)
        assert phi[0] == pytest.approx(a, rel=1e-15)                   # centre: a
        assert phi[1] == pytest.approx(a * math.exp(-beta), rel=1e-12)  # q = 1/2: a e^-beta
        assert phi[2] == 0.0 and phi[3] == 0.0                          # on / outside the sphere
        assert list(inside) == [True, True, False, False]


def test_bump_beta_limits():
    # beta -> 0: the bump becomes a times the indicator of its ball;
    # beta -> infinity: it vanishes away from the centre (a delta function).
    rng = np.random.default_rng(0)
    x = rng.uniform(-1, 1, (500, 3))
    c, r, a = np.zeros(3), 0.8, 2.5
    phi0, inside = O.bump_phi(x, c, r, a, beta=1e-15)
    assert np.allclose(phi0, a * inside, rtol=1e-9, atol=0)
    far = np.linalg.norm(x, axis=1) > 0.05
    phi_inf, _ = O.bump_phi(x, c, r, a, beta=1e4)
    assert np.max(np.abs(phi_inf[far])) < 1e-300 or np.all(phi_inf[far] == 0)


def test_bump_gradients_fd():
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 1, (400, 3))
    c, r, a = np.array([0.5, 0.45, 0.55]), 0.37, 0.8
    d_c, d_r, d_a = O.bump_phi_grads(x, c, r, a, beta=1.3)
    eps = 1e-6
    for k in range(3):
        e = np.zeros(3)
        e[k] = eps
        fd = (O.bump_phi(x, c + e, r, a, 1.3)[0] - O.bump_phi(x, c - e, r, a, 1.3)[0]) / (2 * eps)
        assert np.max(np.abs(fd - d_c[:, k])) < 1e-7
    fd = (O.bump_phi(x, c, r + eps, a, 1.3)[0] - O.bump_phi(x, c, r - eps, a, 1.3)[0]) / (2 * eps)
    assert np.max(np.abs(fd - d_r)) < 1e-7
    fd = (O.bump_phi(x, c, r, a + eps, 1.3)[0] - O.bump_phi(x, c, r, a - eps, 1.3)[0]) / (2 * eps)
    assert np.max(np.abs(fd - d_a)) < 1e-8


def test_bump_table_sums_and_mask():
    x, y, h, dim, n1, n2 = small_problem()
    p = O.unpack_h(h, dim, n1, n2)
    F, mask = O.bump_table(x, h, dim, n1, n2)
    for m in range(n1):
        tot = np.zeros(len(x))
        ins = np.zeros(len(x), bool)
        for b in range(n2):
            # pure-python evaluation of one bump, point by point
            for i, xi in enumerate(x):
                q = sum((xi[k] - p["centres"][m, b, k]) ** 2 for k in range(dim)) / p["radii"][m, b] ** 2
                if q < 1:
                    tot[i] += p["amps"][m, b] * math.exp(1.0 - 1.0 / (1.0 - q))
                    ins[i] = True
        assert np.allclose(F[:, m], tot, rtol=1e-13, atol=0)
        assert np.array_equal(((mask >> m) & 1).astype(bool), ins)


# --------------------------------------------------------------------- K

def test_param_count_matches_climate_example():
    g = golden()
    # n1 = 2, n2 = 4, dim = 3 without the noise variance: 42 (Sec. 3)
    assert O.n_params(3, 2, 4) - 1 == g["climate_param_count_without_noise"]
    assert O.n_params(3, 4, 8) == 163


def test_pattern_matches_pure_python_brute_force():
    x, y, h, dim, n1, n2 = small_problem(n=90, r_s=0.25)
    p = O.unpack_h(h, dim, n1, n2)
    _, mask = O.bump_table(x, h, dim, n1, n2)
    row_ptr, col, val = O.assemble_csr(x, h, dim, n1, n2, chunk=17)
    for i in range(len(x)):
        expect = [j for j in range(len(x))
                  if j == i or (math.dist(x[i], x[j]) ** 2 < p["r_s"] ** 2 and (mask[i] & mask[j]) != 0)]
        assert list(col[row_ptr[i]:row_ptr[i + 1]]) == expect


def test_K_symmetric_psd_and_unit_bump_separation():
    for dim in (1, 2, 3):
        x, y, h, _, n1, n2 = small_problem(seed=20 + dim, n=300, dim=dim, r_s=0.4)
        K = O.dense_K(x, h, dim, n1, n2)
        assert np.array_equal(K, K.T)
        ev = np.linalg.eigvalsh(K)
        assert ev[0] > -1e-12 * ev[-1]
    # n1 = n2 = 1: K_ij / (f_i f_j) = A k~(d/r_s) wherever f_i f_j != 0
    x, y, h, dim, n1, n2 = small_problem(seed=5, n=200, n1=1, n2=1, radii=(0.6, 0.7))
    p = O.unpack_h(h, dim, n1, n2)
    K = O.dense_K(x, h, dim, n1, n2) - p["sigma2"] * np.eye(len(x))
    F, _ = O.bump_table(x, h, dim, n1, n2)
    f = F[:, 0]
    nz = np.abs(np.outer(f, f)) > 1e-8
    d = np.sqrt(np.sum((x[:, None] - x[None]) ** 2, axis=2))
    rr = np.minimum(d / p["r_s"], 1.0)
    expect = p["A"] * series_kstat(rr.ravel(), terms=4000).reshape(d.shape)
    expect[d >= p["r_s"]] = 0
    far = nz & (rr >= 0.3)                 # where the series has converged
    ratio = K[far] / np.outer(f, f)[far]
    assert np.allclose(ratio, expect[far], rtol=1e-9, atol=1e-13)
    on = np.abs(f) > 1e-4                  # diagonal: A k~(0) f_i^2
    assert np.allclose(np.diag(K)[on] / f[on] ** 2, p["A"] * golden()["kstat_at_zero"], rtol=1e-13)


def test_disjoint_supports_give_exact_zeros():
    # f_0 lives on the left half, f_1 on the right; points near x = 0.5 are
    # within r_s of each other but share no function: K must be exactly 0.
    rng = np.random.default_rng(3)
    x = np.column_stack([rng.uniform(0.3, 0.7, 400), rng.uniform(0.4, 0.6, 400)])
    c = np.array([[[0.25, 0.5]], [[0.75, 0.5]]])
    r = np.array([[0.249], [0.249]])
    a = np.array([[1.0], [1.0]])
    h = W.pack_h(c, r, a, 0.2, 1.0, 1e-3)
    K = O.dense_K(x, h, 2, 2, 1)
    _, mask = O.bump_table(x, h, 2, 2, 1)
    cross = (mask[:, None] == 1) & (mask[None, :] == 2)
    assert cross.sum() > 1000
    assert np.all(K[cross] == 0.0)
    near = cross & (np.sum((x[:, None] - x[None]) ** 2, axis=2) < 0.04)
    assert near.sum() > 100


def test_sparsity_bound_holds_for_uniform_points():
    rng = np.random.default_rng(9)
    dim, n1, n2 = 2, 2, 3
    c = rng.uniform(0.25, 0.75, (n1, n2, dim))
    r = rng.uniform(0.05, 0.12, (n1, n2))
    a = np.ones((n1, n2))
    h = W.pack_h(c, r, a, 2.0, 1.0, 1e-3)   # r_s > sqrt(2): stationary term never cuts
    x = rng.uniform(0, 1, (3000, dim))
    row_ptr, col, _ = O.assemble_csr(x, h, dim, n1, n2)
    frac = (row_ptr[-1] - len(x)) / len(x) ** 2
    bound = O.sparsity_upper_bound(h, dim, n1, n2)
    assert 0 < frac <= bound * 1.05
    g = golden()
    assert O.ball_volume(3, 1.0) == pytest.approx(g["ball_volume_dim3_r1"], rel=1e-15)


# --------------------------------------------------------------------- LML

def test_lml_closed_forms():
    # N = 1: -y^2/(2k) - log(k)/2
    assert O.lml_exact(np.array([[2.5]]), np.array([1.5])) == pytest.approx(-1.5 ** 2 / 5 - 0.5 * math.log(2.5))
    # N = 2 via the adjugate inverse and det = ad - b^2
    a, b, d = 2.0, 0.7, 1.3
    y = np.array([0.4, -1.1])
    det = a * d - b * b
    quad = (d * y[0] ** 2 - 2 * b * y[0] * y[1] + a * y[1] ** 2) / det
    K = np.array([[a, b], [b, d]])
    assert O.lml_exact(K, y) == pytest.approx(-0.5 * quad - 0.5 * math.log(det), rel=1e-14)


def test_all_inactive_is_exact_noise_model():
    x, y, h, dim, n1, n2 = small_problem()
    p = O.unpack_h(h, dim, n1, n2)
    c = np.full((n1, n2, dim), 5.0)              # every bump far outside the data
    h2 = W.pack_h(c, p["radii"], p["amps"], p["r_s"], p["A"], p["sigma2"])
    s2 = p["sigma2"]
    expect = -0.5 * float(y @ y) / s2 - 0.5 * len(y) * math.log(s2)
    assert O.lml_exact(O.dense_K(x, h2, dim, n1, n2), y) == pytest.approx(expect, rel=1e-13)
    lml, grad, info = O.lml_grad_same_probes(x, y, h2, dim, n1, n2, 4, 10, 7)
    assert lml == pytest.approx(expect, rel=1e-13)
    assert grad[-1] == pytest.approx(0.5 * float(y @ y) / s2 ** 2 - 0.5 * len(y) / s2, rel=1e-12)
    assert np.all(grad[:-1] == 0.0)


@pytest.mark.parametrize("core", [False, True])
def test_exact_gradient_matches_central_fd(core):
    x, y, h, dim, n1, n2 = small_problem(n=120)
    if core:
        h = np.append(h, 0.2)     # squared-exponential core, l = 0.2 against r_s = 0.35
    lml, grad = O.lml_grad_exact(x, y, h, dim, n1, n2)
    eps = 1e-6
    for i in range(len(h)):
        e = np.zeros_like(h)
        e[i] = eps
        fp = O.lml_exact(O.dense_K(x, h + e, dim, n1, n2), y)
        fm = O.lml_exact(O.dense_K(x, h - e, dim, n1, n2), y)
        fd = (fp - fm) / (2 * eps)
        assert fd == pytest.approx(grad[i], rel=2e-5, abs=1e-4 * (1 + abs(lml)) * 1e-3), i


def test_exact_gradient_homogeneity_identities():
    # K = A k~ o (F F^T) + s2 I is homogeneous of degree 1 in (A, s2) and F is
    # linear in the amplitudes, so (Euler):
    #   A dL/dA + s2 dL/ds2 = 1/2 y^T K^-1 y - N/2
    #   sum_b a_b dL/da_b  = 2 A dL/dA
    x, y, h, dim, n1, n2 = small_problem(n=160)
    p = O.unpack_h(h, dim, n1, n2)
    lml, g = O.lml_grad_exact(x, y, h, dim, n1, n2)
    K = O.dense_K(x, h, dim, n1, n2)
    quad = float(y @ np.linalg.solve(K, y))
    A, s2 = p["A"], p["sigma2"]
    assert A * g[-2] + s2 * g[-1] == pytest.approx(0.5 * quad - 0.5 * len(y), rel=1e-10)
    amp_idx = [(m * n2 + b) * (dim + 2) + dim + 1 for m in range(n1) for b in range(n2)]
    lhs = sum(h[i] * g[i] for i in amp_idx)
    assert lhs == pytest.approx(2 * A * g[-2], rel=1e-9, abs=1e-9)


# --------------------------------------------------------------------- estimators

def test_splitmix64_published_stream():
    # SplitMix64 with state 0: the first three outputs of the reference stream
    assert [int(O.splitmix64(0, k)) for k in range(3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_rademacher_balanced():
    Z = O.rademacher(42, 8, np.arange(20000))
    assert set(np.unique(Z)) == {-1.0, 1.0}
    assert abs(Z.mean()) < 0.02
    assert np.abs(np.corrcoef(Z.T) - np.eye(8)).max() < 0.05


def test_lanczos_quadrature_exact_when_krylov_space_is_full():
    rng = np.random.default_rng(4)
    B = rng.normal(size=(40, 40))
    M = B @ B.T / 40 + 0.5 * np.eye(40)
    z = np.sign(rng.normal(size=40))
    lam, V = np.linalg.eigh(M)
    exact = float(np.sum((V.T @ z) ** 2 * np.log(lam)))
    assert O.lanczos_quadrature(M, z, 40) == pytest.approx(exact, rel=1e-10)
    # only 3 distinct eigenvalues: Lanczos stops after 3 steps and is exact
    Q, _ = np.linalg.qr(rng.normal(size=(40, 40)))
    lam3 = np.repeat([0.5, 1.0, 4.0], [10, 15, 15])
    M3 = (Q * lam3) @ Q.T
    exact3 = float(np.sum((Q.T @ z) ** 2 * np.log(lam3)))
    assert O.lanczos_quadrature(M3, z, 30) == pytest.approx(exact3, rel=1e-9)


def test_same_probe_estimator_identities_and_statistics():
    x, y, h, dim, n1, n2 = small_problem(n=200, sigma2=5e-2)
    p = O.unpack_h(h, dim, n1, n2)
    lml, g, info = O.lml_grad_same_probes(x, y, h, dim, n1, n2, 16, 30, 99)
    # exact for any probe set: the estimator is linear in dK and dK/dA*A + dK/ds2*s2 = K
    assert p["A"] * g[-2] + p["sigma2"] * g[-1] == pytest.approx(0.5 * info["quad_form"] - 0.5 * len(y), rel=1e-9)
    # statistical: SLQ and Hutchinson within 5 standard errors of the exact values
    K = O.dense_K(x, h, dim, n1, n2)
    lml_x, g_x = O.lml_grad_exact(x, y, h, dim, n1, n2)
    nv = 400
    lml_s, g_s, info_s = O.lml_grad_same_probes(x, y, h, dim, n1, n2, nv, 60, 5)
    se = np.std(info_s["slq_terms"]) / math.sqrt(nv)
    assert abs(info_s["logdet"] - 2 * np.sum(np.log(np.diag(np.linalg.cholesky(K))))) < 5 * se + 1e-8
    assert np.median(np.abs(g_s - g_x) / (np.abs(g_x) + 1e-3)) < 0.2


# --------------------------------------------------------------------- posterior mean

def test_cross_K_matches_pure_python_brute_force():
    # pair by pair with plain loops: bump sums with math.exp, the strict
    # support tests, k~ from the independent series where it has converged
    x, y, h, dim, n1, n2 = small_problem(seed=31, n=40)
    rng = np.random.default_rng(32)
    xs = rng.uniform(-0.1, 1.1, (15, dim))
    p = O.unpack_h(h, dim, n1, n2)
    kappa = O.cross_K(xs, x, h, dim, n1, n2)

    def f(pt, m):
        tot = 0.0
        for b in range(n2):
            q = sum((pt[k] - p["centres"][m, b][k]) ** 2 for k in range(dim)) / p["radii"][m, b] ** 2
            if q < 1.0:
                tot += p["amps"][m, b] * math.exp(1.0 - 1.0 / (1.0 - q))
        return tot

    kappa_hp = O.cross_K_hp(xs, x, h, dim, n1, n2)
    checked = 0
    for a in range(len(xs)):
        for i in range(len(x)):
            d = math.dist(xs[a], x[i])
            S = sum(f(xs[a], m) * f(x[i], m) for m in range(n1))
            if d >= p["r_s"] or S == 0.0:
                assert kappa[a, i] == 0.0 and kappa_hp[a, i] == 0.0
                continue
            rho = d / p["r_s"]
            # k~ from the independent positive series where it has converged
            # (no cancellation), the printed form nearer the centre
            k = series_kstat(np.array([rho]), terms=4000)[0] if rho >= 0.3 else O.kstat(np.array([rho]))[0]
            # the full-accuracy route agrees everywhere; the float64 printed
            # form only where it does not cancel
            assert kappa_hp[a, i] == pytest.approx(p["A"] * k * S, rel=1e-9)
            if rho < 0.9:
                assert kappa[a, i] == pytest.approx(p["A"] * k * S, rel=1e-9)
            checked += 1
    assert checked > 20


def test_predict_mean_at_training_points_and_outside_supports():
    # K alpha = y with K = Kf + sigma2 I gives Kf alpha = y - sigma2 alpha:
    # the posterior mean at the training inputs is y - sigma2 K^-1 y
    x, y, h, dim, n1, n2 = small_problem(seed=33, n=120)
    p = O.unpack_h(h, dim, n1, n2)
    K = O.dense_K(x, h, dim, n1, n2)
    alpha = np.linalg.solve(K, y)
    m_train = O.predict_mean(x, y, h, x, dim, n1, n2)
    assert np.allclose(m_train, y - p["sigma2"] * alpha, rtol=1e-10, atol=1e-12 * np.abs(y).max())
    # points outside every bump, or farther than r_s from every training point,
    # have an exactly zero mean
    far = np.array([[5.0, 5.0], [-3.0, 0.5]])
    assert np.array_equal(O.predict_mean(x, y, h, far, dim, n1, n2), np.zeros(2))
    _, mask = O.bump_table(x, h, dim, n1, n2)
    outside = x[mask == 0][:3]
    if len(outside):
        assert np.array_equal(O.predict_mean(x, y, h, outside, dim, n1, n2), np.zeros(len(outside)))


# --------------------------------------------------------------------- Taylor log-determinant

def test_taylor_logdet_exact_traces_match_the_eigenvalue_series():
    # probes = the N basis vectors give exact traces: the estimator is then
    # N ln a - sum_i sum_{k<=m} c_i^k / k with c_i = 1 - lambda_i / a, written
    # here from the eigenvalues instead of matrix powers
    x, y, h, dim, n1, n2 = small_problem(seed=51, n=120)
    K = O.dense_K(x, h, dim, n1, n2)
    D = np.diag(K)
    Khat = K / np.sqrt(np.outer(D, D))
    a = O.gershgorin_bound(Khat)
    lam = np.linalg.eigvalsh(Khat)
    assert lam[-1] <= a * (1 + 1e-12)
    c = 1.0 - lam / a
    for m in (1, 5, 40):
        series = len(lam) * math.log(a) - sum(np.sum(c ** k) / k for k in range(1, m + 1))
        got = O.taylor_logdet_terms(Khat, np.eye(len(lam)), m, a)
        assert np.sum(got) - (len(lam) - 1) * len(lam) * math.log(a) == pytest.approx(series, rel=1e-10)
    # the full series is ln|Khat|: a well-conditioned matrix converges fast
    Kw = Khat + 2.0 * np.eye(len(lam))
    aw = O.gershgorin_bound(Kw)
    gw = O.taylor_logdet_terms(Kw, np.eye(len(lam)), 400, aw)
    exact = np.linalg.slogdet(Kw)[1]
    assert np.sum(gw) - (len(lam) - 1) * len(lam) * math.log(aw) == pytest.approx(exact, rel=1e-9)


def test_taylor_logdet_same_probes_split_and_statistics():
    # the same split as SLQ: all-inactive data give the exact noise model
    x, y, h, dim, n1, n2 = small_problem(seed=52, n=150)
    p = O.unpack_h(h, dim, n1, n2)
    far = h.copy()
    per = dim + 2
    for b in range(n1 * n2):
        far[b * per: b * per + dim] = 40.0
    ld, gam, a = O.logdet_taylor_same_probes(x, far, dim, n1, n2, 8, 10, 3)
    assert ld == pytest.approx(len(x) * math.log(p["sigma2"]), rel=1e-14)
    # with many terms and probes the estimate is within its standard error of
    # ln|K| (the truncation bias shrinks as c^m for the well-separated spectrum
    # this small problem has; checked against the eigenvalue series above)
    ld, gam, a = O.logdet_taylor_same_probes(x, h, dim, n1, n2, 64, 300, 4)
    exact = np.linalg.slogdet(O.dense_K(x, h, dim, n1, n2))[1]
    se = np.std(gam, ddof=1) / math.sqrt(len(gam))
    assert abs(ld - exact) <= 5 * se + 1e-3 * abs(exact)


# --------------------------------------------------------------------- augmented objective

def test_sparsity_gradient_and_augmented_objective_against_finite_differences():
    # d s / d h by central differences of the bound (only radii move it), and
    # the augmented objective's product rule on a smooth stand-in for ln L
    rng = np.random.default_rng(61)
    for dim in (1, 2, 3):
        n1, n2 = 3, 4
        h = W.pack_h(rng.uniform(0, 1, (n1, n2, dim)), rng.uniform(0.05, 0.3, (n1, n2)),
                     rng.normal(0, 1, (n1, n2)), 0.1, 1.0, 1e-3)
        vol = 1.7
        g = O.sparsity_upper_bound_grad(h, dim, n1, n2, vol)
        eps = 1e-6
        for q in range(len(h)):
            hp, hm = h.copy(), h.copy()
            hp[q] += eps
            hm[q] -= eps
            fd = (O.sparsity_upper_bound(hp, dim, n1, n2, vol) - O.sparsity_upper_bound(hm, dim, n1, n2, vol)) / (2 * eps)
            assert g[q] == pytest.approx(fd, rel=1e-6, abs=1e-12)

        def f(hh):  # smooth stand-in for ln L with a known gradient
            return -float(np.sum(hh ** 2)) - 3.0, -2.0 * hh

        val, gr, s = O.augmented_objective(*f(h), h, dim, n1, n2, vol)
        assert val == pytest.approx((2 - s) * f(h)[0], rel=1e-15)
        for q in range(len(h)):
            hp, hm = h.copy(), h.copy()
            hp[q] += eps
            hm[q] -= eps
            vp = O.augmented_objective(*f(hp), hp, dim, n1, n2, vol)[0]
            vm = O.augmented_objective(*f(hm), hm, dim, n1, n2, vol)[0]
            assert gr[q] == pytest.approx((vp - vm) / (2 * eps), rel=1e-6, abs=1e-9)


# --------------------------------------------------------------------- core kernel k_c * k_s

def test_core_kernel_entries_psd_and_limits():
    # K with a squared-exponential core: pair by pair against plain loops
    # (math.exp, the independent k~ series where it has converged), symmetric
    # and PSD (a Schur product of PSD kernels), the diagonal untouched, and
    # the plain kernel recovered as l -> infinity
    for dim in (1, 2, 3):
        x, y, h, _, n1, n2 = small_problem(seed=70 + dim, n=160, dim=dim, r_s=0.4)
        hc = np.append(h, 0.15)
        p = O.unpack_h(hc, dim, n1, n2)
        assert p["ell"] == 0.15 and O.unpack_h(h, dim, n1, n2)["ell"] is None
        K = O.dense_K(x, hc, dim, n1, n2)
        K0 = O.dense_K(x, h, dim, n1, n2)
        assert np.array_equal(K, K.T)
        ev = np.linalg.eigvalsh(K)
        assert ev[0] > -1e-12 * ev[-1]
        assert np.array_equal(np.diag(K), np.diag(K0))
        F, _ = O.bump_table(x, h, dim, n1, n2)
        checked = 0
        for i in range(0, len(x), 7):
            for j in range(len(x)):
                if i == j or K0[i, j] == 0.0:
                    assert K[i, j] == K0[i, j]
                    continue
                d2 = sum((x[i][k] - x[j][k]) ** 2 for k in range(dim))
                rho = math.sqrt(d2) / p["r_s"]
                if rho < 0.3:
                    continue
                kt = series_kstat(np.array([rho]), terms=4000)[0]
                S = sum(F[i, m] * F[j, m] for m in range(n1))
                expect = p["A"] * kt * math.exp(-d2 / (2 * 0.15 ** 2)) * S
                assert K[i, j] == pytest.approx(expect, rel=1e-9, abs=1e-15 * abs(p["A"] * S)), (i, j)
                checked += 1
        assert checked > 50
        Kinf = O.dense_K(x, np.append(h, 1e9), dim, n1, n2)
        assert np.allclose(Kinf, K0, rtol=1e-15, atol=1e-300)


def test_core_kernel_full_accuracy_entries_and_cross_covariance():
    # the decimal route with the core against the float64 brute force where
    # neither cancels, and the test-point cross-covariance likewise
    x, y, h, dim, n1, n2 = small_problem(seed=81, n=100, dim=2, r_s=0.45)
    hc = np.append(h, 0.2)
    rp, col, val = O.assemble_csr(x, hc, dim, n1, n2)
    rows = np.repeat(np.arange(len(x)), np.diff(rp))
    hp = O.entries_hp(x, hc, dim, n1, n2, rows, col)
    d2 = np.sum((x[rows] - x[col]) ** 2, axis=1)
    F, _ = O.bump_table(x, h, dim, n1, n2)
    S_abs = np.sum(np.abs(F[rows] * F[col]), axis=1)
    p = O.unpack_h(hc, dim, n1, n2)
    assert np.all(np.abs(hp - val) <= 1e-14 * p["A"] * O.KSTAT_PREFACTOR * S_abs + 1e-10 * np.abs(val))
    # away from every edge (rho < 0.9, both points well inside their bumps or
    # outside all) the float64 form is accurate to rounding
    q = np.stack([np.sum((x - p["centres"][m, b]) ** 2, axis=1) / p["radii"][m, b] ** 2
                  for m in range(n1) for b in range(n2)], axis=1)
    deep = np.all((q < 0.8) | (q > 1.0), axis=1)
    good = (d2 < (0.9 * p["r_s"]) ** 2) & deep[rows] & deep[col] \
        & (np.abs(val) > 1e-3 * p["A"] * O.KSTAT_PREFACTOR * S_abs)
    assert good.sum() > 50
    assert np.allclose(hp[good], val[good], rtol=1e-12, atol=0)
    xs = np.random.default_rng(82).uniform(0, 1, (20, dim))
    k64, khp = O.cross_K(xs, x, hc, dim, n1, n2), O.cross_K_hp(xs, x, hc, dim, n1, n2)
    assert np.array_equal(k64 == 0, khp == 0)
    assert np.allclose(khp, k64, rtol=1e-9, atol=1e-15 * np.abs(k64).max())


# --------------------------------------------------------------------- posterior variance

def test_predict_var_identities():
    # at a training input x_i, kappa = K_:i - s2 e_i and k(x_i, x_i) = K_ii - s2,
    # so the posterior variance is s2 - s2^2 (K^-1)_ii (an identity the dense
    # solve does not use); elsewhere 0 <= var <= prior, var = prior where no
    # training point is within r_s, and 0 outside every bump; with and without
    # the core kernel
    for core in (None, 0.2):
        x, y, h, dim, n1, n2 = small_problem(seed=91, n=120)
        if core is not None:
            h = np.append(h, core)
        p = O.unpack_h(h, dim, n1, n2)
        K = O.dense_K(x, h, dim, n1, n2)
        v_train = O.predict_var(x, h, x, dim, n1, n2)
        expect = p["sigma2"] - p["sigma2"] ** 2 * np.diag(np.linalg.inv(K))
        assert np.allclose(v_train, expect, rtol=1e-9, atol=1e-13 * p["sigma2"])
        rng = np.random.default_rng(92)
        xs = rng.uniform(-0.2, 1.2, (200, dim))
        v = O.predict_var(x, h, xs, dim, n1, n2)
        prior = O.prior_var(xs, h, dim, n1, n2)
        assert np.all(v >= -1e-12 * (1 + prior)) and np.all(v <= prior + 1e-12 * (1 + prior))
        d2min = np.min(np.sum((xs[:, None, :] - x[None, :, :]) ** 2, axis=2), axis=1)
        far = d2min >= p["r_s"] ** 2
        assert np.array_equal(v[far], prior[far])
        _, mask = O.bump_table(xs, h, dim, n1, n2)
        assert np.all(v[mask == 0] == 0.0)
        # the full-accuracy prior agrees with the float64 one to the bumps' rounding
        assert np.allclose(O.prior_var_hp(xs, h, dim, n1, n2), prior, rtol=1e-10, atol=0)
