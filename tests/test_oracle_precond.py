"""Pins for the oracle's block-Jacobi preconditioned estimator and its row
order.  The estimator is pinned by exact identities: over the full set of
2^n sign vectors E[z z^T] = I holds exactly, and with at least n Lanczos
steps Gauss quadrature is exact, so the preconditioned log-determinant and
gradient must equal the dense closed forms for every block size."""

import itertools
import os

import numpy as np
import pytest

from oracle import gp_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "zorder_2d.txt")


def test_zorder_matches_z_curve_fixture():
    want = np.loadtxt(GOLDEN, dtype=np.int64)
    # one point per unit cell, a corner point at the origin fixes the grid
    # origin and one at (3.9, 3.9) its extent (4 x 4 cells of edge r_s = 1)
    cells = [(i, j) for j in range(4) for i in range(4)]
    rng = np.random.default_rng(0)
    rng.shuffle(cells)
    pts = [(0.0, 0.0), (3.9, 3.9)] + [(i + 0.3, j + 0.3) for i, j in cells]
    x = np.asarray(pts)
    act = np.arange(2, x.shape[0])
    order = O.zorder_active(x, act, 1.0, 2)
    got = np.floor(x[order]).astype(np.int64)
    np.testing.assert_array_equal(got, want)


def test_zorder_sub_cells_and_ties():
    # inside one cell the 4 x 4 sub-cells follow their own Z-curve; equal keys
    # keep ascending original index
    x = np.array([[0.0, 0.0], [3.9, 3.9], [0.1, 0.6], [0.6, 0.1], [0.62, 0.12], [0.05, 0.05]])
    order = O.zorder_active(x, np.arange(x.shape[0]), 1.0, 2)
    # sub-cells: 0 -> (0,0), 5 -> (0,0), 3 -> (2,0), 4 -> (2,0), 2 -> (0,2); 1 is in cell (3,3)
    np.testing.assert_array_equal(order, [0, 5, 3, 4, 2, 1])


def test_zorder_is_a_permutation_with_cells_contiguous():
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, (400, 3))
    act = np.sort(rng.choice(400, 250, replace=False))
    order = O.zorder_active(x, act, 0.1, 3)
    assert sorted(order.tolist()) == act.tolist()
    cell = [tuple(np.floor((x[i] - x.min(0)) / (0.1 * (1 + 1e-9))).astype(int)) for i in order]
    seen = set()
    for a, b in zip(cell, cell[1:] + [None]):
        if a != b:
            assert a not in seen, "a cell's points must be contiguous"
            seen.add(a)


def tiny_problem(seed):
    rng = np.random.default_rng(seed)
    n, dim = 12, 2
    x = rng.uniform(0, 1, (n, dim))
    y = rng.normal(0, 1, n)
    h = np.array([0.5, 0.5, 0.42, 1.3, 0.6, 0.9, 0.05])  # centre, r, a; r_s, A, sigma^2
    return x, y, h, dim


def exhaustive_signs(n):
    return np.array(list(itertools.product([1.0, -1.0], repeat=n))).T


@pytest.mark.parametrize("B", [2, 3, 5, 64])
def test_preconditioned_estimator_exact_over_all_signs(B):
    x, y, h, dim = tiny_problem(8)
    _, mask = O.bump_table(x, h, dim, 1, 1)
    n_act = int(np.count_nonzero(mask))
    assert 5 <= n_act <= 11
    Z = exhaustive_signs(n_act)
    lml, grad, info = O.lml_grad_same_probes(x, y, h, dim, 1, 1, 0, n_act + 2, 0,
                                             precond_block=B, probes=Z)
    lml_ex, grad_ex = O.lml_grad_exact(x, y, h, dim, 1, 1)
    assert abs(lml - lml_ex) < 1e-9 * max(1.0, abs(lml_ex))
    np.testing.assert_allclose(grad, grad_ex, rtol=1e-8, atol=1e-9 * np.max(np.abs(grad_ex)))


def test_block_size_one_is_the_unpreconditioned_estimator():
    x, y, h, dim = tiny_problem(7)
    a = O.lml_grad_same_probes(x, y, h, dim, 1, 1, 6, 5, 123, precond_block=0)
    b = O.lml_grad_same_probes(x, y, h, dim, 1, 1, 6, 5, 123, precond_block=1)
    assert abs(a[0] - b[0]) < 1e-12 * max(1.0, abs(a[0]))
    np.testing.assert_allclose(a[1], b[1], rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(a[2]["slq_terms"], b[2]["slq_terms"], rtol=1e-10)
    assert b[2]["logdet_precond"] == pytest.approx(0.0, abs=1e-12)


def test_one_block_covering_all_rows_is_exact_logdet():
    # M = Khat: the preconditioned operator is I, every quadrature term is 0
    x, y, h, dim = tiny_problem(8)
    lml, _, info = O.lml_grad_same_probes(x, y, h, dim, 1, 1, 4, 6, 9, with_grad=False,
                                          precond_block=1000)
    assert np.max(np.abs(info["slq_terms"])) < 1e-10
    lml_ex, _ = O.lml_grad_exact(x, y, h, dim, 1, 1)
    assert abs(lml - lml_ex) < 1e-10 * max(1.0, abs(lml_ex))
