"""CPU pins of the oracle's training loop (Sec. 2.4 objectives, Adam as the
reading of Sec. 4's gradient-based training): closed-form Adam steps, the
maximiser of a concave quadratic, feasibility under the Eq. eq:constrained
requirement, and the objective values of the trace."""

import math

import numpy as np
import pytest

from oracle import gp_oracle as O
from paper_2205_09070_gb300 import workloads as W


def test_positive_entries_follow_the_parameter_layout():
    dim, n1, n2 = 2, 2, 3
    p = n1 * n2 * (dim + 2) + 3
    pos = O.positive_entries(p, dim, n1, n2)
    want = np.zeros(p, dtype=bool)
    want[[b * 4 + 2 for b in range(6)]] = True        # radii
    want[-3:] = True                                   # r_s, A, sigma_n^2
    assert np.array_equal(pos, want)
    assert O.positive_entries(p + 1, dim, n1, n2)[-1]  # a core length scale


def test_first_step_is_lr_times_the_gradient_sign():
    # m_1 / (1 - beta1) = g and v_1 / (1 - beta2) = g^2, so the first step in
    # theta is lr g / (|g| + eps): + lr up the gradient, multiplicative (e^lr)
    # on the positive entries
    a = np.array([3.0, -2.0, 0.5, -7.0])
    pos = np.array([False, False, True, True])
    h0 = np.array([1.0, 2.0, 0.5, 4.0])

    def obj(h):
        return float(a @ h), a.copy(), None

    lr, eps = 0.1, 1e-8
    h1, trace = O.adam_ascent(obj, h0, pos, 1, lr, eps=eps)
    g = np.where(pos, h0 * a, a)
    step = lr * g / (np.abs(g) + eps)
    assert np.allclose(h1[:2], h0[:2] + step[:2], rtol=0, atol=1e-15)
    assert np.allclose(h1[2:], h0[2:] * np.exp(step[2:]), rtol=1e-15)
    assert h1[0] > h0[0] and h1[1] < h0[1] and h1[2] > h0[2] and h1[3] < h0[3]   # ascent
    assert len(trace) == 2 and trace[0][0] == pytest.approx(a @ h0)


def test_constant_gradient_gives_equal_steps():
    # f = a . theta with theta = h on the free entries and ln h on the positive
    # ones (d f / d h = a / h there): d f / d theta is the constant a, the
    # bias-corrected moments are exactly a and a^2 at every step, and n steps
    # move theta by n lr a / (|a| + eps)
    a = np.array([1.5, -0.25, 4.0, -0.6, 2.0])
    pos = np.array([False, False, False, True, True])
    h0 = np.array([0.3, -1.0, 2.0, 0.8, 5.0])

    def obj(h):
        th = h.copy()
        th[pos] = np.log(h[pos])
        grad = a.copy()
        grad[pos] /= h[pos]
        return float(a @ th), grad, None

    n, lr, eps = 25, 0.01, 1e-8
    move = n * lr * a / (np.abs(a) + eps)
    for b1, b2 in ((0.9, 0.999), (0.5, 0.9), (0.0, 0.0)):
        h, _ = O.adam_ascent(obj, h0, pos, n, lr, b1, b2, eps)
        assert np.allclose(h[~pos], h0[~pos] + move[~pos], rtol=1e-12, atol=1e-14), (b1, b2)
        assert np.allclose(h[pos], h0[pos] * np.exp(move[pos]), rtol=1e-12), (b1, b2)


def test_maximiser_of_a_concave_quadratic():
    # f = -sum w (theta - c)^2 with theta = h (free) or ln h (positive): the
    # iterates end within a few lr of the maximiser
    c = np.array([0.7, -1.2, math.log(3.0), math.log(0.2)])
    w = np.array([1.0, 4.0, 0.5, 2.0])
    pos = np.array([False, False, True, True])

    def theta(h):
        th = h.copy()
        th[pos] = np.log(h[pos])
        return th

    def obj(h):
        th = theta(h)
        value = -float(np.sum(w * (th - c) ** 2))
        grad = -2.0 * w * (th - c)                    # d f / d theta
        grad[pos] /= h[pos]                            # d f / d h = (d f / d theta) / h there
        return value, grad, None

    h, trace = O.adam_ascent(obj, np.array([0.0, 0.0, 1.0, 1.0]), pos, 4000, 2e-3)
    th = theta(h)
    assert np.max(np.abs(th - c)) < 1e-2
    assert trace[-1][0] > trace[0][0]


def test_constrained_iterates_stay_feasible_and_reach_the_boundary():
    # an objective that grows the radii pushes s up; every iterate keeps
    # s < s_max and the steps, halved at the boundary, end close to it
    dim, n1, n2 = 2, 1, 3
    p = W.small_2d(seed=1, n=10)
    h0 = np.asarray(p.h[: n1 * n2 * (dim + 2)].tolist() + list(p.h[-3:]))
    h0[[b * 4 + 2 for b in range(3)]] = 0.1
    pos = O.positive_entries(len(h0), dim, n1, n2)
    radii = pos.copy()
    radii[-3:] = False

    def obj(h):
        return float(np.sum(h[radii])), radii.astype(np.float64), None

    s0 = O.sparsity_upper_bound(h0, dim, n1, n2)
    s_max = 4.0 * s0

    def feasible(h):
        return O.sparsity_upper_bound(h, dim, n1, n2) < s_max

    h, _ = O.adam_ascent(obj, h0, pos, 200, 0.05, feasible=feasible)
    s_end = O.sparsity_upper_bound(h, dim, n1, n2)
    assert 0.9 * s_max < s_end < s_max
    # unconstrained, the same steps pass the requirement
    h_free, _ = O.adam_ascent(obj, h0, pos, 200, 0.05)
    assert O.sparsity_upper_bound(h_free, dim, n1, n2) > s_max
    # a step that cannot be made feasible is not taken
    h_stuck, _ = O.adam_ascent(obj, h0, pos, 3, 0.05, feasible=lambda h: False)
    assert np.array_equal(h_stuck, h0)


def test_training_trace_objectives():
    # trace rows (objective, ln L, s): the augmented row is (2 - s) ln L; ln L
    # is the same-probe estimator's value at that iterate
    p = W.small_2d(seed=2, n=150)
    kw = dict(n_probes=4, lanczos_steps=10, seed=5, n_steps=2, lr=0.02)
    h_aug, tr = O.train_same_probes(p.x, p.y, p.h, p.dim, p.n1, p.n2, objective="augmented", **kw)
    assert np.allclose(tr[:, 0], (2.0 - tr[:, 2]) * tr[:, 1], rtol=1e-14)
    lml_end, _, _ = O.lml_grad_same_probes(p.x, p.y, h_aug, p.dim, p.n1, p.n2, 4, 10, 5, with_grad=False)
    assert tr[-1, 1] == pytest.approx(lml_end, rel=1e-13)
    h_lml, tr2 = O.train_same_probes(p.x, p.y, p.h, p.dim, p.n1, p.n2, objective="lml", **kw)
    assert np.array_equal(tr2[:, 0], tr2[:, 1])
    assert tr2[0, 1] == tr[0, 1]                       # same start, same estimator
    assert not np.array_equal(h_aug, h_lml)            # the objectives' gradients differ
