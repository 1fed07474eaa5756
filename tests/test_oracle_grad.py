"""Pins of the oracle's vector-Jacobian products against finite differences."""
import numpy as np
import pytest

import oracle
import synth


def _functional(acc, pot, gA, gP):
    return float(np.sum(acc * gA) + np.sum(pot * gP))


def test_direct_grad_matches_central_differences():
    N = 64
    x, m, h = synth.make_particles("plummer", N, 11, "loguniform10", n_neigh=20)
    rng = np.random.default_rng(1)
    gA, gP = rng.standard_normal((N, 3)), rng.standard_normal(N)
    gx, gm = oracle.direct_grad(x, m, h, gA, gP)
    for trial in range(3):
        u = rng.standard_normal((N, 3))
        v = rng.standard_normal(N) * m
        eps = 1e-6
        Lp = _functional(*oracle.direct(x + eps * u, m + eps * v, h), gA, gP)
        Lm = _functional(*oracle.direct(x - eps * u, m - eps * v, h), gA, gP)
        fd = (Lp - Lm) / (2 * eps)
        an = np.sum(gx * u) + np.sum(gm * v)
        assert an == pytest.approx(fd, rel=2e-6)


@pytest.fixture(scope="module")
def tree600():
    x, m, h = synth.make_particles("plummer", 600, 12, "loguniform10")
    T = oracle.OracleTree(x, m, h)
    T.walk(0.5)
    assert T.lists()["far_ids"].size > 0
    return x, m, h, T


def _frozen_forward(T, x, m):
    T.refit(x, m)
    return T.gravity()


def test_tree_backward_matches_frozen_structure_differences(tree600):
    # a(x, m) with the tree's particle sets and interaction lists held fixed: moments are
    # refitted from the displaced particles (Sec. 2.1.8) and the lists are not re-walked.
    x, m, h, T = tree600
    N = x.shape[0]
    rng = np.random.default_rng(2)
    gA, gP = rng.standard_normal((N, 3)), rng.standard_normal(N)
    T.refit(x, m)
    gx, gm = T.gravity_backward(gA, gP)
    for trial in range(4):
        u = rng.standard_normal((N, 3)) if trial != 1 else np.zeros((N, 3))
        v = rng.standard_normal(N) * m if trial != 0 else np.zeros(N)
        eps = 1e-6
        Lp = _functional(*_frozen_forward(T, x + eps * u, m + eps * v), gA, gP)
        Lm = _functional(*_frozen_forward(T, x - eps * u, m - eps * v), gA, gP)
        fd = (Lp - Lm) / (2 * eps)
        an = np.sum(gx * u) + np.sum(gm * v)
        assert an == pytest.approx(fd, rel=1e-6)
    T.refit(x, m)


def test_tree_backward_loss_of_config5_form(tree600):
    # loss = sum |a - a_t|^2 with a_t from jittered positions: gA = 2 (a - a_t), gPhi = 0
    x, m, h, T = tree600
    T.refit(x, m)
    acc, _ = T.gravity()
    at, _ = oracle.direct(synth.jitter(x, 1e-3, 5), m, h)
    gA = 2 * (acc - at)
    gx, gm = T.gravity_backward(gA, None)
    u = synth.random_unit_vectors(x.shape, 9)
    eps = 1e-6

    def loss(xx):
        a, _ = _frozen_forward(T, xx, m)
        return float(np.sum((a - at) ** 2))

    fd = (loss(x + eps * u) - loss(x - eps * u)) / (2 * eps)
    assert np.sum(gx * u) == pytest.approx(fd, rel=1e-5)
    T.refit(x, m)


def test_tree_backward_at_theta_zero_equals_direct_gradient():
    x, m, h = synth.make_particles("sphere", 400, 13, "loguniform10")
    T = oracle.OracleTree(x, m, h)
    T.walk(0.0)
    rng = np.random.default_rng(3)
    gA, gP = rng.standard_normal((400, 3)), rng.standard_normal(400)
    gx, gm = T.gravity_backward(gA, gP)
    dx, dm = oracle.direct_grad(x, m, h, gA, gP)
    assert np.max(np.abs(gx - dx)) <= 1e-10 * np.max(np.abs(dx))
    assert np.max(np.abs(gm - dm)) <= 1e-10 * np.max(np.abs(dm))
