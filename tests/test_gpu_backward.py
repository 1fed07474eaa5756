"""GPU backward pass against the oracle's vector-Jacobian product and the direct-sum gradient."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _gpu(*arrays):
    import torch
    dev = torch.device("cuda:0")
    return tuple(torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in arrays)


def _close(g, o, rtol):
    scale = np.max(np.abs(o)) + 1e-300
    err = np.max(np.abs(g - o)) / scale
    nerr = np.linalg.norm(g - o) / (np.linalg.norm(o) + 1e-300)
    return err, nerr


@pytest.mark.parametrize("kind,N,theta,precision", [("plummer", 3000, 0.5, "fp64"), ("sphere", 8000, 0.7, "fp64"),
                                                     ("plummer", 3000, 0.5, "mixed")])
def test_backward_matches_oracle_vjp(kind, N, theta, precision):
    import paper_1108_0028_gb300 as rcb
    x, m, h = synth.make_particles(kind, N, synth.seed_for(5, 7), "loguniform10")
    rng = np.random.default_rng(4)
    gA, gP = rng.standard_normal((N, 3)), rng.standard_normal(N)
    ref = oracle.OracleTree(x, m, h)
    ref.walk(theta)
    ox, om = ref.gravity_backward(gA, gP)
    tree = rcb.RCBTree(*_gpu(x, m, h), theta=theta, precision=precision)
    tree.gravity()
    gx, gm = tree.gravity_backward(*_gpu(gA, gP))
    gx, gm = gx.cpu().numpy(), gm.cpu().numpy()
    ex, nx = _close(gx, ox, 1e-9)
    em, nm = _close(gm, om, 1e-9)
    print(f"{precision} {kind} N={N}: dx max {ex:.2e} norm {nx:.2e}; dm max {em:.2e} norm {nm:.2e}")
    tol = 1e-9 if precision == "fp64" else 1e-5
    assert ex < tol and em < tol and nx < tol and nm < tol
    # a second call reuses the transposed lists and gives the same result up to the order of
    # atomic additions: FP64 node adjoints in the FP64 form; in the mixed form the far part first
    # merges node adjoints in float32 shared-memory sums, so the order shows at float32 level
    gx2, gm2 = tree.gravity_backward(*_gpu(gA, gP))
    rep = 1e-12 if precision == "fp64" else 1e-6
    assert np.allclose(gx2.cpu().numpy(), gx, rtol=0, atol=rep * np.abs(gx).max())
    assert np.allclose(gm2.cpu().numpy(), gm, rtol=0, atol=rep * np.abs(gm).max())


def test_backward_theta_zero_equals_direct_gradient():
    import paper_1108_0028_gb300 as rcb
    N = 2048
    x, m, h = synth.make_particles("plummer", N, 91, "equal")
    at, _ = oracle.direct(synth.jitter(x, 1e-3, 3), m, h)
    tree = rcb.RCBTree(*_gpu(x, m, h), theta=0.0, precision="fp64")
    acc, _ = tree.gravity()
    gA = 2.0 * (acc.cpu().numpy() - at)          # loss = sum |a - a_target|^2
    gx, gm = tree.gravity_backward(*_gpu(gA))
    dx, dm = oracle.direct_grad(x, m, h, gA, None)
    ex, nx = _close(gx.cpu().numpy(), dx, 1e-9)
    em, nm = _close(gm.cpu().numpy(), dm, 1e-9)
    assert ex < 1e-9 and em < 1e-9


def test_autograd_function():
    import torch

    import paper_1108_0028_gb300 as rcb
    N = 2500
    x, m, h = synth.make_particles("sphere", N, 92, "loguniform10")
    xt, mt, ht = _gpu(x, m, h)
    xt.requires_grad_(True)
    mt.requires_grad_(True)
    acc, pot = rcb.rcb_gravity_fn(xt, mt, ht, 12, 0.6, "fp64")
    loss = (acc * acc).sum() + pot.sum()
    loss.backward()
    ref = oracle.OracleTree(x, m, h)
    ref.walk(0.6)
    a, p = ref.gravity()
    ox, om = ref.gravity_backward(2 * a, np.ones(N))
    ex, _ = _close(xt.grad.cpu().numpy(), ox, 1e-9)
    em, _ = _close(mt.grad.cpu().numpy(), om, 1e-9)
    assert ex < 1e-9 and em < 1e-9


def test_autograd_function_mixed():
    # the torch.autograd.Function in the mixed form: its gradient matches the oracle's FP64 VJP to
    # the mixed backward's tolerance (1e-5 of the largest component)
    import paper_1108_0028_gb300 as rcb
    N = 2500
    x, m, h = synth.make_particles("sphere", N, 93, "loguniform10")
    xt, mt, ht = _gpu(x, m, h)
    xt.requires_grad_(True)
    mt.requires_grad_(True)
    acc, pot = rcb.rcb_gravity_fn(xt, mt, ht, 12, 0.6, "mixed")
    loss = (acc * acc).sum() + pot.sum()
    loss.backward()
    ref = oracle.OracleTree(x, m, h)
    ref.walk(0.6)
    a, p = ref.gravity()
    ox, om = ref.gravity_backward(2 * a, np.ones(N))
    ex, _ = _close(xt.grad.cpu().numpy(), ox, 1e-5)
    em, _ = _close(mt.grad.cpu().numpy(), om, 1e-5)
    assert ex < 1e-5 and em < 1e-5, (ex, em)
