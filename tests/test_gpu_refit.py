"""GPU refit (Sec. 2.1.8) and the gradient check of the differentiation workload."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _gpu(*arrays):
    import torch
    dev = torch.device("cuda:0")
    return tuple(torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in arrays)


def test_refit_matches_oracle_refit():
    import paper_1108_0028_gb300 as rcb
    N = 6000
    x, m, h = synth.make_particles("plummer", N, 61, "loguniform10")
    x2 = synth.jitter(x, 1e-4, 62)
    m2 = m * (1.0 + 0.01 * np.random.default_rng(63).random(N))
    ref = oracle.OracleTree(x, m, h)
    ref.walk(0.6)
    ref.refit(x2, m2)
    oa, op = ref.gravity()
    tree = rcb.RCBTree(*_gpu(x, m, h), theta=0.6, precision="fp64")
    tree.refit(*_gpu(x2, m2))
    ga, gp = tree.gravity()
    e = np.linalg.norm(ga.cpu().numpy() - oa, axis=1) / np.linalg.norm(oa, axis=1)
    assert e.max() < 1e-10
    g = tree.export_topology()
    o = ref.nodes()
    live = o["count"] > 0
    live[0] = False
    assert np.array_equal(g["sums"][live], o["sums"][live])
    for k in ("com", "bmin", "bmax", "rg", "hint"):
        assert np.array_equal(g[k][live].view(np.int64), o[k][live].view(np.int64)), k


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_gradient_central_differences_config5(precision):
    # N = 262144 Plummer; loss = sum |a(x, m) - a_t|^2, a_t from positions jittered by N(0, 1e-3^2);
    # backward through the frozen tree vs central differences (step 1e-6) of the FP64 forward
    # with the same frozen tree (refit), along random directions in x and in m.
    # FP64: the two agree to the finite-difference truncation (bound 1e-6 relative).
    # Mixed: the backward is seeded with the mixed forward's residuals a - a_t; their relative
    # error is the force error (~1e-7 RMS, up to ~6e-6) over the residual size (~1e-4 of |a|
    # for a 1e-3 jitter), i.e. ~1e-3 at worst, so the bound is 1e-3.
    import torch

    import paper_1108_0028_gb300 as rcb
    N = 262144
    x, m, h = synth.make_particles("plummer", N, synth.seed_for(5), "equal")
    xt_np = synth.jitter(x, 1e-3, synth.seed_for(5, 1))
    tx, tm, th = _gpu(x, m, h)
    ttx, = _gpu(xt_np)
    target = rcb.RCBTree(ttx, tm, th, theta=0.5, precision="fp64")
    at, _ = target.gravity()
    tree = rcb.RCBTree(tx, tm, th, theta=0.5, precision=precision)
    acc, _ = tree.gravity()
    gx, gm = tree.gravity_backward(2.0 * (acc - at))
    tree.set_precision("fp64")

    def loss(xx, mm):
        tree.refit(xx, mm)
        a, _ = tree.gravity()
        return float(torch.sum((a - at) ** 2).item())

    rng = np.random.default_rng(7)
    eps = 1e-6
    for trial in range(2):
        u = rng.standard_normal((N, 3))
        u /= np.linalg.norm(u)
        ut, = _gpu(u)
        fd = (loss(tx + eps * ut, tm) - loss(tx - eps * ut, tm)) / (2 * eps)
        an = float(torch.sum(gx * ut).item())
        print(f"{precision} x-direction: analytic {an:.10e} fd {fd:.10e}")
        assert an == pytest.approx(fd, rel=1e-3 if precision == "mixed" else 1e-6)
    v = rng.standard_normal(N) * m
    v /= np.linalg.norm(v) / np.linalg.norm(m)
    vt, = _gpu(v)
    fd = (loss(tx, tm + eps * vt) - loss(tx, tm - eps * vt)) / (2 * eps)
    an = float(torch.sum(gm * vt).item())
    print(f"{precision} m-direction: analytic {an:.10e} fd {fd:.10e}")
    assert an == pytest.approx(fd, rel=1e-3 if precision == "mixed" else 1e-6)


@pytest.mark.parametrize("sigma", [1e-9, 3e-2])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_update_with_integrity_check(sigma, precision):
    # Sec. 2.1.8 time step: new positions, masses and smoothing lengths.  With a tiny move every
    # particle stays in its ll-cell, so the tree is refitted and walked again; with a large one
    # particles leave their cells and the tree is rebuilt.  Either way the result equals the
    # oracle's update (or fresh build): topology, node data, lists, neighbours, forces.
    import paper_1108_0028_gb300 as rcb
    N = 6000
    x, m, h = synth.make_particles("plummer", N, 81, "loguniform10")
    x2 = synth.jitter(x, sigma, 82)
    m2 = m * (1.0 + 0.01 * np.random.default_rng(83).random(N))
    h2 = h * (1.0 + 0.05 * np.random.default_rng(84).random(N))
    ref = oracle.OracleTree(x, m, h)
    outside = ref.update(x2, m2, h2)
    if sigma < 1e-6:
        assert outside == 0
    else:
        assert outside > 0
        ref = oracle.OracleTree(x2, m2, h2)
    ref.walk(0.6)
    tree = rcb.RCBTree(*_gpu(x, m, h), theta=0.6, precision=precision)
    rebuilt = tree.update(*_gpu(x2, m2, h2))
    assert rebuilt == (outside > 0)
    g = tree.export_topology()
    assert np.array_equal(g["leaf_of"], ref.leaf_of())
    o = ref.nodes()
    live = o["count"] > 0
    live[0] = False
    for k in ("com", "bmin", "bmax", "rg", "hint"):
        assert np.array_equal(g[k][live].view(np.int64), o[k][live].view(np.int64)), k
    gl, ol = tree.export_lists(), ref.lists()
    for j in range(ref.nleaves):
        a, b = gl["near_off"][j], gl["near_off"][j + 1]
        c, d = ol["near_off"][j], ol["near_off"][j + 1]
        assert sorted(zip(gl["near_ids"][a:b].tolist(), gl["near_reach"][a:b].tolist())) == \
            sorted(zip(ol["near_ids"][c:d].tolist(), ol["near_reach"][c:d].tolist())), j
        a, b = gl["far_off"][j], gl["far_off"][j + 1]
        c, d = ol["far_off"][j], ol["far_off"][j + 1]
        assert sorted(gl["far_ids"][a:b].tolist()) == sorted(ol["far_ids"][c:d].tolist()), j
    ro, ri = ref.neighbours()
    go, gi = tree.neighbours()
    assert np.array_equal(go.cpu().numpy(), ro) and np.array_equal(gi.cpu().numpy(), ri)
    oa, _ = ref.gravity()
    ga, _ = tree.gravity()
    e = np.linalg.norm(ga.cpu().numpy() - oa, axis=1) / np.linalg.norm(oa, axis=1)
    assert np.sqrt(np.mean(e * e)) < (1e-10 if precision == "fp64" else 2e-6)
