"""SPH density over the neighbour CSR (next-4) against the oracle's FP64 sum."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _gpu(*arrays):
    import torch
    dev = torch.device("cuda:0")
    return tuple(torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in arrays)


@pytest.mark.parametrize("kind,N,mass", [("plummer", 6000, "loguniform10"), ("sphere", 20000, "equal"),
                                         ("cube", 30000, "loguniform10")])
def test_density_matches_oracle(kind, N, mass):
    import paper_1108_0028_gb300 as rcb
    x, m, h = synth.make_particles(kind, N, synth.seed_for(8, N), mass)
    ref = oracle.OracleTree(x, m, h)
    ref.walk(0.6)
    ro, ri = ref.neighbours()
    want = oracle.density(x, m, h, ro, ri)
    tree = rcb.RCBTree(*_gpu(x, m, h), theta=0.6)
    off, idx = tree.neighbours()
    assert np.array_equal(off.cpu().numpy(), ro) and np.array_equal(idx.cpu().numpy(), ri)
    rho = tree.density(off, idx).cpu().numpy()
    err = np.abs(rho - want) / want
    assert err.max() < 1e-6, err.max()
    # the fused pass's lists give the same density
    _, _, off2, idx2 = tree.gravity_neighbours()
    assert np.array_equal(tree.density(off2, idx2).cpu().numpy(), rho)


def test_density_after_update():
    # the density follows the tree's current positions, masses and smoothing lengths
    import paper_1108_0028_gb300 as rcb
    N = 8000
    x, m, h = synth.make_particles("sphere", N, 95, "loguniform10")
    x2 = synth.jitter(x, 1e-9, 96)
    m2 = m * (1.0 + 0.01 * np.random.default_rng(97).random(N))
    h2 = h * (1.0 + 0.05 * np.random.default_rng(98).random(N))
    tree = rcb.RCBTree(*_gpu(x, m, h), theta=0.6)
    assert not tree.update(*_gpu(x2, m2, h2))
    off, idx = tree.neighbours()
    ro, ri = oracle.brute_neighbours(x2, h2)
    assert np.array_equal(off.cpu().numpy(), ro) and np.array_equal(idx.cpu().numpy(), ri)
    want = oracle.density(x2, m2, h2, ro, ri)
    rho = tree.density(off, idx).cpu().numpy()
    assert (np.abs(rho - want) / want).max() < 1e-6
