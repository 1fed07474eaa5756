"""Parity at the full sizes of the benchmark configurations, on sampled sinks.

The GPU runs each configuration whole, in the launch configuration bench.py times (the fused
forces + neighbour entry point in the mixed form, then the FP64 form on the same tree); the
oracle builds the same tree on the host and walks a seeded sample of sinks, whose interaction
lists, neighbour rows and forces are compared.  The tree topology is compared for every
particle.
"""
import numpy as np
import pytest

import oracle
import synth
from test_gpu_forces import (FP64_P999, FP64_RMS, MIXED_P999, MIXED_RMS, _gpu, _particles_of, _sample_sinks,
                             rel_errors)

pytestmark = pytest.mark.gpu

FULL = [
    # kind, N, masses, theta, config, case
    ("sphere", 4194304, "loguniform10", 0.7, 3, 0),   # the headline workload
    ("sphere", 4194304, "loguniform10", 0.5, 3, 2),
    ("plummer", 4194304, "loguniform10", 0.5, 3, 1),
    ("plummer", 4194304, "loguniform10", 0.7, 3, 3),  # long far lists: the paired walk at full size
    ("plummer", 1000000, "equal", 0.5, 2, 0),
    ("cube", 10000000, "equal", 0.7, 4, 0),
    ("plummer", 10000000, "equal", 0.7, 4, 1),        # the Plummer half of the scaling sweep
    ("cube", 100000000, "equal", 0.7, 4, 2),          # the largest size of the scaling sweep
]


@pytest.mark.parametrize("kind,N,mass,theta,cfg,case", FULL)
def test_full_size_sampled_parity(kind, N, mass, theta, cfg, case):
    import paper_1108_0028_gb300 as rcb
    x, m, h = synth.make_particles(kind, N, synth.seed_for(cfg, case), mass)
    tree = rcb.RCBTree(*_gpu(x, m, h), n_ll=12, theta=theta, precision="mixed")
    acc, pot, off, idx = tree.gravity_neighbours()
    acc, pot, off, idx = acc.cpu().numpy(), pot.cpu().numpy(), off.cpu().numpy(), idx.cpu().numpy()
    g_lists = tree.export_lists()
    leaf_of = tree.export_topology()["leaf_of"]
    tree.set_precision("fp64")
    acc64, _ = tree.gravity()
    acc64 = acc64.cpu().numpy()

    ref = oracle.OracleTree(x, m, h)
    assert np.array_equal(leaf_of, ref.leaf_of())
    sinks = _sample_sinks(ref, 200, 100 * cfg + case)
    ref.walk(theta, sinks)
    o_lists = ref.lists()
    for j in sinks:
        a, b = g_lists["near_off"][j], g_lists["near_off"][j + 1]
        c, d = o_lists["near_off"][j], o_lists["near_off"][j + 1]
        assert sorted(zip(g_lists["near_ids"][a:b].tolist(), g_lists["near_reach"][a:b].tolist())) == \
            sorted(zip(o_lists["near_ids"][c:d].tolist(), o_lists["near_reach"][c:d].tolist())), j
        a, b = g_lists["far_off"][j], g_lists["far_off"][j + 1]
        c, d = o_lists["far_off"][j], o_lists["far_off"][j + 1]
        assert sorted(g_lists["far_ids"][a:b].tolist()) == sorted(o_lists["far_ids"][c:d].tolist()), j
    parts = _particles_of(ref, sinks)
    ro, ri = ref.neighbours()
    for p in parts:
        assert np.array_equal(idx[off[p]:off[p + 1]], ri[ro[p]:ro[p + 1]]), p
    oa, _ = ref.gravity()
    e_mixed = rel_errors(acc[parts], oa[parts])
    e_fp64 = rel_errors(acc64[parts], oa[parts])
    print(f"{kind} N={N}: {len(sinks)} sinks, {len(parts)} particles; mixed rms {np.sqrt(np.mean(e_mixed ** 2)):.2e} "
          f"p99.9 {np.quantile(e_mixed, 0.999):.2e}; fp64 rms {np.sqrt(np.mean(e_fp64 ** 2)):.2e}")
    assert np.sqrt(np.mean(e_fp64 ** 2)) < FP64_RMS and np.quantile(e_fp64, 0.999) < FP64_P999
    assert np.sqrt(np.mean(e_mixed ** 2)) < MIXED_RMS and np.quantile(e_mixed, 0.999) < MIXED_P999
