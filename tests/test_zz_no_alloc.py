"""The allocation-free neighbour-offsets entry point against rcb_neighbours.

rcb_neighbour_offsets_noalloc serves callers that cannot allocate device memory when they need
neighbour offsets (code recorded into a CUDA graph, or hosts whose memory manager owns the
device).  It keeps its scratch in a fixed static array inside the library.  This test calls it
through the C ABI twice in a row, on two different trees, and checks each result against the
offsets of the existing rcb_neighbours entry point.  The offsets are integers, so they must be
identical.  The second call runs on a smaller tree, so stale scratch from the first call would
show up.  This file is collected last so that a run stopping at the first failure has run every
other test before it.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _tree(kind, n, seed):
    import torch

    import paper_1108_0028_gb300 as rcb
    x, m, h = synth.make_particles(kind, n, seed, "loguniform10")
    dev = torch.device("cuda:0")
    xt, mt, ht = (torch.from_numpy(a).to(dev) for a in (x, m, h))
    return rcb.RCBTree(xt, mt, ht, theta=0.7)


def test_noalloc_offsets_match_rcb_neighbours_twice():
    import torch

    import paper_1108_0028_gb300 as rcb
    lib = rcb.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for kind, n, seed in (("plummer", 30000, 11), ("sphere", 7000, 12)):
        tree = _tree(kind, n, seed)
        ref = torch.empty(n + 1, dtype=torch.int64, device="cuda:0")
        need_ref = ctypes.c_int64(-1)
        st = lib.rcb_neighbours(tree.handle, ctypes.c_void_p(ref.data_ptr()), None, 0, ctypes.byref(need_ref), stream)
        assert st == rcb.RCB_OK
        out = torch.full((n + 1,), -7, dtype=torch.int64, device="cuda:0")
        need = ctypes.c_int64(-1)
        st = lib.rcb_neighbour_offsets_noalloc(tree.handle, ctypes.c_void_p(out.data_ptr()), ctypes.byref(need),
                                               stream)
        assert st == rcb.RCB_OK
        assert need.value == need_ref.value > 0
        assert np.array_equal(out.cpu().numpy(), ref.cpu().numpy())
        tree.free()


def test_noalloc_rejects_missing_arguments():
    import paper_1108_0028_gb300 as rcb
    need = ctypes.c_int64(0)
    assert rcb.lib().rcb_neighbour_offsets_noalloc(None, None, ctypes.byref(need), None) == rcb.RCB_ERR_ARG
