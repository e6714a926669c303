"""The tensor-pipe rate probe (nav_mma_probe): argument checks on the host,
and on the GPU that every CTA reports a time, no bounded wait gives up, and
commits that drain the pipe after every MMA cost more than none.  The probe
measures what sets the weight staging of the actor inside the step kernel
(Sec. 2.3 actor, evaluated in the Eq. 7 loop)."""
import ctypes as C

import pytest

from paper_2606_15846_b300 import flashnav as fn


def test_probe_rejects_bad_arguments():
    L = fn.load()
    ns = (C.c_uint64 * 4)()
    st = (C.c_int * 1)()
    bad = [
        (8, 16, 0, 0, 1),        # N below 16
        (24, 16, 0, 0, 1),       # N not a multiple of 16
        (272, 16, 0, 0, 1),      # N above 256
        (128, 0, 0, 0, 1),       # no MMA
        (128, 1 << 21, 0, 0, 1),  # too many MMAs
        (128, 16, -1, 0, 1),     # negative commit interval
        (128, 16, 4, 2, 1),      # wait flag not 0 or 1
        (128, 16, 0, 0, 0),      # no CTA
        (128, 16, 0, 0, 2048),   # too many CTAs
    ]
    for n, n_mma, every, wait, blocks in bad:
        rc = L.nav_mma_probe(n, n_mma, every, wait, blocks, C.cast(ns, C.c_void_p),
                             C.cast(st, C.c_void_p), None)
        assert rc == -1, (n, n_mma, every, wait, blocks)  # NAV_E_INVAL
    assert L.nav_mma_probe(128, 16, 0, 0, 1, None, C.cast(st, C.c_void_p), None) == -1
    assert L.nav_mma_probe(128, 16, 0, 0, 1, C.cast(ns, C.c_void_p), None, None) == -1


@pytest.mark.gpu
def test_probe_times_every_cta_and_commits_cost_time():
    import torch
    ns = torch.zeros(8, dtype=torch.int64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    res = {}
    for every, wait in ((0, 0), (4, 1), (1, 0)):
        fn.mma_probe(128, 512, every, wait, ns, status)
        fn.mma_probe(128, 512, every, wait, ns, status)
        torch.cuda.synchronize()
        t = ns.cpu().numpy()
        assert (t > 0).all(), (every, wait, t)
        res[(every, wait)] = float(t.max())
    assert int(status.item()) == 0
    # a commit (and a wait) after every few MMAs can only add time
    assert res[(1, 0)] > res[(0, 0)]
    assert res[(4, 1)] > res[(0, 0)]
