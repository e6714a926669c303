"""The random-gather rate probe (nav_gather_probe): its checksums against a
numpy restatement of the documented generator and tables, and its argument
checks.  The probe measures the memory ceiling of the beam traversal
(Sec. 2.2.1), so it must read exactly the bytes its contract names."""
import ctypes as C

import numpy as np
import pytest

from paper_2606_15846_b300 import flashnav as fn

M32 = 0xFFFFFFFF


def expected_sums(table: np.ndarray, n_blocks: int, iters: int) -> np.ndarray:
    nbytes = table.size
    sh = 32 - (nbytes.bit_length() - 1)
    g = np.arange(n_blocks * 256, dtype=np.uint64)
    c = np.arange(8, dtype=np.uint64)
    s = ((g[:, None] * 8 + c[None, :]) * 2654435761 + 0x9E3779B9) & M32
    acc = np.zeros(n_blocks * 256, dtype=np.uint64)
    t = table.astype(np.uint64)
    for _ in range(iters):
        s = (s * 1664525 + 1013904223) & M32
        acc += t[s >> np.uint64(sh)].sum(axis=1)
    return (acc.reshape(n_blocks, 256).sum(axis=1) & M32).astype(np.uint32)


def shared_table(nbytes: int) -> np.ndarray:
    j = np.arange(nbytes, dtype=np.uint64)
    return (((j * 2654435761) & M32) >> 24).astype(np.uint8)


def test_probe_rejects_bad_arguments():
    L = fn.load()
    sums = (C.c_uint32 * 4)()
    bad = [
        (2, None, 4096, 1, 1),        # unknown table kind
        (0, None, 3000, 1, 1),        # not a power of two
        (0, None, 512, 1, 1),         # below 1024 bytes
        (0, None, 1 << 18, 1, 1),     # larger than a CTA's shared memory
        (1, None, 4096, 1, 1),        # global table missing
        (0, None, 4096, 0, 1),        # no CTA
        (0, None, 4096, 1, -1),       # negative iteration count
    ]
    for where, table, nbytes, n_blocks, iters in bad:
        rc = L.nav_gather_probe(where, table, nbytes, n_blocks, iters, C.cast(sums, C.c_void_p),
                                None)
        assert rc == -1, (where, nbytes, n_blocks, iters)  # NAV_E_INVAL
    assert L.nav_gather_probe(0, None, 4096, 1, 1, None, None) == -1


@pytest.mark.gpu
@pytest.mark.parametrize("nbytes,n_blocks,iters", [(4096, 3, 5), (1 << 17, 2, 3)])
def test_shared_probe_reads_the_documented_bytes(nbytes, n_blocks, iters):
    import torch
    sums = torch.zeros(n_blocks, dtype=torch.int32, device="cuda")
    fn.gather_probe(0, None, nbytes, n_blocks, iters, sums)
    torch.cuda.synchronize()
    got = sums.cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(got, expected_sums(shared_table(nbytes), n_blocks, iters))


@pytest.mark.gpu
@pytest.mark.parametrize("nbytes,n_blocks,iters", [(1024, 1, 2), (1 << 20, 4, 7)])
def test_global_probe_reads_the_documented_bytes(nbytes, n_blocks, iters):
    import torch
    rng = np.random.default_rng(nbytes)
    host = rng.integers(0, 256, size=nbytes, dtype=np.uint8)
    table = torch.from_numpy(host).cuda()
    sums = torch.zeros(n_blocks, dtype=torch.int32, device="cuda")
    fn.gather_probe(1, table, nbytes, n_blocks, iters, sums)
    torch.cuda.synchronize()
    got = sums.cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(got, expected_sums(host, n_blocks, iters))
