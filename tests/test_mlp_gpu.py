"""GPU tests of the tensor-core MLP kernels against the FP64 reference.

The GEMM computes C = act(A B^T + bias) with BF16 inputs and FP32
accumulation; the reference is the binary64 product of the same BF16
values, so the only error is FP32 accumulation order (bounded by
K * 2^-23 * sum |a||b|) and, for BF16 outputs, one BF16 rounding.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_15846_b300 import flashnav
    return flashnav, torch


def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


@pytest.mark.parametrize("m,n,k,lda,act", [
    (128, 256, 64, 64, 0), (4096, 256, 364, 368, 1), (200, 40, 100, 104, 0),
    (1, 4, 256, 256, 0), (333, 256, 256, 256, 1), (4096, 2, 256, 256, 0),
    (129, 17, 16, 16, 1), (4096, 256, 256, 264, 0)])
def test_gemm_matches_fp64(env, m, n, k, lda, act):
    flashnav, torch = env
    lib = flashnav.load()
    g = torch.Generator(device="cuda").manual_seed(m * 7 + n * 3 + k)
    A = torch.randn(m, lda, device="cuda", generator=g).to(torch.bfloat16)
    ldb = (k + 7) // 8 * 8
    B = torch.randn(n, ldb, device="cuda", generator=g).to(torch.bfloat16)
    bias = torch.randn(n, device="cuda", generator=g)
    c32 = torch.full((m, n), float("nan"), device="cuda")
    c16 = torch.zeros(m, n, dtype=torch.bfloat16, device="cuda")
    c16t = torch.zeros(n, m, dtype=torch.bfloat16, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = lib.nav_gemm_bf16(_p(A), lda, _p(B), ldb, m, n, k, _p(bias), act, _p(c32), n, _p(c16), n,
                           _p(c16t), m, _p(status), None)
    assert rc == 0
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    a64 = A[:, :k].double().cpu().numpy()
    b64 = B[:, :k].double().cpu().numpy()
    ref = a64 @ b64.T + bias.double().cpu().numpy()
    if act:
        ref = np.where(ref > 0, ref, 0.01 * ref)
    bound = (np.abs(a64) @ np.abs(b64).T) * (k * 2.0 ** -23) + 1e-6
    got = c32.double().cpu().numpy()
    assert np.isfinite(got).all()
    assert (np.abs(got - ref) <= bound + 1e-5).all(), np.abs(got - ref).max()
    g16 = c16.double().cpu().numpy()
    assert np.abs(g16 - got).max() <= np.abs(got).max() * 2.0 ** -8 + 1e-6
    assert torch.equal(c16t, c16.t())
