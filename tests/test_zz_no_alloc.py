"""nav_step_host_noalloc: the host-buffer step for callers that may not
allocate device memory after start-up (a control loop or embedded process
that fixes its GPU memory once, or an application whose allocator must own
every allocation).  It stages through a fixed array inside the library
instead of the buffers nav_step_host allocates on first use; its results must
be the ones nav_step_host gives for the same handle state.

Kept in its own file, collected last, so that a run stopping at the first
failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2606_15846_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fn():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2606_15846_b300 import flashnav
    return flashnav


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _buffers(sim, want_final):
    n = sim.obs_size
    return (np.zeros(n, np.float32), np.zeros(sim.n_envs, np.float32),
            np.zeros(sim.n_envs, np.uint8), np.zeros(n, np.float32) if want_final else None)


@pytest.mark.parametrize("want_final", [False, True])
def test_no_alloc_step_matches_step_host(fn, want_final):
    lib = fn.load()
    wl = W.config_throughput(n_envs=1024, n_maps=4)
    ref = fn.NavSim.from_workload(wl)   # driven by nav_step_host
    sim = fn.NavSim.from_workload(wl)   # driven by nav_step_host_noalloc
    ref.reset(31)
    sim.reset(31)
    acts = W.uniform_actions(31, 2, wl.n_envs)
    off = sim.obs_offsets
    for t in range(2):  # two calls in a row share the fixed staging array
        a = np.ascontiguousarray(acts[t])
        ro, rr, rd, rf = _buffers(ref, want_final)
        ref.step_host(a, ro, rr, rd, rf)
        so, sr, sd, sf = _buffers(sim, want_final)
        sim._bind_stream()
        rc = lib.nav_step_host_noalloc(sim._h, _ptr(a), _ptr(so), _ptr(sr), _ptr(sd), _ptr(sf))
        assert rc == 0, lib.nav_last_error(sim._h)
        assert np.array_equal(sd, rd)
        assert np.abs(sr - rr).max() <= 1e-5
        assert np.abs(so - ro).max() <= 1e-4
        if want_final:
            ended = np.flatnonzero(sd & 3)
            for e in ended:
                assert np.abs(sf[off[e]:off[e + 1]] - rf[off[e]:off[e + 1]]).max() <= 1e-4
            live = np.ones(wl.n_envs, bool)
            live[ended] = False
            for e in np.flatnonzero(live)[:64]:
                assert not sf[off[e]:off[e + 1]].any()


def test_no_alloc_rejects_handles_beyond_its_buffer(fn):
    lib = fn.load()
    wl = W.config_small(n_envs=8192)
    wl.env_beams[:] = 360  # 8192 x 364 floats of obs: more than the fixed 8 MiB
    sim = fn.NavSim.from_workload(wl)
    sim.reset(1)
    a = np.zeros((wl.n_envs, 2), np.float32)
    o, r, d, _ = _buffers(sim, False)
    sim._bind_stream()
    rc = lib.nav_step_host_noalloc(sim._h, _ptr(a), _ptr(o), _ptr(r), _ptr(d), None)
    assert rc == -1
    assert b"staging bytes" in lib.nav_last_error(sim._h)


def _noalloc_step(lib, sim, acts, want_final):
    o, r, d, f = _buffers(sim, want_final)
    sim._bind_stream()
    rc = lib.nav_step_host_noalloc(sim._h, _ptr(np.ascontiguousarray(acts)), _ptr(o), _ptr(r),
                                   _ptr(d), _ptr(f))
    assert rc == 0, lib.nav_last_error(sim._h)


def test_no_alloc_calls_allocate_no_device_memory(fn):
    """After one warm-up call on the device (start-up: under lazy module
    loading that call places the fixed array on the device), a fresh handle's
    calls leave the device's free memory unchanged, with and without final
    observations.  The same measurement sees nav_step_host's first call on a
    fresh handle allocate its staging buffers."""
    import torch
    lib = fn.load()
    wl = W.config_throughput(n_envs=1024, n_maps=4)
    acts = W.uniform_actions(7, 6, wl.n_envs)
    warm = fn.NavSim.from_workload(wl)
    warm.reset(3)
    _noalloc_step(lib, warm, acts[0], True)
    sim = fn.NavSim.from_workload(wl)  # a fresh handle
    sim.reset(5)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for t in range(4):
        _noalloc_step(lib, sim, acts[t], t % 2 == 1)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0, "nav_step_host_noalloc allocated device memory"
    # contrast: nav_step_host allocates on its first call on a fresh handle
    other = fn.NavSim.from_workload(wl)
    other.reset(5)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    o, r, d, f = _buffers(other, True)
    other.step_host(np.ascontiguousarray(acts[0]), o, r, d, f)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] < free1
