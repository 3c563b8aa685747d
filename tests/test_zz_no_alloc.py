"""The allocation-free CIC deposit (sim_deposit_cic_static) against sim_deposit_cic.

Some callers cannot allocate device memory: code running while a framework's caching
allocator holds the device memory, deployments with a fixed device footprint, and
latency-critical loops that cannot take cudaFree's synchronisation. For them the library
keeps the deposit's fixed-point accumulator in a static device array. This test calls both
entry points through the C ABI on the same inputs, twice in a row with different particles
(the shared array keeps the first call's contents and must be cleared by the second), and
also checks that oversize grids are refused. It is named to be collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth
from gpu_helpers import f32, lib, need_gpu

pytestmark = pytest.mark.gpu


def _deposit(L, fn, s, vals, n, box, grid0=None):
    grid = torch.zeros(n, n, n, dtype=torch.float32, device="cuda") if grid0 is None else grid0.clone()
    st = fn(ctypes.c_void_p(s.data_ptr()),
            None if vals is None else ctypes.c_void_p(vals.data_ptr()), n, box,
            ctypes.c_void_p(grid.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, L.sim_last_error(None)
    return grid


def test_static_deposit_matches_allocating_deposit_twice():
    need_gpu()
    dh = lib()
    L = dh.lib
    for call, (n, box, seed) in enumerate(((32, 32.0, 1), (24, 30.0, 2))):
        s, _ = f32(synth.displacements(n, seed, 2.0 * box / n))
        vals, _ = f32(synth.rng(seed + 10).uniform(0.5, 2.0, size=n ** 3))
        want = _deposit(L, L.sim_deposit_cic, s, vals, n, box)
        got = _deposit(L, L.sim_deposit_cic_static, s, vals, n, box)
        torch.cuda.synchronize()
        # the same fixed-point arithmetic: the deposit tests' tolerance, met exactly here
        assert (got - want).abs().max().item() <= 2e-6 * want.abs().max().item(), call
        assert torch.equal(got, want), call


def test_static_deposit_accumulates_and_takes_the_largest_grid():
    """The output grid is accumulated (grid += deposit), and n = 128 (exactly the static
    array's SIM_DEPOSIT_STATIC_MAX_CELLS) is accepted and matches the allocating deposit."""
    need_gpu()
    dh = lib()
    L = dh.lib
    for n, box in ((20, 20.0), (128, 128.0)):
        s, _ = f32(synth.displacements(n, 30 + n, 1.5 * box / n))
        grid0, _ = f32(synth.field(n, 31 + n))
        want = _deposit(L, L.sim_deposit_cic, s, None, n, box, grid0)
        got = _deposit(L, L.sim_deposit_cic_static, s, None, n, box, grid0)
        fresh = _deposit(L, L.sim_deposit_cic_static, s, None, n, box)
        torch.cuda.synchronize()
        assert torch.equal(got, want), n
        # accumulated, not overwritten: the result is grid0 plus the deposit alone
        assert (got - (grid0 + fresh)).abs().max().item() <= 1e-6 * got.abs().max().item(), n
        assert abs(fresh.double().sum().item() / n ** 3 - 1.0) < 1e-6   # unit mass per particle


def test_static_deposit_rejects_oversize_grid():
    need_gpu()
    dh = lib()
    L = dh.lib
    n = 129
    s = torch.zeros(3, n ** 3, dtype=torch.float32, device="cuda")
    grid = torch.zeros(n ** 3, dtype=torch.float32, device="cuda")
    st = L.sim_deposit_cic_static(ctypes.c_void_p(s.data_ptr()), None, n, float(n),
                                  ctypes.c_void_p(grid.data_ptr()), None)
    assert st == dh._lib.SIM_EINVAL
    assert b"static scratch" in L.sim_last_error(None)
