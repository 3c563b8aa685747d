"""Shared helpers of the GPU parity tests (imported by tests marked gpu only)."""
import numpy as np
import pytest
import torch

import synth


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2502_02294_gb300 as dh
    return dh


def rel_l2(got, want):
    got = torch.as_tensor(got).double().cpu()
    want = torch.as_tensor(want).double().cpu()
    den = want.norm().item()
    return (got - want).norm().item() / (den if den > 0 else 1.0)


def f32(x):
    """Round an array to float32 and return (cuda float32 tensor, cpu float64 tensor)."""
    a = np.asarray(x, dtype=np.float32)
    return torch.from_numpy(a.copy()).cuda(), torch.from_numpy(a.astype(np.float64))


def gas(n, seed, **kw):
    return synth.gas_state(n, seed, **kw)


def oracle_params(p):
    """oracle.sim parameter dict from a SimParams (same numbers, oracle's own names)."""
    from oracle.sim import Params
    d = Params().as_dict()
    for k in d:
        if k == "kdk_mode":
            d[k] = "fastpm" if p.kdk_mode == 0 else "plain"
        elif hasattr(p, k):
            d[k] = getattr(p, k)
    return d
