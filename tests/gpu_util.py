"""Helpers for the GPU parity tests: device detection, the library context,
and numpy <-> torch moves.  The CUDA path is reached only through the C-ABI
binding paper_1104_3870_gb300.laph."""
import functools

import numpy as np
import pytest


def has_gpu():
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


@functools.lru_cache(maxsize=1)
def lib():
    from paper_1104_3870_gb300 import build
    build.build()
    from paper_1104_3870_gb300 import laph
    return laph


@functools.lru_cache(maxsize=1)
def context():
    return lib().Context(0)


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


def empty(shape, dtype):
    import torch
    return torch.empty(shape, dtype=dtype, device="cuda")


def rel_err(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@functools.lru_cache(maxsize=2)
def oracle_links(workload):
    """The oracle's own stout smearing of a workload's seeded field (4D links, 3D links);
    cached because it takes about a minute at 16^3 x 32."""
    import synth
    from oracle import gauge
    wl = synth.WORKLOADS[workload]
    return gauge.prepare_links(wl.gauge(), wl.rho_stout, wl.n_stout4d, wl.n_stout3d)


requires_gpu = pytest.mark.skipif(not has_gpu(), reason="needs a CUDA GPU")
