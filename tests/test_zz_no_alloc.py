"""fmm_evaluate_noalloc: the uniform-octree FMM for callers that cannot
allocate device memory -- programs that give all device memory to their own
pool allocator up front, or that cannot afford the device-wide
synchronisation cudaMalloc/cudaFree may cause in the middle of a time step.

The entry point works in one fixed __device__ array and must return what the
plan-based fmm_evaluate returns.  This file is collected last on purpose, so
a run that stops at its first failure has already run every other test; it
also passes on its own in a fresh process (the first call does the set-up).
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1811_06332_gb300 import inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
MAX_N = 65536


@pytest.fixture(scope="module")
def F():
    import __graft_entry__ as g
    g.build()
    from paper_1811_06332_gb300 import fmm
    return fmm


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _noalloc(F, p, basis, depth, X, out):
    s = torch.cuda.current_stream().cuda_stream
    return F.lib().fmm_evaluate_noalloc(p, basis, depth, X[0].numel(), *[t.data_ptr() for t in X],
                                        *[out[k].data_ptr() for k in range(4)], s)


def test_noalloc_matches_fmm_evaluate_twice_in_a_row(F):
    # two calls in a row with different sizes, orders and bases, each checked
    # against fmm_evaluate with the same tolerance as the other FP64 tests
    cases = [(4, 0, 3, 4096, 1), (6, 1, 3, 20000, 2)]
    free = []
    for p, basis, depth, n, seed in cases:
        x, y, z = inputs.uniform_cube(n, seed)
        q = inputs.masses_open_unit(n, seed)
        X = [_dev(a) for a in (x, y, z, q)]
        out = torch.full((4, n), 3.0, dtype=torch.float64, device=DEV)
        plan = F.Plan(p=p, basis=basis, prec=F.FP64, depth=depth)
        pot, acc = plan.evaluate(*X)
        torch.cuda.synchronize()
        plan.close()
        rc = _noalloc(F, p, basis, depth, X, out)
        assert rc == F.OK, F.lib().fmm_last_error(None)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        ep = (torch.linalg.norm(out[0] - pot) / torch.linalg.norm(pot)).item()
        ea = (torch.linalg.norm(out[1:] - acc) / torch.linalg.norm(acc)).item()
        assert ep < 1e-12 and ea < 1e-12, (p, basis, ep, ea)


def test_noalloc_repeat_and_limits(F):
    n = 5000
    x, y, z = inputs.uniform_cube(n, 9)
    q = inputs.masses_open_unit(n, 9)
    X = [_dev(a) for a in (x, y, z, q)]
    o1 = torch.zeros((4, n), dtype=torch.float64, device=DEV)
    o2 = torch.zeros((4, n), dtype=torch.float64, device=DEV)
    assert _noalloc(F, 5, 1, 3, X, o1) == F.OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    assert _noalloc(F, 5, 1, 3, X, o2) == F.OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0    # nothing was allocated
    assert torch.equal(o1, o2)
    # sizes beyond the stated maxima are rejected before any work is queued
    L = F.lib()
    big = MAX_N + 1
    assert L.fmm_evaluate_noalloc(4, 0, 3, big, *[X[0].data_ptr()] * 8, None) == F.ERR_ARG
    assert b"FMM_NOALLOC_MAX_N" in L.fmm_last_error(None)
    assert L.fmm_evaluate_noalloc(7, 0, 3, n, *[X[0].data_ptr()] * 8, None) == F.ERR_ARG
    assert L.fmm_evaluate_noalloc(4, 0, 4, n, *[X[0].data_ptr()] * 8, None) == F.ERR_ARG
