"""fmm_evaluate_noalloc: the uniform-octree FMM for callers that cannot
allocate device memory -- programs that give all device memory to their own
pool allocator up front, or that cannot afford the device-wide
synchronisation cudaMalloc/cudaFree may cause in the middle of a time step.

The entry point works in one fixed __device__ array and must agree with the
plan-based fmm_evaluate (FP64, 1e-12 relative, the tolerance of the other
FP64 tests).  This file is collected last on purpose, so a run that stops at
its first failure has already run every other test; it also passes on its
own in a fresh process (the first call does the set-up).
"""
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


def _noalloc(F, p, basis, depth, X, out, stream=None):
    s = (stream or torch.cuda.current_stream()).cuda_stream
    return F.lib().fmm_evaluate_noalloc(p, basis, depth, X[0].numel(), *[t.data_ptr() for t in X],
                                        *[out[k].data_ptr() for k in range(4)], s)


def _inputs(n, seed):
    x, y, z = inputs.uniform_cube(n, seed)
    q = inputs.masses_open_unit(n, seed)
    return [_dev(a) for a in (x, y, z, q)]


def _reference(F, p, basis, depth, X):
    plan = F.Plan(p=p, basis=basis, prec=F.FP64, depth=depth)
    pot, acc = plan.evaluate(*X)
    torch.cuda.synchronize()
    plan.close()
    return pot, acc


def _rel(a, b):
    den = torch.linalg.norm(b)
    return (torch.linalg.norm(a - b) / den).item() if den > 0 else torch.linalg.norm(a).item()


def test_noalloc_matches_fmm_evaluate_twice_in_a_row(F):
    # calls in a row with different sizes, orders, bases and depths (depth 1
    # and 2 have no M2L level to run, or no L2L), each compared with
    # fmm_evaluate; a call that changes (p, basis) rebuilds the matrices in
    # the fixed array and must leave the device's free memory unchanged
    cases = [(4, 0, 3, 4096, 1), (6, 1, 3, 20000, 2), (3, 1, 2, 3000, 3), (5, 0, 1, 777, 4)]
    # The first call in a process may load the library's device module that
    # holds the fixed array (lazy module loading), which takes the array's
    # own memory; every call after it must allocate nothing.
    w = _inputs(64, 30)
    assert _noalloc(F, 2, 1, 1, w, torch.zeros((4, 64), dtype=torch.float64, device=DEV)) == F.OK
    torch.cuda.synchronize()
    for p, basis, depth, n, seed in cases:
        X = _inputs(n, seed)
        pot, acc = _reference(F, p, basis, depth, X)
        out = torch.full((4, n), 3.0, dtype=torch.float64, device=DEV)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        rc = _noalloc(F, p, basis, depth, X, out)
        assert rc == F.OK, F.lib().fmm_last_error(None)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, (p, basis, depth)   # nothing was allocated
        ep, ea = _rel(out[0], pot), _rel(out[1:], acc)
        assert ep < 1e-12 and ea < 1e-12, (p, basis, depth, ep, ea)


def test_noalloc_empty_input(F):
    e = torch.zeros((0,), dtype=torch.float64, device=DEV)
    out = torch.zeros((4, 0), dtype=torch.float64, device=DEV)
    for depth in (0, 3):
        assert _noalloc(F, 4, 1, depth, [e, e, e, e], out) == F.OK, F.lib().fmm_last_error(None)
    torch.cuda.synchronize()


def test_noalloc_repeat_and_limits(F):
    n = 5000
    X = _inputs(n, 9)
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


def test_noalloc_rebuild_refused_while_capturing(F):
    # a call that would rebuild the matrices (another p) while its stream is
    # being captured returns FMM_ERR_STATE and queues nothing
    n = 2000
    X = _inputs(n, 12)
    out = torch.zeros((4, n), dtype=torch.float64, device=DEV)
    assert _noalloc(F, 4, 0, 2, X, out) == F.OK
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    pad = torch.zeros(4, device=DEV)
    with torch.cuda.graph(g, stream=s, capture_error_mode="thread_local"):
        pad.add_(1.0)
        rc = _noalloc(F, 5, 0, 2, X, out, stream=s)
    assert rc == F.ERR_STATE
    assert b"captured" in F.lib().fmm_last_error(None)
    torch.cuda.synchronize()
    # the state is unchanged: the next call at the held (p, basis) still agrees
    pot, acc = _reference(F, 4, 0, 2, X)
    assert _noalloc(F, 4, 0, 2, X, out) == F.OK
    torch.cuda.synchronize()
    assert _rel(out[0], pot) < 1e-12 and _rel(out[1:], acc) < 1e-12
