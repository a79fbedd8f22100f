"""The bounded waits of the tensor-core kernels give up, report and leave the
context usable (tested without a GPU fault: a wait on an mbarrier that
nothing arrives at, with a short poll limit)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1811_06332_gb300 import inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def F():
    import __graft_entry__ as g
    g.build()
    from paper_1811_06332_gb300 import fmm
    return fmm


def test_bounded_wait_gives_up_and_the_context_stays_usable(F):
    F.fmm_selftest_wait(1 << 12, 1)                    # arrived on: completes
    with pytest.raises(F.FMMError) as e:
        F.fmm_selftest_wait(1 << 12, 0)                # nothing arrives: gives up
    assert e.value.code == -5                          # FMM_ERR_TIMEOUT
    with pytest.raises(F.FMMError):
        F.fmm_selftest_wait(0, 1)                      # FMM_ERR_ARG
    F.fmm_selftest_wait(1 << 12, 1)
    # the context still runs the library's kernels correctly
    n, depth, p = 2048, 2, 4
    x, y, z = inputs.uniform_cube(n, 61)
    q = inputs.masses_open_unit(n, 61)
    plan = F.Plan(p=p, basis=F.BASIS_SYM, prec=F.FP64, depth=depth)
    pot, acc = plan.evaluate(*[torch.from_numpy(a).to(DEV) for a in (x, y, z, q)])
    plan.sync_status()
    plan.close()
    pref, aref = oracle.fmm_uniform(x, y, z, q, depth, p, 0)
    assert np.linalg.norm(acc.cpu().numpy() - aref) / np.linalg.norm(aref) < 1e-12
