"""Failure detection on the GPU without a fault: the bounded waits of the kernels
(look-back record, bulk-copy mbarrier) are made to run out on purpose by
lb_selftest; each must give up, report LB_ERR_TIMEOUT, and leave the context
usable for the next SpMV."""
import numpy as np
import pytest

import oracle
import workloads as W
from helpers import assert_within_bound, to_dev

pytestmark = pytest.mark.gpu

LB_ERR_TIMEOUT = 5


@pytest.fixture(scope="module")
def lbmod():
    import paper_2301_04792_gb300 as lb
    lb.build()
    return lb


def test_bounded_waits_give_up_and_context_survives(lbmod):
    from paper_2301_04792_gb300 import _lib
    lib = _lib.load()
    for which in (1, 2):
        assert lib.lb_selftest(which, None) == LB_ERR_TIMEOUT, which
        assert b"gave up as designed" in lib.lb_last_error()
    m = W.powerlaw(3000, 3000, 60_000, lmax=3000, plant_long=False, seed=4)
    x = W.x_for(m)
    y64, b = oracle.spmv(m.rp, m.ci, m.v, x)
    rp, ci, v, xd = to_dev(m.rp, m.ci, m.v, x)
    for var in (0, 2, 3):
        plan = lbmod.Plan(rp, m.nnz, "merge_path", mp_variant=var)
        assert_within_bound(plan.spmv(ci, v, xd).cpu().numpy(), y64, b, f"after self-test, variant {var}")
        plan.status()  # no timeout recorded by a normal run
