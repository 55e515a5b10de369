"""Host-side fault injection (the paper itself has no failure handling): an allocation made to
fail on the host makes the call return UF_ENOMEM and leaves none of its allocations behind, and
the hook disarms itself after firing.  A host-only operator (device -1) makes one allocation, the
operator object, so these tests need no GPU."""
import pytest

import workloads
from paper_2404_07911_gb300 import (UnfittedError, UnfittedOperator, debug_fail_allocation,
                                    debug_live_allocations)
from paper_2404_07911_gb300.binding import UF_ENOMEM

CFG = workloads.small(p=1, N=4, dim=2)


@pytest.fixture(autouse=True)
def _disarm():
    yield
    debug_fail_allocation(-1)


def test_operator_allocation_failure_leaves_nothing():
    base = debug_live_allocations()
    debug_fail_allocation(0)
    with pytest.raises(UnfittedError) as ei:
        UnfittedOperator(CFG, device=-1)
    assert ei.value.status == UF_ENOMEM
    assert debug_live_allocations() == base
    op = UnfittedOperator(CFG, device=-1)  # the hook fired once and is disarmed
    assert debug_live_allocations() == base + 1
    op.close()
    assert debug_live_allocations() == base


def test_hook_counts_allocations_and_can_be_disarmed():
    base = debug_live_allocations()
    debug_fail_allocation(1)
    op = UnfittedOperator(CFG, device=-1)  # the first allocation succeeds
    with pytest.raises(UnfittedError) as ei:
        UnfittedOperator(CFG, device=-1)  # the second fails
    assert ei.value.status == UF_ENOMEM
    op.close()
    debug_fail_allocation(3)
    debug_fail_allocation(-1)
    ops = [UnfittedOperator(CFG, device=-1) for _ in range(5)]
    assert debug_live_allocations() == base + 5
    for o in ops:
        o.close()
    assert debug_live_allocations() == base
