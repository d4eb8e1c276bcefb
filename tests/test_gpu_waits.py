"""Failure path of the persistent batched kernel's bounded waits, tested
without a GPU fault.

A task of the batch waits for the tasks it depends on with a bounded spin
(a device-time limit and an iteration cap). rr_debug_wait_probe runs that
same wait on a counter nothing ever increments: it must give up after its
limit with RR_ETIMEDOUT (or at once when the batch's abort flag is set), and
the context must stay usable -- a query afterwards still matches the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2010_08423_gb300 import capi
from paper_2010_08423_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_wait_on_a_flag_nothing_sets_times_out():
    capi.load()
    st, ns = capi.rr_debug_wait_probe(2_000_000)
    assert st == capi.RR_ETIMEDOUT
    assert 2_000_000 <= ns < 200_000_000


def test_abort_flag_ends_the_wait_at_once():
    st, ns = capi.rr_debug_wait_probe(2_000_000_000, abort_preset=True)
    assert st == capi.RR_ETIMEDOUT
    assert ns < 1_000_000


def test_context_usable_after_timed_out_waits():
    oracle.build()
    for _ in range(3):
        st, _ = capi.rr_debug_wait_probe(1_000_000)
        assert st == capi.RR_ETIMEDOUT
    g = W.uniform(600, 6_000, 15, 0, 4, 17)
    with capi.Graph(g) as G:
        _, w = G.reach(3, 5, 11)
        assert np.array_equal(w, oracle.sieve(g, 3, 5, 11))


def test_probe_argument_errors():
    with pytest.raises(capi.RRError) as ei:
        capi.rr_debug_wait_probe(20_000_000_000)
    assert ei.value.status == capi.RR_EINVAL
