"""The allocation-free wa-tor comparators (per-cell SOA and AOS arrays) match
the oracle, and the allocator-based form, step by step."""
import numpy as np
import pytest

import oracle as O
from paper_1809_07444_gb300 import workloads as WL
from paper_1809_07444_gb300.apps import Wator, WatorStatic

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("aos", [False, True])
@pytest.mark.parametrize("W,H,seed,steps", [(64, 64, 1, 120), (17, 9, 3, 80), (257, 129, 4, 40), (3, 3, 2, 20)])
def test_static_wator_matches_oracle(aos, W, H, seed, steps):
    k0 = WL.wator_initial(W, H, seed)
    st, ref, dyn = WatorStatic(W, H, k0, seed, aos=aos), O.Wator(W, H, k0, seed=seed), Wator(W, H, k0, seed)
    assert st.hash() == ref.hash()
    for t in range(1, steps + 1):
        st.step(1)
        ref.step(1)
        dyn.step(1)
        assert st.hash() == ref.hash(), "step %d" % t
        if t % 10 == 0 or t == steps:
            f, s = st.dump()
            fr, sr = ref.dump()
            assert np.array_equal(f, fr) and np.array_equal(s, sr), "step %d" % t
            assert np.array_equal(st.grid(), ref.grid())
    # the same objects visited as by the allocator-based do-alls
    assert st.visits() == dyn.heap.counters()["visits"]


def test_static_wator_full_size():
    W = H = 2048
    k0 = WL.wator_initial(W, H, 1)
    soa, aos, ref = WatorStatic(W, H, k0, 1), WatorStatic(W, H, k0, 1, aos=True), O.Wator(W, H, k0, seed=1)
    for t in range(1, 21):
        soa.step(1)
        aos.step(1)
        ref.step(1)
        h = ref.hash()
        assert soa.hash() == h and aos.hash() == h, "step %d" % t
