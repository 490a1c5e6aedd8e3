"""Failure detection without a GPU fault.

Every device-side wait of the library (the mbarrier waits of the tensor-core
kernels) is bounded by globaltimer. A kernel whose wait gives up sets the
context's error word, the call returns SLAG_ERR_TIMEOUT, and the context stays
usable. slag_check_wait_timeout runs that path on demand, with nothing else in
flight: one role waits on an mbarrier that nothing completes, a second role
gives up through the first one's abort flag. Nothing here traps or faults the
GPU; the wait runs out because nobody arrives on the barrier."""
import time

import numpy as np
import pytest

import synth
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def slag():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2505_08124_b300 import build
    build.build()
    from paper_2505_08124_b300 import slag as S
    S.load_library()
    return S


def test_bounded_wait_times_out_and_the_context_stays_usable(slag):
    s = synth.small_scene(17, 4000, 3, 128, 96, 6, dim=128, surfaces=3)
    views = [s.view(i) for i in range(s.n_views)]
    with slag.Lifter(s.gaussians, dim=128) as L:
        L.add_view(views[0].camera, views[0].seg, views[0].table)
        # the control case: the barrier is completed, both roles finish
        assert L.check_wait_timeout(20_000, complete=True) == slag.OK
        t0 = time.perf_counter()
        assert L.check_wait_timeout(20_000) == slag.ERR_TIMEOUT
        dt = time.perf_counter() - t0
        # the second role left through the abort flag, not through its own ~1 s bound
        assert dt < 0.9, dt
        assert "wait" in L._lib.slag_last_error(L._h).decode()
        # twice in a row: the error word was cleared after the first report
        assert L.check_wait_timeout(5_000) == slag.ERR_TIMEOUT
        assert L.check_wait_timeout(5_000, complete=True) == slag.OK
        # the context still works: the views added before and after, against the oracle
        for v in views[1:]:
            L.add_view(v.camera, v.seg, v.table)
        E, w = L.finalize()
        ids, _ = L.query(views[1].table[0] / np.linalg.norm(views[1].table[0]), 3)
    num, den, _ = O.lift(s.gaussians, views)
    Eo = O.normalise(num, den)
    assert np.linalg.norm(E - Eo) / np.linalg.norm(Eo) <= 1e-4
    assert len(ids) == 3


def test_wait_check_argument_errors(slag):
    s = synth.small_scene(18, 500, 1, 32, 32, 2, dim=128)
    with slag.Lifter(s.gaussians, dim=128) as L:
        assert L.check_wait_timeout(0) == slag.ERR_INVALID_ARG
        assert L.check_wait_timeout(2_000_000) == slag.ERR_INVALID_ARG
