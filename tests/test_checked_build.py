"""The checked build (libslag_checks.so, compiled with -DSLAG_CHECKS).

Index checks are compiled into pair emission, the sort's scatter, compositing and
aggregation; a refused index sets an error word, and the next synchronising call
returns SLAG_ERR_CAPACITY. The test runs the checked library in a process of its own:
a whole job gives the oracle's result (no false alarm), a pair capacity forced below a
view's pair count (possible only in this build) is caught by the emission's checks and
reported, and the context works again after slag_reset."""
import os
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = textwrap.dedent("""
    import sys
    import numpy as np
    sys.path.insert(0, %r)
    from paper_2505_08124_b300 import slag as S
    lib = S.load_library(S.CHECKED_LIB_PATH)
    assert lib.slag_is_checked_build() == 1
    import synth
    from oracle import oracle as O
    s = synth.small_scene(23, 5000, 3, 160, 104, 7, dim=128, surfaces=4)
    views = [s.view(i) for i in range(s.n_views)]
    num, den, _ = O.lift(s.gaussians, views)
    Eo = O.normalise(num, den)
    with S.Lifter(s.gaussians, dim=128) as L:
        for v in views:
            L.add_view(v.camera, v.seg, v.table)
        E, w = L.finalize()
        assert np.linalg.norm(E - Eo) / np.linalg.norm(Eo) <= 1e-4
        lst, _ = L.bin_view_bins(views[1].camera, 2)
        P = len(lst)
        assert P > 100
        # a forced overflow: the second view's pair buffers hold half of its pairs
        L.reset()
        L.add_view(views[0].camera, views[0].seg, views[0].table)
        assert L.debug_force_pair_capacity(P // 2) == S.OK
        L.add_view(views[1].camera, views[1].seg, views[1].table)
        try:
            L.finalize()
            raise SystemExit("no error reported")
        except S.SlagError as e:
            assert e.status == S.ERR_CAPACITY, e
            assert "pair emission" in str(e), e
        assert L.debug_force_pair_capacity(0) == S.OK
        L.reset()
        for v in views:
            L.add_view(v.camera, v.seg, v.table)
        E2, w2 = L.finalize()
        assert np.linalg.norm(E2 - Eo) / np.linalg.norm(Eo) <= 1e-4
    print("checked build ok: %%d pairs, forced capacity %%d" %% (P, P // 2))
""") % ROOT


@pytest.mark.gpu
def test_checked_build_catches_a_forced_overflow():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2505_08124_b300 import build
    build.build(checks=True)
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "checked build ok" in r.stdout


def test_regular_and_checked_builds_say_which_they_are():
    from paper_2505_08124_b300 import build
    build.build()
    build.build(checks=True)
    code = ("import sys; sys.path.insert(0, %r); from paper_2505_08124_b300 import slag as S; "
            "a = S.load_library(sys.argv[1]); print(a.slag_is_checked_build())" % ROOT)
    from paper_2505_08124_b300 import slag as S
    for path, want in ((S.LIB_PATH, "0"), (S.CHECKED_LIB_PATH, "1")):
        r = subprocess.run([sys.executable, "-c", code, path], capture_output=True, text=True, timeout=120)
        assert r.returncode == 0, r.stderr[-2000:]
        assert r.stdout.strip() == want
