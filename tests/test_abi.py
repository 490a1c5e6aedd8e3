"""CPU-side checks of the C-ABI library: it builds, loads and exports every declared entry point.

No compute call is made here (this machine may have no GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(slag_[a-z_0-9]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2505_08124_b300 import build
    build.build()
    from paper_2505_08124_b300 import slag
    return slag.load_library()


def test_header_declares_the_path():
    d = _declared()
    for name in ("slag_create", "slag_add_view", "slag_finalize", "slag_query"):
        assert name in d


def test_every_declared_symbol_is_exported(lib):
    for name in sorted(_declared()):
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_binding_lists_every_export(lib):
    from paper_2505_08124_b300 import slag
    assert set(slag.EXPORTS) <= _declared()
    assert _declared() <= set(slag.EXPORTS)


def test_struct_layouts_match_header():
    from paper_2505_08124_b300 import slag
    # slag_camera: 4 floats, 2 int32, 9 + 3 floats, 2 floats
    assert ctypes.sizeof(slag.CCamera) == 4 * (4 + 2 + 9 + 3 + 2)
    assert ctypes.sizeof(slag.CGaussians) == 8 + 4 * 8 + 8
    assert ctypes.sizeof(slag.COptions) == 16 + 8
    hdr = open(os.path.join(ROOT, "include", "slag.h")).read()
    body = re.search(r"typedef struct \{([^{}]*)\} slag_stats;", re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)).group(1)
    fields = re.findall(r"int64_t\s+(\w+);", body)
    assert [f for f, _ in slag.CStats._fields_] == fields
    assert ctypes.sizeof(slag.CStats) == 8 * len(fields)
    # slag_profile: ms, spans, busy_ms per stage
    assert ctypes.sizeof(slag.CProfile) == 3 * 7 * 8


def test_launch_counter_reads_without_a_gpu(lib):
    # a running count of the library's kernel launches: plain host state
    from paper_2505_08124_b300 import slag
    n = slag.kernel_launches()
    assert isinstance(n, int) and n >= 0


def test_missing_library_fails_loudly(tmp_path):
    from paper_2505_08124_b300 import slag
    saved = slag._lib
    slag._lib = None
    try:
        with pytest.raises(RuntimeError):
            slag.load_library(str(tmp_path / "nope.so"))
    finally:
        slag._lib = saved


def test_null_arguments_rejected_without_a_gpu(lib):
    # every entry point checks its context and pointers before any CUDA call, so a NULL context
    # or missing output is INVALID_ARG on any machine, GPU or not
    from paper_2505_08124_b300 import slag as S
    I = S.ERR_INVALID_ARG
    assert lib.slag_add_view(None, None, None, None, 4, 0) == I
    assert lib.slag_finalize(None, None, None, 0) == I
    assert lib.slag_finalize_async(None, None, None, 0) == I
    assert lib.slag_wait_outputs(None) == I
    assert lib.slag_query(None, None, 10, None, None, None) == I
    assert lib.slag_query_batch(None, None, 1, 10, None, None, None, 0) == I
    assert lib.slag_reset(None) == I
    assert lib.slag_get_stats(None, None) == I
    assert lib.slag_bin_view(None, None, None, None, None, 0, None) == I
    assert lib.slag_render_debug(None, None, None, None, None) == I
    assert lib.slag_set_profiling(None, 1) == I
    assert lib.slag_set_profiling_stages(None, 4) == I
    assert lib.slag_get_profile(None, None, 0) == I
    assert lib.slag_export_partitions(None, b"x", 1, 1, 0, None) == I
    assert lib.slag_set_latent(None, None) == I
    assert lib.slag_set_autotune(None, 1) == I
    assert lib.slag_add_views_batched(-1, None, None, None, None) == I
    assert lib.slag_noalloc_query_topk(None, 10, 128, None, None, 1, 10, None, None, None, None) == I
    out = ctypes.c_void_p(1)
    assert lib.slag_create(None, None, ctypes.byref(out)) == I and out.value is None
    assert lib.slag_create(None, None, None) == I
    assert lib.slag_last_error(None) == b"no context"
    lib.slag_destroy(None)   # a no-op
