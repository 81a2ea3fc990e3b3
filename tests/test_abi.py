"""C ABI checks that need no GPU: the library loads, exports every symbol the
header declares, and host-side argument checks reject bad calls before any
CUDA work is enqueued."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gpa.h")


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"GPA_API\s+(?:const\s+)?\w+\*?\s+\*?(\w+)\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2104_05372_b300 import build
    build.build()
    from paper_2104_05372_b300 import _lib
    return _lib.load()


def test_header_declares_entry_points():
    names = _declared()
    for n in ("gmm_objective", "gmm_vjp", "reproj_residual", "reproj_vjp", "accum_scatter_add"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2104_05372_b300 import _lib
    assert sorted(_lib.exported_symbols()) == _declared()


def test_status_strings(lib):
    from paper_2104_05372_b300 import _lib
    for code in range(8):
        assert _lib.status_string(code).startswith("GPA_")
    assert _lib.version() >= 100


def test_workspace_queries(lib):
    from paper_2104_05372_b300 import _lib
    small = _lib.gpa_gmm_workspace_bytes(1000, 10, 5, 0, 128)
    full = _lib.gpa_gmm_workspace_bytes(1000, 10, 5, 0, 0)
    assert 0 < small < full
    assert _lib.gpa_gmm_workspace_bytes(0, 10, 5, 0, 0) == 0
    assert _lib.gpa_gmm_workspace_bytes(10, 129, 5, 0, 0) == 0
    assert _lib.gpa_reproj_workspace_bytes(8192, 500000, 4000000) >= 8192 * 32 * 4
    assert _lib.gpa_plan_bytes(100, 10) >= 256 + 3 * 400 + 44
    assert _lib.gpa_plan_workspace_bytes(0, 10) == 0


def test_host_argument_errors_return_before_any_launch(lib):
    fake = C.c_void_p(256)  # never dereferenced: every call below fails its host checks
    # null x
    assert lib.gmm_objective(None, fake, fake, fake, fake, 10, 3, 2, 1.0, 0, 0, fake, None, None, fake, 1 << 20,
                             None, None) == 1
    # D out of range
    assert lib.gmm_objective(fake, fake, fake, fake, fake, 10, 129, 2, 1.0, 0, 0, fake, None, None, fake, 1 << 20,
                             None, None) == 1
    # gamma <= 0
    assert lib.gmm_vjp(fake, fake, fake, fake, fake, 10, 3, 2, 0.0, 0, 0, None, None, 1.0, fake, fake, fake, fake,
                       None, fake, 1 << 20, None, None) == 1
    # workspace too small
    assert lib.gmm_objective(fake, fake, fake, fake, fake, 10, 3, 2, 1.0, 0, 0, fake, None, None, fake, 16,
                             None, None) == 4
    # misaligned workspace
    assert lib.gmm_objective(fake, fake, fake, fake, fake, 10, 3, 2, 1.0, 0, 0, fake, None, None, C.c_void_p(260),
                             1 << 20, None, None) == 7
    # reprojection: non-positive sizes, bad strategy, SORT without a plan
    assert lib.reproj_residual(fake, fake, fake, fake, 0, 1, 1, fake, fake, 1 << 20, None, None) == 1
    assert lib.reproj_vjp(fake, fake, fake, fake, 2, 2, 2, fake, fake, 9, None, 0, fake, 1 << 20, None, None) == 1
    assert lib.reproj_vjp(fake, fake, fake, fake, 2, 2, 2, fake, fake, 3, None, 0, fake, 1 << 20, None, None) == 1
    # plan-ordered cotangents need the SORT strategy; orders other than 0, 1
    assert lib.reproj_vjp(fake, fake, fake, fake, 2, 2, 2, fake, fake, 1, None, 1, fake, 1 << 20, None, None) == 1
    assert lib.reproj_vjp(fake, fake, fake, fake, 2, 2, 2, fake, fake, 3, fake, 2, fake, 1 << 20, None, None) == 1
    assert lib.reproj_residual_vjp(fake, fake, fake, fake, 2, 2, 2, 1.0, fake, fake, fake, 2, None, 1, fake,
                                   1 << 20, None, None) == 1
    # scatter: w out of range, bad dtype
    assert lib.accum_scatter_add(fake, fake, 10, 65, 0, fake, 4, 1, None, None, None) == 1
    assert lib.accum_scatter_add(fake, fake, 10, 1, 2, fake, 4, 1, None, None, None) == 1
    # plans: workspace too small
    assert lib.gpa_index_plan_build(fake, 100, 10, fake, 16, fake, 1 << 20, None, None) == 4


def test_bounded_wait_check_rejects_bad_arguments(lib):
    fake = C.c_void_p(256)
    assert lib.gpa_check_bounded_wait(0, fake, fake, None) == 1
    assert lib.gpa_check_bounded_wait(1_000_000_001, fake, fake, None) == 1
    assert lib.gpa_check_bounded_wait(1000, None, fake, None) == 1
    assert lib.gpa_check_bounded_wait(1000, fake, None, None) == 1


def test_host_streaming_entry_checks(lib):
    """gmm_vjp_host: the workspace query and the host-side rejections, all
    before its first CUDA call."""
    from paper_2104_05372_b300 import _lib
    q = _lib.gpa_gmm_vjp_host_workspace_bytes
    assert q(1000, 10, 5, 0, 256) > 0
    assert q(1000, 64, 5, 1, 256) > 0
    assert q(0, 10, 5, 0, 256) == 0        # no points
    assert q(1000, 129, 5, 0, 256) == 0    # D out of range
    assert q(1000, 10, 5, 2, 256) == 0     # unknown precision
    big = q(1 << 20, 64, 200, 0, 0)
    assert q(1 << 20, 64, 200, 0, 4096) < big  # smaller chunks, smaller staging
    fake = C.c_void_p(256)
    args = [fake] * 5 + [1000, 10, 5, 1.0, 0, 0, 1.0] + [fake] * 5 + [256]
    # null x
    assert lib.gmm_vjp_host(None, *args[1:], fake, 1 << 30, None, None) == 1
    # gamma <= 0
    bad = list(args)
    bad[8] = 0.0
    assert lib.gmm_vjp_host(*bad, fake, 1 << 30, None, None) == 1
    # tensor cores below their dimension range
    tc = list(args)
    tc[10] = 1
    assert lib.gmm_vjp_host(*tc, fake, 1 << 30, None, None) == 6
    # misaligned workspace, then a workspace smaller than the query
    assert lib.gmm_vjp_host(*args, C.c_void_p(260), 1 << 30, None, None) == 7
    assert lib.gmm_vjp_host(*args, fake, 16, None, None) == 4


def test_batched_workspace_query_and_settings_checks(lib):
    """The batched form's workspace query works from the instance shapes
    alone (the device pointers are not read) and rejects bad per-class
    settings and out-of-range tensor-core instances with 0 bytes."""
    from paper_2104_05372_b300 import _lib

    def inst(n, d, k, prec=0):
        i = _lib.GmmInstance()
        for f in ("x", "alpha", "mu", "q", "l", "d_alpha", "d_mu", "d_q", "d_l"):
            setattr(i, f, 256)
        i.n, i.d, i.k, i.gamma, i.m, i.seed, i.prec = n, d, k, 1.0, 0, 1.0, prec
        return i

    arr = (_lib.GmmInstance * 3)(inst(1000, 8, 5), inst(5000, 30, 40), inst(3000, 64, 20, 1))
    ok = _lib.BatchedOpts.make({})
    size = lib.gpa_gmm_batched_workspace_bytes_opts(arr, 3, C.byref(ok))
    assert size > 0
    assert lib.gpa_gmm_batched_workspace_bytes(arr, 3, 4096) == size  # uniform settings = the default opts
    assert lib.gpa_gmm_batched_workspace_bytes_opts(arr, 3, None) == 0
    assert lib.gpa_gmm_batched_workspace_bytes_opts(
        arr, 3, C.byref(_lib.BatchedOpts.make({1: {"chunk_points": 32}}))) == 0
    assert lib.gpa_gmm_batched_workspace_bytes_opts(
        arr, 3, C.byref(_lib.BatchedOpts.make({2: {"ctas_per_sm": -1}}))) == 0
    tc_small = (_lib.GmmInstance * 1)(inst(1000, 32, 5, 1))  # tensor cores need 32 < D
    assert lib.gpa_gmm_batched_workspace_bytes_opts(tc_small, 1, C.byref(ok)) == 0
