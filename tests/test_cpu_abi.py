"""Host-only checks of the C ABI: the library builds, loads without a GPU and
exports every entry point that include/apm.h declares; argument errors are
rejected on the host before any launch."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "apm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(apm_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2104_07638_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_four_paper_calls():
    syms = declared_symbols()
    for s in ("apm_all_minors", "apm_cdet_connected", "apm_keldysh_sum", "apm_perm_minors"):
        assert s in syms


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_host_side_argument_errors(lib):
    P, i32, i64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
    f = lib.apm_all_minors
    f.argtypes = [P, i32, i64, P, P, P, P, sz, P]
    f.restype = ctypes.c_int
    fake = ctypes.c_void_p(1 << 20)           # never dereferenced: the call must fail first
    assert f(fake, 0, 1, fake, None, None, None, 0, None) == 2      # n out of range
    assert f(fake, 25, 1, fake, None, None, None, 0, None) == 2
    assert f(fake, 17, 1, fake, None, None, None, 0, None) == 6     # orders 17..24 need the workspace
    assert f(fake, 8, -1, fake, None, None, None, 0, None) == 1     # negative batch
    assert f(None, 8, 1, fake, None, None, None, 0, None) == 1      # null input
    assert f(ctypes.c_void_p((1 << 20) + 8), 8, 1, fake, None, None, None, 0, None) == 1  # misaligned
    assert f(None, 8, 0, None, None, None, None, 0, None) == 0      # empty batch: no launch
    g = lib.apm_cdet_connected
    g.argtypes = [P, P, i32, i64, i32, P, P, P, P, P, sz, P]
    g.restype = ctypes.c_int
    assert g(fake, fake, 8, 1, 1, fake, None, None, None, None, 0, None) == 1  # single-det with A_dn
    assert g(fake, None, 8, 1, 4, fake, None, None, None, None, 0, None) == 1  # unknown flag
    h = lib.apm_cdet_connected_host
    h.argtypes = [P, P, i32, i64, i32, P, P, P, P, i64, i32, P, sz, P]
    h.restype = ctypes.c_int
    assert h(fake, None, 0, 1, 0, fake, None, None, None, 8, 2, fake, 1 << 20, None) == 2   # n out of range
    assert h(fake, None, 8, 1, 0, fake, None, None, None, 0, 2, fake, 1 << 20, None) == 1   # chunk 0
    assert h(fake, None, 8, 1, 0, fake, None, None, None, 8, 0, fake, 1 << 20, None) == 1   # no stream
    assert h(fake, None, 8, 1, 0, fake, None, None, None, 8, 9, fake, 1 << 20, None) == 1   # > 8 streams
    assert h(fake, None, 8, 1, 4, fake, None, None, None, 8, 2, fake, 1 << 20, None) == 1   # unknown flag
    assert h(fake, fake, 8, 1, 1, fake, None, None, None, 8, 2, fake, 1 << 20, None) == 1   # single-det, A_dn
    assert h(None, None, 8, 1, 0, fake, None, None, None, 8, 2, fake, 1 << 20, None) == 1   # null input
    assert h(None, None, 8, 0, 0, None, None, None, None, 8, 2, None, 0, None) == 0         # empty batch
    hw = lib.apm_cdet_connected_host_workspace_size
    hw.argtypes = [i32, i64, i32, i32, ctypes.POINTER(sz)]
    hw.restype = ctypes.c_int
    nb = sz(7)
    assert hw(8, 16, 2, 0, None) == 1
    assert hw(17, 16, 2, 0, ctypes.byref(nb)) == 2 and nb.value == 0
    assert hw(8, 0, 2, 0, ctypes.byref(nb)) == 1
    assert hw(8, 16, 9, 0, ctypes.byref(nb)) == 1
    lib.apm_status_string.restype = ctypes.c_char_p
    assert b"WORKSPACE" in lib.apm_status_string(6)
    lib.apm_version.restype = ctypes.c_int
    assert lib.apm_version() >= 100


def test_tune_tables_host_side(lib):
    """The cost-model lane-group table is valid for every order, and invalid
    tables are rejected on the host."""
    P = ctypes.c_void_p
    lib.apm_cdet_tune_get.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]
    lib.apm_cdet_tune_get.restype = ctypes.c_int
    lib.apm_cdet_tune_set.argtypes = [P]
    lib.apm_cdet_tune_set.restype = ctypes.c_int
    for n in range(17):
        out = ctypes.c_uint64(0)
        assert lib.apm_cdet_tune_get(n, ctypes.byref(out)) == 0
        for k in range(17):
            r = (out.value >> (3 * k)) & 7
            assert r <= 5 and (r == 0 or 2 <= k <= n) and r <= max(k - 1, 0)
    bad = (ctypes.c_uint64 * 17)(*([0] * 17))
    bad[4] = 7 << (3 * 3)           # r = 7 > 5
    assert lib.apm_cdet_tune_set(ctypes.cast(bad, P)) == 1
    bad[4] = 3 << (3 * 2)           # layer k = 2 allows r <= 1
    assert lib.apm_cdet_tune_set(ctypes.cast(bad, P)) == 1
    assert lib.apm_cdet_tune_set(None) == 0


def test_xnor_and_nambu_argument_errors(lib):
    P, i32, i64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
    fake = ctypes.c_void_p(1 << 20)           # never dereferenced: the call must fail first
    x = lib.apm_xnor_minors
    x.argtypes = [P, i32, i64, P, P, P, sz, P]
    x.restype = ctypes.c_int
    assert x(fake, 0, 1, fake, None, None, 0, None) == 2            # n out of range
    assert x(fake, 17, 1, fake, None, None, 0, None) == 2
    assert x(fake, 6, -1, fake, None, None, 0, None) == 1           # negative batch
    assert x(None, 6, 1, fake, None, None, 0, None) == 1            # null input
    assert x(fake, 6, 1, ctypes.c_void_p((1 << 20) + 8), None, None, 0, None) == 1  # misaligned output
    assert x(None, 6, 0, None, None, None, 0, None) == 0            # empty batch: no launch
    nb = lib.apm_nambu_cdet
    nb.argtypes = [P, i32, i64, P, P, P, P, sz, P]
    nb.restype = ctypes.c_int
    assert nb(fake, 17, 1, fake, fake, None, None, 0, None) == 2
    assert nb(fake, 6, 1, fake, None, None, None, 0, None) == 1     # null c
    assert nb(None, 6, 0, None, None, None, None, 0, None) == 0


def test_nand_and_two_type_argument_errors(lib):
    P, i32, i64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
    fake = ctypes.c_void_p(1 << 20)
    f = lib.apm_nand_minors
    f.argtypes = [P, i32, i64, P, P, P, P, sz, P]
    f.restype = ctypes.c_int
    assert f(fake, 14, 1, fake, None, None, None, 0, None) == 2     # 3^14 per matrix: beyond the limit
    assert f(fake, 0, 1, fake, None, None, None, 0, None) == 2
    assert f(None, 5, 1, fake, None, None, None, 0, None) == 1
    assert f(None, 5, 0, None, None, None, None, 0, None) == 0
    g = lib.apm_two_type_cdet
    g.argtypes = [P, i32, i64, P, P, P, P, P, sz, P]
    g.restype = ctypes.c_int
    assert g(fake, 17, 1, fake, fake, None, None, None, 0, None) == 2
    assert g(fake, 16, -1, fake, fake, None, None, None, 0, None) == 1
    assert g(fake, 6, 1, fake, None, None, None, None, 0, None) == 1


def test_keldysh2_argument_errors(lib):
    P, i32, i64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
    fake = ctypes.c_void_p(1 << 20)
    f = lib.apm_keldysh2_sum
    f.argtypes = [P, P, i32, i64, i32, P, P, P, P, sz, P]
    f.restype = ctypes.c_int
    assert f(fake, fake, 17, 1, 0, fake, None, None, None, 0, None) == 2
    assert f(fake, None, 6, 1, 0, fake, None, None, None, 0, None) == 1      # missing second spin
    assert f(fake, fake, 6, 1, 2, fake, None, None, None, 0, None) == 1      # unknown flag
    assert f(None, None, 6, 0, 0, None, None, None, None, 0, None) == 0


def test_mlp_gemm_and_status_argument_errors(lib):
    P, i32, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    fake = ctypes.c_void_p(1 << 20)
    ws = ctypes.c_size_t(0)
    lib.apm_mlp_workspace_size.argtypes = [i32, ctypes.POINTER(sz)]
    assert lib.apm_mlp_workspace_size(0, ctypes.byref(ws)) == 0 and ws.value > 0
    f = lib.apm_mlp_gemm_tn
    f.argtypes = [P, P, P, P, P, i32, i32, i32, i32, P, sz, P]
    f.restype = ctypes.c_int
    assert f(fake, fake, None, fake, None, 128, 96, 64, 0, fake, ws.value, None) == 1     # N not a multiple of 64
    assert f(fake, fake, None, fake, None, 128, 64, 80, 0, fake, ws.value, None) == 1     # K not a multiple of 64
    assert f(fake, fake, None, fake, None, 0, 64, 64, 0, fake, ws.value, None) == 1       # empty M
    assert f(fake, fake, None, None, None, 128, 64, 64, 0, fake, ws.value, None) == 1     # no output
    assert f(ctypes.c_void_p((1 << 20) + 8), fake, None, fake, None, 128, 64, 64, 0, fake, ws.value, None) == 1
    assert f(fake, fake, None, fake, None, 128, 64, 64, 0, None, 0, None) == 6            # no workspace
    assert f(fake, fake, None, fake, None, 128, 64, 64, 0, fake, ws.value - 1, None) == 6
    g = lib.apm_mlp_status
    g.argtypes = [P, sz, ctypes.POINTER(ctypes.c_uint32), P]
    g.restype = ctypes.c_int
    assert g(None, 0, None, None) == 6


def test_host_call_workspace_layout(lib):
    """apm_cdet_connected_host's workspace for n <= 12 (no kernel scratch): per
    slot the chunk's matrices (one or two), connected sums, minors (one or two
    rows) and status words, each rounded up to 256 bytes; times the streams."""
    sz = ctypes.c_size_t
    hw = lib.apm_cdet_connected_host_workspace_size
    hw.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.POINTER(sz)]
    hw.restype = ctypes.c_int
    r256 = lambda x: (x + 255) // 256 * 256
    for n, chunk, ns, two in ((10, 100, 3, 0), (12, 2048, 4, 0), (7, 33, 1, 1), (1, 5, 8, 1)):
        out = sz(0)
        assert hw(n, chunk, ns, two, ctypes.byref(out)) == 0
        mats, N = (2 if two else 1), 1 << n
        slot = (mats * r256(chunk * n * n * 8) + r256(chunk * N * 8) + r256(chunk * mats * N * 8)
                + r256(chunk * 4))
        assert out.value == ns * slot, (n, chunk, ns, two)


def test_tune_options_host_side(lib):
    """apm_tune_options_set/get keep host state only: range checks, defaults
    (0 selects the hand-off at 16, all resident CTAs, 12 Keldysh warps), and a
    rejected call changes nothing."""
    i32, P = ctypes.c_int, ctypes.c_void_p
    lib.apm_tune_options_set.argtypes = [i32, i32, i32]
    lib.apm_tune_options_set.restype = ctypes.c_int
    lib.apm_tune_options_get.argtypes = [P, P, P]
    lib.apm_tune_options_get.restype = ctypes.c_int

    def get():
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        assert lib.apm_tune_options_get(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)) == 0
        return a.value, b.value, c.value

    try:
        assert lib.apm_tune_options_set(0, 0, 0) == 0 and get() == (16, 0, 0)
        assert lib.apm_tune_options_set(14, 2, 6) == 0 and get() == (14, 2, 6)
        for bad in ((12, 0, 0), (18, 0, 0), (16, 4, 0), (16, -1, 0), (16, 0, 2), (16, 0, 13)):
            assert lib.apm_tune_options_set(*bad) == 1
            assert get() == (14, 2, 6)
        assert lib.apm_tune_options_set(17, 3, 12) == 0 and get() == (17, 3, 12)
    finally:
        lib.apm_tune_options_set(0, 0, 0)


def test_exchange_and_split_training_argument_errors(lib):
    """apm_order_sums and the split training step reject bad arguments on the
    host, before any launch."""
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    f = lib.apm_order_sums
    f.argtypes = [P, i32, P, P, i64, i32, P, P]
    f.restype = ctypes.c_int
    fake = ctypes.c_void_p(1 << 20)
    assert f(fake, 8, None, None, 4, 0, fake, None) == 1        # n_max out of range
    assert f(fake, 8, None, None, 4, 17, fake, None) == 1
    assert f(fake, 9, None, None, 4, 8, fake, None) == 1        # fixed order above n_max
    assert f(fake, 0, fake, None, 4, 8, fake, None) == 1        # n_arr without c_off
    assert f(fake, 8, None, None, -1, 8, fake, None) == 1       # negative batch
    assert f(fake, 8, None, None, 4, 8, None, None) == 1        # no output
    assert f(None, 8, None, None, 4, 8, fake, None) == 1        # rows missing
    g = lib.apm_mlp_adam_step
    g.argtypes = [P, ctypes.c_float, i32, P]
    g.restype = ctypes.c_int
    assert g(None, ctypes.c_float(1e-3), 1, None) == 1
    h = lib.apm_mlp_gradient
    h.argtypes = [P, P, P, i32, i32, P, P, ctypes.c_size_t, P]
    h.restype = ctypes.c_int
    assert h(None, fake, fake, 64, 64, fake, fake, 1 << 20, None) == 1
