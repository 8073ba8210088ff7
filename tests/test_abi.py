"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point declared in include/p3t.h; host-only argument checks work."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "p3t.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(p3t_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1506_04553_b300 import build
    path = build.build()
    return C.CDLL(path)


def test_header_declares_the_hot_path():
    names = declared_functions()
    for f in ("p3t_build_tree", "p3t_long_force", "p3t_neighbours", "p3t_kick",
              "p3t_drift", "p3t_create", "p3t_destroy", "p3t_energy",
              "p3t_status_string"):
        assert f in names


def test_every_declared_symbol_is_exported(lib):
    missing = [f for f in declared_functions() if not hasattr(lib, f)]
    assert not missing, missing


def test_host_only_paths(lib):
    lib.p3t_status_string.restype = C.c_char_p
    assert lib.p3t_status_string(0) == b"ok"
    assert lib.p3t_status_string(2) == b"capacity exceeded"
    buf = (C.c_double * 8)()
    assert lib.p3t_default_params(buf) == 0
    assert buf[0] == 0.4  # theta
    assert lib.p3t_default_params(None) == 1
    # argument validation happens before any device call
    lib.p3t_kick.argtypes = [C.c_int64, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p]
    assert lib.p3t_kick(0, None, None, 0.1, None) == 0
    assert lib.p3t_kick(-1, None, None, 0.1, None) == 1
    assert lib.p3t_kick(5, None, None, 0.1, None) == 1
    lib.p3t_create.argtypes = [C.c_void_p, C.c_void_p]
    assert lib.p3t_create(None, None) == 1
    # parameters are checked before any device call; r_out below
    # P3T_R_OUT_MIN (1e-15) is refused
    ctx = C.c_void_p()
    buf[1] = 1e-16  # r_out
    assert lib.p3t_create(C.byref(ctx), buf) == 1 and not ctx.value


def test_binding_imports_without_gpu():
    import paper_1506_04553_b300 as P
    assert P.Params().n_group == 64
    assert os.path.exists(P.library_path())


def test_noalloc_energy_limits_fit_the_kernel_index():
    """The largest index the energy kernel forms is below n + blocks x 256
    with at most P3T_ENERGY_NOALLOC_MAX_PARTIALS blocks; at the largest
    accepted n it must fit the kernel's 64-bit index (and the entry point
    must reject 2^31, the first n the library cannot index)."""
    src = open(HEADER).read()
    max_n = int(re.search(r"#define P3T_ENERGY_NOALLOC_MAX_N (\d+)LL", src).group(1))
    parts = int(re.search(r"#define P3T_ENERGY_NOALLOC_MAX_PARTIALS (\d+)", src).group(1))
    assert max_n + parts * 256 < 2 ** 63
    assert max_n == 2 ** 31 - 1
    misc = open(os.path.join(ROOT, "paper_1506_04553_b300", "csrc", "p3t_misc.cu")).read()
    body = misc[misc.index("k_energy_part(long long n"):]
    body = body[:body.index("block_sum")]
    assert "for (long long i" in body
