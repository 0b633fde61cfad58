"""The C-ABI library builds for sm_103a, loads, and exports what include/fd.h declares (no GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "fd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fd_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    return __graft_entry__._build_module().build()


def test_header_declares_hot_path():
    names = _declared()
    for n in ["fd_build_matrix", "fd_filter", "fd_orthonormalize", "fd_rayleigh_ritz", "fd_solve",
              "fd_kpm_moments", "fd_spectral_bounds", "fd_matrix_to_csr"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib):
    import paper_2209_01974_gb300 as fd
    assert sorted(_declared()) == fd.EXPORTED


def test_library_is_built_for_sm_103a(lib):
    out = subprocess.run(["cuobjdump", "--list-elf", lib], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


def test_null_arguments_are_rejected_without_device_work(lib):
    L = ctypes.CDLL(lib)
    L.fd_filter.restype = ctypes.c_int
    assert L.fd_filter(None, None, 0, None, 0, 0, 0, None, ctypes.c_double(0), ctypes.c_double(0),
                       None, None, 0) == 1          # FD_ERR_ARG
    L.fd_last_error.restype = ctypes.c_char_p
    assert L.fd_last_error(None) == b"null context"


def test_options_and_result_structs_follow_the_header(lib):
    """The binding's ctypes mirrors of fd_options, fd_result and fd_checkpoint
    have the header's fields in the header's order (a mismatch would shift
    every later field), and the option strings map to the header's enums."""
    import paper_2209_01974_gb300 as fd
    src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "fd.h")).read(), flags=re.S)

    def fields(name):
        body = re.search(r"typedef struct \{([^}]*)\} " + name + ";", src).group(1)
        out = []
        for decl in body.split(";"):
            decl = decl.strip()
            if decl:
                out += [n.strip() for n in decl.split(None, 1)[1].split(",")]
        return out

    assert [f for f, _ in fd.fd_options._fields_] == fields("fd_options")
    assert [f for f, _ in fd.fd_result._fields_] == fields("fd_result")
    assert [f for f, _ in fd.fd_checkpoint._fields_] == fields("fd_checkpoint")
    assert [f for f, _ in fd.fd_problem._fields_] == fields("fd_problem")
    o = fd._options({"precision": "ff", "finish": "ff", "intervals": "lehmann"})
    assert (o.precision, o.finish, o.intervals) == (fd.FD_FF, fd.FD_FINISH_FF, fd.FD_INTERVALS_LEHMANN)
    o = fd._options({"precision": "f32", "finish": "f64"})
    assert (o.precision, o.finish) == (fd.FD_F32, fd.FD_FINISH_F64)
    for name, value in (("FD_F64", 0), ("FD_F32", 1), ("FD_FF", 2)):
        assert re.search(r"\b%s = %d\b" % (name, value), src) and getattr(fd, name) == value
    for name, value in (("FD_FINISH_F64", 0), ("FD_FINISH_FF", 1)):
        assert re.search(r"\b%s = %d\b" % (name, value), src) and getattr(fd, name) == value
