"""CPU checks of the C ABI: the library builds, loads and exports every
function declared in include/tetra.h; host-side argument checks answer
without a GPU."""
import ctypes
import os
import re

import pytest

import paper_1710_10789_gb300 as T

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "tetra.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(tetra_[a-z_0-9]+)\s*\(",
                       src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built():
    T.build()
    return T.lib()


def test_header_declares_the_binding_symbols():
    assert sorted(T.EXPORTED_SYMBOLS) == declared_functions()


def test_library_exports_every_declared_symbol(built):
    for name in declared_functions():
        assert hasattr(built, name), name


def test_strerror_and_version_without_gpu(built):
    assert T.tetra_version() == "0.1.0"
    assert T.tetra_strerror(T.TETRA_OK) == "TETRA_OK"
    assert "invalid" in T.tetra_strerror(T.TETRA_EINVAL)


def test_plan_rejects_bad_descriptions(built):
    bad = [
        T.TetraDesc(0, 4, 4, 1, 1, 10, 0, 0, 0, 0),
        T.TetraDesc(4, 4, 4, 0, 1, 10, 0, 0, 0, 0),
        T.TetraDesc(4, 4, 4, 1, 17, 10, 0, 0, 0, 0),
        T.TetraDesc(4, 4, 4, 1, 1, 0, 0, 0, 0, 0),
        T.TetraDesc(4, 4, 4, 1, 1, 10, 3, 0, 0, 0),
        T.TetraDesc(4, 4, 4, 1, 1, 10, 0, 3, 0, 0),
        T.TetraDesc(4, 4, 4, 1, 1, 10, 0, 0, 3, 2),
        T.TetraDesc(4, 4, 4, 1, 1, 10, 0, 0, 0, 9),
    ]
    for d in bad:
        h = ctypes.c_void_p()
        assert built.tetra_plan(ctypes.byref(h), ctypes.byref(d), 0) == T.TETRA_EINVAL
        assert h.value is None


def test_null_arguments_are_rejected(built):
    assert built.tetra_plan(None, None, 0) == T.TETRA_EINVAL
    assert built.tetra_dos(None, None, None, None, None, None, 0, None) == T.TETRA_EINVAL
    assert built.tetra_dos_backward(None, None, None, None, None, None, None, None, 0, None) == T.TETRA_EINVAL
    assert built.tetra_eig(None, None, None, None, None) == T.TETRA_EINVAL
    assert built.tetra_workspace_bytes(None) == 0
    assert built.tetra_plan_destroy(None) == T.TETRA_OK


def test_batched_plan_rejects_bad_batches(built):
    good = T.TetraDesc(8, 8, 8, 8, 8, 100, 0, 0, 0, 0)
    h = ctypes.c_void_p()
    for descs in ([], [good] * (T.TETRA_MAX_BATCH + 1),
                  [good, T.TetraDesc(8, 8, 8, 4, 8, 100, 0, 0, 0, 0)],     # n_bands differ
                  [good, T.TetraDesc(8, 8, 8, 8, 4, 100, 0, 0, 0, 0)],     # n_orb differ
                  [good, T.TetraDesc(8, 8, 8, 8, 8, 100, 1, 0, 0, 0)],     # mode differs
                  [good, T.TetraDesc(8, 8, 8, 8, 8, 100, 0, 1, 0, 0)]):    # dtype differs
        arr = (T.TetraDesc * max(1, len(descs)))(*descs)
        assert built.tetra_plan_batched(ctypes.byref(h), arr, len(descs), None, 0) == T.TETRA_EINVAL
        assert h.value is None
    assert built.tetra_batch_workspace_bytes(None) == 0
    assert built.tetra_batch_plan_destroy(None) == T.TETRA_OK
