"""The C ABI library builds for sm_103a and exports every entry point include/pb.h declares.
CPU only: nothing here touches a GPU."""
import ctypes
import os
import re

import pytest

from paper_2110_13778_gb300 import build, pb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    txt = open(os.path.join(ROOT, "include", "pb.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pb_[a-z_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpb():
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(libpb):
    names = declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(libpb, n), n


def test_binding_covers_the_header():
    assert sorted(pb.EXPORTS) == declared()


def test_missing_library_fails_loudly(monkeypatch):
    monkeypatch.setattr(pb, "LIB_PATH", "/nonexistent/libpb.so")
    monkeypatch.setattr(pb, "_lib", None)
    with pytest.raises(ImportError):
        pb.lib()


def test_params_struct_matches_header():
    # field order and count of pb_params as declared in the header
    txt = open(os.path.join(ROOT, "include", "pb.h")).read()
    body = re.search(r"typedef struct pb_params \{(.*?)\} pb_params;", txt, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b(?:double|int)\s+(\w+);", body)
    assert fields == [f for f, _ in pb.pb_params._fields_]


@pytest.mark.parametrize("bad", [dict(eps_in=0.0), dict(eps_out=-1.0), dict(kappa=-0.1), dict(eta0=1.0),
                                 dict(eta0=0.0), dict(p=11), dict(qs=0), dict(qs=9), dict(precision=2),
                                 dict(precond=3), dict(singular=3), dict(leaf_size=0), dict(levels=11)])
def test_create_rejects_bad_parameters(bad):
    # argument checks run before any CUDA call, so they are testable without a GPU
    h = ctypes.c_void_p()
    rc = pb.lib().pb_create(ctypes.byref(pb.params(**bad)), None, ctypes.byref(h))
    assert rc == pb.PB_ERR_ARG and not h.value


@pytest.mark.parametrize("shape", [(0, 128, 3, 2), (18, 100, 3, 2), (18, 8, 3, 2), (18, 128, 0, 2),
                                   (18, 128, 8, 2), (18, 128, 3, 0), (18, 128, 3, 65)])
def test_mlp_create_rejects_bad_shapes(shape):
    h = ctypes.c_void_p()
    rc = pb.lib().pb_mlp_create(*shape, 0, None, ctypes.byref(h))
    assert rc == pb.PB_ERR_ARG and not h.value


def test_null_handles_are_rejected():
    L = pb.lib()
    assert L.pb_destroy(None) == pb.PB_OK
    assert L.pb_mlp_destroy(None) == pb.PB_OK
    n = ctypes.c_longlong()
    assert L.pb_get_launch_count(None, ctypes.byref(n)) == pb.PB_ERR_ARG
    assert L.pb_matvec_multi(None, None, None, 1) == pb.PB_ERR_ARG
    assert L.pb_learned_guess(None, None, None) == pb.PB_ERR_ARG
    assert L.pb_autotune(None, 1e-4, 10, 1, None) == pb.PB_ERR_ARG
