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
