"""The C-ABI library builds, loads and exports every symbol include/lbmpcd.h
declares (no GPU needed); without a GPU every handle creation fails loudly."""
import os
import re

import pytest

import paper_2004_00304_gb300 as lb
from paper_2004_00304_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "lbmpcd.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|long long|const char\*)\s+(lbmpcd_\w+)\s*\(", txt, re.M)))


def test_library_exports_every_declared_symbol():
    libbuild.build()
    L = lb.load_library()
    names = _declared()
    assert len(names) >= 8
    for n in names:
        assert hasattr(L, n), n
    assert sorted(lb.EXPORTED) == sorted(n for n in names if n in lb.EXPORTED)


def test_params_struct_matches_header():
    """The ctypes mirror of lbmpcd_params has the header's field order."""
    txt = open(os.path.join(ROOT, "include", "lbmpcd.h")).read()
    body = txt[txt.index("typedef struct {"):txt.index("} lbmpcd_params;")]
    fields = re.findall(r"^\s*(?:int|double|uint64_t)\s+([^;]+);", body, re.M)
    names = []
    for f in fields:
        for part in f.split(","):
            names.append(part.strip().split("[")[0])
    assert names == [f[0] for f in lb.lbmpcd_params._fields_]


def test_create_fails_loudly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lb.LbmpcdError):
        lb.lbmpcd_create(dict(nx=8, ny=8, tau=1.0))
