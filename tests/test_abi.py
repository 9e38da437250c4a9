"""The C-ABI library builds, loads and exports every function include/stab.h
declares (no GPU needed: nothing here launches work)."""
import os
import re

import numpy as np
import pytest

from paper_2507_03092_gb300 import binding as B
from paper_2507_03092_gb300 import build as BLD
from paper_2507_03092_gb300 import circuit as C

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "stab.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(stab_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    BLD.build()
    L = B.lib()
    names = declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(B.EXPORTED)


def test_op_record_layout_matches_header():
    src = open(os.path.join(ROOT, "include", "stab.h")).read()
    assert C.OP_DTYPE.itemsize == 16
    for kind, name in ((C.H, "STAB_H"), (C.CX, "STAB_CX"), (C.M, "STAB_M"), (C.R, "STAB_R"),
                       (C.DEP2, "STAB_DEP2"), (C.PC1, "STAB_PC1"), (C.RESET_ERR, "STAB_RESET_ERR")):
        m = re.search(name + r"\s*=\s*(\d+)", src)
        assert m and int(m.group(1)) == kind, name


def test_create_without_gpu_fails_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(B.StabError):
        B.stab_create(0, None)
