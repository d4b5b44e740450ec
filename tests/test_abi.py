"""The C-ABI library loads and exports every entry point declared in include/fetipe.h; host
validation rejects bad input without touching the GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2509_06673_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def _declared():
    src = open(os.path.join(ROOT, "include", "fetipe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fp_[A-Za-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 17
    for n in names:
        assert hasattr(lib, n), n
    from paper_2509_06673_gb300 import fetipe
    assert sorted(fetipe.EXPORTED) == names


def test_invalid_input_rejected_on_host(lib):
    from paper_2509_06673_gb300 import fetipe as F
    from paper_2509_06673_gb300 import workloads as W
    bad = W.small_case(2, 2, 4).with_(order_k=3)
    with pytest.raises(F.FetipeError) as e:
        F.Solver(bad)
    assert e.value.status == 1 and "order_k" in str(e.value)
    bad = W.small_case(2, 2, 4).with_(lame_lambda=-1.0)
    with pytest.raises(F.FetipeError) as e:
        F.Solver(bad)
    assert e.value.status == 1
    bad = W.small_case(2, 2, 4).with_(source="point", src_node=(4, 2))  # on an interface line
    with pytest.raises(F.FetipeError) as e:
        F.Solver(bad)
    assert e.value.status == 1 and "point source" in str(e.value)
