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


_CTYPE = {"int": ctypes.c_int, "long long": ctypes.c_longlong,
          "unsigned long long": ctypes.c_ulonglong, "double": ctypes.c_double}


def _signatures():
    src = open(os.path.join(ROOT, "include", "fetipe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"(fp_status|const char \*|void)\s*(fp_\w+)\s*\(([^)]*)\)\s*;", src):
        args = []
        for a in m.group(3).split(","):
            a = " ".join(a.split())
            if "*" in a:
                args.append(ctypes.c_void_p)
            else:
                args.append(_CTYPE[a.rsplit(" ", 1)[0].replace("const ", "")])
        out[m.group(2)] = (m.group(1), args)
    return out


def test_null_handle_rejected_without_gpu(lib):
    """Every call that takes a handle returns FP_ERR_INVALID (1) for a NULL handle before it
    touches the device; fp_create rejects NULL arguments; fp_destroy(NULL) is a no-op and
    fp_last_error(NULL) reports the last fp_create failure."""
    sigs = _signatures()
    assert len(sigs) == len(_declared())
    for name, (ret, args) in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        zeros = [None if a is ctypes.c_void_p else a(0) for a in args]
        if name == "fp_destroy":
            fn.restype = None
            fn(*zeros)
        elif name == "fp_last_error":
            fn.restype = ctypes.c_char_p
            assert fn(None) is not None
        elif name == "fp_create":
            fn.restype = ctypes.c_int
            assert fn(None, None, None, None) == 1
            out = ctypes.c_void_p(1)
            assert fn(None, None, None, ctypes.byref(out)) == 1 and out.value is None
        else:
            fn.restype = ctypes.c_int
            if name == "fp_run":
                zeros[1] = ctypes.c_int(1)
            assert fn(*zeros) == 1, name


def test_bad_permeability_rejected_on_host(lib):
    from paper_2509_06673_gb300 import fetipe as F
    from paper_2509_06673_gb300 import workloads as W
    case = W.small_case(2, 2, 4)
    case = case.with_(perm=W.lognormal_perm(case, sigma=1.0, seed=3))
    case.perm[1] = case.perm[1].copy()
    case.perm[1][5] = -1.0
    with pytest.raises(F.FetipeError) as e:
        F.Solver(case)
    assert e.value.status == 1 and "perm" in str(e.value)


def test_no_host_fallback_without_gpu(lib):
    """A valid problem on a host without a CUDA device fails loudly (FP_ERR_CUDA): the
    library has no CPU path."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2509_06673_gb300 import fetipe as F
    from paper_2509_06673_gb300 import workloads as W
    with pytest.raises(F.FetipeError) as e:
        F.Solver(W.small_case(2, 2, 4))
    assert e.value.status == 3 and "no usable CUDA device" in str(e.value)


def test_partition_limits_rejected_on_host(lib):
    from paper_2509_06673_gb300 import fetipe as F
    from paper_2509_06673_gb300 import workloads as W
    for bad, word in ((W.small_case(2, 2, 4).with_(cells_x=[4, 0]), "cells_x"),
                      (W.small_case(2, 2, 4).with_(cells_y=[4, 5000]), "cells_y"),
                      (W.small_case(2, 2, 4).with_(poro_rows=2), "poro_rows"),
                      (W.small_case(5000, 2, 1), "4096")):
        with pytest.raises(F.FetipeError) as e:
            F.Solver(bad)
        assert e.value.status == 1 and word in str(e.value), (word, str(e.value))


_STRUCTS = {"fp_mesh_desc": "MeshDesc", "fp_params": "Params", "fp_sizes": "Sizes",
            "fp_step_stats": "StepStats", "fp_kernel_stats": "KernelStats", "fp_tuning": "Tuning"}


def _header_structs():
    """{struct name: [field names in order]} from the typedefs of include/fetipe.h."""
    src = open(os.path.join(ROOT, "include", "fetipe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"typedef struct\s*\{(.*?)\}\s*(\w+)\s*;", src, flags=re.S):
        names = []
        for decl in m.group(1).split(";"):
            decl = " ".join(decl.split())
            if not decl:
                continue
            first = re.match(r"(?:const\s+)?(?:unsigned\s+)?(?:long long|int|double|float|char)\s*\**\s*", decl)
            for d in decl[first.end():].split(","):
                names.append(re.match(r"\s*\**\s*(\w+)", d).group(1))
        out[m.group(2)] = names
    return out


def test_struct_layouts_match_the_c_compiler(tmp_path):
    """Every struct of include/fetipe.h has, in the ctypes binding, the same fields in the same
    order at the offsets and with the total size that the C compiler gives (gcc, this host)."""
    import shutil
    import subprocess
    from paper_2509_06673_gb300 import fetipe
    structs = _header_structs()
    assert set(structs) == set(_STRUCTS)
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fetipe.h"', "int main(void) {"]
    for cname, fields in structs.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for f in fields:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines += ["return 0;", "}"]
    (tmp_path / "layout.c").write_text("\n".join(lines))
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(tmp_path / "layout"),
                    str(tmp_path / "layout.c")], check=True)
    got = subprocess.run([str(tmp_path / "layout")], check=True, capture_output=True, text=True).stdout.split("\n")
    c = {}
    for ln in got:
        if ln:
            a, b, v = ln.split()
            c[(a, b)] = int(v)
    for cname, pyname in _STRUCTS.items():
        cls = getattr(fetipe, pyname)
        assert [f[0] for f in cls._fields_] == structs[cname], cname
        assert ctypes.sizeof(cls) == c[(cname, "size")], cname
        for f in structs[cname]:
            assert getattr(cls, f).offset == c[(cname, f)], (cname, f)


@pytest.mark.parametrize("lang", ["c", "c++"])
def test_header_compiles_alone_pedantic(tmp_path, lang):
    """include/fetipe.h is self-contained and warning-free as strict C11 and as C++17."""
    import shutil
    import subprocess
    cc, std = ("gcc", "-std=c11") if lang == "c" else ("g++", "-std=c++17")
    if shutil.which(cc) is None:
        pytest.skip("no " + cc)
    src = tmp_path / ("h.c" if lang == "c" else "h.cpp")
    src.write_text('#include "fetipe.h"\nint main(void) { fp_sizes s; (void)s; return 0; }\n')
    subprocess.run([cc, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                    "-c", str(src), "-o", str(tmp_path / "h.o")], check=True)


def test_every_option_key_is_documented():
    """The keys fp_set_option accepts (csrc/api.cu) are exactly the keys the header documents."""
    api = open(os.path.join(ROOT, "paper_2509_06673_gb300", "csrc", "api.cu")).read()
    i = api.index("fp_status fp_set_option(fp_handle *h, const char *key, double value) {")
    accepted = set(re.findall(r'k == "(\w+)"', api[i: api.index("\n}\n", i)]))
    hdr = open(os.path.join(ROOT, "include", "fetipe.h")).read()
    doc = hdr[hdr.index("Tunables of the solve"): hdr.index("fp_status fp_set_option")]
    documented = set(re.findall(r'^\s*\*\s+"(\w+)"\s*\[', doc, flags=re.M))
    assert accepted and accepted == documented, accepted ^ documented


def test_binding_argtypes_match_the_header():
    """Every ctypes prototype of the binding has the header's parameter count, a pointer where
    the header has a pointer and the same scalar type where it has a scalar."""
    from paper_2509_06673_gb300 import fetipe
    ptr_like = (ctypes.c_void_p, ctypes.c_char_p)
    for name, (ret, args) in _signatures().items():
        fn = getattr(fetipe._lib, name)
        bound = fn.argtypes
        assert bound is not None and len(bound) == len(args), name
        for i, (want, got) in enumerate(zip(args, bound)):
            if want is ctypes.c_void_p:
                assert got in ptr_like or issubclass(got, ctypes._Pointer), (name, i, got)
            else:
                assert got is want, (name, i, got, want)
        if ret == "void":
            assert fn.restype is None, name
        elif ret == "fp_status":
            assert fn.restype is ctypes.c_int, name
