"""The C ABI used from plain C: tests/c/abi_steps.c is compiled with gcc against
include/fetipe.h and linked to libfetipe.so.  Without a CUDA device it must fail cleanly with
FP_ERR_CUDA (no host fallback); on the GPU its multipliers must match the oracle."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("no C compiler")
    from paper_2509_06673_gb300 import build
    lib = build.build()
    libdir = os.path.dirname(lib)
    cudalib = os.path.join(os.path.dirname(os.path.dirname(build.NVCC)), "lib64")   # libcudart of the toolkit
    exe = str(tmp_path_factory.mktemp("cclient") / "abi_steps")
    subprocess.run(["gcc", "-std=c11", "-O1", "-Wall", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "abi_steps.c"), "-o", exe, "-L", libdir, "-lfetipe",
                    "-L", cudalib, "-lcudart", "-Wl,-rpath," + libdir, "-Wl,-rpath," + cudalib], check=True)
    return exe


def _run(exe, *args):
    return subprocess.run([exe] + [str(a) for a in args], capture_output=True, text=True, timeout=600)


def test_c_client_without_gpu_fails_with_cuda_status(client):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    r = _run(client, 2, 2, 4, 2, 1, 0, 1e-12)
    assert r.returncode == 3, (r.returncode, r.stdout, r.stderr)
    assert "fp_create" in r.stderr and "no usable CUDA device" in r.stderr


def test_c_client_rejects_bad_mesh_on_host(client):
    r = _run(client, 2, 2, 5000, 2, 1, 0, 1e-12)   # 5000 cells per direction: above the limit
    assert r.returncode == 1 and "cells_x" in r.stderr, (r.returncode, r.stderr)


@pytest.mark.gpu
def test_c_client_steps_match_oracle(client):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_06673_gb300 import workloads as W
    from oracle.monolithic import Discretization, solve_monolithic
    r = _run(client, 3, 4, 4, 2, 2, 0, 1e-13)
    assert r.returncode == 0, (r.returncode, r.stderr)
    lines = r.stdout.split("\n")
    k = next(i for i, ln in enumerate(lines) if ln.startswith("lambda "))
    n = int(lines[k].split()[1])
    lam = np.array([float(v) for v in lines[k + 1: k + 1 + n]])
    assert sum(ln.startswith("step ") for ln in lines[:k]) == 2
    case = W.small_case(3, 4, 4, k=2, n_steps=2, tol=1e-13)
    ref = solve_monolithic(case, Discretization(case))[-1]["lambda"]
    assert lam.shape == ref.shape
    assert np.abs(lam - ref).max() / np.abs(ref).max() < 1e-10
