"""The C ABI used from plain C (tests/c_client.c, built with gcc against include/mbc.h and
libmbc.so): planning in a host-only context on the CPU (FP32 guard and shape settings
included), and a proton correlator on the GPU in FP64 and in FP32 with guards checked
against the oracle."""
import os
import subprocess

import numpy as np
import pytest

import mbc_inputs as mi
from oracle import correlator as ocor
from oracle import operators as oops

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    from paper_2201_04269_gb300 import build
    build.build()
    lib_dir = os.path.join(ROOT, "paper_2201_04269_gb300")
    exe = str(tmp_path_factory.mktemp("c") / "c_client")
    cmd = ["gcc", "-O2", "-std=c99", "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA, "include"),
           os.path.join(ROOT, "tests", "c_client.c"), "-o", exe, "-L", lib_dir, "-lmbc",
           "-L", os.path.join(CUDA, "lib64"), "-lcudart", "-Wl,-rpath," + lib_dir,
           "-Wl,-rpath," + os.path.join(CUDA, "lib64")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        pytest.fail("c_client did not build: " + r.stderr[-2000:])
    return exe


def run(exe, *args):
    r = subprocess.run([exe, *map(str, args)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    return r.stdout.splitlines()


def test_c_client_plans_on_the_host(client):
    out = run(client, -1)
    op = oops.build("proton")
    assert out[0] == f"terms {sum(len(t) for t in op.terms)}"
    assert out[1] == f"canonical {ocor.CanonicalPlan(op).n_terms}"
    assert out[2] == "guard 3 5e-07"
    assert out[3] == "shape 384 1 2"


@pytest.mark.gpu
def test_c_client_evaluates_on_the_gpu(client, tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    U, D = mi.workload_fields("proton_4x8")
    T, V3 = U.shape[:2]
    path = str(tmp_path / "fields.bin")
    with open(path, "wb") as f:
        f.write(np.ascontiguousarray(U).tobytes())
        f.write(np.ascontiguousarray(D).tobytes())
    out = run(client, 0, path, T, V3)
    want = ocor.correlator(ocor.CanonicalPlan(oops.build("proton")).site_values, U, D)
    for tag, tol in (("C", 1e-12), ("H", 1e-12), ("F", 5e-7)):
        got = np.array([complex(float(l.split()[2]), float(l.split()[3])) for l in out if l.startswith(tag + " ")])
        assert len(got) == T
        assert np.max(np.abs(got - want) / np.abs(want)) <= tol, tag
