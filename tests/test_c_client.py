"""The C ABI without Python: tests/c_client/masw_client.c, a plain C11
program, compiles against include/masw.h with -std=c11 -pedantic -Werror and
links against libmasw.so (CPU); on a GPU its dispersion, leaky and misfit
outputs equal the Python binding's for the same models."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2003_02256_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_client", "masw_client.c")


def compile_client(tmp_path):
    from paper_2003_02256_gb300 import build
    so = build.build()
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no gcc")
    out = os.path.join(str(tmp_path), "masw_client")
    libdir = os.path.dirname(so)
    subprocess.run([gcc, "-std=c11", "-Wall", "-Wextra", "-Werror", "-pedantic",
                    "-I", os.path.join(ROOT, "include"), SRC, "-L", libdir, "-lmasw",
                    "-Wl,-rpath," + libdir, "-o", out], check=True)
    return out


def test_client_compiles_as_c11_and_links(tmp_path):
    assert os.path.exists(compile_client(tmp_path))


@pytest.mark.gpu
def test_client_results_equal_the_python_binding(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2003_02256_gb300 import masw
    out = subprocess.run([compile_client(tmp_path)], capture_output=True, text=True, check=True)
    rec = {}
    for line in out.stdout.splitlines():
        f = line.split()
        rec.setdefault(f[0], []).append(f[1:])
    m = W.Models(np.array([2, 1], np.int32), np.array([2.0, 4.0, 3.0]),
                 np.array([400.0, 600.0, 800.0, 450.0, 900.0]),
                 np.array([180.0, 260.0, 380.0, 200.0, 420.0]),
                 np.array([1850.0, 1900.0, 2000.0, 1800.0, 2000.0]),
                 np.array([3, 2], np.int32), np.array([2.0, 10.0, 40.0, 5.0, 25.0]))
    with masw.Batch(m, W.Grid(50.0, 0.5, 1500)) as b:
        ct, idx, st = b.dispersion()
        phi = b.misfit(ct + 1.0)
        _, idx_l, st_l = b.leaky()
    assert [int(r[1]) for r in rec["idx"]] == idx.tolist()
    assert [int(r[2]) for r in rec["idx"]] == st.tolist()
    assert [int(r[1]) for r in rec["leaky"]] == idx_l.tolist()
    assert [int(r[2]) for r in rec["leaky"]] == st_l.tolist()
    assert np.allclose([float(r[1]) for r in rec["misfit"]], phi, rtol=1e-12)
    assert (st == 0).all()


def test_header_compiles_as_cpp_with_c_linkage(tmp_path):
    """include/masw.h also serves C++ callers: its extern "C" block keeps the
    symbols unmangled, so a C++ translation unit links against libmasw."""
    from paper_2003_02256_gb300 import build
    so = build.build()
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    src = tmp_path / "client.cpp"
    src.write_text('#include "masw.h"\nint main() { return masw_strerror(0) ? 0 : 1; }\n')
    out = str(tmp_path / "client_cpp")
    libdir = os.path.dirname(so)
    subprocess.run([gxx, "-std=c++17", "-Wall", "-Wextra", "-Werror", "-I",
                    os.path.join(ROOT, "include"), str(src), "-L", libdir, "-lmasw",
                    "-Wl,-rpath," + libdir, "-o", out], check=True)
    assert subprocess.run([out]).returncode == 0
