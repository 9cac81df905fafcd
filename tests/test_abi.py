"""CPU checks of the C ABI library: it builds, loads without a GPU, and
exports every function that the public header declares."""
import ctypes
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1007_3432_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_symbols_exported(lib):
    from paper_1007_3432_gb300.binding import header_symbols
    names = header_symbols()
    assert "hh_create" in names and "hh_trajectory" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_and_defaults_need_no_gpu(lib):
    from paper_1007_3432_gb300 import binding
    L = binding.load()
    assert L.hh_strerror(-4).decode().startswith("CG did not converge")
    p = binding.hh_params()
    L.hh_default_params(ctypes.byref(p))
    assert p.cg_tol == 1e-10 and p.n_pf == 2 and p.A == 0.5 and p.dtau == 0.05
    assert L.hh_nsites(None) == 0
    assert L.hh_destroy(None) == 0


def test_create_rejects_bad_shapes_before_touching_the_device(lib):
    from paper_1007_3432_gb300 import binding
    L = binding.load()
    p = binding.hh_params()
    L.hh_default_params(ctypes.byref(p))
    h = ctypes.c_void_p()
    for d, nx, nt in [(2, 4, 4), (1, 1, 4), (3, 4, 1), (3, 1400, 1000)]:
        lat = binding.hh_lattice(d, nx, nt)
        assert L.hh_create(ctypes.byref(h), ctypes.byref(lat), ctypes.byref(p), None) == -1
    lat = binding.hh_lattice(1, 8, 8)
    p.precision = 7
    assert L.hh_create(ctypes.byref(h), ctypes.byref(lat), ctypes.byref(p), None) == -1


def test_fast_division_matches_integer_division(tmp_path):
    import shutil
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "fastdiv_check")
    subprocess.check_call([nvcc, "-O2", "-std=c++17", os.path.join(ROOT, "tests", "native", "fastdiv_check.cu"),
                           "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr


def test_host_logic_tiling_and_md_schedules(tmp_path):
    """Engine tiling covers every site once in 32-aligned chunks; leapfrog and
    Omelyan schedules kick and drift n_md * dt in total (host-only build)."""
    import shutil
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "host_logic_check")
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "native", "host_logic_check.cu"), "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
