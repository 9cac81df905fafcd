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


def test_bounds_check_is_off_in_the_default_build(lib):
    """The default library compiles the index checks out: hh_bounds_check
    reports them disabled, with no record, without touching the device, and
    refuses an unknown op."""
    from paper_1007_3432_gb300 import binding
    L = binding.load()
    en, rec = ctypes.c_int(7), ctypes.c_longlong(7)
    assert L.hh_bounds_check(binding.HH_BOUNDS_READ, ctypes.byref(en), ctypes.byref(rec)) == binding.HH_OK
    assert en.value == 0 and rec.value == 0
    assert L.hh_bounds_check(5, None, None) == binding.HH_EINVAL
    assert L.hh_strerror(binding.HH_EBOUNDS).decode().startswith("an index check")


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


def test_chebyshev_table_matches_oracle_polynomial(tmp_path):
    """The engine's Chebyshev table (Leja-ordered real factors, Sec. 4.2),
    evaluated factor by factor on the host, against the oracle's P(z) of
    Eq. (13) on [eps, 1]: the same polynomial to 1e-11 relative."""
    import shutil
    import numpy as np
    import oracle
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = str(tmp_path / "cheb_table_dump")
    subprocess.check_call([nvcc, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"),
                           os.path.join(ROOT, "tests", "native", "cheb_table_dump.cu"),
                           os.path.join(ROOT, "paper_1007_3432_gb300", "csrc", "hh_engine_host.cu"), "-o", exe])
    for n, eps in [(4, 1e-3), (8, 1e-4), (32, 1e-5), (64, 1e-6)]:
        zs = np.concatenate([np.geomspace(eps, 1.0, 25), np.linspace(0.0, 1.0, 11)])
        out = subprocess.run([exe, str(n), repr(eps)] + [repr(float(z)) for z in zs],
                             capture_output=True, text=True, check=True)
        got = np.array([float(v) for v in out.stdout.split()])
        ref = np.array([oracle.cheb_poly(n, eps, float(z)) for z in zs])
        assert np.all(np.abs(got - ref) <= 1e-11 * np.abs(ref)), (n, eps, np.max(np.abs(got - ref) / np.abs(ref)))


def test_public_header_compiles_as_c99_and_cxx11():
    """include/hubhmc.h is a plain C header: no CUDA or C++ types leak into it."""
    hdr = os.path.join(ROOT, "include", "hubhmc.h")
    for cmd in (["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-fsyntax-only", "-x", "c", hdr],
                ["g++", "-std=c++11", "-Wall", "-Werror", "-fsyntax-only", "-x", "c++", hdr]):
        subprocess.check_call(cmd)


def build_c_consumer(out_dir):
    """Compile tests/native/c_consumer.c as C99 and link it against the built
    library and the CUDA runtime; returns (executable, library directories)."""
    import glob
    import shutil
    from paper_1007_3432_gb300 import build
    build.build()
    cuda = os.path.dirname(os.path.dirname(shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"))
    libdir = next((d for d in glob.glob(os.path.join(cuda, "lib*")) + glob.glob(os.path.join(cuda, "targets", "*", "lib"))
                   if glob.glob(os.path.join(d, "libcudart.so*"))), os.path.join(cuda, "lib64"))
    exe = os.path.join(str(out_dir), "c_consumer")
    subprocess.check_call(["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                           "-I", os.path.join(cuda, "include"), os.path.join(ROOT, "tests", "native", "c_consumer.c"),
                           "-L", os.path.dirname(build.LIB), "-lhubhmc", "-L", libdir, "-lcudart", "-o", exe])
    return exe, [os.path.dirname(build.LIB), libdir]


def test_plain_c_program_links_against_the_library(tmp_path):
    """tests/native/c_consumer.c (a context, a solve, a multi-vector apply,
    the observables and a trajectory through the C ABI) compiles as C99 and
    links against the built library; tests/test_gpu_c_consumer.py runs it."""
    exe, _ = build_c_consumer(tmp_path)
    assert os.path.exists(exe)
