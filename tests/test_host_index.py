"""Host logic of the CUDA path that needs no GPU: the multiply-shift division
every kernel uses to turn a linear node index into grid coordinates (axis 0
fastest).  The check program includes the library's own header, so it tests
the code the kernels compile, on the host."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_fast_division_matches_integer_division(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "fast_div_check")
    subprocess.run([nvcc, "-std=c++17", "-I" + os.path.join(ROOT, "include"), "-o", exe,
                    os.path.join(HERE, "native", "fast_div_check.cu")], check=True, capture_output=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr


def test_double_float_transformations(tmp_path):
    """The double-float primitives of the outer Krylov kernels (two-sum,
    the FMA two-product, the float64 split and the normalisation), compiled
    for the host from the library's own header: exactness where the
    transformations are exact, and a running sum of 256 products within
    256 x 2^-46 of the terms' magnitude sum against an exact long double
    reference."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "df_check")
    subprocess.run([nvcc, "-std=c++17", "-Xcompiler", "-ffp-contract=off", "-o", exe,
                    os.path.join(HERE, "native", "df_check.cu")], check=True, capture_output=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr


def test_arnoldi_scalar_helpers(tmp_path):
    """The single-thread parts of the GMRES iterations (complex Givens
    rotations, the Hessenberg column update with its running residual
    estimate, the back substitution, the breakdown stop and the selective
    second-pass decision from Pythagoras), compiled for the host from the
    library's own header, against a modified Gram-Schmidt least-squares
    solve in long double (Sec. 3.1: FGMRES and the coarsest GMRES)."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "krylov_check")
    subprocess.run([nvcc, "-std=c++17", "-I" + os.path.join(ROOT, "include"), "-o", exe,
                    os.path.join(HERE, "native", "krylov_check.cu")], check=True, capture_output=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
