"""A plain C program calls the library through include/stencil.h alone
(no Python between): it compiles and links here; on a GPU its Jacobi sweeps
match the oracle's."""
import os
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = "/usr/local/cuda"


def build_caller(tmp_path):
    from paper_2310_01882_b300 import build
    libdir = os.path.dirname(build.build())
    exe = tmp_path / "c_abi_jacobi"
    res = subprocess.run(["gcc", "-std=c99", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                          "-I", os.path.join(CUDA, "include"), os.path.join(ROOT, "tests", "c_abi_jacobi.c"),
                          "-o", str(exe), "-L", libdir, "-lstencil", "-L", os.path.join(CUDA, "lib64"), "-lcudart",
                          f"-Wl,-rpath,{libdir}", f"-Wl,-rpath,{os.path.join(CUDA, 'lib64')}"],
                         capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    return exe


def test_c_caller_builds(tmp_path):
    assert build_caller(tmp_path).exists()


@pytest.mark.gpu
@pytest.mark.parametrize("shape,nsweeps", [((30, 21, 17), 12), ((64, 64, 64), 100)])
def test_c_caller_matches_oracle(tmp_path, shape, nsweeps):
    exe = build_caller(tmp_path)
    nx, ny, nz = shape
    rng = np.random.default_rng(sum(shape))
    u = rng.random((nz + 2, ny + 2, nx + 2))
    f = rng.standard_normal(u.shape)
    u.tofile(tmp_path / "u.bin")
    f.tofile(tmp_path / "f.bin")
    res = subprocess.run([str(exe), str(nx), str(ny), str(nz), str(nsweeps), str(tmp_path / "u.bin"),
                          str(tmp_path / "f.bin"), str(tmp_path / "out.bin")], capture_output=True, text=True,
                         timeout=300)
    assert res.returncode == 0, res.stderr
    got = np.fromfile(tmp_path / "out.bin").reshape(u.shape)
    ref = oracle.jacobi(u, f, 1.0 / (nx + 1), nsweeps)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
    # the Dirichlet halo is never written
    for sl in (np.s_[0], np.s_[-1], np.s_[:, 0], np.s_[:, -1], np.s_[:, :, 0], np.s_[:, :, -1]):
        assert np.array_equal(got[sl], u[sl])
