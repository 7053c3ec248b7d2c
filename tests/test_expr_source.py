"""The library's translation of stencil.apply expressions (no GPU needed):
stencil_expr_source accepts what the oracle's parser accepts, rejects what
it rejects, reports the same bounds radius, and produces CUDA C that the
device compiler takes."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import expr as E
from paper_2310_01882_b300 import stencil as S

GOOD = [
    ("a0(0,0,0)", 1),
    ("1.e2*a0(0,0,0) - .5E-1 + 7.", 1),
    ("0.25*(a0(-1,0,0) + a0(1,0,0)) - -a1(0,2,-1)/3", 2),
    ("a0(1,-2,3)*a2(0,0,0) + 1e-3*(a1(0,0,1) - a1(0,0,-1))", 3),
    ("((a0(0,0,0)))", 1),
]
BAD = ["a0(4,0,0)", "a3(0,0,0)", "1 +", "a0(0,0)", "b0(0,0,0)", "((1)", "1e999", "2 3", "", "0x10", "0x1p3",
       "1e", ".", "1.5.2", "inf", "a0(0,0,0) ^ 2"]


@pytest.mark.parametrize("expr,ninputs", GOOD)
def test_accepts_and_reports_the_oracle_radius(expr, ninputs):
    src, r = S.stencil_expr_source(expr, ninputs)
    assert "stencil_expr_kernel" in src and "__dfma" not in src and "fma(" not in src
    assert r == E.parse(expr, ninputs)[1]


@pytest.mark.parametrize("expr", BAD)
def test_rejects_what_the_oracle_rejects(expr):
    with pytest.raises(ValueError):
        E.parse(expr, 3)
    with pytest.raises(S.StencilError) as e:
        S.stencil_expr_source(expr, 3)
    assert e.value.code == -1


def test_input_count_limits():
    for n in (0, 9):
        with pytest.raises(S.StencilError):
            S.stencil_expr_source("1", n)


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="no device compiler")
def test_generated_source_compiles_for_sm_103a(tmp_path):
    src, _ = S.stencil_expr_source(GOOD[1][0], 2)
    f = tmp_path / "gen.cu"
    f.write_text(src)
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    r = subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-fmad=false", "-c", str(f), "-o",
                        str(tmp_path / "gen.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
