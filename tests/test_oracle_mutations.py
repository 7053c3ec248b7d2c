"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake in a copy of oracle.c (on the CPU: a swapped
neighbour, a sign, a transposed axis, a swapped coefficient, a dropped term,
a correction solve that does not restart from zero, a wrong escalation),
builds it into a temporary library and runs the pin suites against it in a
subprocess (ORACLE_LIB).  The pins must fail for every mutant."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")
PINS = ["tests/test_oracle_jacobi.py", "tests/test_oracle_residual.py", "tests/test_oracle_advect.py",
        "tests/test_oracle_rbgs.py", "tests/test_oracle_average2d.py", "tests/test_oracle_apply_linear.py",
        "tests/test_oracle_refine.py"]

MUTANTS = {
    "sweep_z_as_y": ("s += AT(u, i, j, k + 1);\n        s += hh", "s += AT(u, i, j + 1, k);\n        s += hh"),
    "sweep_drop_source": ("s += hh * AT(f, i, j, k);\n        AT(out", "s += 0.0 * AT(f, i, j, k);\n        AT(out"),
    "sweep_div5": ("AT(out, i, j, k) = s / 6.0;", "AT(out, i, j, k) = s / 6.000001;"),
    "residual_sign": ("(6.0 * AT(u, i, j, k) - s) / hh", "(6.0 * AT(u, i, j, k) + s) / hh"),
    "residual_fnorm": ("ff += AT(f, i, j, k) * AT(f, i, j, k);", "ff += AT(f, i, j, k) * AT(u, i, j, k);"),
    "su_v_index": ("(AT(v, i, j - 1, k) + AT(v, i + 1, j - 1, k))", "(AT(v, i, j - 1, k) + AT(v, i - 1, j - 1, k))"),
    "sv_u_index": ("(AT(u, i - 1, j, k) + AT(u, i - 1, j + 1, k)) -", "(AT(u, i - 1, j, k) + AT(u, i, j + 1, k)) -"),
    "sw_tzc_swap": ("c2 * AT(w, i, j, k + 1) * (AT(w, i, j, k) + AT(w, i, j, k + 1))",
                    "c1 * AT(w, i, j, k + 1) * (AT(w, i, j, k) + AT(w, i, j, k + 1))"),
    "su_sign_x": ("tx = tcx * (AT(u, i - 1, j, k) * (AT(u, i, j, k) + AT(u, i - 1, j, k)) -",
                  "tx = tcx * (AT(u, i - 1, j, k) * (AT(u, i, j, k) + AT(u, i - 1, j, k)) +"),
    "sw_drop_y": ("AT(sw, i, j, k) = tx + ty + tz;", "AT(sw, i, j, k) = tx + tz;"),
    "rb_black_first": ("if (((i + j + k) & 1) != color) continue;", "if (((i + j + k + 1) & 1) != color) continue;"),
    "rb_colour_ij": ("if (((i + j + k) & 1) != color) continue;", "if (((i + j) & 1) != color) continue;"),
    "avg2d_y_as_z": ("s += AT(a, i, j + 1, k);\n          AT(b, i, j, k) = s * 0.25;",
                     "s += AT(a, i, j, k + 1);\n          AT(b, i, j, k) = s * 0.25;"),
    "avg2d_third": ("AT(b, i, j, k) = s * 0.25;", "AT(b, i, j, k) = s * 0.3333333333333333;"),
    "apply_axes_swapped": ("AT(in, i + offsets[3 * p], j + offsets[3 * p + 1], k + offsets[3 * p + 2])",
                           "AT(in, i + offsets[3 * p + 1], j + offsets[3 * p], k + offsets[3 * p + 2])"),
    "rb_drop_source": ("s += hh * AT(f, i, j, k);\n            AT(u, i, j, k) = s / 6.0;",
                       "s += 0.0 * AT(f, i, j, k);\n            AT(u, i, j, k) = s / 6.0;"),
    # mixed-precision refinement
    "refine_no_restart_f64": ("memset(e64, 0, len * sizeof(double));", ";"),
    "refine_correction_sign": ("AT(u, i, j, k) = AT(u, i, j, k) + AT(e, i, j, k);",
                               "AT(u, i, j, k) = AT(u, i, j, k) - AT(e, i, j, k);"),
    "refine_absolute_residual": ("double rel = norms[1] > 0.0 ? norms[0] / norms[1] : norms[0];",
                                 "double rel = norms[0];"),
    "refine_escalate_to_f64": ("if (cur == 2) {\n        cur = 1;", "if (cur == 2) {\n        cur = 0;"),
    "refine_f32_start_from_r": ("r32[q] = (float)r[q]; e32[q] = 0.0f;", "r32[q] = (float)r[q]; e32[q] = r32[q];"),
    # reduced-precision storage
    "bf16_truncates": ("x += 0x7fffu + lsb;", "x += 0u * lsb;"),
    "f32_sweep_z_as_y": ("        s += AT(u, i, j, k + 1);\n        s += hh * AT(f, i, j, k);\n        AT(out, i, j, k) = s / 6.0f;",
                         "        s += AT(u, i, j + 1, k);\n        s += hh * AT(f, i, j, k);\n        AT(out, i, j, k) = s / 6.0f;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, name
    mutated = src.replace(old, new, 1)
    csrc = tmp_path / "oracle_mut.c"
    csrc.write_text(mutated)
    lib = tmp_path / "liboracle_mut.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", str(lib),
                    str(csrc), "-lm"], check=True)
    env = dict(os.environ, ORACLE_LIB=str(lib))
    res = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", *PINS],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert res.returncode != 0, f"mutant {name} survived the pins:\n{res.stdout[-2000:]}"


NET_SRC = os.path.join(ROOT, "oracle", "net.py")
NET_MUTANTS = {
    "conv_tap_flipped": ("out += pad[dz:dz + D, dy:dy + H, dx:dx + Wd, :] @ W[dz, dy, dx]",
                         "out += pad[dz:dz + D, dy:dy + H, dx:dx + Wd, :] @ W[2 - dz, dy, dx]"),
    "conv_bwd_wrong_tap": ("dpad[dz:dz + D, dy:dy + H, dx:dx + Wd, :] += g @ W[dz, dy, dx].T",
                           "dpad[dz:dz + D, dy:dy + H, dx:dx + Wd, :] += g @ W[dz, dy, 2 - dx].T"),
    "pool_bwd_scale": ("0), 2, 1), 2, 2) / 8.0", "0), 2, 1), 2, 2) / 4.0"),
    "skip_dropped_in_backward": ("g = g + gskip[l]", "g = g"),
    "relu_mask_of_other_layer": ('g = g * (cache[f"enc{l}b.out"] > 0)', 'g = g * (cache[f"enc{l}a.out"] > 0)'),
    "filter_weights": ("y = 0.25 * p[sl(0, n)] + 0.5 * p[sl(1, n + 1)] + 0.25 * p[sl(2, n + 2)]",
                       "y = 0.25 * p[sl(0, n)] + 0.5 * p[sl(1, n + 1)] + 0.2 * p[sl(2, n + 2)]"),
    "mse_grad_half": ("return float(np.mean(d * d)), 2.0 * d / d.size", "return float(np.mean(d * d)), d / d.size"),
    "adam_eps_inside_sqrt": ("(np.sqrt(v1 / c2) + eps)", "np.sqrt(v1 / c2 + eps)"),
    "adam_no_bias_correction": ("c1 = 1.0 - b1 ** t", "c1 = 1.0"),
}


@pytest.mark.parametrize("name", sorted(NET_MUTANTS))
def test_net_pins_catch_mutant(name, tmp_path):
    """The same for the FP64 network oracle (oracle/net.py): a copy of the
    oracle package with one planted mistake shadows the real one on the
    pins' import path."""
    import shutil
    import oracle
    old, new = NET_MUTANTS[name]
    src = open(NET_SRC).read()
    assert src.count(old) >= 1, name
    pkg = tmp_path / "oracle"
    shutil.copytree(os.path.join(ROOT, "oracle"), pkg,
                    ignore=shutil.ignore_patterns("__pycache__", "*.so", "_build"))
    (pkg / "net.py").write_text(src.replace(old, new, 1))
    env = dict(os.environ, ORACLE_LIB=oracle.lib()._name,
               PYTHONPATH=os.pathsep.join([str(tmp_path), ROOT, os.environ.get("PYTHONPATH", "")]))
    # run from the copy's parent, so that it comes first on the import path
    res = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                          os.path.join(ROOT, "tests", "test_oracle_net.py")], cwd=str(tmp_path), env=env,
                         capture_output=True, text=True, timeout=600)
    assert res.returncode != 0, f"mutant {name} survived the pins:\n{res.stdout[-2000:]}"


def test_net_mutation_harness_passes_unmutated(tmp_path):
    """Control: the shadowing copy without a mutation passes the pins (so a
    failure above is the planted mistake's)."""
    import shutil
    import oracle
    pkg = tmp_path / "oracle"
    shutil.copytree(os.path.join(ROOT, "oracle"), pkg,
                    ignore=shutil.ignore_patterns("__pycache__", "*.so", "_build"))
    env = dict(os.environ, ORACLE_LIB=oracle.lib()._name,
               PYTHONPATH=os.pathsep.join([str(tmp_path), ROOT, os.environ.get("PYTHONPATH", "")]))
    res = subprocess.run([sys.executable, "-c", "import oracle, sys; print(oracle.__file__)"], cwd=str(tmp_path),
                         env=env, capture_output=True, text=True, timeout=120)
    assert str(tmp_path) in res.stdout, res.stdout + res.stderr
    res = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                          os.path.join(ROOT, "tests", "test_oracle_net.py")], cwd=str(tmp_path), env=env,
                         capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stdout[-2000:]
    # and it is the copy that the pins import
    probe = tmp_path / "probe_test.py"
    probe.write_text("import oracle\n\ndef test_probe():\n    assert oracle.__file__.startswith(%r)\n"
                     % str(tmp_path))
    res = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", "-c",
                          os.path.join(ROOT, "pytest.ini"), "--rootdir", ROOT, str(probe)], cwd=str(tmp_path),
                         env=env, capture_output=True, text=True, timeout=120)
    assert res.returncode == 0, res.stdout[-2000:]


EXPR_SRC = os.path.join(ROOT, "oracle", "expr.py")
EXPR_MUTANTS = {
    "operands_swapped": ("node = (op, node, self.term())", "node = (op, self.term(), node)"),
    "product_looser_than_sum": ("node = (op, node, self.unary())", "node = (op, node, self.expr())"),
    "divide_as_multiply": ('"/": np.divide', '"/": np.multiply'),
    "minus_dropped": ("return np.negative(ev(node[1]))", "return ev(node[1])"),
    "y_offset_sign": ("r + dy:ny2 - r + dy", "r - dy:ny2 - r - dy"),
    "x_and_z_swapped": ("dx, dy, dz = d", "dz, dy, dx = d"),
    "radius_ignores_z": ("for d in node[2]:", "for d in node[2][:2]:"),
}


@pytest.mark.parametrize("name", sorted(EXPR_MUTANTS))
def test_expr_pins_catch_mutant(name, tmp_path):
    """The same for the expression oracle (oracle/expr.py)."""
    import shutil
    import oracle
    old, new = EXPR_MUTANTS[name]
    src = open(EXPR_SRC).read()
    assert src.count(old) == 1, name
    pkg = tmp_path / "oracle"
    shutil.copytree(os.path.join(ROOT, "oracle"), pkg,
                    ignore=shutil.ignore_patterns("__pycache__", "*.so", "_build"))
    (pkg / "expr.py").write_text(src.replace(old, new, 1))
    env = dict(os.environ, ORACLE_LIB=oracle.lib()._name,
               PYTHONPATH=os.pathsep.join([str(tmp_path), ROOT, os.environ.get("PYTHONPATH", "")]))
    res = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                          os.path.join(ROOT, "tests", "test_oracle_expr.py")], cwd=str(tmp_path), env=env,
                         capture_output=True, text=True, timeout=600)
    assert res.returncode != 0, f"mutant {name} survived the pins:\n{res.stdout[-2000:]}"


def test_expr_mutation_harness_passes_unmutated(tmp_path):
    """Control: the unmutated copy passes the expression pins."""
    import shutil
    import oracle
    pkg = tmp_path / "oracle"
    shutil.copytree(os.path.join(ROOT, "oracle"), pkg,
                    ignore=shutil.ignore_patterns("__pycache__", "*.so", "_build"))
    env = dict(os.environ, ORACLE_LIB=oracle.lib()._name,
               PYTHONPATH=os.pathsep.join([str(tmp_path), ROOT, os.environ.get("PYTHONPATH", "")]))
    res = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                          os.path.join(ROOT, "tests", "test_oracle_expr.py")], cwd=str(tmp_path), env=env,
                         capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stdout[-2000:]
