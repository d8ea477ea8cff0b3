"""The boundary is a plain C ABI: tests/c_abi_host.c, a C99 program that includes only
include/lsms.h, compiles with gcc -std=c99 -pedantic -Wall -Wextra -Werror, links against liblsms.so
and calls the host-only entry points and lsms_create.  Its printed results equal, to the last bit,
what the Python binding gets from the same library (the inclusion matrix, whose curve is sampled
by C's and NumPy's cos/sin separately, to 1e-13)."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1407_3868_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1407_3868_gb300 import build as b
    b.build()
    from paper_1407_3868_gb300 import lsms
    return lsms


@pytest.fixture(scope="module")
def c_results(lib, tmp_path_factory):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path_factory.mktemp("c_abi") / "c_abi_host")
    libdir = os.path.dirname(lib.LIB_PATH)
    cmd = [gcc, "-std=c99", "-pedantic", "-Wall", "-Wextra", "-Werror", "-I" + os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c_abi_host.c"), "-o", exe, "-L" + libdir, "-llsms", "-lm",
           "-Wl,-rpath," + libdir]
    res = subprocess.run(cmd, capture_output=True, text=True)
    assert res.returncode == 0, res.stderr
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    vals, text = {}, {}
    for line in out.stdout.splitlines():
        name, _, rest = line.partition(" ")
        text[name] = rest
        try:
            vals[name] = np.array([float(v) for v in rest.split()])
        except ValueError:
            pass
    return vals, text


def cplx(v):
    return v[0::2] + 1j * v[1::2]


def test_c_program_sees_the_same_host_results(lib, c_results):
    v, _ = c_results
    k1, k2, k3, kp, R, p = 2 * math.pi, 3 * math.pi, 4 * math.pi, 2.4 * math.pi, 0.25, 6
    assert v["build_contour_rc"][0] == 0
    lam, wt = lib.build_contour(256, k1, k2, k3, 0.2, 40.0, 16)
    assert np.array_equal(cplx(v["nodes_head"]), lam[:4])
    assert np.array_equal(cplx(v["weights_tail"]), wt[-4:])
    assert v["mie_rc"][0] == 0
    assert np.array_equal(cplx(v["mie"]), lib.scattering_diagonal(p, k2, kp, R))
    assert np.array_equal(cplx(v["mie_absorbing"]), lib.scattering_diagonal(p, k2, kp + 0.5j, R))
    assert np.array_equal(cplx(v["pec"]), lib.pec_scattering_diagonal(p, k2, R))
    assert v["mie_absorbing_bad_rc"][0] == -1
    assert v["geometry_ok"][0] == 0 and v["geometry_close"][0] == -2
    assert v["layer_response_rc"][0] == 0
    want = lib.layer_response([1.0, 2.5, 3.0, 1.5], [0.7, 2.0], 3, np.array([0.5 - 0.1j, 2.7 - 0.1j]))
    assert np.array_equal(cplx(v["layer_response"]), np.asarray(want).ravel())


def test_c_program_inclusion_matrices(lib, c_results):
    v, _ = c_results
    k2, kp, R = 3 * math.pi, 2.4 * math.pi, 0.25
    assert v["inclusion_rc"][0] == 0
    cur = inputs.star_curve(0.2, 0.0, 0, 64)
    for key, k in (("inclusion", kp), ("inclusion_absorbing", kp + 0.5j)):
        got = cplx(v[key]).reshape(5, 5)
        want = lib.inclusion_scattering_matrix(2, k2, k, R, cur)
        assert np.abs(got - want).max() < 1e-13 * np.abs(want).max(), key


def test_c_program_create_reports_the_missing_gpu(c_results):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    v, text = c_results
    assert v["create_rc"][0] == -6
    assert "CUDA" in text["create_error"] or "cuda" in text["create_error"]
