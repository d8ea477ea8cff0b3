"""Host-side checks of the C ABI that need no GPU: the library loads, exports every symbol the
header declares, and its host logic (contour, disc scattering matrix, geometry validation) agrees
with the oracle and with the stated rules."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from oracle import lsms_oracle as O
from paper_1407_3868_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MED_K = (inputs.MEDIUM["k1"], inputs.MEDIUM["k2"], inputs.MEDIUM["k3"])


@pytest.fixture(scope="module")
def lib():
    from paper_1407_3868_gb300 import build as b
    b.build()
    from paper_1407_3868_gb300 import lsms
    return lsms


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lsms.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lsms_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    so = ctypes.CDLL(lib.LIB_PATH)
    for name in names:
        assert hasattr(so, name), name
    assert set(lib.EXPORTS) == set(names)


def test_library_links_no_vendor_fft_or_blas(lib):
    # every step of the path runs in the library's own kernels: no cuFFT / cuBLAS dependency or
    # symbol in the shared library (tool output: its dynamic section and dynamic symbol table)
    import shutil
    import subprocess
    readelf, nm = shutil.which("readelf"), shutil.which("nm")
    if not readelf or not nm:
        pytest.skip("binutils not installed")
    needed = subprocess.run([readelf, "-d", lib.LIB_PATH], capture_output=True, text=True, check=True).stdout
    syms = subprocess.run([nm, "-D", lib.LIB_PATH], capture_output=True, text=True, check=True).stdout
    for name in ("cufft", "cublas", "cusparse", "cudnn"):
        assert name not in needed.lower(), name
        assert name not in syms.lower(), name


@pytest.mark.parametrize("name", ["disc16_p10_ns256", "disc1000_p12_ns512", "disc5000_p14_ns1024",
                                  "disc2000_p12_ns768_src64"])
def test_library_contour_equals_oracle_contour(lib, name):
    w = inputs.WORKLOADS[name]
    m = w.medium
    lam, wt = lib.build_contour(w.n_nodes, m["k1"], m["k2"], m["k3"], w.b, w.t_max, 16)
    lam_o, wt_o = O.contour(w.n_nodes, m["k1"], m["k2"], m["k3"], w.b, w.t_max)
    assert np.max(np.abs(lam - lam_o)) <= 1e-12 * w.t_max
    assert np.max(np.abs(wt - wt_o)) <= 1e-14 * w.t_max


@pytest.mark.parametrize("ks,b,n_nodes,t_max", [((1.0, 6.0, 1.0), 0.2, 1024, 40.0),
                                              ((1.0, 20.0, 1.0), 0.19, 2048, 40.0),
                                              ((2.0, 3.0, 2.5), 0.05, 768, 25.0)])
def test_library_contour_equals_oracle_contour_in_guided_media(lib, ks, b, n_nodes, t_max):
    lam, wt = lib.build_contour(n_nodes, *ks, b, t_max, 16)
    lam_o, wt_o = O.contour(n_nodes, *ks, b, t_max)
    assert np.max(np.abs(lam - lam_o)) <= 1e-12 * t_max
    assert np.max(np.abs(wt - wt_o)) <= 1e-14 * t_max
    # the band refines the panels between max(k1, k3) and k2 (where it is wider than the panels)
    if ks[1] - max(ks[0], ks[2]) > 20 * b:
        lam_p, _ = O.contour(n_nodes, *ks, b, t_max, guided=False)
        assert np.max(np.abs(lam - lam_p)) > 1e-3


@pytest.mark.parametrize("ks,b,n_nodes,t_max", [(MED_K, 0.2, 256, 141.0), (MED_K, 9.4e-4, 1024, 163.0),
                                              ((1.0, 6.0, 1.0), 0.2, 1024, 40.0)])
def test_library_greedy_contour_equals_oracle(lib, ks, b, n_nodes, t_max):
    # panel_rule = 1: the length / (b + distance) rule in every medium (the default in guided media)
    lam, wt = lib.build_contour(n_nodes, *ks, b, t_max, 16, 1)
    lam_o, wt_o = O.contour(n_nodes, *ks, b, t_max, greedy=True)
    assert np.max(np.abs(lam - lam_o)) <= 1e-12 * t_max
    assert np.max(np.abs(wt - wt_o)) <= 1e-14 * t_max
    lam_d, _ = lib.build_contour(n_nodes, *ks, b, t_max, 16, 0)
    guided = ks[1] > max(ks[0], ks[2])
    assert (np.array_equal(lam, lam_d)) == guided
    with pytest.raises(lib.LsmsError) as e:
        lib.build_contour(n_nodes, *ks, b, t_max, 16, 2)
    assert e.value.code == -1


def test_contour_defaults_follow_the_paper(lib):
    # b = 0.2, t_max = max k + 20, 16-point panels (Sec. 6)
    lam, wt = lib.build_contour(500, 1.0, 3.0, 1.0)
    assert np.isclose(lam[-1].imag, -0.2) and lam[-1].real < 23.0
    lam_o, wt_o = O.contour(500, 1.0, 3.0, 1.0, 0.2, 23.0)
    assert np.allclose(lam, lam_o, atol=1e-13) and np.allclose(wt, wt_o, atol=1e-14)


def test_contour_rejects_too_few_nodes(lib):
    with pytest.raises(lib.LsmsError) as e:
        lib.build_contour(40, 1.0, 3.0, 1.0, 0.2, 20.0, 16)
    assert e.value.code == -1


@pytest.mark.parametrize("p", [0, 5, 10, 14, 15])
def test_library_scattering_matrix_equals_oracle(lib, p):
    m = inputs.MEDIUM
    s = lib.scattering_diagonal(p, m["k2"], m["kp"], m["radius"])
    s_o = O.mie_coefficients(p, m["k2"], m["kp"], m["radius"])
    assert np.allclose(s, s_o, rtol=1e-11, atol=0)


def test_geometry_rules(lib):
    d, R = 2.0, 0.25
    ok = np.array([[0.0, -1.0], [0.6, -1.0], [0.3, -0.3]])
    assert lib.check_geometry(d, R, ok) == 0
    # gap below 0.2 R
    assert lib.check_geometry(d, R, [[0.0, -1.0], [0.54, -1.0]]) == -2
    # touching the top interface
    assert lib.check_geometry(d, R, [[0.0, -0.25]]) == -2
    # crossing the bottom interface
    assert lib.check_geometry(d, R, [[0.0, -1.8]]) == -2
    # non-finite
    assert lib.check_geometry(d, R, [[math.nan, -1.0]]) == -1
    assert lib.check_geometry(d, R, np.zeros((0, 2))) == 0
    # every generated workload layout is valid
    assert lib.check_geometry(d, R, inputs.WORKLOADS["disc1000_p12_ns512"].centres()) == 0


def test_create_without_a_gpu_reports_an_error(lib):
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(lib.LsmsError) as e:
        lib.Context(1.0, 3.0, 1.0, 2.0, 2.0, 0.25, 5, 128)
    assert e.value.code == -6


def test_seeded_layouts_respect_the_geometry():
    c = inputs.layout(200, -50.0, 50.0, 9)
    assert c.shape == (200, 2)
    assert np.all(c[:, 1] >= -1.7) and np.all(c[:, 1] <= -0.3)
    dd = np.hypot(c[:, None, 0] - c[None, :, 0], c[:, None, 1] - c[None, :, 1]) + np.eye(200) * 9
    assert dd.min() >= 0.6
    assert np.array_equal(c, inputs.layout(200, -50.0, 50.0, 9))
    assert len(inputs.sweep_sizes()) == 128
    assert min(inputs.sweep_sizes()) >= 200 and max(inputs.sweep_sizes()) <= 4000


def test_layer_stack_arguments_are_validated_before_any_device_work(lib):
    two_pi = 2 * math.pi
    ks, ds = [two_pi, 2.6 * math.pi, 3 * math.pi, 3.4 * math.pi, 4 * math.pi], [0.5, 2.0, 0.7]
    bad = [
        (ks[:2], [], 2),                 # fewer than three layers
        (ks, ds, 1),                     # discs in the top half-space
        (ks, ds, 5),                     # discs in the bottom half-space
        (ks, [0.5, -2.0, 0.7], 3),       # negative thickness
        (ks, [0.5, 0.4, 0.7], 3),        # radius 0.25 not below half the disc layer (0.2)
        ([two_pi, -1.0] + ks[2:], ds, 3),
        (ks, ds[:2], 3),                 # wrong number of thicknesses
    ]
    for stack in bad:
        with pytest.raises(lib.LsmsError) as e:
            lib.Context(0, 0, 0, 0, 2.4 * math.pi, 0.25, 6, 128, stack=stack)
        assert e.value.code == -1, stack
    try:
        import torch
        if torch.cuda.is_available():
            return
    except ImportError:
        pass
    with pytest.raises(lib.LsmsError) as e:         # valid: fails only for want of a GPU
        lib.Context(0, 0, 0, 0, 2.4 * math.pi, 0.25, 6, 128, stack=(ks, ds, 3))
    assert e.value.code == -6


@pytest.mark.parametrize("p,n_pts,shape,kp,k2", [(10, 256, (0.15, 0.05, 5), 2.4 * math.pi, MED_K[1]),
                                                 (14, 128, (0.2, 0.0, 0), 2.4 * math.pi, MED_K[1]),
                                                 (8, 96, (0.12, 0.04, 3), 2.0 * math.pi, MED_K[1]),
                                                 (10, 256, (0.12, 0.04, 3), 2.0, 20.0)])   # Example 2's contrast
def test_library_inclusion_matrix_equals_oracle(lib, p, n_pts, shape, kp, k2):
    # host-only helper (Sec. 4): the library's Nystrom solve against the oracle's
    from oracle import lsms_oracle as O
    cur = inputs.star_curve(*shape, n_pts, rotation=0.3)
    s_lib = lib.inclusion_scattering_matrix(p, k2, kp, 0.25, cur)
    s_o = O.inclusion_scattering_matrix(cur, p, k2, kp)
    assert np.abs(s_lib - s_o).max() < 1e-13 * np.abs(s_o).max()


@pytest.mark.parametrize("kp", [7.54 + 0.5j, 7.54 + 7.54j, 20 + 10j, 3 + 23.9j, 0.5 + 5j])
@pytest.mark.parametrize("shape", [(0.18, 0.05, 5), (0.15, 0.06, 3), (0.2, 0.0, 0)])
def test_library_absorbing_inclusion_matrix_equals_oracle(lib, kp, shape):
    # complex k_p (absorbing interior): the library's complex-argument J_0, J_1, Y_0, Y_1 (Miller,
    # Neumann) against the oracle's AMOS values in the same Nystrom system, up to the loss bound
    # Im k_p * 2R <= 12 (R = 0.25); a centred circle also equals the library's own absorbing Mie
    # diagonal (the log-derivative route)
    k2, p = inputs.MEDIUM["k2"], 10
    cur = inputs.star_curve(*shape, 256, rotation=0.3)
    s_lib = lib.inclusion_scattering_matrix(p, k2, kp, 0.25, cur)
    s_o = O.inclusion_scattering_matrix(cur, p, k2, kp)
    assert np.abs(s_lib - s_o).max() < 1e-12 * np.abs(s_o).max()
    if shape[1] == 0.0:
        mie = lib.scattering_diagonal(p, k2, kp, shape[0])
        assert np.abs(s_lib - np.diag(mie)).max() < 1e-12 * np.abs(mie).max()


def test_library_absorbing_inclusion_arguments(lib):
    s = inputs.STAR5
    cur = inputs.star_curve(s["a1"], s["a2"], s["a3"], 128)
    k2 = inputs.MEDIUM["k2"]
    real = lib.inclusion_scattering_matrix(6, k2, 7.5, 0.25, cur)
    assert np.array_equal(lib.inclusion_scattering_matrix(6, k2, 7.5 + 0j, 0.25, cur), real)
    for bad in (7.5 - 0.1j, -1 + 1j, 0j, complex(7.5, np.nan), 3 + 24.1j, 2.1e4 + 1j):  # Im: 24.1 * 0.5 > 12
        with pytest.raises(lib.LsmsError):
            lib.inclusion_scattering_matrix(6, k2, bad, 0.25, cur)


def test_library_inclusion_matrix_rejects_bad_curves(lib):
    k2, kp = inputs.MEDIUM["k2"], inputs.MEDIUM["kp"]
    x, dx, ddx = inputs.star_curve(0.15, 0.05, 5, 64)
    cases = [((x, dx, ddx), 0.15, -2),                      # outside the enclosing disc
             ((x[::-1], -dx[::-1], ddx[::-1]), 0.25, -1),   # clockwise
             ((x[:63], dx[:63], ddx[:63]), 0.25, -1),       # odd number of points
             ((x * np.nan, dx, ddx), 0.25, -1)]
    for cur, radius, code in cases:
        with pytest.raises(lib.LsmsError) as e:
            lib.inclusion_scattering_matrix(10, k2, kp, radius, cur)
        assert e.value.code == code
    with pytest.raises(lib.LsmsError) as e:
        lib.inclusion_scattering_matrix(16, k2, kp, 0.25, (x, dx, ddx))
    assert e.value.code == -1


def test_lossy_stack_arguments_are_validated_before_any_device_work(lib):
    kp, R = 2.4 * math.pi, 0.25
    for ks in ([2 * math.pi + 0.1j, 3 * math.pi, 4 * math.pi],      # lossy source half-space
               [2 * math.pi, 3 * math.pi + 0.1j, 4 * math.pi],      # lossy particle layer
               [2 * math.pi, 3 * math.pi, 4 * math.pi - 0.1j],      # gain
               [2 * math.pi, 3 * math.pi, -4 * math.pi + 0.1j]):    # Re k <= 0
        with pytest.raises(lib.LsmsError) as e:
            lib.Context(0, 0, 0, 0, kp, R, 6, 128, stack=(np.array(ks), [2.0], 2))
        assert e.value.code == -1, ks


def test_library_pec_diagonal_equals_oracle(lib):
    from oracle import lsms_oracle as O
    for p, k2, R in ((10, inputs.MEDIUM["k2"], 0.25), (15, 2.0, 0.17)):
        s = lib.pec_scattering_diagonal(p, k2, R)
        s_o = O.pec_coefficients(p, k2, R)
        assert np.abs(s - s_o).max() < 1e-13 * np.abs(s_o).max()
    with pytest.raises(lib.LsmsError):
        lib.pec_scattering_diagonal(16, 2.0, 0.2)


@pytest.mark.parametrize("kp", [7.54 + 0.5j, 7.54 + 7.54j, 40 + 1j, 0.1 + 20j, 2 + 1e-3j, 5j, 1e-3 + 0.01j,
                                300 + 300j])
def test_library_absorbing_disc_diagonal_equals_oracle(lib, kp):
    # complex k_p: the library's log-derivative route against the oracle's 2x2 solve with SciPy's
    # complex-argument Bessel functions
    for p in (0, 5, 10, 15):
        for k2, R in ((inputs.MEDIUM["k2"], 0.25), (1.0, 0.1), (20.0, 0.5)):
            s = lib.scattering_diagonal(p, k2, kp, R)
            s_o = O.mie_coefficients(p, k2, kp, R)
            assert np.abs(s - s_o).max() < 1e-12 * np.abs(s_o).max(), (p, k2, R)


def test_library_absorbing_disc_beyond_the_oracle_range(lib):
    # Im(k_p R) = 800, where J_n(k_p R) overflows (the oracle's 2x2 solve gives NaN): the library's
    # diagonal stays finite and sits at the good-conductor gap O(1/|k_p|) from the perfectly
    # conducting disc, half the gap at half the |k_p|
    k2, R, p = 20.0, 0.5, 12
    pec = O.pec_coefficients(p, k2, R)
    gap = {s: np.abs(lib.scattering_diagonal(p, k2, s * (1 + 1j), R) - pec).max() / np.abs(pec).max()
           for s in (800.0, 1600.0)}
    assert gap[1600.0] < 2e-2 and 1.9 < gap[800.0] / gap[1600.0] < 2.1
    real = lib.scattering_diagonal(p, k2, 7.5, R)
    assert np.array_equal(lib.scattering_diagonal(p, k2, 7.5 + 0j, R), real)   # Im k_p = 0: the real route
    for bad in (7.5 - 0.1j, -1 + 1j, 0j, complex(np.nan, 1.0), 1e6 + 1e6j):
        with pytest.raises(lib.LsmsError):
            lib.scattering_diagonal(p, k2, bad, R)


@pytest.mark.parametrize("ks,b,n_nodes,t_max", [
    (inputs.STACK5["ks"], 0.2, 512, 80.0),                                # five layers, no guided band
    ([1.0, 2.5, 6.0, 3.0, 1.5], 0.2, 1024, 40.0),                          # guided band (1.5, 6)
    ([2.0 * math.pi, 3.0 * math.pi, 3.4 * math.pi, 4.0 * math.pi], 0.1, 768, 60.0),
    ([1.0, 1.0, 3.0, 1.0], 0.15, 2048, 45.0),                               # Example 1's medium, split
])
def test_library_stack_contour_equals_oracle_contour(lib, ks, b, n_nodes, t_max):
    # the contour lsms_create_stack builds (host only) against the oracle's, node for node
    lam, wt = lib.build_contour_stack(n_nodes, ks, b, t_max, 16)
    lam_o, wt_o = O.contour(n_nodes, ks[0], ks[1], ks[-1], b, t_max, branch_points=ks)
    assert np.max(np.abs(lam - lam_o)) <= 1e-12 * t_max
    assert np.max(np.abs(wt - wt_o)) <= 1e-14 * t_max
    with pytest.raises(lib.LsmsError):
        lib.build_contour_stack(n_nodes, ks[:2], b, t_max, 16)


@pytest.mark.parametrize("ks,ds,m", [
    ([MED_K[0], MED_K[1], MED_K[2]], [2.0], 2),                                      # the bench medium
    (inputs.STACK5["ks"], inputs.STACK5["ds"], 3),                                   # five layers
    ([2 * math.pi, 3 * math.pi, 3.4 * math.pi + 0.5j, 4 * math.pi], [2.0, 0.7], 2),  # absorbing film
    ([1.0, 3.0, 1.0], [32.0], 2),                                                    # Example 1 (guided)
])
def test_library_layer_response_equals_oracle(lib, ks, ds, m):
    # the per-node interface solve every context precomputes (host only) against the oracle's Stack
    lam, _ = O.contour(256, complex(ks[0]).real, complex(ks[m - 1]).real, complex(ks[-1]).real, 0.2, 40.0,
                       branch_points=[complex(k).real for k in ks])
    lam = lam[::7]
    r = lib.layer_response(ks, ds, m, lam)
    st = O.Stack(ks, ds, m, 2.4 * math.pi, 0.25)
    one = np.ones(lam.size, dtype=complex)
    zero = np.zeros(lam.size, dtype=complex)
    for s, (inc, pp, qm) in enumerate(((one, zero, zero), (zero, one, zero), (zero, zero, one))):
        o = st.solve_layers(lam, inc=inc, p_plus=pp, q_minus=qm)           # (sigma_1, s+, s-, sigma_L)
        scale = np.abs(o).max(axis=1, keepdims=True) + 1e-300
        assert np.max(np.abs(r[:, :, s] - o) / scale) < 1e-11, s


def test_library_contour_equals_oracle_contour_on_random_stacks(lib):
    # both panel rules (graded; greedy in guided-mode media), random stacks of 3-5 layers, random
    # offsets, lengths and node counts (including budgets too small for every branch point)
    rng = np.random.default_rng(2024)
    guided = 0
    for _ in range(60):
        L = int(rng.integers(3, 6))
        ks = list(rng.uniform(0.5, 25.0, L))
        b = float(rng.uniform(0.01, 0.4))
        t_max = float(max(ks) + rng.uniform(5.0, 80.0))
        n_nodes = int(rng.integers(64, 3000))
        guided += O.guided_band(ks) is not None
        lam, wt = lib.build_contour_stack(n_nodes, ks, b, t_max, 16)
        lam_o, wt_o = O.contour(n_nodes, ks[0], ks[1], ks[-1], b, t_max, branch_points=ks)
        assert np.max(np.abs(lam - lam_o)) <= 1e-12 * t_max, (ks, b, t_max, n_nodes)
        assert np.max(np.abs(wt - wt_o)) <= 1e-14 * t_max, (ks, b, t_max, n_nodes)
    assert 10 < guided < 60                      # both rules exercised


def test_library_layer_response_on_random_stacks(lib):
    # random stacks of 3-6 layers, random thicknesses, absorbing layers anywhere but layer 1 and the
    # particle layer, nodes on and off the real axis: the library's per-node solve against the oracle
    rng = np.random.default_rng(77)
    for _ in range(30):
        L = int(rng.integers(3, 7))
        m = int(rng.integers(2, L))
        ks = [complex(k) for k in rng.uniform(1.0, 15.0, L)]
        for j in range(1, L):
            if j != m - 1 and rng.random() < 0.4:
                ks[j] += 1j * rng.uniform(0.05, 2.0)
        ds = list(rng.uniform(0.3, 4.0, L - 2))
        lam = rng.uniform(-30.0, 30.0, 12) + 1j * rng.choice([-0.2, 0.0, 0.2], 12)
        lam[lam.imag == 0] += 0.013            # off the real branch points
        r = lib.layer_response(ks, ds, m, lam)
        st = O.Stack(ks, ds, m, 2.0, 0.1)
        one, zero = np.ones(lam.size, dtype=complex), np.zeros(lam.size, dtype=complex)
        for s, (inc, pp, qm) in enumerate(((one, zero, zero), (zero, one, zero), (zero, zero, one))):
            o = st.solve_layers(lam, inc=inc, p_plus=pp, q_minus=qm)
            # per node, relative to its largest response, floored at 1e-2 of this input's largest
            # response: where a response vanishes (a nearly homogeneous stack scatters nothing) both
            # sides hold cancellation noise — in one case a 50-digit solve gives 1.5e-48, the
            # library 7.6e-15, LAPACK in the oracle 3.5e-13 — so there the check is absolute, ~1e-12
            scale = np.maximum(np.abs(o).max(axis=1, keepdims=True), 1e-2 * np.abs(o).max())
            assert np.max(np.abs(r[:, :, s] - o) / scale) < 1e-10, (ks, ds, m, s)


def test_library_inclusion_matrix_on_random_shapes(lib):
    # random star-shaped inclusions (lobes, amplitude, rotation, offset from the enclosing disc's
    # centre) and contrasts: the library's Nystrom solve against the oracle's
    rng = np.random.default_rng(11)
    for _ in range(4):
        a1 = float(rng.uniform(0.08, 0.15))
        a2 = float(rng.uniform(0.0, 0.4 * a1))
        a3 = int(rng.integers(2, 7))
        off = rng.uniform(-0.03, 0.03, 2)
        k2, kp = float(rng.uniform(2.0, 12.0)), float(rng.uniform(1.0, 15.0))
        p = int(rng.integers(4, 12))
        cur = inputs.star_curve(a1, a2, a3, 128, rotation=float(rng.uniform(0, 6.3)), centre=off)
        s_lib = lib.inclusion_scattering_matrix(p, k2, kp, 0.25, cur)
        s_o = O.inclusion_scattering_matrix(cur, p, k2, kp)
        assert np.abs(s_lib - s_o).max() < 1e-12 * np.abs(s_o).max(), (a1, a2, a3, k2, kp, p)


def test_library_absorbing_inclusion_matrix_on_random_shapes(lib):
    # random star-shaped inclusions and random lossy interiors up to the loss bound
    # (Im k_p * 2R <= 12, R = 0.25): the library's complex-argument Bessel functions in the Nystrom
    # solve against the oracle's (AMOS)
    rng = np.random.default_rng(12)
    for _ in range(5):
        a1 = float(rng.uniform(0.08, 0.15))
        a2 = float(rng.uniform(0.0, 0.4 * a1))
        a3 = int(rng.integers(2, 7))
        off = rng.uniform(-0.03, 0.03, 2)
        k2 = float(rng.uniform(2.0, 12.0))
        kp = complex(rng.uniform(0.5, 15.0), rng.uniform(0.01, 23.0))
        p = int(rng.integers(4, 12))
        cur = inputs.star_curve(a1, a2, a3, 128, rotation=float(rng.uniform(0, 6.3)), centre=off)
        s_lib = lib.inclusion_scattering_matrix(p, k2, kp, 0.25, cur)
        s_o = O.inclusion_scattering_matrix(cur, p, k2, kp)
        assert np.abs(s_lib - s_o).max() < 1e-12 * np.abs(s_o).max(), (a1, a2, a3, k2, kp, p)
