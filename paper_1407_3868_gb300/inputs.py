"""Seeded synthetic inputs shared by the CUDA path's tests and benchmark and by the CPU oracle.

This module only draws random numbers and lays out points. It contains none of the method's
arithmetic (no Bessel/Hankel functions, no contour quadrature, no scattering matrices): the two
independent implementations (the CUDA library and the CPU oracle) both consume what it returns.

Geometry follows the paper's setting (Sec. 1, Sec. 6): a three-layer medium with the middle layer
-d < y < 0, identical dielectric discs of radius R inside it, a line source in the top layer
(Sec. 2, Eq. "sommer"), and observation points in the top layer.  The paper places its particles
by a "bin sorting" perturbation scheme (Sec. 6); here discs are placed by seeded rejection
sampling (a documented substitution), keeping a minimum gap of 0.1 between discs and 0.05
between a disc edge and either interface.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Medium shared by every workload: k1 = 2 pi, k2 = 3 pi, k3 = 4 pi, d = 2, discs kp = 2.4 pi, R = 0.25.
MEDIUM = dict(k1=2.0 * math.pi, k2=3.0 * math.pi, k3=4.0 * math.pi, d=2.0,
              kp=2.4 * math.pi, radius=0.25)
# Five layers (top to bottom): the three-layer medium's k1 and k3 at the ends, two extra layers
# (k = 2.6 pi above, 3.4 pi below) around the disc layer (k2, thickness d); discs in layer 3, whose
# top interface lies 0.5 below y = 0, so layout centres move down by STACK5_DEPTH.
STACK5 = dict(ks=[2.0 * math.pi, 2.6 * math.pi, 3.0 * math.pi, 3.4 * math.pi, 4.0 * math.pi],
              ds=[0.5, 2.0, 0.7], layer=3)
STACK5_DEPTH = 0.5
GAP = 0.1            # minimum edge-to-edge gap between discs
CLEARANCE = 0.05     # minimum distance from a disc edge to either interface
AREA_FRACTION = 0.2  # area fraction used to widen the large layouts


def widened_half_width(n: int, radius: float = MEDIUM["radius"], d: float = MEDIUM["d"],
                       fraction: float = AREA_FRACTION) -> float:
    """Half-width of a layout holding n discs at the given area fraction of the middle layer."""
    return 0.5 * n * math.pi * radius * radius / (fraction * d)


def contour_b(width: float) -> float:
    """Offset b of the deformed Sommerfeld contour from the real axis (Sec. 5.1, Eq. "sommerseg").

    The paper uses b = 0.2 for layouts a few wavelengths wide (Sec. 6).  Every contour term carries
    |exp(i lambda dx)| = exp(b |dx|), so for wide layouts b is reduced to ln(10)/width, which bounds
    that growth by a factor of 10 across the whole layout.
    """
    return min(0.2, math.log(10.0) / width)


@dataclass
class Workload:
    """One synthetic problem: medium, discs, contour size, sources and targets."""
    name: str
    n: int
    p: int
    n_nodes: int
    t_max: float
    x_lo: float
    x_hi: float
    seed: int
    sources: np.ndarray                 # (n_src, 2) source positions in layer 1
    targets: np.ndarray                 # (n_tgt, 2) observation points in layer 1
    tol: float
    medium: dict = field(default_factory=lambda: dict(MEDIUM))

    @property
    def b(self) -> float:
        return contour_b(self.x_hi - self.x_lo)

    def centres(self) -> np.ndarray:
        return layout(self.n, self.x_lo, self.x_hi, self.seed)


def _targets(x_lo: float, x_hi: float, n: int = 64, y: float = 1.5) -> np.ndarray:
    xs = np.linspace(x_lo, x_hi, n)
    return np.stack([xs, np.full(n, y)], axis=1)


def _workloads() -> dict[str, Workload]:
    w = {}
    # 16 discs in x in [-2, 2], p = 10, 256 contour nodes, one source at (0, 1).
    w["disc16_p10_ns256"] = Workload("disc16_p10_ns256", 16, 10, 256, 141.0, -2.0, 2.0, 0,
                                     np.array([[0.0, 1.0]]), _targets(-2.0, 2.0), 1e-12)
    h = widened_half_width(1000)
    w["disc1000_p12_ns512"] = Workload("disc1000_p12_ns512", 1000, 12, 512, 152.0, -h, h, 1,
                                       np.array([[0.0, 1.0]]), _targets(-h, h), 1e-10)
    h = widened_half_width(5000)
    w["disc5000_p14_ns1024"] = Workload("disc5000_p14_ns1024", 5000, 14, 1024, 163.0, -h, h, 2,
                                        np.array([[0.0, 1.0]]), _targets(-h, h), 1e-10)
    h = widened_half_width(2000)
    src = np.stack([np.linspace(-h, h, 64), np.full(64, 1.0)], axis=1)
    w["disc2000_p12_ns768_src64"] = Workload("disc2000_p12_ns768_src64", 2000, 12, 768, 152.0,
                                             -h, h, 3, src, _targets(-h, h), 1e-10)
    return w


WORKLOADS = _workloads()


def sweep_sizes(n_layouts: int = 128, seed: int = 5, n_min: int = 200, n_max: int = 4000) -> list[int]:
    """Disc counts of a design sweep, log-uniform in [n_min, n_max]."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(math.log(n_min), math.log(n_max), size=n_layouts)
    return [int(round(math.exp(v))) for v in u]


def sweep_layouts(n_layouts: int = 128, seed: int = 5) -> list[np.ndarray]:
    """Centres of every layout of the sweep; layout l uses seed 1000 + l and the widened width."""
    out = []
    for l, n in enumerate(sweep_sizes(n_layouts, seed)):
        h = widened_half_width(n)
        out.append(layout(n, -h, h, 1000 + l))
    return out


def layout(n: int, x_lo: float, x_hi: float, seed: int,
           radius: float = MEDIUM["radius"], d: float = MEDIUM["d"],
           gap: float = GAP, clearance: float = CLEARANCE, max_draws: int = 10_000_000) -> np.ndarray:
    """n disc centres by seeded rejection sampling.

    Each candidate draws x ~ U(x_lo, x_hi) then y ~ U(-d + R + clearance, -R - clearance) from
    numpy's PCG64 generator; it is accepted when its distance to every accepted centre is at
    least 2R + gap (checked on a cell grid).  Returns an (n, 2) float64 array in acceptance order.
    """
    if n == 0:
        return np.zeros((0, 2))
    rng = np.random.default_rng(seed)
    y_lo, y_hi = -d + radius + clearance, -radius - clearance
    dmin = 2.0 * radius + gap
    cell = dmin
    grid: dict[tuple[int, int], list[int]] = {}
    pts = np.zeros((n, 2))
    count = 0
    draws = 0
    while count < n:
        if draws >= max_draws:
            raise RuntimeError(f"layout: could not place {n} discs in {max_draws} draws")
        draws += 1
        u = rng.random(2)
        x = x_lo + (x_hi - x_lo) * u[0]
        y = y_lo + (y_hi - y_lo) * u[1]
        cx, cy = int(math.floor(x / cell)), int(math.floor(y / cell))
        ok = True
        for i in range(cx - 1, cx + 2):
            for j in range(cy - 1, cy + 2):
                for q in grid.get((i, j), ()):
                    if (pts[q, 0] - x) ** 2 + (pts[q, 1] - y) ** 2 < dmin * dmin:
                        ok = False
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            pts[count] = (x, y)
            grid.setdefault((cx, cy), []).append(count)
            count += 1
    return pts


def random_coefficients(n: int, p: int, nrhs: int = 1, seed: int = 0) -> np.ndarray:
    """Complex standard-normal coefficients, shape (nrhs, n, 2p+1), complex128."""
    rng = np.random.default_rng(seed)
    shape = (nrhs, n, 2 * p + 1)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2.0)


def observation_points(x_lo: float, x_hi: float, n: int, y: float) -> np.ndarray:
    """n points evenly spaced on the horizontal line at height y, endpoints included."""
    return _targets(x_lo, x_hi, n, y)


# ------------------------------------------------------------------------------------------------
# Inclusion shapes (the star-shaped family of Sec. 6, Eq. "par1") and orientations
# ------------------------------------------------------------------------------------------------
# The pentagon-like inclusion used with the bench layout: radius 0.15 +- 0.05 (inside the
# enclosing disc of radius 0.25), five lobes, 256 boundary points.
STAR5 = dict(a1=0.15, a2=0.05, a3=5, n_pts=256)


def star_curve(a1: float, a2: float, a3: int, n_pts: int, rotation: float = 0.0,
               centre=(0.0, 0.0)):
    """Points, first and second derivatives of x(t) = c + (a1 + a2 cos(a3 t)) (cos(t + rot),
    sin(t + rot)) at t_j = 2 pi j / n_pts (counterclockwise).  Returns three (n_pts, 2) arrays."""
    t = 2.0 * np.pi * np.arange(n_pts) / n_pts
    r = a1 + a2 * np.cos(a3 * t)
    dr = -a2 * a3 * np.sin(a3 * t)
    ddr = -a2 * a3 * a3 * np.cos(a3 * t)
    ct, st = np.cos(t + rotation), np.sin(t + rotation)
    x = np.stack([centre[0] + r * ct, centre[1] + r * st], axis=1)
    dx = np.stack([dr * ct - r * st, dr * st + r * ct], axis=1)
    ddx = np.stack([ddr * ct - 2.0 * dr * st - r * ct, ddr * st + 2.0 * dr * ct - r * st], axis=1)
    return x, dx, ddx


def orientations(n: int, seed: int) -> np.ndarray:
    """n rotation angles, uniform on [0, 2 pi) (NumPy PCG64, default_rng(seed))."""
    return np.random.default_rng(seed).uniform(0.0, 2.0 * np.pi, n)


# ------------------------------------------------------------------------------------------------
# Contrast sweep (Sec. 6, Example 2): 200 three-lobed inclusions (Eq. "par1" with a1 = 0.12,
# a2 = 0.04, a3 = 3; enclosing radius 0.17) with kp = 2 in a layer of thickness 12 between two
# half-spaces of k = 1, the layer's k2 swept from 1 to 20 (k2 > 1: a guided-mode layer); p = 10,
# GMRES to 1e-6.  The layout (20 wide, centres at least 1 from the interfaces) stands in for the
# paper's random placement.
# ------------------------------------------------------------------------------------------------
CONTRAST = dict(k1=1.0, k3=1.0, d=12.0, kp=2.0, radius=0.17, n=200, p=10, n_nodes=2048,
                x_lo=-10.0, x_hi=10.0, clearance=1.0, seed=21, tol=1e-6,
                shape=dict(a1=0.12, a2=0.04, a3=3, n_pts=256),
                k2_values=[1.0, 2.0, 4.0, 6.0, 8.0, 10.0, 12.0, 14.0, 16.0, 18.0, 20.0])


def contrast_layout(n: int = CONTRAST["n"], x_lo: float = CONTRAST["x_lo"], x_hi: float = CONTRAST["x_hi"],
                    seed: int = CONTRAST["seed"]) -> np.ndarray:
    c = CONTRAST
    return layout(n, x_lo, x_hi, seed, radius=c["radius"], d=c["d"], clearance=c["clearance"])


def contrast_t_max(k2: float) -> float:
    """Gamma1 length for the contrast sweep: the integrands decay like exp(-2 t) beyond k2 (centres
    at least 1.17 from the interfaces), so 30 past the largest wavenumber."""
    return max(CONTRAST["k1"], k2) + 30.0


# ------------------------------------------------------------------------------------------------
# Sec. 6, Example 1: 5000 three-lobed inclusions (a1 = 0.12, a2 = 0.04, a3 = 3; enclosing radius
# 0.17) with kp = 2 in a layer of thickness 32 between half-spaces of k = 1, k2 = 3 (a guided-mode
# layer); p = 10; GMRES to 1e-6.  The layout (71 wide, ~21% area fraction, centres at least 0.67
# from the interfaces) stands in for the paper's random placement.
# ------------------------------------------------------------------------------------------------
EXAMPLE1 = dict(k1=1.0, k2=3.0, k3=1.0, d=32.0, kp=2.0, radius=0.17, n=5000, p=10, n_nodes=2048,
                t_max=45.0, x_lo=-35.5, x_hi=35.5, clearance=0.5, seed=31, tol=1e-6,
                shape=dict(a1=0.12, a2=0.04, a3=3, n_pts=256))


def example1_layout(n: int = EXAMPLE1["n"], x_lo: float = EXAMPLE1["x_lo"], x_hi: float = EXAMPLE1["x_hi"],
                    seed: int = EXAMPLE1["seed"]) -> np.ndarray:
    e = EXAMPLE1
    return layout(n, x_lo, x_hi, seed, radius=e["radius"], d=e["d"], clearance=e["clearance"])
