"""Seeded synthetic geometries and surface potentials for the boundary-integral solver.

This module only *generates inputs*: node positions zeta_k(alpha_km), their
alpha-derivatives zeta', zeta'' (analytic), obstacle centres z_j, the flow
parameters V1 and a_j, and the surface potential phi~.  It holds none of the
method's arithmetic (no kernels, no solves), so that the CPU oracle and the CUDA
path can both be fed from it without sharing any computation.

Conventions (paper Sec. 2, eqs per0/per1/per2N, zeta:cx):
  * boundary 0 is the free surface, parameterised left to right,
    zeta_0(alpha + 2pi) = zeta_0(alpha) + 2pi;
  * boundary 1 is the bottom, also left to right;
  * boundaries 2..N are obstacles, closed curves traversed **clockwise** so that
    the normal (-eta', xi') points into the fluid;
  * nodes are alpha_kl = 2 pi l / M_k, l = 0..M_k-1 (Sec. 3.3).

Ellipses follow the paper's problem data (Sec. 7.1) with the reading
zeta_j = z_j + e^{i theta_j}(q_j cos(alpha) - i b_j sin(alpha)): the printed
form has a '+' (counter-clockwise) and no centre, which contradicts the
clockwise convention of Sec. 2.

Workload recipes (all seeded with numpy.random.default_rng(seed)):
  one_ellipse_640  -- 640 unknowns: surface 0.1cos x + 0.02cos 3x (256), flat bottom y=-1
              (256), one ellipse at (pi,-0.5), semi-axes 0.2 x 0.1, tilt 0.3 (128),
              a_2 = 0.5, V1 = 1, phi~ = 0.05 randn filtered to |k| <= 20.
  three_ellipses_16383  -- 16383 unknowns: random smooth surface (amplitude 0.15, |k| <= 64,
              k^-2 spectrum, 8192), Gaussian-bump bottom -1 + 0.3 exp(-(x-pi)^2/0.2)
              (4096), three random ellipses (1365 each), V1 = 1,
              a_j ~ U[-0.5, 0.5], phi~ filtered to |k| <= 64.
  random_batch  -- batch of random geometries with N ~ U{1024..12288}.
  two_ellipses_4096  -- 4096 unknowns: surface 2048, bottom 1024, two ellipses of 512.
  four_ellipses_32768  -- 32768 unknowns: steep surface (16384), sinusoidal bottom (8192),
              four ellipses of 2048; targets: ~10^6 points of a uniform grid of
              the fluid plus 10^5 points within 2 node spacings of a boundary.
  problem1..3 -- the paper's problems 1-3 at t = 0 (Sec. 7.1): flat surface,
              flat bottom y = -3, three ellipses from the ellipse table.
  problem4_bottom -- the basin bottom of problem 4 (Sec. 7.2).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np

TWO_PI = 2.0 * np.pi


@dataclass
class Geometry:
    """Boundary nodes in block order 0 (surface), 1 (bottom), 2..N (obstacles).

    zeta, dzeta, d2zeta are complex128 arrays of length sum(M), concatenated in
    block order.  zc[j-2] is the centre z_j of obstacle j (j >= 2).
    """

    M: List[int]
    zeta: np.ndarray
    dzeta: np.ndarray
    d2zeta: np.ndarray
    zc: np.ndarray
    # shape parameters of each obstacle (x, y, q, b, theta), for reference
    ellipses: List[tuple] = field(default_factory=list)

    @property
    def nb(self) -> int:
        return len(self.M)

    @property
    def N(self) -> int:
        return int(sum(self.M))

    def offsets(self) -> np.ndarray:
        return np.concatenate([[0], np.cumsum(self.M)]).astype(np.int64)

    def block(self, k: int):
        o = self.offsets()
        s = slice(int(o[k]), int(o[k + 1]))
        return self.zeta[s], self.dzeta[s], self.d2zeta[s]


@dataclass
class Flow:
    """Background current V1 and circulation parameters a_j (j = 2..N)."""

    V1: float
    a: np.ndarray  # length nb - 2


def alphas(M: int) -> np.ndarray:
    return TWO_PI * np.arange(M) / M


# ----------------------------------------------------------------------------
# curve families (analytic derivatives)
# ----------------------------------------------------------------------------

def graph_curve(M: int, f, df, d2f):
    """zeta = alpha + i f(alpha), a graph over the horizontal (surface or bottom)."""
    a = alphas(M)
    return a + 1j * f(a), 1.0 + 1j * df(a), 1j * d2f(a)


def fourier_graph(M: int, offset: float, A: np.ndarray, B: np.ndarray):
    """eta(alpha) = offset + sum_k A_k cos(k alpha) + B_k sin(k alpha), k = 1..K."""
    k = np.arange(1, len(A) + 1)
    a = alphas(M)[:, None]
    c, s = np.cos(k * a), np.sin(k * a)
    eta = offset + c @ A + s @ B
    deta = (-s * k) @ A + (c * k) @ B
    d2eta = (-c * k * k) @ A + (-s * k * k) @ B
    return alphas(M) + 1j * eta, 1.0 + 1j * deta, 1j * d2eta


def ellipse(M: int, x: float, y: float, q: float, b: float, theta: float):
    """Clockwise ellipse z_j + e^{i theta}(q cos alpha - i b sin alpha)."""
    a = alphas(M)
    r = np.exp(1j * theta)
    z = (x + 1j * y) + r * (q * np.cos(a) - 1j * b * np.sin(a))
    dz = r * (-q * np.sin(a) - 1j * b * np.cos(a))
    d2z = r * (-q * np.cos(a) + 1j * b * np.sin(a))
    return z, dz, d2z


def assemble_geometry(curves, ellipses) -> Geometry:
    M = [len(c[0]) for c in curves]
    zeta = np.concatenate([c[0] for c in curves]).astype(np.complex128)
    dzeta = np.concatenate([c[1] for c in curves]).astype(np.complex128)
    d2zeta = np.concatenate([c[2] for c in curves]).astype(np.complex128)
    zc = np.array([e[0] + 1j * e[1] for e in ellipses], dtype=np.complex128)
    return Geometry(M=M, zeta=zeta, dzeta=dzeta, d2zeta=d2zeta, zc=zc,
                    ellipses=[tuple(map(float, e)) for e in ellipses])


def filtered_noise(rng, M: int, amp: float, kmax: int) -> np.ndarray:
    """amp * randn(M), band-limited to |k| <= kmax (mode 0 kept)."""
    v = amp * rng.standard_normal(M)
    vh = np.fft.rfft(v)
    vh[kmax + 1:] = 0.0
    return np.fft.irfft(vh, n=M)


# ----------------------------------------------------------------------------
# geometric sanity (input validation for generators only)
# ----------------------------------------------------------------------------

def _dense_curve(kind, params, n=4096):
    a = TWO_PI * np.arange(n) / n
    if kind == "ellipse":
        x, y, q, b, th = params
        return (x + 1j * y) + np.exp(1j * th) * (q * np.cos(a) - 1j * b * np.sin(a))
    f = params
    return a + 1j * f(a)


def min_gap(curves_dense) -> float:
    """Smallest distance between distinct curves, including periodic images."""
    best = np.inf
    for i in range(len(curves_dense)):
        for j in range(i + 1, len(curves_dense)):
            zi, zj = curves_dense[i], curves_dense[j]
            for shift in (-TWO_PI, 0.0, TWO_PI):
                d = np.abs(zi[:, None] - (zj[None, :] + shift))
                best = min(best, float(d.min()))
    return best


def _curve_gap(f_surf, f_bot, ells, n=1024):
    dense = [_dense_curve("graph", f_surf, n), _dense_curve("graph", f_bot, n)]
    dense += [_dense_curve("ellipse", e, n) for e in ells]
    return min_gap(dense)


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

def one_ellipse_640(seed: int = 0):
    """640 unknowns (256 + 256 + 128); see module docstring."""
    rng = np.random.default_rng(seed)
    surf = graph_curve(256,
                       lambda a: 0.1 * np.cos(a) + 0.02 * np.cos(3 * a),
                       lambda a: -0.1 * np.sin(a) - 0.06 * np.sin(3 * a),
                       lambda a: -0.1 * np.cos(a) - 0.18 * np.cos(3 * a))
    bot = graph_curve(256, lambda a: -1.0 + 0 * a, lambda a: 0 * a, lambda a: 0 * a)
    e = (np.pi, -0.5, 0.2, 0.1, 0.3)
    g = assemble_geometry([surf, bot, ellipse(128, *e)], [e])
    flow = Flow(V1=1.0, a=np.array([0.5]))
    phit = filtered_noise(rng, 256, 0.05, 20)
    return g, flow, phit


def _random_surface(rng, M, amp, kmax, power):
    k = np.arange(1, kmax + 1, dtype=np.float64)
    A = rng.standard_normal(kmax) * k ** (-power)
    B = rng.standard_normal(kmax) * k ** (-power)
    a = TWO_PI * np.arange(8192) / 8192
    eta = np.cos(np.outer(a, k)) @ A + np.sin(np.outer(a, k)) @ B
    s = amp / np.abs(eta).max()
    return A * s, B * s


def _random_ellipses(rng, n, fsurf, fbot, yrange, srange, gap=0.05, tries=2000):
    ells = []
    for _ in range(n):
        for _t in range(tries):
            x = rng.uniform(0.0, TWO_PI)
            y = rng.uniform(*yrange)
            q, b = rng.uniform(*srange), rng.uniform(*srange)
            th = rng.uniform(0.0, np.pi)
            cand = ells + [(x, y, q, b, th)]
            if _curve_gap(fsurf, fbot, cand, n=512) >= gap:
                ells.append((x, y, q, b, th))
                break
        else:
            raise RuntimeError("could not place a non-overlapping ellipse")
    return ells


def three_ellipses_16383(seed: int = 0, M0=8192, M1=4096, Me=1365):
    """16383 unknowns (8192 + 4096 + 3 x 1365); see module docstring."""
    rng = np.random.default_rng(seed)
    A, B = _random_surface(rng, M0, 0.15, 64, 2.0)
    k = np.arange(1, 65)
    fs = lambda a: np.cos(np.outer(a, k)) @ A + np.sin(np.outer(a, k)) @ B
    bump = lambda a: -1.0 + 0.3 * np.exp(-(a - np.pi) ** 2 / 0.2)
    dbump = lambda a: 0.3 * np.exp(-(a - np.pi) ** 2 / 0.2) * (-2.0 * (a - np.pi) / 0.2)
    d2bump = lambda a: 0.3 * np.exp(-(a - np.pi) ** 2 / 0.2) * (
        (2.0 * (a - np.pi) / 0.2) ** 2 - 2.0 / 0.2)
    ells = _random_ellipses(rng, 3, fs, bump, (-0.8, -0.3), (0.1, 0.25))
    surf = fourier_graph(M0, 0.0, A, B)
    bot = graph_curve(M1, bump, dbump, d2bump)
    g = assemble_geometry([surf, bot] + [ellipse(Me, *e) for e in ells], ells)
    flow = Flow(V1=1.0, a=rng.uniform(-0.5, 0.5, size=3))
    phit = filtered_noise(rng, M0, 0.05, 64)
    return g, flow, phit


def random_geometry(rng, N: int):
    """A random geometry with N unknowns split ~50/25/25 (1-4 ellipses)."""
    M0 = 2 * (N // 4)
    M1 = N // 4
    ne = int(rng.integers(1, 5))
    rest = N - M0 - M1
    Me = [rest // ne] * ne
    Me[-1] += rest - sum(Me)
    amp = 0.1
    A, B = _random_surface(rng, M0, amp, 8, 2.0)
    k = np.arange(1, 9)
    fs = lambda a: np.cos(np.outer(a, k)) @ A + np.sin(np.outer(a, k)) @ B
    fb = lambda a: -1.0 + 0 * a
    ells = _random_ellipses(rng, ne, fs, fb, (-0.75, -0.35), (0.08, 0.15))
    surf = fourier_graph(M0, 0.0, A, B)
    bot = graph_curve(M1, fb, lambda a: 0 * a, lambda a: 0 * a)
    g = assemble_geometry([surf, bot] + [ellipse(m, *e) for m, e in zip(Me, ells)], ells)
    flow = Flow(V1=1.0, a=rng.uniform(-0.5, 0.5, size=ne))
    phit = filtered_noise(rng, M0, 0.05, 20)
    return g, flow, phit


def random_batch(seed: int = 0, nbatch: int = 96, nmin: int = 1024, nmax: int = 12288):
    """A batch of random problems with N ~ U{nmin..nmax}."""
    rng = np.random.default_rng(seed)
    Ns = rng.integers(nmin, nmax + 1, size=nbatch)
    return [random_geometry(rng, int(n)) for n in Ns]


def two_ellipses_4096(seed: int = 0):
    """4096 unknowns: surface 2048, flat bottom 1024, two ellipses of 512."""
    rng = np.random.default_rng(seed)
    surf = graph_curve(2048,
                       lambda a: 0.1 * np.cos(a) + 0.02 * np.cos(3 * a),
                       lambda a: -0.1 * np.sin(a) - 0.06 * np.sin(3 * a),
                       lambda a: -0.1 * np.cos(a) - 0.18 * np.cos(3 * a))
    bot = graph_curve(1024, lambda a: -1.0 + 0 * a, lambda a: 0 * a, lambda a: 0 * a)
    ells = [(2.0, -0.5, 0.2, 0.1, 0.3), (4.3, -0.6, 0.15, 0.12, -0.4)]
    g = assemble_geometry([surf, bot] + [ellipse(512, *e) for e in ells], ells)
    flow = Flow(V1=1.0, a=np.array([0.5, -0.3]))
    phit = filtered_noise(rng, 2048, 0.05, 20)
    return g, flow, phit


def four_ellipses_32768(seed: int = 0):
    """32768 unknowns: steep surface 16384, sinusoidal bottom 8192, 4 x 2048 ellipses."""
    rng = np.random.default_rng(seed)
    A, B = _random_surface(rng, 16384, 0.3, 128, 1.5)
    k = np.arange(1, 129)
    fs = lambda a: np.cos(np.outer(a, k)) @ A + np.sin(np.outer(a, k)) @ B
    fb = lambda a: -1.0 + 0.15 * np.sin(a)
    ells = _random_ellipses(rng, 4, fs, fb, (-0.75, -0.45), (0.08, 0.16))
    surf = fourier_graph(16384, 0.0, A, B)
    bot = graph_curve(8192, fb, lambda a: 0.15 * np.cos(a), lambda a: -0.15 * np.sin(a))
    g = assemble_geometry([surf, bot] + [ellipse(2048, *e) for e in ells], ells)
    flow = Flow(V1=1.0, a=rng.uniform(-0.5, 0.5, size=4))
    phit = filtered_noise(rng, 16384, 0.05, 64)
    return g, flow, phit


# the paper's problems 1-3 at t = 0 (Sec. 7.1, ellipse table and parameter table)
PAPER_ELLIPSES_123 = [(np.pi, -1.00, 0.5, 0.5, 0.0),
                      (4.0, -1.75, 0.6, 0.4, 1.0),
                      (2.3, -1.60, 0.7, 0.3, -0.5)]
PAPER_CIRCULATION_123 = {1: (1.0, [-1.0, 0.0, 0.0]),
                         2: (1.0, [0.0, 0.0, 0.0]),
                         3: (1.0, [1.0, 0.0, 0.0])}


def paper_problem(problem: int, M0=256, M1=96, Me=128):
    """Problems 1-3 at t=0: flat surface (eta = 0), flat bottom y = -3, phi~ = 0."""
    surf = graph_curve(M0, lambda a: 0 * a, lambda a: 0 * a, lambda a: 0 * a)
    bot = graph_curve(M1, lambda a: -3.0 + 0 * a, lambda a: 0 * a, lambda a: 0 * a)
    ells = PAPER_ELLIPSES_123
    g = assemble_geometry([surf, bot] + [ellipse(Me, *e) for e in ells], ells)
    V1, a = PAPER_CIRCULATION_123[problem]
    return g, Flow(V1=V1, a=np.array(a, dtype=np.float64)), np.zeros(M0)


def problem4_bottom_eta(alpha: np.ndarray) -> np.ndarray:
    """eta_1 with eta_1(0) = -1/2 and eta_1' = -5 sin^63 (Sec. 7.2), by quadrature.

    The antiderivative of sin^63 is evaluated with Gauss-Legendre quadrature on
    [0, alpha] (the integrand is a polynomial in sin, so 64 points are exact to
    rounding for the pieces used here).
    """
    x, w = np.polynomial.legendre.leggauss(64)
    alpha = np.atleast_1d(np.asarray(alpha, dtype=np.float64))
    out = np.empty_like(alpha)
    for i, a in enumerate(alpha):
        # split [0, a] into unit-ish panels so the rule stays exact
        npan = max(1, int(np.ceil(a / 0.5)))
        edges = np.linspace(0.0, a, npan + 1)
        tot = 0.0
        for lo, hi in zip(edges[:-1], edges[1:]):
            t = 0.5 * (hi - lo) * x + 0.5 * (hi + lo)
            tot += 0.5 * (hi - lo) * np.sum(w * np.sin(t) ** 63)
        out[i] = -0.5 - 5.0 * tot
    return out


def simple_channel(M0=128, M1=128, h=1.0, surface=None, seed=0):
    """No obstacles: flat bottom y = -h and a graph surface (default: a smooth wave)."""
    rng = np.random.default_rng(seed)
    if surface is None:
        A = np.array([0.08, 0.0, 0.02]) * (1 + 0.1 * rng.standard_normal(3))
        B = np.array([0.03, 0.01, 0.0])
        surf = fourier_graph(M0, 0.0, A, B)
    else:
        surf = surface
    bot = graph_curve(M1, lambda a: -h + 0 * a, lambda a: 0 * a, lambda a: 0 * a)
    return assemble_geometry([surf, bot], [])


def _height(g, k, x):
    o = g.offsets()
    zk = g.zeta[o[k]:o[k + 1]]
    return np.interp(x, np.concatenate([zk.real, [zk.real[0] + TWO_PI]]),
                     np.concatenate([zk.imag, [zk.imag[0]]]))


def fluid_grid(g, nx, ny, margin=0.0):
    """Uniform grid of the period cell restricted to the fluid (below the
    surface, above the bottom, outside every ellipse), shrunk by `margin`."""
    ymin = min(g.zeta[g.offsets()[1]:g.offsets()[2]].imag.min(), -1.0)
    ymax = g.zeta[: g.M[0]].imag.max()
    xs = (np.arange(nx) + 0.5) * TWO_PI / nx
    ys = ymin + (np.arange(ny) + 0.5) * (ymax - ymin) / ny
    Z = (xs[None, :] + 1j * ys[:, None]).ravel()
    ok = (Z.imag < _height(g, 0, Z.real) - margin) & (Z.imag > _height(g, 1, Z.real) + margin)
    for (x, y, q, b, th) in g.ellipses:
        w = (Z - (x + 1j * y)) * np.exp(-1j * th)
        ok &= (w.real / (q + margin)) ** 2 + (w.imag / (b + margin)) ** 2 > 1.0
    return Z[ok]


def near_boundary_targets(g, n, seed=0, max_spacings=2.0):
    """n points within `max_spacings` local node spacings of a boundary, on the
    fluid side: a random node, offset along the normal by U(0.05, max) spacings
    and along the tangent by U(-0.5, 0.5) spacings."""
    rng = np.random.default_rng(seed)
    o = g.offsets()
    k = rng.integers(0, g.nb, n)
    M = np.asarray(g.M)
    i = (rng.random(n) * M[k]).astype(np.int64)
    l = o[k] + i
    dz = g.dzeta[l]
    t = dz / np.abs(dz)
    h = np.abs(dz) * TWO_PI / M[k]
    side = np.where(k == 0, -1.0, 1.0)          # fluid below the surface, left of solids
    a = rng.uniform(0.05, max_spacings, n)
    s = rng.uniform(-0.5, 0.5, n)
    return g.zeta[l] + h * (side * a * 1j * t + s * t)


def targets_32768(g, seed=0, n_grid=1_000_000, n_near=100_000):
    """About n_grid points of a uniform grid of the fluid plus n_near points
    within 2 node spacings of the boundaries."""
    area_frac = 0.67
    side = int(np.sqrt(n_grid / area_frac))
    grid = fluid_grid(g, 2 * side, side // 2)
    return grid, near_boundary_targets(g, n_near, seed=seed + 1)


def smooth_density(g, seed=0, kmax=24):
    """A seeded smooth density omega (band-limited on each boundary)."""
    rng = np.random.default_rng(seed)
    return np.concatenate([filtered_noise(rng, m, 0.3, kmax) for m in g.M])


def adjoint_direction(g, seed=0, kmax=6, amp=1e-2):
    """A seeded direction in the inputs of U: (dzeta, d(zeta'), d(zeta''), d z_j,
    d phi~), each band-limited on every boundary, for directional-derivative checks."""
    rng = np.random.default_rng(seed)

    def cnoise():
        return np.concatenate([filtered_noise(rng, m, amp, kmax) + 1j * filtered_noise(rng, m, amp, kmax)
                               for m in g.M])
    dz, ddz, dd2z = cnoise(), cnoise(), cnoise()
    dzc = amp * (rng.standard_normal(len(g.zc)) + 1j * rng.standard_normal(len(g.zc)))
    dphit = filtered_noise(rng, g.M[0], amp, kmax)
    return dz, ddz, dd2z, dzc, dphit


def perturbed(g, d, t):
    """Geometry moved by t times a direction from adjoint_direction."""
    dz, ddz, dd2z, dzc, _ = d
    return Geometry(M=g.M, zeta=g.zeta + t * dz, dzeta=g.dzeta + t * ddz,
                    d2zeta=g.d2zeta + t * dd2z, zc=g.zc + t * dzc, ellipses=g.ellipses)


CONFIGS = {"one_ellipse_640": one_ellipse_640, "three_ellipses_16383": three_ellipses_16383, "two_ellipses_4096": two_ellipses_4096, "four_ellipses_32768": four_ellipses_32768}
