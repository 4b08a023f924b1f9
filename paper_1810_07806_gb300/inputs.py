"""Seeded synthetic initial states shaped like the paper's test problems.

This module holds only input construction (initial conditions and request
traces); none of the scheme's arithmetic lives here.  It depends on numpy
alone, so the CUDA library and the CPU oracle can both be fed from it.

All states are returned as float64 numpy arrays in SoA layout
U[var][z][y][x] (x fastest) with conserved variables
(rho, rho*u_1, ..., rho*u_nd, E), E = p/(gamma-1) + rho |u|^2 / 2.

Grid convention: transmissive axes place node i at lo + i*h with
h = (hi - lo)/(n - 1) (both end points are nodes); periodic axes place node i
at lo + i*h with h = (hi - lo)/n (the end point is the image of node 0); axes
with a reflecting wall or a fixed-state side place node i at the cell centre
lo + (i + 1/2) h with h = (hi - lo)/n (walls sit on the outer faces).

Boundary kinds (the library's codes): 0 transmissive, 1 periodic,
2 reflecting wall, 3 fixed state.
"""
import math
from dataclasses import dataclass, field

import numpy as np


def prim_to_cons(rho, vel, p, gamma):
    """rho, p: arrays of one shape; vel: list of nd arrays of that shape."""
    nd = len(vel)
    out = np.empty((nd + 2,) + np.shape(rho), dtype=np.float64)
    out[0] = rho
    ke = np.zeros_like(out[0])
    for a, v in enumerate(vel):
        out[1 + a] = rho * v
        ke += v * v
    out[nd + 1] = p / (gamma - 1.0) + 0.5 * rho * ke
    return out


def cons_to_prim(U, gamma):
    nd = U.shape[0] - 2
    rho = U[0]
    vel = [U[1 + a] / rho for a in range(nd)]
    ke = sum(v * v for v in vel)
    p = (gamma - 1.0) * (U[nd + 1] - 0.5 * rho * ke)
    return rho, vel, p


def axis_nodes(n, lo, hi, periodic):
    h = (hi - lo) / n if periodic else (hi - lo) / (n - 1)
    return lo + h * np.arange(n), h


@dataclass
class Problem:
    """A synthetic initial state together with the grid it lives on."""
    name: str
    ndim: int
    n: tuple
    lo: tuple
    hi: tuple
    periodic: tuple
    gamma: float
    U0: np.ndarray
    t_end: float = 0.0
    h: tuple = field(default=())
    bc_lo: tuple = (0, 0, 0)          # boundary kind of the low side of each axis
    bc_hi: tuple = (0, 0, 0)
    bc_state: tuple = None            # [axis][side] conserved state of fixed sides
    gravity: tuple = (0.0, 0.0, 0.0)  # body force per unit mass

    @property
    def nv(self):
        return self.ndim + 2

    @property
    def cells(self):
        return int(np.prod(self.n[: self.ndim]))


def _finish(name, ndim, n, lo, hi, periodic, gamma, U0, t_end):
    h = tuple(((hi[a] - lo[a]) / n[a]) if periodic[a] else ((hi[a] - lo[a]) / (n[a] - 1))
              for a in range(ndim))
    return Problem(name, ndim, tuple(n), tuple(lo), tuple(hi), tuple(periodic), gamma,
                   np.ascontiguousarray(U0), t_end, h)


# ---------------------------------------------------------------- 1D shock tubes
SOD = ((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))            # Sec. 3.4
LAX = ((0.445, 0.698, 3.528), (0.5, 0.0, 0.571))      # Sec. 3.4


def shock_tube(n=400, states=SOD, x0=0.5, gamma=1.4, t_end=0.2, name="sod"):
    x, _ = axis_nodes(n, 0.0, 1.0, False)
    left = x <= x0
    rho = np.where(left, states[0][0], states[1][0])
    u = np.where(left, states[0][1], states[1][1])
    p = np.where(left, states[0][2], states[1][2])
    U = prim_to_cons(rho, [u], p, gamma)
    return _finish(name, 1, (n,), (0.0,), (1.0,), (0,), gamma, U, t_end)


def density_wave_1d(n, amp=0.2, gamma=1.4):
    """rho = 1 + amp sin(2 pi x), u = 1, p = 1 on periodic [0, 1): a smooth
    solution that translates with unit speed."""
    x, _ = axis_nodes(n, 0.0, 1.0, True)
    rho = 1.0 + amp * np.sin(2 * np.pi * x)
    U = prim_to_cons(rho, [np.ones_like(x)], np.ones_like(x), gamma)
    return _finish("density_wave", 1, (n,), (0.0,), (1.0,), (1,), gamma, U, 0.0)


# ---------------------------------------------------------------- 2D four quadrants
LAX_LIU_3 = ((1.5, 0.0, 0.0, 1.5), (0.5323, 1.206, 0.0, 0.3),
             (0.138, 1.206, 1.206, 0.029), (0.5323, 0.0, 1.206, 0.3))   # NE, NW, SW, SE
LAX_LIU_6 = ((1.0, 0.75, -0.5, 1.0), (2.0, 0.75, 0.5, 1.0),
             (1.0, -0.75, 0.5, 1.0), (3.0, -0.75, -0.5, 1.0))


def four_quadrant(n=1024, ny=None, quads=LAX_LIU_3, gamma=1.4, t_end=0.3, name="lax_liu_3"):
    """Quadrant states (rho, u, v, p) in the order NE, NW, SW, SE; interfaces
    at x = y = 1/2 on [0, 1]^2, transmissive boundaries."""
    ny = n if ny is None else ny
    x, _ = axis_nodes(n, 0.0, 1.0, False)
    y, _ = axis_nodes(ny, 0.0, 1.0, False)
    X = np.broadcast_to(x[None, :], (ny, n))
    Y = np.broadcast_to(y[:, None], (ny, n))
    east, north = X >= 0.5, Y >= 0.5
    sel = [east & north, (~east) & north, (~east) & (~north), east & (~north)]
    prim = np.zeros((4, ny, n))
    for q, m in zip(quads, sel):
        for c in range(4):
            prim[c][m] = q[c]
    U = prim_to_cons(prim[0], [prim[1], prim[2]], prim[3], gamma)
    return _finish(name, 2, (n, ny), (0.0, 0.0), (1.0, 1.0), (0, 0), gamma, U, t_end)


# ---------------------------------------------------------------- 3D Taylor-Green
def taylor_green(n=256, gamma=1.4):
    """Inviscid Taylor-Green vortex on periodic [0, 2 pi)^3 (n unique nodes per axis)."""
    x, _ = axis_nodes(n, 0.0, 2 * np.pi, True)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    u = np.sin(X) * np.cos(Y) * np.cos(Z)
    v = -np.cos(X) * np.sin(Y) * np.cos(Z)
    w = np.zeros_like(u)
    p = 100.0 / gamma + (np.cos(2 * X) + np.cos(2 * Y)) * (np.cos(2 * Z) + 2.0) / 16.0
    U = prim_to_cons(np.ones_like(u), [u, v, w], p, gamma)
    return _finish("taylor_green", 3, (n, n, n), (0.0,) * 3, (2 * np.pi,) * 3, (1, 1, 1),
                   gamma, U, 0.0)


# ---------------------------------------------------------------- batched Shu-Osher type
def normal_shock_post(mach, rho1=1.0, p1=1.0, gamma=1.4):
    """State behind a normal shock of Mach `mach` running into gas at rest
    (rho1, 0, p1) (Rankine-Hugoniot relations).  Mach 3 gives the paper's
    (3.857, 2.629, 10.333) of the shock-density wave case."""
    g, M2 = gamma, mach * mach
    rho2 = rho1 * (g + 1) * M2 / ((g - 1) * M2 + 2)
    p2 = p1 * (2 * g * M2 - (g - 1)) / (g + 1)
    s = mach * math.sqrt(g * p1 / rho1)
    u2 = s * (1.0 - rho1 / rho2)
    return rho2, u2, p2


def shu_osher_like(n, mach, eps, k, gamma=1.4, lo=-5.0, hi=5.0, x_shock=-4.0):
    x, _ = axis_nodes(n, lo, hi, False)
    r2, u2, p2 = normal_shock_post(mach, 1.0, 1.0, gamma)
    post = x < x_shock
    rho = np.where(post, r2, 1.0 + eps * np.sin(k * x))
    u = np.where(post, u2, 0.0)
    p = np.where(post, p2, 1.0)
    U = prim_to_cons(rho, [u], p, gamma)
    return _finish("shu_osher_like", 1, (n,), (lo,), (hi,), (0,), gamma, U, 1.8)


def shu_osher_batch(count=4096, seed=1810, n_lo=200, n_hi=4000, gamma=1.4):
    """Instances with N log-uniform in [n_lo, n_hi], Mach U[1.5, 5],
    eps U[0.1, 0.3], k U[3, 8]."""
    rng = np.random.default_rng(seed)
    ns = np.rint(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), count))).astype(int)
    mach = rng.uniform(1.5, 5.0, count)
    eps = rng.uniform(0.1, 0.3, count)
    kk = rng.uniform(3.0, 8.0, count)
    return [shu_osher_like(int(ns[i]), mach[i], eps[i], kk[i], gamma) for i in range(count)]


def density_wave_batch(count=4096, seed=1811, n_lo=200, n_hi=4000, gamma=1.4, t_end=0.2):
    """Smooth counterparts of the Shu-Osher batch, for the FP32 error where
    no discontinuity is present: periodic [0, 1), N log-uniform in
    [n_lo, n_hi], rho = 1 + a sin(2 pi k x + phi), a U[0.05, 0.3], k in
    1..4, u U[0.5, 1.5], p = 1 (each an exact translation at speed u)."""
    rng = np.random.default_rng(seed)
    ns = np.rint(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), count))).astype(int)
    amp = rng.uniform(0.05, 0.3, count)
    kk = rng.integers(1, 5, count)
    phi = rng.uniform(0.0, 2 * np.pi, count)
    vel = rng.uniform(0.5, 1.5, count)
    out = []
    for i in range(count):
        x, _ = axis_nodes(int(ns[i]), 0.0, 1.0, True)
        rho = 1.0 + amp[i] * np.sin(2 * np.pi * kk[i] * x + phi[i])
        U = prim_to_cons(rho, [np.full_like(x, vel[i])], np.ones_like(x), gamma)
        out.append(_finish("density_wave", 1, (int(ns[i]),), (0.0,), (1.0,), (1,), gamma, U, t_end))
    return out


# ---------------------------------------------------------------- serving trace
@dataclass
class Request:
    arrival_s: float
    side: int
    quads: tuple
    t_end: float
    fp32: bool

    def problem(self, gamma=1.4):
        return four_quadrant(self.side, quads=self.quads, gamma=gamma, t_end=self.t_end,
                             name="quadrant_request")


def serving_trace(count=2000, rate=200.0, seed=7806, side_lo=128, side_hi=1024):
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, count)
    t = np.cumsum(gaps)
    out = []
    for i in range(count):
        side = int(round(math.exp(rng.uniform(math.log(side_lo), math.log(side_hi)))))
        quads = tuple((float(rng.uniform(0.1, 2.0)), float(rng.uniform(-1.5, 1.5)),
                       float(rng.uniform(-1.5, 1.5)), float(rng.uniform(0.03, 2.0)))
                      for _ in range(4))
        t_end = float(rng.uniform(0.1, 0.3))
        fp32 = bool(rng.uniform() < 0.5)
        out.append(Request(float(t[i]), side, quads, t_end, fp32))
    return out


def random_smooth_state(ndim, n, seed, gamma=1.4, amp=0.1, periodic=True):
    """A smooth random state (low Fourier modes) for RHS parity tests."""
    rng = np.random.default_rng(seed)
    shape = tuple(reversed(n[:ndim]))
    grids = np.meshgrid(*[np.linspace(0, 2 * np.pi, s, endpoint=not periodic) for s in shape],
                        indexing="ij")

    def field_(base, scale):
        f = np.full(shape, base, dtype=np.float64)
        for _ in range(3):
            ph = rng.uniform(0, 2 * np.pi, ndim)
            kv = rng.integers(1, 3, ndim)
            term = np.ones(shape)
            for a in range(ndim):
                term = term * np.cos(kv[a] * grids[a] + ph[a])
            f += scale * rng.uniform(-1, 1) * term
        return f

    rho = field_(1.0, amp)
    vel = [field_(0.0, 0.5) for _ in range(ndim)]
    p = field_(1.0, amp)
    return prim_to_cons(rho, vel, p, gamma)


def random_rough_state(ndim, n, seed, gamma=1.4):
    """Piecewise-constant random blocks plus noise: exercises stencil cuts."""
    rng = np.random.default_rng(seed)
    shape = tuple(reversed(n[:ndim]))
    blocks = [max(1, s // 4) for s in shape]

    def field_(lo, hi):
        coarse = rng.uniform(lo, hi, [-(-s // b) for s, b in zip(shape, blocks)])
        f = coarse
        for a, b in enumerate(blocks):
            f = np.repeat(f, b, axis=a)
        f = f[tuple(slice(0, s) for s in shape)]
        return f * (1.0 + 0.01 * rng.standard_normal(shape))

    rho = field_(0.2, 2.0)
    vel = [field_(-1.0, 1.0) for _ in range(ndim)]
    p = field_(0.1, 2.0)
    return prim_to_cons(rho, vel, p, gamma)


# ---------------------------------------------------------------- Rayleigh-Taylor
BC_TRANSMISSIVE, BC_PERIODIC, BC_REFLECTING, BC_FIXED = 0, 1, 2, 3


def rayleigh_taylor(nx=128, ny=None, amp=0.025, gamma=5.0 / 3.0, t_end=1.95):
    """Sec. 3.9: [0, 0.25] x [0, 1], heavy fluid (rho = 2, p = 1 + 2y) below
    y = 1/2, light fluid (rho = 1, p = y + 3/2, the reading of the garbled
    upper pressure that keeps p continuous and hydrostatic) above, v =
    -amp a cos(8 pi x) with a the local sound speed, u = 0, gamma = 5/3.
    Reflecting walls at x = 0, 0.25; fixed states (2, 0, 0, 1) below y = 0 and
    (1, 0, 0, 2.5) above y = 1; body force g = (0, 1), i.e. the source
    (0, 0, rho, rho v).  Cell-centred nodes, ny = 4 nx (square cells)."""
    ny = 4 * nx if ny is None else ny
    hx, hy = 0.25 / nx, 1.0 / ny
    x = (np.arange(nx) + 0.5) * hx
    y = (np.arange(ny) + 0.5) * hy
    Y, X = np.meshgrid(y, x, indexing="ij")
    lower = Y < 0.5
    rho = np.where(lower, 2.0, 1.0)
    p = np.where(lower, 1.0 + 2.0 * Y, Y + 1.5)
    a = np.sqrt(gamma * p / rho)
    v = -amp * a * np.cos(8.0 * np.pi * X)
    U = prim_to_cons(rho, [np.zeros_like(rho), v], p, gamma)
    bottom = prim_to_cons(np.array(2.0), [np.array(0.0), np.array(0.0)], np.array(1.0), gamma)
    top = prim_to_cons(np.array(1.0), [np.array(0.0), np.array(0.0)], np.array(2.5), gamma)
    return Problem("rayleigh_taylor", 2, (nx, ny), (0.0, 0.0), (0.25, 1.0), (0, 0), gamma,
                   np.ascontiguousarray(U), t_end, (hx, hy),
                   bc_lo=(BC_REFLECTING, BC_FIXED, 0), bc_hi=(BC_REFLECTING, BC_FIXED, 0),
                   bc_state=((None, None), (tuple(bottom), tuple(top)), (None, None)),
                   gravity=(0.0, 1.0, 0.0))
