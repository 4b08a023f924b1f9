"""Exact solutions used to pin the oracle (test infrastructure only).

* Exact solution of the Riemann problem for the 1D Euler equations of an
  ideal gas (the shock-tube reference of the Sod and Lax cases, Sec. 3.4):
  the star pressure solves f_L(p) + f_R(p) + (u_R - u_L) = 0, where f_K is
  the shock (Rankine-Hugoniot) branch for p > p_K and the isentropic
  rarefaction branch for p <= p_K; the solution is then sampled on x/t.
* Exact solution of the inviscid Burgers equation before shock formation
  (Sec. 3.3): u = u0(x - u t), solved per point by Newton's method.
"""
import math

import numpy as np


def _fK(p, rho, pk, c, g):
    if p > pk:   # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        f = (p - pk) * math.sqrt(A / (p + B))
        df = math.sqrt(A / (B + p)) * (1.0 - (p - pk) / (2.0 * (B + p)))
    else:        # rarefaction
        f = 2.0 * c / (g - 1.0) * ((p / pk) ** ((g - 1.0) / (2.0 * g)) - 1.0)
        df = 1.0 / (rho * c) * (p / pk) ** (-(g + 1.0) / (2.0 * g))
    return f, df


def riemann_star(left, right, gamma=1.4, tol=1e-15):
    """Star-region (p*, u*) of the Riemann problem with primitive states
    left = (rho, u, p), right = (rho, u, p)."""
    rl, ul, pl = left
    rr, ur, pr = right
    g = gamma
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    # start from the two-rarefaction approximation
    z = (g - 1.0) / (2.0 * g)
    p = ((cl + cr - 0.5 * (g - 1.0) * (ur - ul)) / (cl / pl ** z + cr / pr ** z)) ** (1.0 / z)
    p = max(p, 1e-12)
    for _ in range(200):
        fl, dfl = _fK(p, rl, pl, cl, g)
        fr, dfr = _fK(p, rr, pr, cr, g)
        pn = p - (fl + fr + ur - ul) / (dfl + dfr)
        if pn <= 0:
            pn = 0.5 * p
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _fK(p, rl, pl, cl, g)
    fr, _ = _fK(p, rr, pr, cr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def riemann_sample(left, right, x, t, x0=0.5, gamma=1.4):
    """Primitive (rho, u, p) arrays of the exact solution at positions x, time t."""
    rl, ul, pl = left
    rr, ur, pr = right
    g = gamma
    ps, us = riemann_star(left, right, g)
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros((3, x.size))
    for i, xi in enumerate(x):
        s = (xi - x0) / t
        if s <= us:  # left of contact
            if ps > pl:  # left shock
                sl = ul - cl * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                if s <= sl:
                    w = (rl, ul, pl)
                else:
                    rs = rl * (ps / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pl + 1)
                    w = (rs, us, ps)
            else:        # left rarefaction
                shl = ul - cl
                csl = cl * (ps / pl) ** ((g - 1) / (2 * g))
                stl = us - csl
                if s <= shl:
                    w = (rl, ul, pl)
                elif s >= stl:
                    w = (rl * (ps / pl) ** (1 / g), us, ps)
                else:
                    c = 2 / (g + 1) * (cl + (g - 1) / 2 * (ul - s))
                    u = 2 / (g + 1) * (cl + (g - 1) / 2 * ul + s)
                    rho = rl * (c / cl) ** (2 / (g - 1))
                    w = (rho, u, pl * (c / cl) ** (2 * g / (g - 1)))
        else:            # right of contact
            if ps > pr:  # right shock
                sr = ur + cr * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                if s >= sr:
                    w = (rr, ur, pr)
                else:
                    rs = rr * (ps / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pr + 1)
                    w = (rs, us, ps)
            else:        # right rarefaction
                shr = ur + cr
                csr = cr * (ps / pr) ** ((g - 1) / (2 * g))
                str_ = us + csr
                if s >= shr:
                    w = (rr, ur, pr)
                elif s <= str_:
                    w = (rr * (ps / pr) ** (1 / g), us, ps)
                else:
                    c = 2 / (g + 1) * (cr - (g - 1) / 2 * (ur - s))
                    u = 2 / (g + 1) * (-cr + (g - 1) / 2 * ur + s)
                    rho = rr * (c / cr) ** (2 / (g - 1))
                    w = (rho, u, pr * (c / cr) ** (2 * g / (g - 1)))
        out[:, i] = w
    return out


def burgers_exact(x, t, u0, du0, tol=1e-15):
    """u(x, t) of u_t + (u^2/2)_x = 0 with smooth u0 (t below breaking time)."""
    x = np.asarray(x, dtype=np.float64)
    u = u0(x)
    for _ in range(100):
        xi = x - u * t
        g = u - u0(xi)
        dg = 1.0 + du0(xi) * t
        un = u - g / dg
        if np.max(np.abs(un - u)) <= tol:
            u = un
            break
        u = un
    return u
