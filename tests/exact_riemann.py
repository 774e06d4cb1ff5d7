"""Exact solution of the Riemann problem of the 1-D Euler equations for an
ideal gas (Toro, "Riemann Solvers and Numerical Methods for Fluid Dynamics",
ch. 4: pressure function, Newton iteration for p*, self-similar sampling).
Written independently of the oracle; used to pin its hydro limit."""
import math

import numpy as np


def _f_and_df(p, rho, pk, ck, g):
    if p > pk:   # shock
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        q = math.sqrt(A / (p + B))
        return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (B + p))
    # rarefaction
    pr = p / pk
    f = 2.0 * ck / (g - 1.0) * (pr ** ((g - 1.0) / (2.0 * g)) - 1.0)
    df = 1.0 / (rho * ck) * pr ** (-(g + 1.0) / (2.0 * g))
    return f, df


def star_state(rl, ul, pl, rr, ur, pr, g):
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    p = max(1e-12, 0.5 * (pl + pr))
    for _ in range(200):
        fl, dfl = _f_and_df(p, rl, pl, cl, g)
        fr, dfr = _f_and_df(p, rr, pr, cr, g)
        dp = (fl + fr + ur - ul) / (dfl + dfr)
        pn = max(1e-14, p - dp)
        if abs(pn - p) < 1e-15 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _f_and_df(p, rl, pl, cl, g)
    fr, _ = _f_and_df(p, rr, pr, cr, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    return p, u


def sample(x, t, left, right, g, x0=0.0):
    """Density, velocity, pressure at positions x (array) and time t."""
    rl, ul, pl = left
    rr, ur, pr = right
    ps, us = star_state(rl, ul, pl, rr, ur, pr, g)
    cl = math.sqrt(g * pl / rl)
    cr = math.sqrt(g * pr / rr)
    out = np.zeros((3, len(x)))
    for n, xx in enumerate(x):
        s = (xx - x0) / t
        if s <= us:   # left of contact
            if ps > pl:  # left shock
                sl = ul - cl * math.sqrt((g + 1) / (2 * g) * ps / pl + (g - 1) / (2 * g))
                if s <= sl:
                    w = (rl, ul, pl)
                else:
                    r = rl * (ps / pl + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pl + 1)
                    w = (r, us, ps)
            else:
                shl = ul - cl
                csl = cl * (ps / pl) ** ((g - 1) / (2 * g))
                stl = us - csl
                if s <= shl:
                    w = (rl, ul, pl)
                elif s >= stl:
                    w = (rl * (ps / pl) ** (1 / g), us, ps)
                else:
                    c = 2 / (g + 1) * (cl + (g - 1) / 2 * (ul - s))
                    r = rl * (c / cl) ** (2 / (g - 1))
                    u = 2 / (g + 1) * (cl + (g - 1) / 2 * ul + s)
                    w = (r, u, pl * (c / cl) ** (2 * g / (g - 1)))
        else:
            if ps > pr:
                sr = ur + cr * math.sqrt((g + 1) / (2 * g) * ps / pr + (g - 1) / (2 * g))
                if s >= sr:
                    w = (rr, ur, pr)
                else:
                    r = rr * (ps / pr + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pr + 1)
                    w = (r, us, ps)
            else:
                shr = ur + cr
                csr = cr * (ps / pr) ** ((g - 1) / (2 * g))
                str_ = us + csr
                if s >= shr:
                    w = (rr, ur, pr)
                elif s <= str_:
                    w = (rr * (ps / pr) ** (1 / g), us, ps)
                else:
                    c = 2 / (g + 1) * (cr - (g - 1) / 2 * (ur - s))
                    r = rr * (c / cr) ** (2 / (g - 1))
                    u = 2 / (g + 1) * (-cr + (g - 1) / 2 * ur + s)
                    w = (r, u, pr * (c / cr) ** (2 * g / (g - 1)))
        out[:, n] = w
    return out


# ------------------------------------------------------------- isothermal
# Isothermal gas (p = c^2 rho): across a shock into state k the velocity
# changes by c (rho* - rho_k) / sqrt(rho* rho_k); across a rarefaction by
# c ln(rho* / rho_k); inside a left (right) fan u -+ c = x/t and
# rho = rho_k exp(-+(u - u_k)/c).

def _iso_f(rs, rk, c):
    if rs > rk:
        return c * (rs - rk) / math.sqrt(rs * rk), c * (rs + rk) / (2 * rs * math.sqrt(rs * rk))
    return c * math.log(rs / rk), c / rs


def iso_star(rl, ul, rr, ur, c):
    """Star density and velocity of the isothermal Riemann problem (Newton
    on f_L(rho*) + f_R(rho*) + u_R - u_L = 0)."""
    rs = math.sqrt(rl * rr)
    for _ in range(100):
        fl, dfl = _iso_f(rs, rl, c)
        fr, dfr = _iso_f(rs, rr, c)
        g = fl + fr + ur - ul
        step = g / (dfl + dfr)
        rs_new = max(rs - step, 1e-3 * rs)
        if abs(rs_new - rs) < 1e-14 * rs:
            rs = rs_new
            break
        rs = rs_new
    fl, _ = _iso_f(rs, rl, c)
    return rs, ul - fl


def iso_sample(x, t, left, right, c, x0=0.0):
    """rho(x, t), u(x, t) of the isothermal Riemann problem; left/right =
    (rho, u)."""
    rl, ul = left
    rr, ur = right
    rs, us = iso_star(rl, ul, rr, ur, c)
    xi = (np.asarray(x, dtype=float) - x0) / t
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    for q, s in enumerate(xi):
        if s <= us:   # left of the contact-free middle: left wave
            if rs > rl:
                sh = ul - c * math.sqrt(rs / rl)
                rho[q], u[q] = (rl, ul) if s < sh else (rs, us)
            else:
                head, tail = ul - c, us - c
                if s < head:
                    rho[q], u[q] = rl, ul
                elif s > tail:
                    rho[q], u[q] = rs, us
                else:
                    u[q] = s + c
                    rho[q] = rl * math.exp(-(u[q] - ul) / c)
        else:
            if rs > rr:
                sh = ur + c * math.sqrt(rs / rr)
                rho[q], u[q] = (rr, ur) if s > sh else (rs, us)
            else:
                head, tail = ur + c, us + c
                if s > head:
                    rho[q], u[q] = rr, ur
                elif s < tail:
                    rho[q], u[q] = rs, us
                else:
                    u[q] = s - c
                    rho[q] = rr * math.exp((u[q] - ur) / c)
    return rho, u
