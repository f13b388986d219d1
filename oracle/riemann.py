"""Exact solution of the 1-D Riemann problem for an ideal gas (TEST
INFRASTRUCTURE ONLY).

Section V.C compares the lattice Boltzmann shock tube with "the analytical
solution"; this is that solution, written from the wave relations of the
Euler equations: across a shock the Rankine-Hugoniot conditions hold, across a
rarefaction the isentropic Riemann invariant; the star pressure p* is the root
of f_L(p) + f_R(p) + (u_R - u_L) = 0, found by Newton's method.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


@dataclass
class Star:
    p: float
    u: float
    rho_l: float
    rho_r: float


def _f(p, rho, pk, a, g):
    """Velocity jump across the left/right wave as a function of p, and its
    derivative."""
    if p > pk:  # shock: Rankine-Hugoniot
        A = 2.0 / ((g + 1.0) * rho)
        B = (g - 1.0) / (g + 1.0) * pk
        s = math.sqrt(A / (p + B))
        return (p - pk) * s, s * (1.0 - 0.5 * (p - pk) / (p + B))
    # rarefaction: isentropic
    e = (g - 1.0) / (2.0 * g)
    return (2.0 * a / (g - 1.0) * ((p / pk) ** e - 1.0),
            (p / pk) ** (-(g + 1.0) / (2.0 * g)) / (rho * a))


def star_state(left, right, gamma: float = 1.4, tol: float = 1e-14) -> Star:
    """left/right = (rho, u, p).  Returns the star region state."""
    rl, ul, pl = left
    rr, ur, pr = right
    g = gamma
    al, ar = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    if 2.0 * (al + ar) / (g - 1.0) <= ur - ul:
        raise ValueError("vacuum generated: no star state")
    p = max(1e-12, 0.5 * (pl + pr))
    for _ in range(200):
        fl, dl = _f(p, rl, pl, al, g)
        fr, dr = _f(p, rr, pr, ar, g)
        dp = (fl + fr + ur - ul) / (dl + dr)
        pn = max(1e-14, p - dp)
        if abs(pn - p) <= tol * 0.5 * (pn + p):
            p = pn
            break
        p = pn
    fl, _ = _f(p, rl, pl, al, g)
    fr, _ = _f(p, rr, pr, ar, g)
    u = 0.5 * (ul + ur) + 0.5 * (fr - fl)
    gm = (g - 1.0) / (g + 1.0)
    rho_l = (rl * (p / pl + gm) / (gm * p / pl + 1.0) if p > pl
             else rl * (p / pl) ** (1.0 / g))
    rho_r = (rr * (p / pr + gm) / (gm * p / pr + 1.0) if p > pr
             else rr * (p / pr) ** (1.0 / g))
    return Star(p, u, rho_l, rho_r)


def wave_speeds(left, right, gamma: float = 1.4) -> dict:
    """Speeds of the wave edges: left head/tail (or shock), contact, right
    tail/head (or shock)."""
    rl, ul, pl = left
    rr, ur, pr = right
    g = gamma
    st = star_state(left, right, g)
    al, ar = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    out = {"contact": st.u}
    if st.p > pl:
        s = ul - al * math.sqrt((g + 1) / (2 * g) * st.p / pl + (g - 1) / (2 * g))
        out["left_head"] = out["left_tail"] = s
    else:
        out["left_head"] = ul - al
        out["left_tail"] = st.u - al * (st.p / pl) ** ((g - 1) / (2 * g))
    if st.p > pr:
        s = ur + ar * math.sqrt((g + 1) / (2 * g) * st.p / pr + (g - 1) / (2 * g))
        out["right_head"] = out["right_tail"] = s
    else:
        out["right_head"] = ur + ar
        out["right_tail"] = st.u + ar * (st.p / pr) ** ((g - 1) / (2 * g))
    return out


def sample(x, t: float, x_d: float, left, right, gamma: float = 1.4):
    """(rho, u, p) of the exact solution at positions x and time t > 0 for a
    diaphragm at x_d."""
    x = np.asarray(x, dtype=np.float64)
    rl, ul, pl = left
    rr, ur, pr = right
    g = gamma
    st = star_state(left, right, g)
    w = wave_speeds(left, right, g)
    al, ar = math.sqrt(g * pl / rl), math.sqrt(g * pr / rr)
    S = (x - x_d) / t
    rho = np.empty_like(S)
    u = np.empty_like(S)
    p = np.empty_like(S)
    for i, s in enumerate(S):
        if s <= st.u:  # left of the contact
            if st.p > pl:  # left shock
                if s < w["left_head"]:
                    rho[i], u[i], p[i] = rl, ul, pl
                else:
                    rho[i], u[i], p[i] = st.rho_l, st.u, st.p
            else:  # left rarefaction
                if s < w["left_head"]:
                    rho[i], u[i], p[i] = rl, ul, pl
                elif s > w["left_tail"]:
                    rho[i], u[i], p[i] = st.rho_l, st.u, st.p
                else:
                    c = 2.0 / (g + 1) + (g - 1) / ((g + 1) * al) * (ul - s)
                    rho[i] = rl * c ** (2.0 / (g - 1))
                    u[i] = 2.0 / (g + 1) * (al + 0.5 * (g - 1) * ul + s)
                    p[i] = pl * c ** (2.0 * g / (g - 1))
        else:  # right of the contact
            if st.p > pr:  # right shock
                if s > w["right_head"]:
                    rho[i], u[i], p[i] = rr, ur, pr
                else:
                    rho[i], u[i], p[i] = st.rho_r, st.u, st.p
            else:  # right rarefaction
                if s > w["right_head"]:
                    rho[i], u[i], p[i] = rr, ur, pr
                elif s < w["right_tail"]:
                    rho[i], u[i], p[i] = st.rho_r, st.u, st.p
                else:
                    c = 2.0 / (g + 1) - (g - 1) / ((g + 1) * ar) * (ur - s)
                    rho[i] = rr * c ** (2.0 / (g - 1))
                    u[i] = 2.0 / (g + 1) * (-ar + 0.5 * (g - 1) * ur + s)
                    p[i] = pr * c ** (2.0 * g / (g - 1))
    return rho, u, p


def l1_errors(x, t, x_d, left, right, rho, u, p, gamma=1.4) -> dict:
    """Mean absolute error of (rho, u, p) against the exact solution."""
    er, eu, ep = sample(x, t, x_d, left, right, gamma)
    return {"rho": float(np.mean(np.abs(rho - er))),
            "u": float(np.mean(np.abs(u - eu))),
            "p": float(np.mean(np.abs(p - ep)))}
