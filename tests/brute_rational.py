"""Exact rational-arithmetic packet tracer for tiny lattices.

An independent restatement of the tau = 1 step used to pin the FP64 oracle.
It takes a different route to the same quantities so that a slip in one is
not repeated in the other:

* level densities d1, d2 come from solving the two constraints they exist to
  satisfy (Section III.B): total mass  b0 d0 + b1 d1 + b2 d2 = rho  and the
  velocity-spread energy  b1 d1 c1^2 + b2 d2 c2^2 = D (gamma-1) rho e,
  by Cramer's rule, instead of from the closed forms of eqs 24-25;
* c1 = int(sqrt(X)) is taken exactly with integer square roots;
* each packet is followed to its continuous end point x + V + c' and split
  over the surrounding nodes with linear / bilinear (cloud-in-cell) weights
  (eqs 28-29), instead of via floor(V) + c' + k.

All arithmetic is exact (fractions.Fraction), so summation order is
irrelevant and the result is the exact value of one step.
"""
from __future__ import annotations

import math
from fractions import Fraction as F

TRANSMISSIVE, REFLECTING, PERIODIC = 0, 1, 2


def isqrt_floor(x: F) -> int:
    """floor(sqrt(x)) for a non-negative rational x."""
    p, q = x.numerator, x.denominator
    return math.isqrt(p * q) // q


def velocity_set(dim: int, c1: int):
    """(c' vector, level) pairs of Section IV."""
    c2 = c1 + 1
    if dim == 1:
        return [((0,), 0), ((c1,), 1), ((-c1,), 1), ((c2,), 2), ((-c2,), 2)]
    out = []
    for lev, c in ((1, c1), (2, c2)):
        out += [((c, 0), lev), ((-c, 0), lev), ((0, c), lev), ((0, -c), lev)]
    return out


def equilibrium(dim, gamma, theta, rho, m, rhoE):
    """Exact equilibrium of one node: velocity, levels, densities, phi."""
    D = dim
    V = [mi / rho for mi in m]
    e = rhoE / rho - sum(v * v for v in V) / 2
    assert e >= 0
    b0, b = 1, (2 if dim == 1 else 4)
    d0 = theta * rho if dim == 1 else F(0)
    q = D * (gamma - 1) * rho * e
    c1 = isqrt_floor(q / (rho - b0 * d0))
    c2 = c1 + 1
    # b d1 + b d2 = rho - b0 d0 ;  b d1 c1^2 + b d2 c2^2 = q
    a11, a12, r1 = b, b, rho - b0 * d0
    a21, a22, r2 = b * c1 * c1, b * c2 * c2, q
    det = a11 * a22 - a12 * a21
    d1 = (r1 * a22 - a12 * r2) / det
    d2 = (a11 * r2 - a21 * r1) / det
    phi = (1 - F(D, 2) * (gamma - 1)) * e
    return V, c1, (d0, d1, d2), phi


def _map(bc, n, L):
    """(index, sign of the axis momentum) or None when the landing drops."""
    if 0 <= L < n:
        return L, 1
    if bc == TRANSMISSIVE:
        return None
    if bc == PERIODIC:
        return L % n, 1
    # reflecting walls at -1/2 and n - 1/2: the packet bounces until it is
    # inside; each bounce negates its normal momentum (period 2n)
    w = L % (2 * n)
    return (2 * n - 1 - w, -1) if w >= n else (w, 1)


def step(dim, shape, bcs, gamma, theta, state):
    """One exact step.  shape = (nx,) or (nx, ny); bcs per axis; state maps a
    node tuple (x,) / (x, y) to (rho, (m_x[, m_y]), rhoE)."""
    nodes = list(state.keys())
    # generous ghost width: any reach of any node, plus slack
    reach = 0
    for nd in nodes:
        rho, m, rhoE = state[nd]
        if rho == 0:
            continue
        V, c1, _, _ = equilibrium(dim, gamma, theta, rho, m, rhoE)
        reach = max(reach, max(abs(math.floor(v)) + 2 for v in V) + c1 + 1)
    ranges = []
    for a in range(dim):
        lo, hi = (-reach, shape[a] + reach) if bcs[a] == TRANSMISSIVE else (0, shape[a])
        ranges.append(range(lo, hi))
    zero = (F(0), tuple(F(0) for _ in range(dim)), F(0))
    acc = {nd: [F(0), [F(0)] * dim, F(0)] for nd in nodes}

    def sources():
        if dim == 1:
            for x in ranges[0]:
                yield (x,)
        else:
            for y in ranges[1]:
                for x in ranges[0]:
                    yield (x, y)

    for s in sources():
        g = tuple(min(max(s[a], 0), shape[a] - 1) for a in range(dim))
        rho, m, rhoE = state.get(g, zero)
        if rho == 0:
            continue
        V, c1, dl, phi = equilibrium(dim, gamma, theta, rho, m, rhoE)
        for cv, lev in velocity_set(dim, c1):
            d = dl[lev]
            cb = [V[a] + cv[a] for a in range(dim)]
            zeta = sum(c * c for c in cb) / 2 + phi
            end = [s[a] + cb[a] for a in range(dim)]
            base = [math.floor(x) for x in end]
            frac = [end[a] - base[a] for a in range(dim)]
            for corner in range(1 << dim):
                w = F(1)
                L = []
                for a in range(dim):
                    k = (corner >> a) & 1
                    w *= frac[a] if k else 1 - frac[a]
                    L.append(base[a] + k)
                idx, sgn = [], []
                for a in range(dim):
                    r = _map(bcs[a], shape[a], L[a])
                    if r is None:
                        break
                    idx.append(r[0])
                    sgn.append(r[1])
                else:
                    t = acc[tuple(idx)]
                    t[0] += w * d
                    for a in range(dim):
                        t[1][a] += w * d * cb[a] * sgn[a]
                    t[2] += w * d * zeta
    return {nd: (v[0], tuple(v[1]), v[2]) for nd, v in acc.items()}


# ---------------------------------------------------------------------------
# relaxation time tau != 1 (eqs 4-5), per-packet state
# ---------------------------------------------------------------------------

def mirror_slot(dim, axis, j):
    """Slot of packet j after a bounce off a wall normal to `axis`: the entry
    of the velocity set whose c' points the other way along that axis."""
    cv, lev = velocity_set(dim, 1)[j]
    flipped = tuple(-c if a == axis else c for a, c in enumerate(cv))
    for i, (cw, lw) in enumerate(velocity_set(dim, 1)):
        if cw == flipped and lw == lev:
            return i
    raise AssertionError("no mirrored slot")


def equilibrium_slots(dim, gamma, theta, rho, m, rhoE):
    """Equilibrium packets (mass, momentum tuple, energy) in slot order."""
    if rho == 0:
        return [(F(0), tuple(F(0) for _ in range(dim)), F(0))
                for _ in velocity_set(dim, 1)]
    V, c1, dl, phi = equilibrium(dim, gamma, theta, rho, m, rhoE)
    out = []
    for cv, lev in velocity_set(dim, c1):
        d = dl[lev]
        cb = [V[a] + cv[a] for a in range(dim)]
        out.append((d, tuple(d * c for c in cb),
                    d * (sum(c * c for c in cb) / 2 + phi)))
    return out


def step_bgk(dim, shape, bcs, gamma, theta, tau, state):
    """One exact step with relaxation time tau.  state maps a node tuple to
    its list of slots (mass, momentum tuple, energy).  Every packet is
    relaxed towards the equilibrium of its node's moments, f + (f_eq - f)/tau,
    then followed to its end point x + V + c' of its own slot's c' and split
    with cloud-in-cell weights into the same slot of the nodes around it; a
    packet that leaves through a reflecting wall bounces (normal momentum
    negated, slot mirrored)."""
    tau = F(tau)
    nodes = list(state.keys())
    NP = len(velocity_set(dim, 1))

    def moments(slots_):
        rho = sum(s[0] for s in slots_)
        m = tuple(sum(s[1][a] for s in slots_) for a in range(dim))
        return rho, m, sum(s[2] for s in slots_)

    reach = 0
    for nd in nodes:
        rho, m, rhoE = moments(state[nd])
        if rho == 0:
            continue
        V, c1, _, _ = equilibrium(dim, gamma, theta, rho, m, rhoE)
        reach = max(reach, max(abs(math.floor(v)) + 2 for v in V) + c1 + 1)
    ranges = []
    for a in range(dim):
        lo, hi = (-reach, shape[a] + reach) if bcs[a] == TRANSMISSIVE else (0, shape[a])
        ranges.append(range(lo, hi))
    acc = {nd: [[F(0), [F(0)] * dim, F(0)] for _ in range(NP)] for nd in nodes}

    def sources():
        if dim == 1:
            for x in ranges[0]:
                yield (x,)
        else:
            for y in ranges[1]:
                for x in ranges[0]:
                    yield (x, y)

    for s in sources():
        g = tuple(min(max(s[a], 0), shape[a] - 1) for a in range(dim))
        slots_ = state[g]
        rho, m, rhoE = moments(slots_)
        if rho == 0:
            continue
        V, c1, _, _ = equilibrium(dim, gamma, theta, rho, m, rhoE)
        feq = equilibrium_slots(dim, gamma, theta, rho, m, rhoE)
        for j, (cv, lev) in enumerate(velocity_set(dim, c1)):
            f0, f1, f2 = slots_[j]
            e0, e1, e2 = feq[j]
            mass = f0 + (e0 - f0) / tau
            mom = [f1[a] + (e1[a] - f1[a]) / tau for a in range(dim)]
            en = f2 + (e2 - f2) / tau
            end = [s[a] + V[a] + cv[a] for a in range(dim)]
            base = [math.floor(x) for x in end]
            frac = [end[a] - base[a] for a in range(dim)]
            for corner in range(1 << dim):
                w = F(1)
                L = []
                for a in range(dim):
                    k = (corner >> a) & 1
                    w *= frac[a] if k else 1 - frac[a]
                    L.append(base[a] + k)
                idx, sgn = [], []
                for a in range(dim):
                    r = _map(bcs[a], shape[a], L[a])
                    if r is None:
                        break
                    idx.append(r[0])
                    sgn.append(r[1])
                else:
                    jj = j
                    for a in range(dim):
                        if sgn[a] < 0:
                            jj = mirror_slot(dim, a, jj)
                    t = acc[tuple(idx)][jj]
                    t[0] += w * mass
                    for a in range(dim):
                        t[1][a] += w * mom[a] * sgn[a]
                    t[2] += w * en
    return {nd: [(v[0], tuple(v[1]), v[2]) for v in acc[nd]] for nd in nodes}
