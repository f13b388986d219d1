"""Writes the stored expected values that come from the oracle alone.

Run from the repository root:  python tests/golden/make_golden.py
It calls only oracle/ (the FP64 CPU oracle and the exact Riemann solver).
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O, riemann as Rm  # noqa: E402

SOD_L = (1.0, 0.0, 1.0)
SOD_R = (0.125, 0.0, 0.1)


def sod_l1(N, t_end=0.2):
    P = O.Params(dim=1, nx=N, bc_x=O.TRANSMISSIVE)
    n, lam = O.steps_and_lambda(t_end, 1.0 / N)
    s, _ = O.run(P, O.riemann_planar(P, 0, 1, 0.5, SOD_L, SOD_R, lam), n)
    ph = O.lattice_to_physical(1.4, lam, s)
    x = O.node_x(N, 0, 1)
    return Rm.l1_errors(x, t_end, 0.5, SOD_L, SOD_R, ph["rho"], ph["u"],
                        ph["p"])


# A second Riemann problem with a moving left state (Toro's test 1: the
# left state of Sod's problem moving at u = 0.75, diaphragm at x = 0.3), so
# that the conversion of velocities into lattice units is exercised too.
TORO1_L = (1.0, 0.75, 1.0)
TORO1_R = (0.125, 0.0, 0.1)
LAMBDA_CASES = {"sod": (SOD_L, SOD_R, 0.5), "toro1": (TORO1_L, TORO1_R, 0.3)}


def riemann_l1_at_lambda(case, N, lam, t_end=0.2):
    """L1 error against the exact solution of a 1-D tube run with a given
    lambda = dt/dx (t_end / (lambda dx) must be a whole number of steps)."""
    left, right, x_d = LAMBDA_CASES[case]
    P = O.Params(dim=1, nx=N, bc_x=O.TRANSMISSIVE)
    dx = 1.0 / N
    n = int(round(t_end / (lam * dx)))
    if abs(n * lam * dx - t_end) > 1e-12:
        raise ValueError("t_end is not a whole number of steps")
    s, _ = O.run(P, O.riemann_planar(P, 0, 1, x_d, left, right, lam), n)
    ph = O.lattice_to_physical(1.4, lam, s)
    x = O.node_x(N, 0, 1)
    return Rm.l1_errors(x, t_end, x_d, left, right, ph["rho"], ph["u"],
                        ph["p"])


CYL_IN = (1.0, 0.0, 0.0, 1.0)
CYL_OUT = (0.125, 0.0, 0.0, 0.1)


def _as_fp32(st):
    f = lambda a: a.astype("float32").astype("float64")
    return O.State(f(st.rho), f(st.mx), f(st.my), f(st.rhoE))


def cylinder_fp32_floor(n=64, checkpoints=(50, 100, 200, 400, 800)):
    """The periodic cylinder (radius 0.4, Section V.C states) on an n x n
    lattice, run twice by the oracle: in FP64, and in FP64 with the state
    rounded to FP32 after every step.  Returns per checkpoint the mean
    |difference| / range of the FP64 field, and the FP64 run's largest
    departure from the x <-> y mirror symmetry of the problem."""
    import numpy as np
    P = O.Params(dim=2, nx=n, ny=n, bc_x=O.PERIODIC, bc_y=O.PERIODIC)
    a = O.riemann_circle(P, 0, 1, 0, 0.5, 0.5, 0.4, CYL_IN, CYL_OUT, 1.0)
    b = _as_fp32(a)
    rows = []
    for k in range(1, max(checkpoints) + 1):
        a, _, _ = O.step(P, a)
        b = _as_fp32(O.step(P, b)[0])
        if k in checkpoints:
            l1 = []
            for f in ("rho", "mx", "my", "rhoE"):
                x, y = getattr(a, f), getattr(b, f)
                l1.append(float(np.mean(np.abs(x - y)) / (x.max() - x.min())))
            r = a.rho.reshape(n, n)
            rows.append((k, l1, float(np.max(np.abs(r - r.T)))))
    return rows


def write_cylinder_floor(path):
    rows = cylinder_fp32_floor()
    with open(path, "w") as f:
        f.write("# The periodic cylinder (radius 0.4 about the centre, inside (1, 1),\n"
                "# outside (0.125, 0.1), lambda = 1) on a 64 x 64 lattice: the FP64\n"
                "# oracle against the same oracle with its state rounded to FP32 after\n"
                "# every step.  mean |difference| / (max - min) of the FP64 field, and\n"
                "# the FP64 run's largest |rho(x, y) - rho(y, x)|.  The square-lattice\n"
                "# step amplifies round-off, so no FP32 arithmetic can stay within\n"
                "# 1e-5 of FP64 here beyond about 200 steps.  Written by\n"
                "# tests/golden/make_golden.py from oracle/ only.\n"
                "# columns: step rho mx my rhoE fp64_mirror_asymmetry\n")
        for k, l1, sym in rows:
            f.write(f"{k} " + " ".join(f"{v:.6e}" for v in l1) + f" {sym:.6e}\n")


def cylinder_state_hashes(n=128, steps=2000):
    """SHA-256 of the bytes (little-endian FP64) of each lattice-unit field
    of the periodic cylinder on an n x n lattice after `steps` oracle steps;
    the GPU's FP64 path must reproduce them bit for bit."""
    import hashlib
    import numpy as np
    P = O.Params(dim=2, nx=n, ny=n, bc_x=O.PERIODIC, bc_y=O.PERIODIC)
    s = O.riemann_circle(P, 0, 1, 0, 0.5, 0.5, 0.4, CYL_IN, CYL_OUT, 1.0)
    s, _ = O.run(P, s, steps)
    return {f: hashlib.sha256(np.ascontiguousarray(getattr(s, f), "<f8")
                              .tobytes()).hexdigest()
            for f in ("rho", "mx", "my", "rhoE")}


def write_cylinder_hashes(path, n=128, steps=2000):
    h = cylinder_state_hashes(n, steps)
    with open(path, "w") as f:
        f.write("# SHA-256 of each field (lattice units, little-endian FP64, x fastest)\n"
                f"# of the periodic cylinder on a {n} x {n} lattice after {steps} FP64\n"
                "# oracle steps (radius 0.4 about the centre, inside (1, 1), outside\n"
                "# (0.125, 0.1), lambda = 1).  Written by tests/golden/make_golden.py\n"
                "# from oracle/ only.  columns: n steps field sha256\n")
        for k in ("rho", "mx", "my", "rhoE"):
            f.write(f"{n} {steps} {k} {h[k]}\n")


def sod2d_row(nx=4096, t_end=0.2):
    """One row of the 2-D square-lattice Sod tube between reflecting walls
    (x-only data: every row of the 4096 x 512 tube is this row), physical
    units, after the whole solve."""
    P = O.Params(dim=2, nx=nx, ny=1, bc_x=O.TRANSMISSIVE, bc_y=O.REFLECTING)
    n, lam = O.steps_and_lambda(t_end, 1.0 / nx)
    s, _ = O.run(P, O.riemann_planar(P, 0, 1, 0.5, SOD_L, SOD_R, lam), n)
    return n, lam, O.lattice_to_physical(1.4, lam, s)


def write_sod2d_row(path):
    n, lam, ph = sod2d_row()
    with open(path, "w") as f:
        f.write("# One row of the 4096 x 512 square-lattice Sod tube (Section V.C;\n"
                "# transmissive x ends, reflecting y walls, x-only initial jump at\n"
                "# x = 0.5), FP64 oracle, after %d steps to t = 0.2 (lambda = %.17g).\n"
                "# Physical units.  Written by tests/golden/make_golden.py from\n"
                "# oracle/ only.  columns: rho m_x rhoE\n" % (n, lam))
        for r, m, e in zip(ph["rho"], ph["mx"], ph["rhoE"]):
            f.write(f"{float(r)!r} {float(m)!r} {float(e)!r}\n")


BGK_TAUS = (0.8, 1.5, 3.0)
BGK_NS = (200, 400, 800)


def bgk_sod_l1(tau, N, t_end=0.2):
    """L1 error against the exact solution of the 1-D Sod tube run with the
    relaxation-time step (eqs 4-5) from equilibrium."""
    P = O.Params(dim=1, nx=N, bc_x=O.TRANSMISSIVE)
    n, lam = O.steps_and_lambda(t_end, 1.0 / N)
    s = O.riemann_planar(P, 0, 1, 0.5, SOD_L, SOD_R, lam)
    f, _ = O.bgk_run(P, tau, O.bgk_equilibrium(P, s), n)
    ph = O.lattice_to_physical(1.4, lam, O.bgk_moments(P, f))
    x = O.node_x(N, 0, 1)
    return Rm.l1_errors(x, t_end, 0.5, SOD_L, SOD_R, ph["rho"], ph["u"],
                        ph["p"])


def write_bgk_sod_l1(path):
    with open(path, "w") as f:
        f.write("# L1 (mean absolute) error of the 1-D Sod tube run with the\n"
                "# relaxation-time step (eqs 4-5, per-packet state) from\n"
                "# equilibrium, against the exact Riemann solution at t = 0.2\n"
                "# (Section V.C-D), theta = 0.5, lambda from n = ceil(t/dx),\n"
                "# transmissive ends.  Written by tests/golden/make_golden.py\n"
                "# from oracle/ only.  columns: tau N rho u p\n")
        for tau in BGK_TAUS:
            for N in BGK_NS:
                e = bgk_sod_l1(tau, N)
                f.write(f"{tau} {N} {e['rho']:.6e} {e['u']:.6e} {e['p']:.6e}\n")


def main():
    here = os.path.dirname(os.path.abspath(__file__))
    write_bgk_sod_l1(os.path.join(here, "bgk_sod_l1_errors.txt"))
    write_cylinder_floor(os.path.join(here, "cylinder_fp32_storage_floor.txt"))
    write_cylinder_hashes(os.path.join(here, "cylinder128_fp64_2000_sha256.txt"))
    write_sod2d_row(os.path.join(here, "sod2d_row_4096_t0.2.txt"))
    out = os.path.join(here, "sod_l1_errors.txt")
    with open(out, "w") as f:
        f.write("# L1 (mean absolute) error of the 1-D lattice Boltzmann Sod tube\n"
                "# against the exact Riemann solution at t = 0.2 (Section V.C-D),\n"
                "# theta = 0.5, lambda from n = ceil(t/dx), transmissive ends.\n"
                "# Written by tests/golden/make_golden.py from oracle/ only.\n"
                "# columns: N rho u p\n")
        for N in (400, 1000, 4000):
            e = sod_l1(N)
            f.write(f"{N} {e['rho']:.6e} {e['u']:.6e} {e['p']:.6e}\n")
    print(open(out).read())
    out = os.path.join(here, "riemann_l1_lambda_half.txt")
    with open(out, "w") as f:
        f.write("# L1 (mean absolute) error of 1-D lattice Boltzmann tubes run with\n"
                "# lambda = dt/dx = 0.5 against the exact Riemann solution at t = 0.2\n"
                "# (Section V.C-D), theta = 0.5, transmissive ends.  sod: Sod's states,\n"
                "# diaphragm at 0.5; toro1: left (1, 0.75, 1), right (0.125, 0, 0.1),\n"
                "# diaphragm at 0.3.  Written by tests/golden/make_golden.py from\n"
                "# oracle/ only.  columns: case N rho u p\n")
        for case in ("sod", "toro1"):
            for N in (400, 1000):
                e = riemann_l1_at_lambda(case, N, 0.5)
                f.write(f"{case} {N} {e['rho']:.6e} {e['u']:.6e} {e['p']:.6e}\n")
    print(open(out).read())


if __name__ == "__main__":
    main()
