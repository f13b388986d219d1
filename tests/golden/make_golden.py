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


def main():
    here = os.path.dirname(os.path.abspath(__file__))
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
