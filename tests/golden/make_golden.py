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


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                       "sod_l1_errors.txt")
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


if __name__ == "__main__":
    main()
