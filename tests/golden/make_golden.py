"""Write the stored expected values under tests/golden/ from the oracle only.

two_spheres_8200_farfield.txt: far-field pattern u_inf(x^) of the two-sphere
workload (unit spheres at (+-1.5, 0, 0), k = eta = 2, 10 panels x 10 Gauss-Legendre
nodes, 41 azimuthal nodes; plane wave along +z), solved by the oracle's GMRES to a
relative residual of 1e-13, at 8 seeded unit directions.  Columns: x, y, z,
Re u_inf, Im u_inf.

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import Problem, fields, gmres  # noqa: E402

FF_SEED = 812


def main():
    wl = W.two_spheres()
    P = Problem(wl)
    v = fields.plane_wave(P.nodes.x, wl.directions, wl.k)[:, 0]
    res = gmres(P.apply, P.rhs(v), 1e-13)
    assert res.converged
    xh = W.uniform_directions(8, FF_SEED)
    u = fields.far_field(P.nodes, res.x, wl.k, wl.eta, xh)
    out = np.column_stack([xh, u.real, u.imag])
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "two_spheres_8200_farfield.txt")
    np.savetxt(path, out, fmt="%.17e",
               header="oracle far field, two_spheres_8200, plane wave +z, GMRES tol 1e-13 "
                      "(%d iterations); x y z Re Im" % res.iterations)


if __name__ == "__main__":
    main()
