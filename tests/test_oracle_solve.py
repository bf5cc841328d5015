"""Pins of the oracle's full solve against physics (Sec. 6 accuracy protocol and
textbook scattering identities):

  * Mie series for a sound-soft sphere (far field and near field);
  * Green's identity: boundary data from interior point sources reproduces their
    exterior field (the paper's E_inf^rel test);
  * reciprocity u_inf(x^; d) = u_inf(-d; -x^);
  * optical theorem  int |u_inf|^2 = (4 pi / k) Im u_inf(d; d)  (sound-soft);
  * GMRES against a dense LU solve of the full Nystrom system.
"""
import numpy as np

import workloads as W
from oracle import Problem, dense_solve, fields, gauss_legendre, gmres


def _solve_plane(P, d, tol=1e-13):
    v = fields.plane_wave(P.nodes.x, np.atleast_2d(d), P.k)[:, 0]
    res = gmres(P.apply, P.rhs(v), tol)
    assert res.converged
    return res.x


def test_mie_sound_soft_sphere():
    a, k = 1.0, 2.0
    sh = W.ShapeSpec(W.SPHERE, (a,), 8, 10, 25)
    wl = W.Workload("sphere", [W.Body(sh, np.zeros(3), np.eye(3))], k, k, np.array([[0, 0, 1.0]]))
    P = Problem(wl)
    sig = _solve_plane(P, [0, 0, 1.0])
    xh = W.uniform_directions(16, 3)
    uinf = fields.far_field(P.nodes, sig, k, k, xh)
    mie = fields.mie_far_field(a, k, xh[:, 2])
    assert np.abs(uinf - mie).max() < 1e-11 * np.abs(mie).max()
    # near field: the smooth surface rule is evaluated 3 radii out
    pts = 4.0 * W.uniform_directions(8, 4)
    u = fields.field(P.nodes, sig, k, k, pts)
    ref = fields.mie_scattered(a, k, np.linalg.norm(pts, axis=1), pts[:, 2] / 4.0)
    assert np.abs(u - ref).max() < 1e-10 * np.abs(ref).max()


def _green_error(wl, seed=5):
    P = Problem(wl)
    src = W.point_sources(wl, seed)
    tg = W.exterior_targets(wl, 10, seed + 1)
    v = -fields.point_source_field(P.nodes.x, src, wl.k)
    res = gmres(P.apply, P.rhs(v), 1e-13)
    assert res.converged
    u = fields.field(P.nodes, res.x, wl.k, wl.eta, tg)
    ue = fields.point_source_field(tg, src, wl.k)
    return np.abs(u - ue).max() / np.abs(ue).max()


def test_green_identity_two_spheres():
    assert _green_error(W.two_spheres(n_panels=6, gl_order=10, n_modes=25)) < 1e-10


def test_green_identity_spheroid():
    sph = W.ShapeSpec(W.SPHEROID, (1.0, 2.0), 10, 10, 25)
    bodies = [W.Body(sph, np.array([-1.8, 0.2, 0.0]), W.rotation_taking_z_to([0.3, 1.0, 0.2])),
              W.Body(sph, np.array([1.9, -0.1, 0.3]), W.rotation_taking_z_to([-1.0, 0.2, 0.4]))]
    wl = W.Workload("pair", bodies, 2.0, 2.0, np.array([[0, 0, 1.0]]))
    assert _green_error(wl) < 1e-8


def test_green_identity_open_shell_converges_in_azimuth():
    """An open shell's interior source lies in its 0.2-thick wall, 0.1 from the
    surface, so the boundary data is sharply peaked and the error is set by the
    azimuthal resolution: it must fall by more than 10x from N_F = 21 to 41."""
    errs = []
    for nf in (21, 41):
        shell = W.ShapeSpec(W.OPEN_SHELL, (1.0, 0.8, np.pi / 3, 0.1), 12, 10, nf)
        wl = W.Workload("shell", [W.Body(shell, np.zeros(3), W.rotation_taking_z_to([-1.0, 0.2, 0.4]))],
                        2.0, 2.0, np.array([[0, 0, 1.0]]))
        errs.append(_green_error(wl))
    assert errs[1] < 2e-3 and errs[1] < errs[0] / 10


def test_open_shell_optical_theorem_and_reciprocity():
    """Plane-wave scattering by a spheroid and an open shell (cavity with rim)."""
    sph = W.ShapeSpec(W.SPHEROID, (1.0, 2.0), 8, 8, 17)
    shell = W.ShapeSpec(W.OPEN_SHELL, (1.0, 0.8, np.pi / 3, 0.1), 12, 8, 17)
    bodies = [W.Body(sph, np.array([-1.8, 0.2, 0.0]), W.rotation_taking_z_to([0.3, 1.0, 0.2])),
              W.Body(shell, np.array([1.6, -0.1, 0.3]), W.rotation_taking_z_to([-1.0, 0.2, 0.4]))]
    wl = W.Workload("pair", bodies, 1.5, 1.5, np.array([[0, 0, 1.0]]))
    _reciprocity_and_optical(wl, 1e-6)


def test_reciprocity_and_optical_theorem():
    _reciprocity_and_optical(W.two_spheres(n_panels=6, gl_order=8, n_modes=21, k=1.5), 1e-9)


def _reciprocity_and_optical(wl, tol):
    P = Problem(wl)
    k = wl.k
    d = np.array([0.3, -0.5, 0.81]); d /= np.linalg.norm(d)
    xh = np.array([-0.6, 0.2, 0.77]); xh /= np.linalg.norm(xh)
    s_d = _solve_plane(P, d)
    s_mx = _solve_plane(P, -xh)
    u1 = fields.far_field(P.nodes, s_d, k, k, xh[None])[0]
    u2 = fields.far_field(P.nodes, s_mx, k, k, -d[None])[0]
    assert abs(u1 - u2) < tol * abs(u1)
    # optical theorem with a Gauss-Legendre x trapezoid rule on the unit sphere
    x, w = gauss_legendre(40)
    nph = 80
    ph = 2 * np.pi * np.arange(nph) / nph
    st = np.sqrt(1 - x * x)
    dirs = np.stack([st[:, None] * np.cos(ph)[None], st[:, None] * np.sin(ph)[None],
                     np.broadcast_to(x[:, None], (40, nph))], -1).reshape(-1, 3)
    wts = np.repeat(w, nph) * (2 * np.pi / nph)
    uinf = fields.far_field(P.nodes, s_d, k, k, dirs)
    lhs = (wts * np.abs(uinf) ** 2).sum()
    rhs = 4 * np.pi / k * fields.far_field(P.nodes, s_d, k, k, d[None])[0].imag
    assert abs(lhs - rhs) < tol * abs(rhs)


def test_gmres_matches_dense_solve():
    wl = W.tiny_two_spheres()
    P = Problem(wl)
    v = fields.plane_wave(P.nodes.x, wl.directions, wl.k)[:, 0]
    sig_dense = dense_solve(P.dense_matrix(), v)
    res = gmres(P.apply, P.rhs(v), 1e-14)
    assert np.linalg.norm(res.x - sig_dense) < 1e-12 * np.linalg.norm(sig_dense)
    # restarted GMRES reaches the same solution
    res2 = gmres(P.apply, P.rhs(v), 1e-14, restart=3, maxit=200)
    assert res2.converged
    assert np.linalg.norm(res2.x - sig_dense) < 1e-12 * np.linalg.norm(sig_dense)
