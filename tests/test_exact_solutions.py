"""Checks of the closed-form solutions in tests/_exact.py, which the GPU validation
of Sec. 3.1 (plate with a hole) compares against: each displacement field, put
through plane-strain (3D: isotropic) Hooke's law by central differences, gives the
textbook stresses; those stresses are in equilibrium, traction free (or loaded by
the pressure) on the hole and tend to the remote load far away."""
import numpy as np

import _exact as X

E, NU = 1.0, 0.3


def _strain2(fun, x, y, d=1e-5):
    ux1, uy1 = fun(x + d, y)
    ux0, uy0 = fun(x - d, y)
    vx1, vy1 = fun(x, y + d)
    vx0, vy0 = fun(x, y - d)
    exx = (ux1 - ux0) / (2 * d)
    eyy = (vy1 - vy0) / (2 * d)
    exy = 0.5 * ((vx1 - vx0) / (2 * d) + (uy1 - uy0) / (2 * d))
    return exx, eyy, exy


def _points(rng, a, n=400):
    r = a * (1.0 + 4.0 * rng.random(n))
    th = 2 * np.pi * rng.random(n)
    return r * np.cos(th), r * np.sin(th)


def test_kirsch_displacement_gives_kirsch_stress():
    rng = np.random.default_rng(1)
    a, S = 1.0, 0.7
    x, y = _points(rng, a)
    got = X.plane_strain_stress(*_strain2(lambda x, y: X.kirsch_displacement(x, y, a, S, E, NU), x, y), E, NU)
    ref = X.kirsch_stress(x, y, a, S)
    for g, r in zip(got, ref):
        assert np.abs(g - r).max() <= 1e-7 * S


def test_kirsch_stress_is_traction_free_on_the_hole_and_uniaxial_far_away():
    a, S = 1.3, 2.0
    th = np.linspace(0, 2 * np.pi, 73)
    x, y = a * np.cos(th), a * np.sin(th)
    sxx, syy, sxy = X.kirsch_stress(x, y, a, S)
    tx = sxx * np.cos(th) + sxy * np.sin(th)
    ty = sxy * np.cos(th) + syy * np.sin(th)
    assert np.abs(tx).max() < 1e-12 and np.abs(ty).max() < 1e-12
    # the stress concentration 3 S at the top of the hole
    assert np.isclose(X.kirsch_stress(0.0, a, a, S)[0], 3 * S)
    far = X.kirsch_stress(np.array([1e4 * a]), np.array([3e3 * a]), a, S)
    assert np.allclose([far[0][0], far[1][0], far[2][0]], [S, 0, 0], atol=1e-6 * S)


def test_kirsch_stress_is_in_equilibrium():
    rng = np.random.default_rng(2)
    a, S, d = 1.0, 1.0, 1e-5
    x, y = _points(rng, a)
    sx = lambda x, y: X.kirsch_stress(x, y, a, S)
    dsxx = (sx(x + d, y)[0] - sx(x - d, y)[0]) / (2 * d)
    dsxy_y = (sx(x, y + d)[2] - sx(x, y - d)[2]) / (2 * d)
    dsxy_x = (sx(x + d, y)[2] - sx(x - d, y)[2]) / (2 * d)
    dsyy = (sx(x, y + d)[1] - sx(x, y - d)[1]) / (2 * d)
    assert np.abs(dsxx + dsxy_y).max() < 1e-6
    assert np.abs(dsxy_x + dsyy).max() < 1e-6


def test_lame_hole_displacement_gives_the_pressure_field():
    rng = np.random.default_rng(3)
    a, p = 1.0, 0.4
    x, y = _points(rng, a)
    got = X.plane_strain_stress(*_strain2(lambda x, y: X.lame_hole_displacement(x, y, a, p, E, NU), x, y), E, NU)
    ref = X.lame_hole_stress(x, y, a, p)
    for g, r in zip(got, ref):
        assert np.abs(g - r).max() <= 1e-7 * p
    # sigma_rr = -p on the hole
    sxx, syy, sxy = X.lame_hole_stress(np.array([a]), np.array([0.0]), a, p)
    assert np.isclose(sxx[0], -p) and np.isclose(syy[0], p)


def test_cavity_displacement_gives_the_pressure_field():
    rng = np.random.default_rng(4)
    a, p, d = 1.0, 0.5, 1e-5
    lam, mu = X.lame_moduli(E, NU)
    n = 200
    r = a * (1 + 3 * rng.random(n))
    v = rng.normal(size=(3, n))
    v /= np.linalg.norm(v, axis=0)
    P = r * v
    G = np.zeros((3, 3, n))
    for j in range(3):
        e = np.zeros((3, 1))
        e[j] = d
        up = np.array(X.cavity_displacement(*(P + e), a, p, E, NU))
        um = np.array(X.cavity_displacement(*(P - e), a, p, E, NU))
        G[:, j] = (up - um) / (2 * d)
    eps = 0.5 * (G + G.transpose(1, 0, 2))
    sig = lam * np.einsum("iin->n", eps)[None, None] * np.eye(3)[:, :, None] + 2 * mu * eps
    srr = np.einsum("in,ijn,jn->n", v, sig, v)
    assert np.allclose(srr, -p * (a / r) ** 3, atol=1e-7)
    assert np.allclose(np.einsum("iin->n", sig), 0.0, atol=1e-7)      # trace-free: s_tt = -s_rr / 2
