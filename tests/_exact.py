"""Closed-form elasticity solutions used to validate the solver as Sec. 3.1 does
(a plate with a circular hole): Kirsch's uniaxial-tension field and Lame's
pressurised hole, both for an infinite plate in plane strain, and the
pressurised spherical cavity in 3D.  Test infrastructure: the displacements were
derived from the textbook stress fields by integrating the plane-strain strains
(tests/test_exact_solutions.py checks them against those stresses and the
equilibrium and boundary conditions).

All functions take Cartesian coordinates relative to the hole's centre and
return Cartesian components.
"""
import numpy as np


def lame_moduli(E, nu):
    return E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))


def _polar_to_xy(fr, ft, th):
    c, s = np.cos(th), np.sin(th)
    return fr * c - ft * s, fr * s + ft * c


def _polar_tensor_to_xy(srr, stt, srt, th):
    c, s = np.cos(th), np.sin(th)
    sxx = srr * c * c + stt * s * s - 2 * srt * s * c
    syy = srr * s * s + stt * c * c + 2 * srt * s * c
    sxy = (srr - stt) * s * c + srt * (c * c - s * s)
    return sxx, syy, sxy


def kirsch_stress(x, y, a, S):
    """Remote sigma_xx = S, traction-free hole of radius a (Kirsch)."""
    r, th = np.hypot(x, y), np.arctan2(y, x)
    q2, q4 = (a / r) ** 2, (a / r) ** 4
    c2, s2 = np.cos(2 * th), np.sin(2 * th)
    srr = S / 2 * (1 - q2) + S / 2 * (1 - 4 * q2 + 3 * q4) * c2
    stt = S / 2 * (1 + q2) - S / 2 * (1 + 3 * q4) * c2
    srt = -S / 2 * (1 + 2 * q2 - 3 * q4) * s2
    return _polar_tensor_to_xy(srr, stt, srt, th)


def kirsch_displacement(x, y, a, S, E, nu):
    """Plane-strain displacement of the Kirsch field (no rigid motion; symmetric
    about both axes)."""
    _, mu = lame_moduli(E, nu)
    r, th = np.hypot(x, y), np.arctan2(y, x)
    k = S / (4 * mu)
    ur = k * (r * (1 - 2 * nu) + a * a / r + (r + 4 * (1 - nu) * a * a / r - a ** 4 / r ** 3) * np.cos(2 * th))
    ut = -k * (r + 2 * (1 - 2 * nu) * a * a / r + a ** 4 / r ** 3) * np.sin(2 * th)
    return _polar_to_xy(ur, ut, th)


def lame_hole_stress(x, y, a, p):
    """Pressure p in a hole of radius a in an infinite plate, no remote load."""
    r, th = np.hypot(x, y), np.arctan2(y, x)
    q = (a / r) ** 2
    return _polar_tensor_to_xy(-p * q, p * q, 0.0 * r, th)


def lame_hole_displacement(x, y, a, p, E, nu):
    _, mu = lame_moduli(E, nu)
    r, th = np.hypot(x, y), np.arctan2(y, x)
    return _polar_to_xy(p * a * a / (2 * mu * r), 0.0 * r, th)


def cavity_displacement(x, y, z, a, p, E, nu):
    """Pressure p in a spherical cavity of radius a in an infinite solid:
    u_r = p a^3 / (4 mu r^2), sigma_rr = -p a^3 / r^3, sigma_tt = p a^3 / (2 r^3)."""
    _, mu = lame_moduli(E, nu)
    r = np.sqrt(x * x + y * y + z * z)
    ur = p * a ** 3 / (4 * mu * r ** 2)
    return ur * x / r, ur * y / r, ur * z / r


def plane_strain_stress(exx, eyy, exy, E, nu):
    lam, mu = lame_moduli(E, nu)
    tr = exx + eyy
    return lam * tr + 2 * mu * exx, lam * tr + 2 * mu * eyy, 2 * mu * exy
