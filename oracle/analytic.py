"""Closed-form potentials used to pin the oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).  Every function returns
Phi (negative, -G * integral of rho / |r - r'|) in FP64.

* Uniform sphere: the textbook interior/exterior potential.
* Maclaurin spheroid (Sec. 4.1, Eqs. 6-12).  Two printed typos are corrected
  here; both corrections are forced by the mathematics and pinned by tests
  (Laplacian, continuity at the surface, sphere limit, far field):
    - interior: the A_3 term enters with a plus sign,
          V = pi G rho [2 A1 a1^2 - A1 (x^2 + y^2) + A3 (a3^2 - z^2)],
      (with the printed minus sign, V is not the potential of the body: the
      e -> 0 limit misses the sphere's 2 pi G rho (a^2 - r^2/3));
    - exterior: the factor in front of the round bracket is 1/(2 a1 e), not
      1/2 (the printed form is not even dimensionally consistent).
  The paper writes Phi for V = -Phi >= 0; here Phi = -V.
* Uniform rectangular prism: the classical closed form of the integral of
  1/r over a box (sum over the 8 corners of
  xy ln(z+r) + yz ln(x+r) + zx ln(y+r) - x^2/2 atan(yz/(xr)) - ...).
"""
from __future__ import annotations

import numpy as np


def uniform_sphere(x, y, z, centre, radius, rho, G=1.0):
    r = np.sqrt((x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2)
    M = 4.0 / 3.0 * np.pi * radius ** 3 * rho
    inside = -2.0 * np.pi * G * rho * (radius ** 2 - r ** 2 / 3.0)
    with np.errstate(divide="ignore"):
        outside = -G * M / r
    return np.where(r <= radius, inside, outside)


def maclaurin_coefficients(e: float):
    """A1 (= A2) and A3 of an oblate spheroid of eccentricity e (Sec. 4.1)."""
    s = np.sqrt(1.0 - e * e)
    A1 = s / e ** 3 * np.arcsin(e) - (1.0 - e * e) / e ** 2
    A3 = 2.0 / e ** 2 - 2.0 * s / e ** 3 * np.arcsin(e)
    return A1, A3


def maclaurin(x, y, z, centre, a1, e, rho, G=1.0):
    """Potential of a homogeneous oblate spheroid a1 = a2 > a3 = a1 sqrt(1-e^2)."""
    a3 = a1 * np.sqrt(1.0 - e * e)
    X = np.asarray(x, dtype=np.float64) - centre[0]
    Y = np.asarray(y, dtype=np.float64) - centre[1]
    Z = np.asarray(z, dtype=np.float64) - centre[2]
    R2 = X * X + Y * Y
    Z2 = Z * Z
    A1, A3 = maclaurin_coefficients(e)
    v_in = np.pi * G * rho * (2.0 * A1 * a1 ** 2 - A1 * R2 + A3 * (a3 ** 2 - Z2))
    # lambda: positive root of R2/(a1^2+l) + Z2/(a3^2+l) = 1
    b = a1 ** 2 + a3 ** 2 - R2 - Z2
    c = a1 ** 2 * a3 ** 2 - R2 * a3 ** 2 - Z2 * a1 ** 2
    lam = np.maximum(0.5 * (-b + np.sqrt(np.maximum(b * b - 4.0 * c, 0.0))), 0.0)
    h = a1 * e / np.sqrt(a3 ** 2 + lam)
    at = np.arctan(h)
    v_out = (2.0 * a3 / e ** 2) * np.pi * G * rho * (
        a1 * e * at - (1.0 / (2.0 * a1 * e)) * (
            R2 * (at - h / (1.0 + h * h)) + 2.0 * Z2 * (h - at)))
    inside = R2 / a1 ** 2 + Z2 / a3 ** 2 <= 1.0
    return -np.where(inside, v_in, v_out)


def _prism_F(x, y, z):
    r = np.sqrt(x * x + y * y + z * z)
    with np.errstate(divide="ignore", invalid="ignore"):
        def xlog(c, a):                     # c * ln(a + r), zero when c == 0
            return np.where(c == 0.0, 0.0, c * np.log(np.where(c == 0.0, 1.0, a + r)))

        def xatan(a, b, c):                 # a^2/2 * atan(bc/(a r)), zero when a == 0
            safe = np.where(a == 0.0, 1.0, a * r)
            return np.where(a == 0.0, 0.0, 0.5 * a * a * np.arctan(b * c / safe))
        return (xlog(x * y, z) + xlog(y * z, x) + xlog(z * x, y)
                - xatan(x, y, z) - xatan(y, z, x) - xatan(z, x, y))


def prism(x, y, z, lo, hi, rho, G=1.0):
    """Potential of the uniform box [lo, hi] (per axis) at points (x, y, z)."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    total = 0.0
    for i, (ax, sx) in enumerate(((lo[0], -1.0), (hi[0], 1.0))):
        for j, (ay, sy) in enumerate(((lo[1], -1.0), (hi[1], 1.0))):
            for k, (az, sz) in enumerate(((lo[2], -1.0), (hi[2], 1.0))):
                total = total + sx * sy * sz * _prism_F(ax - x, ay - y, az - z)
    return -G * rho * total


def cube_centre_factor() -> float:
    """Integral of 1/r over the unit cube seen from its centre (~2.3800772)."""
    return float(-prism(0.0, 0.0, 0.0, (-0.5,) * 3, (0.5,) * 3, 1.0))


def sphere_in_box(x, y, z, centre, radius, rho_in, rho_out, box_lo=(0, 0, 0), box_len=1.0,
                  G=1.0):
    """A uniform sphere of density rho_in inside a box filled with rho_out."""
    hi = tuple(b + box_len for b in box_lo)
    return (uniform_sphere(x, y, z, centre, radius, rho_in - rho_out, G)
            + prism(x, y, z, box_lo, hi, rho_out, G))


def maclaurin_in_box(x, y, z, centre, a1, e, rho_in, rho_out, box_lo=(0, 0, 0),
                     box_len=1.0, G=1.0):
    hi = tuple(b + box_len for b in box_lo)
    return (maclaurin(x, y, z, centre, a1, e, rho_in - rho_out, G)
            + prism(x, y, z, box_lo, hi, rho_out, G))
