"""Closed-form mid-plane radial forces of the analytic test disks (FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

* D_2 disk (Section 3, after Schulz 2009, Eq. 30 there): surface density
  sigma0 (1 - R^2/alpha^2)^{3/2} inside R < alpha, radial force
      R <= alpha: -(3 pi^2 sigma0 G R / (16 alpha^3)) (4 alpha^2 - 3 R^2)
      R >  alpha: -(3 pi sigma0 G / (8 alpha^3)) [R (4 alpha^2 - 3 R^2) asin(alpha/R)
                                                    - alpha (2 alpha^2 - 3 R^2) sqrt(1 - alpha^2/R^2)]
* Kuzmin disk (not in the paper; the classic potential-density pair): surface
  density a M / (2 pi (R^2 + a^2)^{3/2}), mid-plane radial force
  -G M R / (R^2 + a^2)^{3/2}.

Both forces are negative (towards the centre).
"""
import numpy as np


def d2_radial_force(R, alpha, sigma0=1.0, G=1.0):
    R = np.asarray(R, dtype=np.float64)
    out = np.empty_like(R)
    inside = R <= alpha
    Ri = R[inside]
    out[inside] = -(3.0 * np.pi ** 2 * sigma0 * G * Ri / (16.0 * alpha ** 3)) * (4.0 * alpha ** 2 - 3.0 * Ri ** 2)
    Ro = R[~inside]
    out[~inside] = -(3.0 * np.pi * sigma0 * G / (8.0 * alpha ** 3)) * (
        Ro * (4.0 * alpha ** 2 - 3.0 * Ro ** 2) * np.arcsin(alpha / Ro)
        - alpha * (2.0 * alpha ** 2 - 3.0 * Ro ** 2) * np.sqrt(1.0 - alpha ** 2 / Ro ** 2))
    return out


def d2_force_xy(x, y, alpha, sigma0=1.0, G=1.0, xc=0.0, yc=0.0):
    """Cartesian (Fx, Fy) of a D_2 disk centred at (xc, yc)."""
    dx = np.asarray(x, np.float64) - xc
    dy = np.asarray(y, np.float64) - yc
    R = np.hypot(dx, dy)
    fr = d2_radial_force(R, alpha, sigma0, G)
    with np.errstate(invalid="ignore", divide="ignore"):
        fx = np.where(R > 0, fr * dx / R, 0.0)
        fy = np.where(R > 0, fr * dy / R, 0.0)
    return fx, fy


def kuzmin_radial_force(R, a, M=1.0, G=1.0):
    R = np.asarray(R, dtype=np.float64)
    return -G * M * R / (R * R + a * a) ** 1.5


def kuzmin_force_xy(x, y, a, M=1.0, G=1.0):
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    s = -G * M / (x * x + y * y + a * a) ** 1.5
    return s * x, s * y


def kuzmin_force_xyz(x, y, z, a, M=1.0, G=1.0):
    """Kuzmin disk off the plane: Phi = -G M / sqrt(R^2 + (a + |z|)^2), so
    F = -grad Phi = -G M (x, y, sgn(z) (a + |z|)) / (R^2 + (a + |z|)^2)^{3/2}."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    b = a + abs(z)
    s = -G * M / (x * x + y * y + b * b) ** 1.5
    return s * x, s * y, s * np.sign(z) * b


def d2_potential(R, alpha, sigma0=1.0, G=1.0):
    """Mid-plane potential of the D_2 disk (Section 3, after Schulz 2009, Eq. 29 there):
        R <= alpha: -(3 pi^2 sigma0 G / (64 alpha^3)) (8 alpha^4 - 8 alpha^2 R^2 + 3 R^4)
        R >  alpha: -(3 pi sigma0 G / (32 alpha^3)) [(8 alpha^4 - 8 alpha^2 R^2 + 3 R^4) asin(alpha/R)
                                                      + 3 alpha (2 alpha^2 - R^2) sqrt(R^2 - alpha^2)]"""
    R = np.asarray(R, dtype=np.float64)
    q = 8.0 * alpha ** 4 - 8.0 * alpha ** 2 * R ** 2 + 3.0 * R ** 4
    inside = R <= alpha
    out = np.empty_like(R)
    out[inside] = -(3.0 * np.pi ** 2 * sigma0 * G / (64.0 * alpha ** 3)) * q[inside]
    Ro = R[~inside]
    out[~inside] = -(3.0 * np.pi * sigma0 * G / (32.0 * alpha ** 3)) * (
        q[~inside] * np.arcsin(alpha / Ro) + 3.0 * alpha * (2.0 * alpha ** 2 - Ro ** 2) * np.sqrt(Ro ** 2 - alpha ** 2))
    return out
