"""Level-set descriptions of the synthetic cracks (Section 2.2, Eqs. sgned_distance, polar_coords).

Each crack supplies the normal level set phi (signed distance to the crack
surface) and the tangential level set psi (signed in-surface distance to the
front, negative on the cracked side), plus the tip-enrichment radius r_e.

For the warped surfaces the distances are first-order: phi divides the
height above the surface by sqrt(1 + |grad w|^2), and psi is the in-plane
distance to the front curve, linearised for the ellipse.  Any consistent
choice serves, because the assembled system is the input of both solvers.
"""
import numpy as np


class Crack:
    r_e = 0.0

    def phi_psi(self, x):
        raise NotImplementedError


class PlanarEdgeCrack(Crack):
    """Flat crack phi = z - z0, occupying x < x_front (psi = x - x_front)."""

    def __init__(self, z0, x_front, r_e):
        self.z0, self.x_front, self.r_e = z0, x_front, r_e

    def phi_psi(self, x):
        return x[:, 2] - self.z0, x[:, 0] - self.x_front


class WarpedEdgeCrack(Crack):
    """Crack z = z0 + w(x, y) occupying x < x_front, w = A sin(2 pi y) cos(2 pi x)."""

    def __init__(self, z0, x_front, amp, r_e):
        self.z0, self.x_front, self.amp, self.r_e = z0, x_front, amp, r_e

    def phi_psi(self, x):
        phi = _warped_phi(x, self.z0, self.amp)
        return phi, x[:, 0] - self.x_front


class WarpedPennyCrack(Crack):
    """Penny of radius R in the surface z = z0 + w(x, y), centred over (cx, cy)."""

    def __init__(self, centre, radius, amp, r_e):
        self.c, self.R, self.amp, self.r_e = np.asarray(centre, float), radius, amp, r_e

    def phi_psi(self, x):
        phi = _warped_phi(x, self.c[2], self.amp)
        rho = np.hypot(x[:, 0] - self.c[0], x[:, 1] - self.c[1])
        return phi, rho - self.R


def _warped_phi(x, z0, amp):
    wx = amp * np.sin(2 * np.pi * x[:, 1]) * np.cos(2 * np.pi * x[:, 0])
    gx = -2 * np.pi * amp * np.sin(2 * np.pi * x[:, 1]) * np.sin(2 * np.pi * x[:, 0])
    gy = 2 * np.pi * amp * np.cos(2 * np.pi * x[:, 1]) * np.cos(2 * np.pi * x[:, 0])
    return (x[:, 2] - z0 - wx) / np.sqrt(1.0 + gx * gx + gy * gy)


class TiltedEllipticalCrack(Crack):
    """Elliptical crack, semi-axes (a along local xi, b along local eta), centred at c,
    rotated by `tilt` radians about the global x-axis, its surface warped by
    amp * sin(2 pi x) along the local normal."""

    def __init__(self, centre, a, b, tilt, amp, r_e):
        self.c = np.asarray(centre, float)
        self.a, self.b, self.amp, self.r_e = a, b, amp, r_e
        ct, st = np.cos(tilt), np.sin(tilt)
        self.e1 = np.array([1.0, 0.0, 0.0])
        self.e2 = np.array([0.0, ct, st])
        self.e3 = np.array([0.0, -st, ct])

    def phi_psi(self, x):
        d = x - self.c
        xi, eta, zeta = d @ self.e1, d @ self.e2, d @ self.e3
        xg = x[:, 0]
        w = self.amp * np.sin(2 * np.pi * xg)
        dw = 2 * np.pi * self.amp * np.cos(2 * np.pi * xg)   # d w / d xi (e1 is the x-axis)
        phi = (zeta - w) / np.sqrt(1.0 + dw * dw)
        a, b = self.a, self.b
        rho = np.sqrt((xi / a) ** 2 + (eta / b) ** 2)
        num = np.sqrt((xi / a ** 2) ** 2 + (eta / b ** 2) ** 2)
        safe = rho > 0.0
        grad = np.where(safe, num / np.where(safe, rho, 1.0), 1.0 / max(a, b))
        psi = (rho - 1.0) / grad
        return phi, psi
