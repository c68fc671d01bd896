"""Enrichment functions of the XFEM approximation (Section 2.3).

* Shifted jump function H_J(x) = H(x) - H(x_J), H = +1 for phi >= 0 and -1
  otherwise (Eq. jump_enr_functions).
* Four quasi-orthogonalised, shifted branch functions of node I
  (Eq. orthogonal_tip_enr_func) in the front polar coordinates
  r = sqrt(phi^2 + psi^2), theta = atan2(phi, psi) (Eq. polar_coords).

The fourth branch function carries the coefficient c_I34 whose denominator
36 (1 + cos 3 theta_I) vanishes at theta_I = +-pi/3 and +-pi.  The function is
rescaled by the positive factor B / sqrt(A^2 + B^2), with A the numerator and
B the denominator of c_I34, which leaves the enriched space unchanged where
c_I34 is finite and takes the limit direction -cos(theta/2 + theta_I) at the
points where both vanish.
"""
import numpy as np


def heaviside(phi):
    return np.where(phi >= 0.0, 1.0, -1.0)


def polar(phi, psi):
    """r and theta of Eq. polar_coords; theta = atan2(phi, psi) in (-pi, pi]."""
    return np.sqrt(phi * phi + psi * psi), np.arctan2(phi, psi)


def c34_coefficients(theta_i):
    """(a, b) such that the fourth branch function is
    -2 sqrt(r) sin^2((theta - theta_I)/2) [a cos X + b sin X], X = theta/2 + theta_I."""
    A = 7.0 * np.sin(theta_i) + 11.0 * np.sin(2.0 * theta_i) + 65.0 * np.sin(3.0 * theta_i)
    B = 36.0 * (1.0 + np.cos(3.0 * theta_i))
    rho = np.hypot(A, B)
    if rho * rho < 1e-24:
        return -1.0, 0.0
    return -A / rho, B / rho


def branch_functions(r, theta, grad_r, grad_theta, r_i, theta_i):
    """Values (4, P) and gradients (4, P, 3) of the shifted branch functions of one node.

    r, theta: (P,); grad_r, grad_theta: (P, 3); r_i, theta_i: nodal scalars.
    """
    s = np.sqrt(r)
    ds_dr = 0.5 / s
    h = 0.5 * theta
    sh, ch = np.sin(h), np.cos(h)
    si, ci = np.sqrt(r_i) * np.sin(0.5 * theta_i), np.sqrt(r_i) * np.cos(0.5 * theta_i)
    X = h + theta_i
    sX, cX = np.sin(X), np.cos(X)
    d = 0.5 * (theta - theta_i)
    sd, cd = np.sin(d), np.cos(d)
    a, b = c34_coefficients(theta_i)
    G = a * cX + b * sX
    dG = 0.5 * (-a * sX + b * cX)

    F = np.empty((4,) + r.shape)
    Fr = np.empty_like(F)
    Ft = np.empty_like(F)
    F[0] = s * sh - si
    Fr[0] = ds_dr * sh
    Ft[0] = 0.5 * s * ch
    F[1] = s * ch - ci
    Fr[1] = ds_dr * ch
    Ft[1] = -0.5 * s * sh
    F[2] = 2.0 * s * cX * sd
    Fr[2] = 2.0 * ds_dr * cX * sd
    Ft[2] = s * np.cos(theta + 0.5 * theta_i)
    F[3] = -2.0 * s * sd * sd * G
    Fr[3] = -2.0 * ds_dr * sd * sd * G
    Ft[3] = -2.0 * s * (sd * cd * G + sd * sd * dG)
    dF = Fr[:, :, None] * grad_r[None] + Ft[:, :, None] * grad_theta[None]
    return F, dF
