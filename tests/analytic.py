"""Closed forms used to pin the oracle (independent of oracle/ and of the CUDA path).

Kuzmin disk (Section 3.1): above/below the plane the Newtonian potential is
that of a point mass at (0, -+a): Phi_N = -GM / r', r' = sqrt(R^2 + (a+|z|)^2).
The field has no curl in either half space, so the exact QUMOND field is
nu(|g_N|/a0) g_N (Eq. 3 is exact here), and its potential is the spherical
QUMOND potential F(r') of a point mass, F'(r) = nu(GM/(a0 r^2)) GM/r^2:
  F(r) = -A/(2r) + (1/2) [ -sqrt(A^2 + c r^2)/r + sqrt(c) asinh(sqrt(c) r / A) ],
with A = GM and c = 4 a0 A (differentiate to check; tests do it numerically).
"""
import numpy as np


def nu(y):
    """nu(y) = 1/2 + 1/2 sqrt(1 + 4/y) (Eq. 2)."""
    return 0.5 + 0.5 * np.sqrt(1.0 + 4.0 / y)


def kuzmin_phiN(x, y, z, M, a, G):
    r = np.sqrt(x * x + y * y + (a + np.abs(z)) ** 2)
    return -G * M / r


def kuzmin_phi_mond(x, y, z, M, a, G, a0):
    A = G * M
    c = 4.0 * a0 * A
    r = np.sqrt(x * x + y * y + (a + np.abs(z)) ** 2)
    return -A / (2.0 * r) + 0.5 * (-np.sqrt(A * A + c * r * r) / r + np.sqrt(c) * np.arcsinh(np.sqrt(c) * r / A))


def kuzmin_vc_newton(R, M, a, G):
    """v_c^2 = R g_R with g_R = G M R (R^2+a^2)^-3/2 in the plane (Section 3.1)."""
    return np.sqrt(G * M * R * R / (R * R + a * a) ** 1.5)


def kuzmin_vc_mond(R, M, a, G, a0):
    """g_M,R = nu(|g_N,r| / a0) g_N,R with |g_N,r| = G M / (R^2 + a^2) (Section 3.1)."""
    gNr = G * M / (R * R + a * a)
    return kuzmin_vc_newton(R, M, a, G) * np.sqrt(nu(gNr / a0))


def node_coords(n, L, center=(0.0, 0.0, 0.0)):
    """x, y, z of every node of a box in the flat x-fastest order."""
    h = L / n
    ii = np.arange(n + 1)
    kk, jj, i3 = np.meshgrid(ii, ii, ii, indexing="ij")
    return (center[0] - 0.5 * L + i3.ravel() * h,
            center[1] - 0.5 * L + jj.ravel() * h,
            center[2] - 0.5 * L + kk.ravel() * h)


def boundary_mask(n):
    ii = np.arange(n + 1)
    kk, jj, i3 = np.meshgrid(ii, ii, ii, indexing="ij")
    return ((i3 == 0) | (i3 == n) | (jj == 0) | (jj == n) | (kk == 0) | (kk == n)).ravel()


def laplacian7(u, n, h):
    """7-point Laplacian on interior nodes by array slicing (0 on the boundary)."""
    U = u.reshape(n + 1, n + 1, n + 1)
    out = np.zeros_like(U)
    out[1:-1, 1:-1, 1:-1] = (U[2:, 1:-1, 1:-1] + U[:-2, 1:-1, 1:-1] + U[1:-1, 2:, 1:-1] + U[1:-1, :-2, 1:-1]
                             + U[1:-1, 1:-1, 2:] + U[1:-1, 1:-1, :-2] - 6.0 * U[1:-1, 1:-1, 1:-1]) / (h * h)
    return out.ravel()
