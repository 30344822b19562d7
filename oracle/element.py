"""Reference stiffness of the 8-node trilinear brick (oracle; test infrastructure only).

The paper computes one element matrix K0 (Algorithm 4, step "Compute K0") and
scales it per element by the SIMP law (Eq. K_mod); it never prints K0.  Here
K0 is the isotropic linear-elastic stiffness of a cube of edge h with Young's
modulus E and Poisson ratio nu:

    K0 = integral over the cube of B^T D B,

B the strain-displacement matrix of the trilinear shape functions and D the
isotropic elasticity matrix (Voigt order xx, yy, zz, xy, yz, xz with
engineering shears).  Local nodes are the cube corners (a_x, a_y, a_z) in
{0,1}^3 numbered a = a_x + 2 a_y + 4 a_z; local DOFs are node-major (x, y, z).

Two independent evaluations are provided: Gauss-Legendre quadrature
(element_stiffness) and exact rational integration of the polynomial
integrand (element_stiffness_exact); 2x2x2 Gauss is exact because the
integrand has degree <= 2 in each coordinate.
"""
from __future__ import annotations

from fractions import Fraction
from itertools import product

import numpy as np

CORNERS = [(ax, ay, az) for az in (0, 1) for ay in (0, 1) for ax in (0, 1)]


def lame(E, nu):
    """Lame constants (lambda, mu) of an isotropic solid."""
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    return lam, mu


def elasticity_matrix(E=1.0, nu=0.3) -> np.ndarray:
    lam, mu = lame(E, nu)
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[0, 0] = D[1, 1] = D[2, 2] = lam + 2 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    return D


def _lin(t, a):
    return t if a else 1.0 - t


def _dlin(a):
    return 1.0 if a else -1.0


def strain_displacement(x, y, z, h=1.0) -> np.ndarray:
    """B (6 x 24) at the point (x, y, z) of the cube [0, h]^3."""
    s, t, r = x / h, y / h, z / h
    B = np.zeros((6, 24))
    for a, (ax, ay, az) in enumerate(CORNERS):
        dx = _dlin(ax) * _lin(t, ay) * _lin(r, az) / h
        dy = _lin(s, ax) * _dlin(ay) * _lin(r, az) / h
        dz = _lin(s, ax) * _lin(t, ay) * _dlin(az) / h
        cx, cy, cz = 3 * a, 3 * a + 1, 3 * a + 2
        B[0, cx] = dx
        B[1, cy] = dy
        B[2, cz] = dz
        B[3, cx], B[3, cy] = dy, dx          # gamma_xy
        B[4, cy], B[4, cz] = dz, dy          # gamma_yz
        B[5, cx], B[5, cz] = dz, dx          # gamma_xz
    return B


def element_stiffness(nu=0.3, E=1.0, h=1.0, npts=2) -> np.ndarray:
    """K0 by npts^3-point Gauss-Legendre quadrature on the cube [0, h]^3."""
    xg, wg = np.polynomial.legendre.leggauss(npts)
    pts = 0.5 * h * (xg + 1.0)
    wts = 0.5 * h * wg
    D = elasticity_matrix(E, nu)
    K = np.zeros((24, 24))
    for (i, j, k) in product(range(npts), repeat=3):
        B = strain_displacement(pts[i], pts[j], pts[k], h)
        K += wts[i] * wts[j] * wts[k] * (B.T @ D @ B)
    return K


# ---------------------------------------------------------------------------
# Exact rational integration: polynomials in (x, y, z) as {(px, py, pz): coef}
# ---------------------------------------------------------------------------

def _poly_mul(p, q):
    out = {}
    for (a, ca) in p.items():
        for (b, cb) in q.items():
            key = (a[0] + b[0], a[1] + b[1], a[2] + b[2])
            out[key] = out.get(key, 0) + ca * cb
    return out


def _poly_integrate_unit_cube(p):
    total = Fraction(0)
    for (ex, ey, ez), c in p.items():
        total += c * Fraction(1, (ex + 1) * (ey + 1) * (ez + 1))
    return total


def _shape_grad_polys(a):
    """Gradient of the trilinear shape function of corner a, as polynomials."""
    ax, ay, az = CORNERS[a]

    def lin(axis, on):   # t or 1 - t along `axis`
        e = [0, 0, 0]
        e[axis] = 1
        return {tuple(e): Fraction(1)} if on else {(0, 0, 0): Fraction(1), tuple(e): Fraction(-1)}

    def const(v):
        return {(0, 0, 0): Fraction(v)}

    lx, ly, lz = lin(0, ax), lin(1, ay), lin(2, az)
    gx = _poly_mul(_poly_mul(const(1 if ax else -1), ly), lz)
    gy = _poly_mul(_poly_mul(const(1 if ay else -1), lx), lz)
    gz = _poly_mul(_poly_mul(const(1 if az else -1), lx), ly)
    return gx, gy, gz


def element_stiffness_exact(nu=Fraction(3, 10), E=Fraction(1)):
    """K0 of the unit cube with exact rational arithmetic (list of Fractions).

    Uses the bilinear form a(u, v) = lambda (div u)(div v) + mu grad u : grad v
    + mu grad u : (grad v)^T, which equals eps(u) : C : eps(v) for isotropic C;
    this is a different route to the same matrix than B^T D B.
    """
    nu = Fraction(nu)
    E = Fraction(E)
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    grads = [_shape_grad_polys(a) for a in range(8)]
    # G[p][q][a][b] = integral d_p N_a d_q N_b
    G = [[[[_poly_integrate_unit_cube(_poly_mul(grads[a][p], grads[b][q]))
            for b in range(8)] for a in range(8)] for q in range(3)] for p in range(3)]
    K = [[Fraction(0)] * 24 for _ in range(24)]
    for a in range(8):
        for b in range(8):
            for i in range(3):          # component of the test function v (row)
                for j in range(3):      # component of the trial function u (column)
                    val = lam * G[i][j][a][b] + mu * G[j][i][a][b]
                    if i == j:
                        val += mu * sum(G[p][p][a][b] for p in range(3))
                    K[3 * a + i][3 * b + j] = val
    return K


def rigid_body_modes() -> np.ndarray:
    """Six rigid-body displacement fields of the unit cube's corners (24 x 6)."""
    R = np.zeros((24, 6))
    for a, (x, y, z) in enumerate(CORNERS):
        R[3 * a + 0, 0] = 1.0
        R[3 * a + 1, 1] = 1.0
        R[3 * a + 2, 2] = 1.0
        # infinitesimal rotations omega x r about the axes x, y, z
        R[3 * a + 1, 3], R[3 * a + 2, 3] = -z, y
        R[3 * a + 0, 4], R[3 * a + 2, 4] = z, -x
        R[3 * a + 0, 5], R[3 * a + 1, 5] = -y, x
    return R
