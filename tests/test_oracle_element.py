"""Pins of the oracle's hex8 reference stiffness K0 (Alg. 4 "Compute K0").

K0 is pinned by facts that do not come from the oracle's own quadrature:
hand-derived closed-form entries (1D integrals of the linear shape functions),
an exact rational integration of a different bilinear form, the rigid-body
null space and the spectrum's sign pattern.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import element

NU = 0.3


def _lam_mu(nu=NU):
    return element.lame(1.0, nu)


def test_symmetric():
    K = element.element_stiffness(NU)
    assert np.abs(K - K.T).max() < 1e-15


def test_rigid_body_null_space_and_spectrum():
    K = element.element_stiffness(NU)
    R = element.rigid_body_modes()
    assert np.abs(K @ R).max() < 1e-14
    ev = np.linalg.eigvalsh(K)
    assert np.sum(np.abs(ev) < 1e-12) == 6
    assert np.all(ev[6:] > 1e-3)
    # the null space is exactly the span of the six rigid modes
    Q, _ = np.linalg.qr(R)
    w, V = np.linalg.eigh(K)
    N = V[:, :6]
    assert np.abs(N - Q @ (Q.T @ N)).max() < 1e-12


def test_row_sums_vanish_per_direction():
    K = element.element_stiffness(NU)
    for c in range(3):
        t = np.zeros(24)
        t[c::3] = 1.0
        assert np.abs(K @ t).max() < 1e-15


def test_gauss2_equals_gauss3():
    assert np.abs(element.element_stiffness(NU, npts=2) - element.element_stiffness(NU, npts=3)).max() < 1e-15


def test_exact_rational_integration_matches():
    Kx = np.array([[float(v) for v in row] for row in element.element_stiffness_exact(Fraction(3, 10))])
    assert np.abs(element.element_stiffness(NU) - Kx).max() < 1e-15


def test_hand_derived_entries():
    """Entries from 1D integrals: int l_a l_b = 1/3, 1/6; int l_a' l_b' = +-1;
    int l_a' l_b = s_a / 2 (s = -1 for the corner at 0)."""
    lam, mu = _lam_mu()
    K = element.element_stiffness(NU)
    assert K[0, 0] == pytest.approx((lam + 4 * mu) / 9, rel=1e-14)       # corner 0 x, corner 0 x
    assert K[0, 1] == pytest.approx((lam + mu) / 12, rel=1e-14)          # corner 0 x, corner 0 y
    assert K[0, 3] == pytest.approx(-(lam + mu) / 9, rel=1e-14)          # corner 0 x, corner (1,0,0) x
    assert K[0, 21] == pytest.approx(-(lam + 4 * mu) / 36, rel=1e-14)    # corner 0 x, corner (1,1,1) x
    assert K[0, 22] == pytest.approx(-(lam + mu) / 24, rel=1e-14)        # corner 0 x, corner (1,1,1) y


def test_edge_length_scaling():
    """3D elastic stiffness of a cube scales linearly with its edge h."""
    assert np.abs(element.element_stiffness(NU, h=2.0) - 2.0 * element.element_stiffness(NU)).max() < 1e-14
    assert np.abs(element.element_stiffness(NU, h=4.0) - 4.0 * element.element_stiffness(NU)).max() < 1e-14


def test_uniform_strain_energy():
    """A uniform strain eps gives element energy u^T K0 u = eps:C:eps * volume."""
    lam, mu = _lam_mu()
    K = element.element_stiffness(NU)
    A = np.array([[0.3, 0.1, -0.2], [0.05, -0.4, 0.2], [0.1, 0.25, 0.15]])
    u = np.concatenate([A @ np.array(c, dtype=float) for c in element.CORNERS])
    eps = 0.5 * (A + A.T)
    energy = lam * np.trace(eps) ** 2 + 2 * mu * np.sum(eps * eps)
    assert u @ K @ u == pytest.approx(energy, rel=1e-13)
