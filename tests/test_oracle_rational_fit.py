"""Pins of the oracle's residue fit and its variable-projection objective
(Section 2.3), by brute force on a problem small enough to solve by hand: one
pole pair and three sample points, where the penalised least-squares
residual follows from the 2 x 2 normal equations written out explicitly.
The starting poles of the pole fit are pinned by their defining moduli and
angle.  CPU only."""
import numpy as np

from oracle import rational


def _by_hand(xi, z, t, mu):
    """Residual sum of squares of min || [B; mu diag(1/|xi|)] a - [e; 0] ||
    for one pole: B = [2 Re c, -2 Im c], c = 1 / (z - xi), e = exp(-t z),
    from the normal equations N a = r with N = B^T B + (mu/|xi|)^2 I."""
    c = 1.0 / (z - xi)
    b1, b2 = 2.0 * c.real, -2.0 * c.imag
    e = np.exp(-t * z)
    p = (mu / abs(xi)) ** 2
    n11, n12, n22 = b1 @ b1 + p, b1 @ b2, b2 @ b2 + p
    r1, r2 = b1 @ e, b2 @ e
    det = n11 * n22 - n12 * n12
    a1, a2 = (n22 * r1 - n12 * r2) / det, (n11 * r2 - n12 * r1) / det
    res = e - a1 * b1 - a2 * b2
    return a1 + 1j * a2, float(res @ res + p * (a1 * a1 + a2 * a2))


def test_residue_fit_and_objective_by_hand():
    xi = np.array([-3.0 + 4.0j])
    z = np.array([0.0, 1.0, 2.5])
    for mu in (0.0, 0.3):
        for t in (0.2, 1.0):
            a_ref, f_ref = _by_hand(xi[0], z, t, mu)
            a = rational.fit_alpha(xi, np.array([t]), z=z, mu=mu)
            assert abs(a[0, 0] - a_ref) <= 1e-12 * abs(a_ref)
            assert abs(rational.vp_objective(xi, np.array([t]), z=z, mu=mu) - f_ref) <= 1e-12 * f_ref
    # the objective sums over the times
    f2 = _by_hand(xi[0], z, 0.2, 0.3)[1] + _by_hand(xi[0], z, 1.0, 0.3)[1]
    assert abs(rational.vp_objective(xi, np.array([0.2, 1.0]), z=z, mu=0.3) - f2) <= 1e-12 * f2


def test_a_larger_basis_never_fits_worse():
    """Without the penalty, adding a pole enlarges the least-squares basis, so
    the residual cannot grow."""
    t = np.logspace(-5, -2, 8)
    xi = rational.seed_poles(4)
    f4 = rational.vp_objective(xi, t, mu=0.0)
    f5 = rational.vp_objective(np.append(xi, -50.0 + 900.0j), t, mu=0.0)
    assert f5 <= f4 * (1 + 1e-9)


def test_seed_poles():
    m, t0, t1, ang = 6, 1e-5, 1e-2, 0.7
    x = rational.seed_poles(m, t0, t1, ang)
    assert np.allclose(np.abs(x), np.geomspace(0.3 / t1, 30.0 / t0, m), rtol=1e-14)
    assert np.allclose(np.angle(x), np.pi * ang, rtol=1e-14)
    assert np.all(x.real < 0) and np.all(x.imag > 0)
