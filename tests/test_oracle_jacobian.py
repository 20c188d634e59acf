"""Pins of the oracle's Jacobian products (CPU only).

* brute-force central finite differences of d(m) on seeded earth cells
  (Richardson-extrapolated, O(h^4)) equal J e_c (Section 3.1), to 1e-6 of the
  column plus a floor of 1e-11 of the data (FD round-off on remote cells);
* Taylor remainder test: e0(h) = O(h), e1(h) = O(h^2) (Section 3.1, eqs. e0/e1);
* adjoint test <J dm, dd> = <dm, J^T dd> to near machine precision (Section 3.1).
"""
import numpy as np
import pytest

from oracle.tem import Oracle
from paper_2605_19951_gb300 import inputs


@pytest.fixture(scope="module")
def c1():
    s = inputs.make_config(1)
    xi, al = inputs.load_rational(s.m, s.times)
    o = Oracle(s.xyz, s.tets, s.sigma, s.is_param, s.loops, s.rx, xi, al)
    m0 = s.log_sigma()
    # a non-uniform model so that every cell matters differently
    m0 = m0 + 0.3 * np.random.default_rng(19951).standard_normal(m0.shape)
    o.set_model(m0)
    return s, o, m0



def test_finite_differences(c1):
    s, o, m0 = c1
    cells = np.random.default_rng(19952).choice(len(m0), size=20, replace=False)
    h = 4e-3
    d0 = o.forward()
    jcols = []
    for c in cells:
        e = np.zeros_like(m0)
        e[c] = 1.0
        jcols.append(o.jvp(e))

    def central(c, hh):
        e = np.zeros_like(m0)
        e[c] = hh
        dp = o.set_model(m0 + e).forward()
        dm = o.set_model(m0 - e).forward()
        return (dp - dm) / (2 * hh)

    fd = []
    for c in cells:
        f1, f2 = central(c, h), central(c, h / 2)
        fd.append((4.0 * f2 - f1) / 3.0)
    o.set_model(m0)
    assert np.array_equal(o.forward(), d0)
    floor = 1e-11 * np.abs(d0).max()
    for c, j, f in zip(cells, jcols, fd):
        scale = np.abs(j).max()
        assert scale > 0
        assert np.abs(j - f).max() <= 1e-6 * scale + floor, f"cell {c}"


def test_taylor_remainder(c1):
    s, o, m0 = c1
    dm = np.random.default_rng(19953).standard_normal(m0.shape)
    d0 = o.forward()
    jdm = o.jvp(dm)
    hs = [0.08, 0.04, 0.02, 0.01]
    e0, e1 = [], []
    for h in hs:
        d = o.set_model(m0 + h * dm).forward()
        e0.append(np.linalg.norm(d - d0))
        e1.append(np.linalg.norm(d - d0 - h * jdm))
    o.set_model(m0)
    s0 = np.log2(np.array(e0[:-1]) / np.array(e0[1:]))
    s1 = np.log2(np.array(e1[:-1]) / np.array(e1[1:]))
    assert np.all(np.abs(s0 - 1.0) < 0.1), s0
    assert np.all(np.abs(s1 - 2.0) < 0.15), s1


def test_adjoint(c1):
    s, o, m0 = c1
    rng = np.random.default_rng(19954)
    for _ in range(3):
        v = rng.standard_normal(m0.shape)
        w = rng.standard_normal(o.forward_shape)
        a = np.sum(o.jvp(v) * w)
        b = np.sum(v * o.jtvp(w))
        assert abs(a - b) / max(abs(a), abs(b)) < 1e-11
