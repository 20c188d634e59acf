"""Physics pin of the oracle's whole chain (CPU only): step-off dB_z/dt at the
centre of a 40 m square loop on a 0.1 S/m half-space against the closed form
(vertical-dipole superposition of the circular-loop formula).

Sign and scale only, not parity: the graded Kuhn mesh (10 m cells near the
loop, PEC at ~450 m) and the 8-pair approximant (max error ~3e-4 of exp) limit
the agreement to the early-time band where the response is at least 1% of its
peak; there it must agree to 10%.
"""
import numpy as np

from oracle import halfspace
from oracle.tem import Oracle
from paper_2605_19951_gb300 import inputs


def test_halfspace_central_loop():
    sig_hs, h0 = 0.1, 10.0
    ax = inputs.graded_axis(h0, 3, 1.6, 6)
    xyz, tets = inputs.kuhn_grid(ax, ax, ax)
    earth = xyz[tets].mean(axis=1)[:, 2] < 0
    sig = np.where(earth, sig_hs, inputs.SIGMA_AIR)
    nx = len(ax)
    c = int(np.argmin(np.abs(ax)))

    def vid(i, j):
        return i + nx * (j + nx * c)

    s = 2
    pts = ([(c - s + t, c - s) for t in range(2 * s)] + [(c + s, c - s + t) for t in range(2 * s)]
           + [(c + s - t, c + s) for t in range(2 * s)] + [(c - s, c + s - t) for t in range(2 * s)])
    loop = np.array([vid(i, j) for i, j in pts], dtype=np.int32)
    times = inputs.times_log(24)
    xi, al = inputs.load_rational(8, times)
    o = Oracle(xyz, tets, sig, earth.astype(np.uint8), [loop], np.zeros((1, 3)), xi, al)
    o.set_model(np.log(sig[earth]))
    d = o.forward()[0, 0]
    ref = halfspace.square(s * h0, times, sig_hs)
    assert np.all(ref < 0)
    band = np.abs(ref) >= 1e-2 * np.abs(ref).max()
    assert band.sum() >= 8
    ratio = d[band] / ref[band]
    assert np.all(np.abs(ratio - 1.0) < 0.1), ratio
