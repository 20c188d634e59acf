"""Oracle: transmitter right-hand sides f and the observation operator Q.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Source (Section 2.1, step-off source and initial condition sigma e(0) = q; Section 2.2,
M u(0) = f): for a loop carrying I = 1 A, f_k = int_loop N_k . dl.  For a loop
running along mesh edges the Whitney property (int_edge N_k . t dl = delta)
makes f = +-1 on the loop's edges: +1 where the loop runs along the edge's
orientation (lower to higher vertex index), -1 against it.

Observation (Section 4.2: curl of the field, vertical component, at the receiver):
the measured quantity is dB_z/dt = -(curl e)_z (Faraday).  On a horizontal face
the normal component of the curl of a Whitney field is constant and equals the
circulation of the three edge unknowns divided by the face area (Stokes).  A
receiver on a face uses that face; a receiver on an edge or a vertex of the
horizontal surface uses the area-weighted mean over the surface triangles
whose closure contains it, i.e. -(sum of circulations)/(sum of areas).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def loop_source(fe, loop_verts, current=1.0):
    """f for one closed polyline of mesh vertices (consecutive ids share an edge)."""
    f = np.zeros(fe.N)
    L = len(loop_verts)
    for s in range(L):
        p, q = int(loop_verts[s]), int(loop_verts[(s + 1) % L])
        e = fe.edge_id(p, q)
        if e < 0:
            raise ValueError(f"loop segment {p}-{q} is not a mesh edge")
        d = fe.dof[e]
        if d < 0:
            raise ValueError("loop runs along the PEC boundary")
        f[d] += current * (1.0 if p < q else -1.0)
    return f


def _faces(fe):
    tv = fe.tv
    fl = np.concatenate([tv[:, [0, 1, 2]], tv[:, [0, 1, 3]], tv[:, [0, 2, 3]], tv[:, [1, 2, 3]]])
    return np.unique(fl, axis=0)


def observation_operator(fe, rx, rel_tol=1e-9):
    """Q: [n_rx, N] sparse, dB_z/dt at each receiver (Stokes reading above)."""
    faces = _faces(fe)
    xyz = fe.xyz
    scale = float(np.ptp(xyz, axis=0).max())
    tol = rel_tol * scale
    rows, cols, vals = [], [], []
    zf = xyz[faces][:, :, 2]
    flat = np.abs(zf - zf[:, :1]).max(axis=1) < tol   # horizontal faces
    hfaces = faces[flat]
    hz = zf[flat, 0]
    for r, p in enumerate(np.asarray(rx, dtype=np.float64)):
        cand = np.nonzero(np.abs(hz - p[2]) < tol)[0]
        near = xyz[hfaces[cand]][:, :, :2]
        lo, hi = near.min(axis=1), near.max(axis=1)
        keep = np.all((lo - tol <= p[:2]) & (p[:2] <= hi + tol), axis=1)
        cand = cand[keep]
        circ = {}
        area_sum = 0.0
        for fi in cand:
            v = [int(x) for x in hfaces[fi]]
            P = xyz[v][:, :2]
            a2 = (P[1, 0] - P[0, 0]) * (P[2, 1] - P[0, 1]) - (P[1, 1] - P[0, 1]) * (P[2, 0] - P[0, 0])
            if a2 < 0:                               # make the ordering counter-clockwise
                v = [v[0], v[2], v[1]]
                P = xyz[v][:, :2]
                a2 = -a2
            # barycentric coordinates of the receiver (closure test)
            lam = []
            for k in range(3):
                A, B = P[(k + 1) % 3], P[(k + 2) % 3]
                lam.append(((B[0] - A[0]) * (p[1] - A[1]) - (B[1] - A[1]) * (p[0] - A[0])) / a2)
            if min(lam) < -1e-9:
                continue
            area_sum += 0.5 * a2
            for k in range(3):
                s, t = v[k], v[(k + 1) % 3]
                d = fe.dof[fe.edge_id(s, t)]
                if d >= 0:
                    circ[d] = circ.get(d, 0.0) + (1.0 if s < t else -1.0)
        if area_sum == 0.0:
            raise ValueError(f"receiver {r} lies on no horizontal face")
        for d, c in circ.items():
            if c != 0.0:
                rows.append(r)
                cols.append(d)
                vals.append(-c / area_sum)
    return sp.csr_matrix((vals, (rows, cols)), shape=(len(rx), fe.N))
