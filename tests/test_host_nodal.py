"""Host tables of the gradient-space (nodal) correction against the oracle, on the CPU.

The probe in tests/host/ runs the library's build_mesh and build_nodal
(csrc/host.cpp) without a GPU.  The gradient space of the edge unknowns is
spanned by the discrete gradients G e_a of the interior vertices a; with
K G = 0 (curl grad = 0) the shifted matrices restrict to it as
G^T (K - xi M) G = -xi G^T M(sigma) G.  The library's tables are compared
with the oracle's own node-to-edge incidence G (fem.gradient_matrix) and mass
matrix M(sigma), after mapping unknowns through edge end points and vertex ids:
- the interior vertices are exactly those the oracle's G couples to interior
  edges and that lie off the outer boundary;
- the library's G (edge -> its lower and higher end node) equals the oracle's G;
- its G^T lists (node -> incident edges with signs) are exactly G transposed;
- the nodal Laplacian summed through its contribution lists (sigma_t S_t,
  S_t the P1 stiffness) equals the oracle's G^T M(sigma) G;
- C summed through its lists (sigma_t B_t) equals the oracle's M(sigma) G.
"""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.fem import FEModel
from paper_2605_19951_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2605_19951_gb300", "csrc")


@pytest.fixture(scope="module")
def probe():
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tempfile.mkdtemp(prefix="tem_nodalprobe_")
    exe = os.path.join(d, "nodalprobe")
    subprocess.check_call([gxx, "-O2", "-std=c++17", "-I", CSRC, "-o", exe,
                           os.path.join(HERE, "host", "nodal_probe.cpp"), os.path.join(CSRC, "host.cpp")])
    yield exe, d
    shutil.rmtree(d, ignore_errors=True)


def run_probe(probe, xyz, tets, sigma, is_param):
    exe, d = probe
    src, dst = os.path.join(d, "in.bin"), os.path.join(d, "out.bin")
    with open(src, "wb") as f:
        np.array([xyz.shape[0], tets.shape[0]], np.int64).tofile(f)
        np.ascontiguousarray(xyz, np.float64).tofile(f)
        np.ascontiguousarray(tets, np.int32).tofile(f)
        np.ascontiguousarray(sigma, np.float64).tofile(f)
        np.ascontiguousarray(is_param, np.uint8).tofile(f)
    subprocess.check_call([exe, src, dst])
    raw = open(dst, "rb").read()
    pos = 0

    def take(dtype, count):
        nonlocal pos
        a = np.frombuffer(raw, dtype=dtype, count=int(count), offset=pos)
        pos += a.nbytes
        return a

    nt = tets.shape[0]
    o = {}
    N, ne = (int(x) for x in take(np.int64, 2))
    o["N"] = N
    o["ev"] = take(np.int32, 2 * ne).reshape(ne, 2)
    o["dof_old"] = take(np.int32, ne)
    o["perm"] = take(np.int32, N)
    Nn = int(take(np.int64, 1)[0])
    o["Nn"] = Nn
    o["node_perm"] = take(np.int32, Nn)
    o["rp"] = take(np.int64, Nn + 1)
    nnz = int(take(np.int64, 1)[0])
    o["ci"] = take(np.int32, nnz)
    o["mc_ptr"] = take(np.int64, nnz + 1)
    o["mc_idx"] = take(np.uint32, take(np.int64, 1)[0])
    o["S"] = take(np.float64, 16 * nt)
    o["e_lo"] = take(np.int32, N)
    o["e_hi"] = take(np.int32, N)
    o["g_ptr"] = take(np.int64, Nn + 1)
    ng = int(take(np.int64, 1)[0])
    o["g_edge"] = take(np.int32, ng)
    o["g_sign"] = take(np.int8, ng)
    o["c_rp"] = take(np.int64, N + 1)
    nc = int(take(np.int64, 1)[0])
    o["c_ci"] = take(np.int32, nc)
    o["c_mc_ptr"] = take(np.int64, nc + 1)
    o["c_mc_idx"] = take(np.uint32, take(np.int64, 1)[0])
    o["B"] = take(np.float64, 24 * nt)
    assert pos == len(raw)
    return o


def _sum_lists(ptr, idx, sigma, table, per):
    """value[z] = sum over the contributions idx of z: sigma[idx // per] table[idx]."""
    vals = sigma[idx // per] * table[idx]
    return np.add.reduceat(vals, ptr[:-1]) * (np.diff(ptr) > 0) if len(idx) else np.zeros(len(ptr) - 1)


def _case(name):
    if name == "c1":
        s = inputs.make_config(1)
        return s.xyz, s.tets, s.sigma, s.is_param
    # graded 6^3 box with a conductive block: unequal tetrahedra, three conductivities
    xs = inputs.graded_axis(20.0, 2, 1.5, 1)
    zs = np.concatenate([xs[:4], xs[4:]])
    xyz, tets = inputs.kuhn_grid(xs, xs, zs)
    cent = xyz[tets].mean(axis=1)
    sigma = np.where(cent[:, 2] > 0, 1e-8, 0.01)
    sigma[(np.abs(cent[:, 0]) < 25) & (cent[:, 2] < -5) & (cent[:, 2] > -45)] = 0.3
    return xyz, tets, sigma, (cent[:, 2] < 0).astype(np.uint8)


@pytest.mark.parametrize("name", ["c1", "graded_block"])
def test_nodal_tables_match_oracle(probe, name):
    xyz, tets, sigma, is_param = _case(name)
    o = run_probe(probe, xyz, tets, sigma, is_param)
    fe = FEModel(xyz, tets)
    nv = xyz.shape[0]
    # library edge unknown (elimination numbering) -> oracle interior edge unknown
    edge_of_old = np.empty(o["N"], np.int64)
    ok = o["dof_old"] >= 0
    edge_of_old[o["dof_old"][ok]] = np.nonzero(ok)[0]
    lev = o["ev"][edge_of_old[o["perm"]]]
    okey = fe.edges[:, 0] * nv + fe.edges[:, 1]
    e = np.searchsorted(okey, lev[:, 0].astype(np.int64) * nv + lev[:, 1])
    assert np.array_equal(okey[e], lev[:, 0].astype(np.int64) * nv + lev[:, 1])
    odof = fe.dof[e]
    assert np.all(odof >= 0) and len(np.unique(odof)) == fe.N == o["N"]
    # interior vertices: off every face of the bounding box
    lo, hi = xyz.min(axis=0), xyz.max(axis=0)
    tol = 1e-9 * (hi - lo).max()
    interior = ~np.any((np.abs(xyz - lo) < tol) | (np.abs(xyz - hi) < tol), axis=1)
    verts = o["node_perm"]
    assert np.array_equal(np.sort(verts), np.nonzero(interior)[0])
    Go = fe.gradient_matrix().tocsc()[:, verts].tocsr()             # oracle G in library node order
    # library G from the end nodes of each edge unknown
    Nn = o["Nn"]
    rows = np.arange(o["N"])
    lo_, hi_ = o["e_lo"], o["e_hi"]
    Gl = sp.csr_matrix((np.r_[np.ones((hi_ >= 0).sum()), -np.ones((lo_ >= 0).sum())],
                        (np.r_[rows[hi_ >= 0], rows[lo_ >= 0]], np.r_[hi_[hi_ >= 0], lo_[lo_ >= 0]])),
                       shape=(o["N"], Nn))
    Go_lib_rows = Go[odof]                                            # oracle G, rows in library edge order
    assert (Gl - Go_lib_rows).count_nonzero() == 0 and abs(Gl - Go_lib_rows).max() == 0
    # G^T lists are exactly G transposed
    gr = np.repeat(np.arange(Nn), np.diff(o["g_ptr"]))
    Gt = sp.csr_matrix((o["g_sign"].astype(float), (gr, o["g_edge"])), shape=(Nn, o["N"]))
    assert abs(Gt - Gl.T).max() == 0
    # nodal Laplacian through its contribution lists
    M = fe.mass(sigma)
    Mlib = M[odof][:, odof]
    Lref = (Go_lib_rows.T @ Mlib @ Go_lib_rows).tocsr()
    lr = np.repeat(np.arange(Nn), np.diff(o["rp"]))
    lval = _sum_lists(o["mc_ptr"], o["mc_idx"].astype(np.int64), sigma, o["S"], 16)
    Llib = sp.csr_matrix((lval, (lr, o["ci"])), shape=(Nn, Nn))
    scale = abs(Lref).max()
    assert abs(Llib - Lref).max() <= 1e-12 * scale
    # C = M(sigma) G through its contribution lists
    Cref = (Mlib @ Go_lib_rows).tocsr()
    cr = np.repeat(np.arange(o["N"]), np.diff(o["c_rp"]))
    cval = _sum_lists(o["c_mc_ptr"], o["c_mc_idx"].astype(np.int64), sigma, o["B"], 24)
    Clib = sp.csr_matrix((cval, (cr, o["c_ci"])), shape=(o["N"], Nn))
    assert abs(Clib - Cref).max() <= 1e-12 * abs(Cref).max()
    # the restriction identity behind the correction: K G = 0 (oracle's K)
    assert abs(fe.K[odof][:, odof] @ Go_lib_rows).max() <= 1e-9 * abs(fe.K).max()
