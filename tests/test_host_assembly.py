"""Host assembly, loop sources and observation operator against the oracle, on the CPU.

The probe in tests/host/ runs the library's host code (csrc/host.cpp: edges,
PEC removal, Whitney element matrices, elimination order, CSR of A, loop
right-hand sides f and the observation operator Q) without a GPU.  Its
unknowns are mapped to the oracle's through the edges' end points (both
orient an edge from its lower to its higher vertex id).  Then:
- K (curl-curl) must equal the oracle's element by element;
- f must equal the oracle's exactly (+-1 on the loop's edges);
- Q must equal the oracle's (Stokes reading of dB_z/dt on the surface faces);
- the library's Q^T (the unknowns Q reads, each with its receivers) must be
  exactly Q transposed;
- M(sigma) summed through the library's per-entry contribution lists (what
  the GPU sums) must equal the oracle's mass matrix;
- the unknown -> (tetrahedron, local edge) incidence must list exactly the
  tetrahedra that carry each unknown;
- the regulariser root W must number the parameters like the oracle and give
  the oracle's Laplacian W^T W (its rows may come in another face order).
"""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest
import scipy.sparse as sp

from oracle.fem import FEModel
from oracle.inversion import regulariser
from oracle.survey import loop_source, observation_operator
from paper_2605_19951_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "..", "paper_2605_19951_gb300", "csrc")


@pytest.fixture(scope="module")
def probe():
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tempfile.mkdtemp(prefix="tem_asmprobe_")
    exe = os.path.join(d, "asmprobe")
    subprocess.check_call([gxx, "-O2", "-std=c++17", "-I", CSRC, "-o", exe,
                           os.path.join(HERE, "host", "assembly_probe.cpp"), os.path.join(CSRC, "host.cpp")])
    yield exe, d
    shutil.rmtree(d, ignore_errors=True)


def run_probe(probe, s):
    exe, d = probe
    src, dst = os.path.join(d, "in.bin"), os.path.join(d, "out.bin")
    ptr = np.zeros(len(s.loops) + 1, np.int64)
    ptr[1:] = np.cumsum([len(lp) for lp in s.loops])
    with open(src, "wb") as f:
        np.array([s.xyz.shape[0], s.tets.shape[0]], np.int64).tofile(f)
        np.ascontiguousarray(s.xyz, np.float64).tofile(f)
        np.ascontiguousarray(s.tets, np.int32).tofile(f)
        np.ascontiguousarray(s.sigma, np.float64).tofile(f)
        np.ascontiguousarray(s.is_param, np.uint8).tofile(f)
        np.array([len(s.loops)], np.int32).tofile(f)
        ptr.tofile(f)
        np.concatenate([np.asarray(lp, np.int32) for lp in s.loops]).tofile(f)
        np.array([len(s.rx)], np.int32).tofile(f)
        np.ascontiguousarray(s.rx, np.float64).tofile(f)
    subprocess.check_call([exe, src, dst])
    raw = open(dst, "rb").read()
    pos = 0

    def take(dtype, count):
        nonlocal pos
        a = np.frombuffer(raw, dtype=dtype, count=count, offset=pos)
        pos += a.nbytes
        return a

    N, ne = (int(x) for x in take(np.int64, 2))
    out = {"N": N, "ev": take(np.int32, 2 * ne).reshape(ne, 2), "dof_old": take(np.int32, ne),
           "perm": take(np.int32, N), "rp": take(np.int64, N + 1)}
    nnz = int(take(np.int64, 1)[0])
    out["ci"], out["kval"] = take(np.int32, nnz), take(np.float64, nnz)
    n_tx = int(take(np.int32, 1)[0])
    out["f"] = take(np.float64, N * n_tx).reshape(N, n_tx)
    n_rx = int(take(np.int32, 1)[0])
    out["q_rp"] = take(np.int64, n_rx + 1)
    nq = int(take(np.int64, 1)[0])
    out["q_ci"], out["q_val"] = take(np.int32, nq), take(np.float64, nq)
    nqd = int(take(np.int64, 1)[0])
    out["qt_dof"], out["qt_rp"] = take(np.int32, nqd), take(np.int64, nqd + 1)
    out["qt_ci"], out["qt_val"] = take(np.int32, nq), take(np.float64, nq)
    out["mc_ptr"] = take(np.int64, nnz + 1)
    out["mc_idx"] = take(np.uint32, int(take(np.int64, 1)[0]))
    nt = s.tets.shape[0]
    out["Me1"] = take(np.float64, nt * 36)
    out["inc_ptr"] = take(np.int64, N + 1)
    ninc = int(take(np.int64, 1)[0])
    out["inc_tet"], out["inc_loc"] = take(np.int32, ninc), take(np.int8, ninc)
    out["tdof"] = take(np.int32, nt * 6).reshape(nt, 6)
    nf, P = (int(x) for x in take(np.int64, 2))
    out["P"] = P
    out["w_rp"] = take(np.int64, nf + 1)
    out["w_ci"], out["w_val"] = take(np.int32, int(out["w_rp"][-1])), take(np.float64, int(out["w_rp"][-1]))
    out["pidx"] = take(np.int32, nt)
    assert pos == len(raw)
    return out


@pytest.mark.parametrize("idx,n", [(1, None), (2, 6)])
def test_host_assembly_matches_oracle(probe, idx, n):
    s = inputs.make_config(idx, n=n) if n else inputs.make_config(idx)
    lib = run_probe(probe, s)
    fe = FEModel(s.xyz, s.tets)
    N = lib["N"]
    assert N == fe.N
    # library unknown (elimination order) -> oracle unknown, through the edge's end points
    old_to_edge = np.full(N, -1, np.int64)
    interior = np.nonzero(lib["dof_old"] >= 0)[0]
    old_to_edge[lib["dof_old"][interior]] = interior
    assert (old_to_edge >= 0).all()
    edges = lib["ev"][old_to_edge[lib["perm"]]]
    assert (edges[:, 0] < edges[:, 1]).all()
    to_or = np.array([fe.dof[fe.edge_id(int(a), int(b))] for a, b in edges])
    assert (to_or >= 0).all() and np.unique(to_or).size == N
    # K element by element
    Kl = sp.csr_matrix((lib["kval"], lib["ci"], lib["rp"]), shape=(N, N))
    P = sp.csr_matrix((np.ones(N), (to_or, np.arange(N))), shape=(N, N))   # library -> oracle
    Kmap = (P @ Kl @ P.T).tocsr()
    scale = abs(fe.K).max()
    assert abs(Kmap - fe.K).max() <= 1e-12 * scale
    # loop right-hand sides, exactly
    F = np.stack([loop_source(fe, lp) for lp in s.loops], axis=1)
    np.testing.assert_array_equal(P @ lib["f"], F)
    # observation operator
    Ql = sp.csr_matrix((lib["q_val"], lib["q_ci"], lib["q_rp"]), shape=(len(s.rx), N))
    Qo = observation_operator(fe, s.rx).tocsr()
    qmap = (Ql @ P.T).tocsr()
    assert abs(qmap - Qo).max() <= 1e-12 * abs(Qo).max()
    # Q^T over the distinct unknowns Q reads is exactly Q transposed
    qd = lib["qt_dof"].astype(np.int64)
    assert (np.diff(qd) > 0).all()
    cols = np.repeat(qd, np.diff(lib["qt_rp"]))
    Qt = sp.csr_matrix((lib["qt_val"], (lib["qt_ci"], cols)), shape=(len(s.rx), N))
    assert abs(Qt - Ql).max() == 0.0
    assert np.array_equal(np.unique(lib["q_ci"]), qd)
    # M(sigma) through the per-entry contribution lists (what the GPU sums)
    idx = lib["mc_idx"].astype(np.int64)
    contrib = s.sigma[idx // 36] * lib["Me1"][idx]
    mvals = np.add.reduceat(contrib, lib["mc_ptr"][:-1]) if contrib.size else contrib
    mvals[np.diff(lib["mc_ptr"]) == 0] = 0.0
    Ml = sp.csr_matrix((mvals, lib["ci"], lib["rp"]), shape=(N, N))
    Mo = fe.mass(s.sigma)
    assert abs((P @ Ml @ P.T) - Mo).max() <= 1e-12 * abs(Mo).max()
    # unknown -> (tet, local edge) incidence: exactly the tetrahedra that carry the unknown
    tdof = lib["tdof"]
    t_idx, a_idx = np.nonzero(tdof >= 0)
    want = np.lexsort((a_idx, t_idx, tdof[t_idx, a_idx]))
    want = np.stack([tdof[t_idx, a_idx][want], t_idx[want], a_idx[want]], axis=1)
    dof_of = np.repeat(np.arange(N), np.diff(lib["inc_ptr"]))
    inc_t, inc_a = lib["inc_tet"].astype(np.int64), lib["inc_loc"].astype(np.int64)
    got = np.lexsort((inc_a, inc_t, dof_of))
    got = np.stack([dof_of[got], inc_t[got], inc_a[got]], axis=1)
    np.testing.assert_array_equal(got, want)
    # regulariser root W (faces x parameters): the same parameter numbering and the
    # same Laplacian W^T W as the oracle's (rows may come in another face order)
    param = np.asarray(s.is_param).astype(bool)
    pid = -np.ones(len(param), np.int64)
    pid[param] = np.arange(int(param.sum()))
    np.testing.assert_array_equal(lib["pidx"], pid)
    Wl = sp.csr_matrix((lib["w_val"], lib["w_ci"], lib["w_rp"]), shape=(len(lib["w_rp"]) - 1, lib["P"]))
    Wo = regulariser(s.xyz, s.tets, s.is_param)
    assert Wl.shape == Wo.shape
    Ll, Lo = (Wl.T @ Wl).tocsr(), (Wo.T @ Wo).tocsr()
    assert abs(Ll - Lo).max() <= 1e-12 * abs(Lo).max()
