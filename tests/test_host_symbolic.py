"""Host set-up (nested dissection, assembly tree, update rows) checked on the CPU.

The probe in tests/host/ runs the library's host code (csrc/host.cpp) on a mesh
without a GPU.  The checks rebuild the factor structure independently:
- A's pattern comes from the tetrahedra's unknowns (every pair of unknowns
  of a tetrahedron couples);
- the symbolic Cholesky structure of L, in the library's elimination order,
  comes from the elimination tree with set unions: struct(j) = {i > j : A_ij
  != 0} united with struct(c) - {j} over the children c of j.
Then every nonzero of L must lie inside its front (the front's later pivots
and its update rows), the fronts must partition the unknowns and nest in
their parents, each extend-add relative map must point at exactly the
child's update rows inside the parent front, the memory plan must keep
factor blocks disjoint and simultaneously alive update blocks disjoint,
every lower-triangle entry of A must go once to its factor position, and the
extend-add tasks must cover every child update column once with no two
children of one parent in the same (concurrently launched) child slot.
"""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from paper_2605_19951_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))
MAX_CHILD = 4          # children per front (csrc/tem_internal.h kMaxChild)
AMALG_DEFAULT = 32     # default amalgamation threshold (kAmalgDefault)
CSRC = os.path.join(HERE, "..", "paper_2605_19951_gb300", "csrc")


@pytest.fixture(scope="module")
def probe():
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tempfile.mkdtemp(prefix="tem_symprobe_")
    exe = os.path.join(d, "symprobe")
    subprocess.check_call([gxx, "-O2", "-std=c++17", "-I", CSRC, "-o", exe,
                           os.path.join(HERE, "host", "symbolic_probe.cpp"), os.path.join(CSRC, "host.cpp")])
    yield exe, d
    shutil.rmtree(d, ignore_errors=True)


def run_probe(probe, s, leaf, amalg=AMALG_DEFAULT):
    exe, d = probe
    src, dst = os.path.join(d, "mesh.bin"), os.path.join(d, "sym.bin")
    with open(src, "wb") as f:
        np.array([s.xyz.shape[0], s.tets.shape[0]], np.int64).tofile(f)
        np.array([leaf, amalg], np.int32).tofile(f)
        np.ascontiguousarray(s.xyz, np.float64).tofile(f)
        np.ascontiguousarray(s.tets, np.int32).tofile(f)
        np.ascontiguousarray(s.sigma, np.float64).tofile(f)
        np.ascontiguousarray(s.is_param, np.uint8).tofile(f)
    subprocess.check_call([exe, src, dst])
    raw = open(dst, "rb").read()
    pos = 0

    def take(dtype, count):
        nonlocal pos
        a = np.frombuffer(raw, dtype=dtype, count=count, offset=pos)
        pos += a.nbytes
        return a

    N, nt = (int(x) for x in take(np.int64, 2))
    tdof = take(np.int32, 6 * nt).reshape(nt, 6)
    nf = int(take(np.int64, 1)[0])
    fronts, layout = [], []
    for _ in range(nf):
        k, n, c0, parent, height, ld = (int(x) for x in take(np.int32, 6))
        lofs, uofs = (int(x) for x in take(np.int64, 2))
        rows = take(np.int32, n - k).copy()
        rel = take(np.int32, n - k).copy() if parent >= 0 else None
        fronts.append((k, n, c0, parent, rows, rel))
        layout.append((height, ld, lofs, uofs))
    nnz_l, ltotal, utotal = (int(x) for x in take(np.int64, 3))
    rp = take(np.int64, N + 1)
    ci = take(np.int32, int(take(np.int64, 1)[0]))
    no = int(take(np.int64, 1)[0])
    onz, odst = take(np.int64, no), take(np.int64, no)
    levels = []
    for _ in range(int(take(np.int64, 1)[0])):
        lf = take(np.int32, int(take(np.int64, 1)[0])).copy()
        beg, end = take(np.int64, MAX_CHILD).copy(), take(np.int64, MAX_CHILD).copy()
        levels.append((lf, beg, end))
    nea = int(take(np.int64, 1)[0])
    ea = (take(np.int32, nea).copy(), take(np.int32, nea).copy())
    assert pos == len(raw)
    return N, tdof, fronts, nnz_l, (layout, ltotal, utotal), (rp, ci, onz, odst), (levels, ea)


def symbolic_cholesky(N, tdof):
    """Row structure below the diagonal of every column of L (elimination tree, set unions)."""
    lower = [set() for _ in range(N)]
    for dofs in tdof:
        u = [int(x) for x in dofs if x >= 0]
        for a in u:
            for b in u:
                if b > a:
                    lower[a].add(b)
    children = [[] for _ in range(N)]
    struct = [None] * N
    for j in range(N):
        sj = set(lower[j])
        for c in children[j]:
            sj |= struct[c]
        sj.discard(j)
        struct[j] = sj
        if sj:
            children[min(sj)].append(j)
    return struct


def check_memory_plan(fronts, layout, ltotal, utotal):
    """Factor blocks are disjoint; update blocks alive at the same level are disjoint.

    Front f's n x k factor block (column stride ld = n rounded up to even) sits at
    lofs.  Its b x b update block sits at uofs from its own level until its
    parent's level, where extend-add consumes it while the parent's blocks are
    being filled."""
    spans = []
    for (k, n, c0, parent, rows, rel), (height, ld, lofs, uofs) in zip(fronts, layout):
        assert ld == n + (n & 1)
        spans.append((lofs, lofs + ld * k))
    spans.sort()
    assert spans[0][0] >= 0 and spans[-1][1] <= ltotal
    assert all(a[1] <= b[0] for a, b in zip(spans, spans[1:]))
    H = max(h for h, _, _, _ in layout)
    for level in range(H + 1):
        alive = []
        for (k, n, c0, parent, rows, rel), (height, ld, lofs, uofs) in zip(fronts, layout):
            b = n - k
            if b == 0:
                continue
            assert parent >= 0 and layout[parent][0] > height
            if height <= level <= layout[parent][0]:
                alive.append((uofs, uofs + b * b))
        alive.sort()
        if alive:
            assert alive[0][0] >= 0 and alive[-1][1] <= utotal
            assert all(a[1] <= b[0] for a, b in zip(alive, alive[1:])), level


def check_original_entries(N, fronts, layout, rp, ci, onz, odst):
    """Every lower-triangle entry (row r >= column c) of A goes exactly once to
    the factor position of (r, c) in the front that owns column c: column
    c - c0, row r - c0 among the pivots or k + (r's place among the update
    rows)."""
    owner = np.empty(N, np.int64)
    for q, (k, n, c0, parent, rows, rel) in enumerate(fronts):
        owner[c0:c0 + k] = q
    row_of = np.repeat(np.arange(N), np.diff(rp))
    lower = np.nonzero(ci >= row_of)[0]
    assert np.array_equal(np.sort(onz), lower)
    for z, dst in zip(onz.tolist(), odst.tolist()):
        c, r = int(row_of[z]), int(ci[z])
        k, n, c0, parent, rows, rel = fronts[owner[c]]
        height, ld, lofs, uofs = layout[owner[c]]
        loc = r - c0 if r < c0 + k else k + int(np.searchsorted(rows, r))
        assert loc < n and (r < c0 + k or rows[loc - k] == r)
        assert dst == lofs + (c - c0) * ld + loc
    assert np.unique(odst).size == odst.size


def check_extend_add(fronts, layout, levels, ea):
    """Level h lists the fronts of height h.  Its extend-add tasks (child front,
    child update column) cover every update column of every child of those
    fronts exactly once, and no two children of one parent fall into the same
    child slot (each slot runs as a launch of its own, so the children's
    scatter-adds into a parent never run concurrently)."""
    ea_child, ea_col = ea
    for h, (lf, beg, end) in enumerate(levels):
        assert all(layout[f][0] == h for f in lf.tolist())
        want = set()
        for f in lf.tolist():
            for c, fr in enumerate(fronts):
                if fr[3] == f:
                    want |= {(c, j) for j in range(fr[1] - fr[0])}
        got = []
        for sl in range(MAX_CHILD):
            kids = ea_child[beg[sl]:end[sl]].tolist()
            got += list(zip(kids, ea_col[beg[sl]:end[sl]].tolist()))
            parents = [fronts[c][3] for c in sorted(set(kids))]
            assert len(parents) == len(set(parents)), (h, sl)
        assert len(got) == len(set(got)) and set(got) == want


def check_structure(N, tdof, fronts, nnz_l, plan, entries, ea):
    check_memory_plan(fronts, *plan)
    check_original_entries(N, fronts, plan[0], *entries)
    check_extend_add(fronts, plan[0], *ea)
    # unknowns: tdof covers 0..N-1 (PEC edges are -1)
    used = np.unique(tdof[tdof >= 0])
    assert used.size == N and used[0] == 0 and used[-1] == N - 1
    # pivots of the fronts partition 0..N-1
    cover = np.zeros(N, np.int32)
    for k, n, c0, parent, rows, rel in fronts:
        assert k >= 0 and n >= k
        cover[c0:c0 + k] += 1
    assert (cover == 1).all()
    # update rows: sorted, after the front's pivots, inside the parent's columns, and the
    # extend-add relative map points at exactly those rows of the parent front (pivots
    # first, then its update rows)
    for q, (k, n, c0, parent, rows, rel) in enumerate(fronts):
        assert (np.diff(rows) > 0).all()
        if rows.size:
            assert rows[0] >= c0 + k and rows[-1] < N
            assert parent > q   # children precede parents
        if parent >= 0:
            pk, pn, pc0, _, prows, _ = fronts[parent]
            pglobal = np.concatenate([np.arange(pc0, pc0 + pk), prows])
            assert ((rel >= 0) & (rel < pn)).all()
            np.testing.assert_array_equal(pglobal[rel], rows)
    # every nonzero of L inside its front
    owner = np.empty(N, np.int64)
    for q, (k, n, c0, parent, rows, rel) in enumerate(fronts):
        owner[c0:c0 + k] = q
    struct = symbolic_cholesky(N, tdof)
    true_nnz = 0
    for j in range(N):
        k, n, c0, parent, rows, rel = fronts[owner[j]]
        allowed = set(range(j + 1, c0 + k)) | set(rows.tolist())
        assert struct[j] <= allowed, (j, sorted(struct[j] - allowed)[:5])
        true_nnz += len(struct[j]) + 1
    # the library's count of factor entries: every front's triangle and update block
    lib = sum(k * (k + 1) // 2 + k * (n - k) for k, n, c0, parent, rows, rel in fronts)
    assert lib == nnz_l
    assert nnz_l >= true_nnz


@pytest.mark.parametrize("amalg", [0, AMALG_DEFAULT])
@pytest.mark.parametrize("leaf", [0, 16, 64])
def test_fronts_contain_symbolic_cholesky(probe, leaf, amalg):
    s = inputs.make_config(1)
    check_structure(*run_probe(probe, s, leaf, amalg))


@pytest.mark.parametrize("amalg", [0, AMALG_DEFAULT])
def test_fronts_with_a_conductive_block(probe, amalg):
    s = inputs.make_config(2, n=6)
    check_structure(*run_probe(probe, s, 24, amalg))


def test_amalgamation_merges_small_separators(probe):
    """With amalgamation every internal front of at most AMALG_DEFAULT
    pivots is one whose parent had no room (four children already, counting
    the merged grandchildren), there are fewer fronts, some fronts have three
    or four children, and no front has more than four."""
    s = inputs.make_config(1)
    plain = run_probe(probe, s, 16, 0)[2]
    merged = run_probe(probe, s, 16, AMALG_DEFAULT)[2]
    assert len(merged) < len(plain)
    nkids = np.zeros(len(merged), np.int64)
    for k, n, c0, parent, rows, rel in merged:
        if parent >= 0:
            nkids[parent] += 1
    assert nkids.max() <= MAX_CHILD and (nkids >= 3).any()
    for q, (k, n, c0, parent, rows, rel) in enumerate(merged):
        if nkids[q] > 0 and k <= AMALG_DEFAULT and parent >= 0:
            assert nkids[parent] - 1 + nkids[q] > MAX_CHILD, q
