"""Oracle: ordering + ctypes binding of the plain C sparse LDL^T (ldlt.c).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Ordering: recursive coordinate bisection of the tetrahedra (split at the
median centroid along the longest extent).  An unknown whose supporting
tetrahedra lie on both sides is a separator unknown; the two halves share no
tetrahedron and hence no matrix entry.  Unknowns are numbered left half,
right half, separator (nested dissection), which keeps the fill of the
up-looking factorisation moderate.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np
import scipy.sparse as sp

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ldlt.c")
_LIB = os.path.join(_HERE, "_ldlt.so")
_lock = threading.Lock()
_lib = None


def build():
    """Compile the oracle's C factorisation (plain gcc, no GPU code)."""
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", _LIB, _SRC])


def _load():
    global _lib
    with _lock:
        if _lib is None:
            if (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
                build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            lib.ldl_symbolic.argtypes = [ctypes.c_int64, P, P, P, P, P, P]
            lib.ldl_symbolic.restype = ctypes.c_int64
            lib.ldl_numeric.argtypes = [ctypes.c_int64, P, P, P, P, P, P, P, P, P]
            lib.ldl_numeric.restype = ctypes.c_int64
            lib.ldl_solve.argtypes = [ctypes.c_int64, ctypes.c_int64, P, P, P, P, P]
            lib.ldl_solve.restype = None
            _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def nested_dissection(tdof, N, centroids, leaf=48):
    """Permutation (new -> old unknown) from recursive coordinate bisection."""
    T = tdof.shape[0]
    mask = tdof >= 0
    d = tdof[mask]
    t = np.nonzero(mask)[0]
    o = np.argsort(d, kind="stable")
    inc_t = t[o]
    ptr = np.searchsorted(d[o], np.arange(N + 1))
    side = np.zeros(T, dtype=np.int8)
    out = []

    def rec(dofs, tets):
        if len(dofs) <= leaf or len(tets) < 2:
            out.append(dofs)
            return
        c = centroids[tets]
        ax = int(np.argmax(c.max(axis=0) - c.min(axis=0)))
        med = np.median(c[:, ax])
        left = c[:, ax] < med
        if left.all() or (~left).all():
            out.append(dofs)
            return
        side[tets] = np.where(left, 0, 1)
        lens = ptr[dofs + 1] - ptr[dofs]
        starts = np.concatenate([[0], np.cumsum(lens)[:-1]])
        flat = np.repeat(ptr[dofs] - starts, lens) + np.arange(lens.sum())
        sl = side[inc_t[flat]]
        nl = np.add.reduceat((sl == 0).astype(np.int64), starts)
        has_l = nl > 0
        has_r = nl < lens
        sep = dofs[has_l & has_r]
        rec(dofs[has_l & ~has_r], tets[left])
        rec(dofs[has_r & ~has_l], tets[~left])
        out.append(sep)

    rec(np.arange(N), np.arange(T))
    perm = np.concatenate(out)
    assert len(perm) == N and len(np.unique(perm)) == N
    return perm


class LDLT:
    """A = L D L^T of a complex symmetric sparse matrix under a fixed ordering."""

    def __init__(self, A, perm):
        lib = _load()
        self.n = n = A.shape[0]
        self.perm = np.asarray(perm, dtype=np.int64)
        Ap = sp.csr_matrix(A)[self.perm][:, self.perm]
        U = sp.triu(Ap).tocsc()
        U.sort_indices()
        self.Ap = U.indptr.astype(np.int64)
        self.Ai = U.indices.astype(np.int64)
        Ax = np.ascontiguousarray(U.data.astype(np.complex128))
        self.Lp = np.zeros(n + 1, dtype=np.int64)
        self.parent = np.zeros(n, dtype=np.int64)
        lnz = np.zeros(n, dtype=np.int64)
        flag = np.zeros(n, dtype=np.int64)
        nnz = lib.ldl_symbolic(n, _ptr(self.Ap), _ptr(self.Ai), _ptr(self.Lp),
                               _ptr(self.parent), _ptr(lnz), _ptr(flag))
        self.Li = np.zeros(max(nnz, 1), dtype=np.int64)
        self.Lx = np.zeros(max(nnz, 1), dtype=np.complex128)
        self.D = np.zeros(n, dtype=np.complex128)
        st = lib.ldl_numeric(n, _ptr(self.Ap), _ptr(self.Ai), _ptr(Ax), _ptr(self.Lp),
                             _ptr(self.parent), _ptr(lnz), _ptr(self.Li), _ptr(self.Lx),
                             _ptr(self.D))
        if st != n:
            raise ZeroDivisionError(f"zero pivot at permuted row {st}")
        self.nnz_L = int(nnz)

    def solve(self, B):
        """X = A^-1 B for B [n] or [n, k]."""
        lib = _load()
        B = np.asarray(B)
        vec = B.ndim == 1
        Bm = B.reshape(self.n, -1)
        X = np.asfortranarray(Bm[self.perm].astype(np.complex128))
        lib.ldl_solve(self.n, X.shape[1], _ptr(self.Lp), _ptr(self.Li), _ptr(self.Lx),
                      _ptr(self.D), _ptr(X))
        out = np.empty_like(X)
        out[self.perm] = X
        return out[:, 0] if vec else out


def symbolic_nnz(A, perm):
    """Entries of L (below the diagonal) of the up-looking factorisation of A's
    pattern under the ordering perm, from the elimination tree alone."""
    lib = _load()
    n = A.shape[0]
    Ap = sp.csr_matrix(A)[np.asarray(perm)][:, np.asarray(perm)]
    U = sp.triu(Ap).tocsc()
    U.sort_indices()
    up = U.indptr.astype(np.int64)
    ui = U.indices.astype(np.int64)
    Lp = np.zeros(n + 1, dtype=np.int64)
    parent = np.zeros(n, dtype=np.int64)
    lnz = np.zeros(n, dtype=np.int64)
    flag = np.zeros(n, dtype=np.int64)
    return int(lib.ldl_symbolic(n, _ptr(up), _ptr(ui), _ptr(Lp), _ptr(parent), _ptr(lnz), _ptr(flag)))
