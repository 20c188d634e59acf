"""Seeded synthetic survey generators (shared by the oracle tests and the CUDA path).

This module only builds inputs: a tensor-product box of Kuhn tetrahedra, a
conductivity model, square loop transmitters given as closed polylines of mesh
vertices, receiver coordinates, observation times and the rational-approximant
table.  It holds none of the method's arithmetic (no finite-element matrices,
no solves, no response): both the oracle and the GPU library derive everything
else from these arrays on their own.

The workloads follow the structure of the paper's synthetic experiment
(Section 4.2: half-space under air, embedded blocks, surface square loops,
surface receiver grid, log-spaced times); the paper's own Gmsh mesh is not
available, so uniform Kuhn meshes stand in for it.
"""
from __future__ import annotations

import json
import os
from dataclasses import dataclass, field
from itertools import permutations

import numpy as np

SIGMA_AIR = 1e-8
_DATA = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data")


@dataclass
class Survey:
    name: str
    n: int                       # cubes per side
    h: float                     # cube size (m)
    n_air: int                   # air layers at the top
    xyz: np.ndarray              # [n_vert, 3] float64
    tets: np.ndarray             # [n_tet, 4] int32 (Kuhn path order)
    sigma: np.ndarray            # [n_tet] float64, true model (air included)
    is_param: np.ndarray         # [n_tet] uint8, 1 = earth cell (inverted)
    loops: list                  # n_tx closed polylines, int32 vertex ids, CCW from +z
    rx: np.ndarray               # [n_rx, 3] float64
    times: np.ndarray            # [K] float64 (s)
    m: int                       # number of conjugate pole pairs
    sigma_start: np.ndarray = field(default=None)  # start model for inversion

    @property
    def n_tet(self):
        return self.tets.shape[0]

    @property
    def n_param(self):
        return int(self.is_param.sum())

    def log_sigma(self, sigma=None):
        s = self.sigma if sigma is None else sigma
        return np.log(s[self.is_param.astype(bool)])


def vertex_id(n, i, j, k):
    return i + (n + 1) * (j + (n + 1) * k)


def kuhn_grid(xs, ys, zs):
    """Kuhn tetrahedra of the tensor-product grid xs x ys x zs (any spacing).
    Vertex (i, j, k) has id i + nx (j + ny k) with nx = len(xs), ny = len(ys);
    cube (i, j, k) has id i + cx (j + cy k) and owns tets 6*cube .. 6*cube+5."""
    xs, ys, zs = (np.asarray(a, dtype=np.float64) for a in (xs, ys, zs))
    nx, ny, nz = len(xs), len(ys), len(zs)
    v = np.arange(nx * ny * nz)
    vi, vj, vk = v % nx, (v // nx) % ny, v // (nx * ny)
    xyz = np.stack([xs[vi], ys[vj], zs[vk]], axis=1)
    cx, cy, cz = nx - 1, ny - 1, nz - 1
    c = np.arange(cx * cy * cz)
    ci, cj, ck = c % cx, (c // cx) % cy, c // (cx * cy)
    tets = []
    for perm in permutations(range(3)):
        step = np.zeros(3, dtype=np.int64)
        path = [ci + nx * (cj + ny * ck)]
        for ax in perm:
            step[ax] += 1
            path.append((ci + step[0]) + nx * ((cj + step[1]) + ny * (ck + step[2])))
        tets.append(np.stack(path, axis=1))
    tets = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    return xyz, tets


def kuhn_box(n, h, n_air):
    """Vertices and Kuhn tetrahedra of an n^3 cube grid, centred at x=y=0,
    surface at z=0, n_air air layers above it.  Each cube is cut into the six
    tetrahedra v000 -> ... -> v111 (one per ordering of the x, y, z steps)."""
    g = np.arange(n + 1, dtype=np.float64)
    return kuhn_grid((g - n / 2.0) * h, (g - n / 2.0) * h, (g - (n - n_air)) * h)


def graded_axis(h0, n_fine, growth, n_grow):
    """Symmetric axis: n_fine cells of size h0 on each side of 0, then n_grow
    cells growing geometrically by `growth`."""
    inner = np.arange(0, n_fine + 1) * h0
    out = [inner]
    x, d = inner[-1], h0
    for _ in range(n_grow):
        d *= growth
        x += d
        out.append([x])
    half = np.concatenate(out)
    return np.concatenate([-half[::-1], half[1:]])


def _cube_of_tet(n):
    return np.repeat(np.arange(n ** 3), 6)


def square_loop(n, n_air, i0, j0, side):
    """Closed CCW (seen from +z) polyline of vertex ids around the square whose
    lower-left corner is grid vertex (i0, j0) and whose side is `side` cubes."""
    k = n - n_air
    pts = []
    for t in range(side):
        pts.append((i0 + t, j0))
    for t in range(side):
        pts.append((i0 + side, j0 + t))
    for t in range(side):
        pts.append((i0 + side - t, j0 + side))
    for t in range(side):
        pts.append((i0, j0 + side - t))
    return np.array([vertex_id(n, i, j, k) for i, j in pts], dtype=np.int32)


def _grid_index(n, h, x):
    v = x / h + n / 2.0
    iv = int(round(v))
    assert abs(v - iv) < 1e-9, "coordinate not on a grid line"
    return iv


def _surface_rx(n, h, xs, ys):
    return np.array([[x, y, 0.0] for y in ys for x in xs], dtype=np.float64)


def load_rational(m, times):
    """Poles xi_i (one per conjugate pair) and coefficients alpha_i^[j] for the
    requested times, read from the stored table (see Section 2.3)."""
    with open(os.path.join(_DATA, f"rational_m{m}.json")) as fh:
        tab = json.load(fh)
    xi = np.array(tab["xi_re"]) + 1j * np.array(tab["xi_im"])
    key = _times_key(times)
    ent = tab["alpha"].get(key)
    if ent is None:
        raise KeyError(f"no alpha table for times {key}; regenerate the table")
    alpha = np.array(ent["re"]) + 1j * np.array(ent["im"])  # [m][K]
    return xi, alpha


def _times_key(times):
    t = np.asarray(times)
    return f"{len(t)}:{t[0]:.6e}:{t[-1]:.6e}"


def times_log(K, t0=1e-5, t1=1e-2):
    return np.logspace(np.log10(t0), np.log10(t1), K)


def _earth_mask(n, n_air):
    ck = _cube_of_tet(n) // (n * n)
    return ck < (n - n_air)


def _block_sigma(n, n_air, sig, blocks):
    """Assign conductivity to the tets of axis-aligned cube blocks
    (i0, j0, k0, di, dj, dk, value)."""
    cube = _cube_of_tet(n)
    ci, cj, ck = cube % n, (cube // n) % n, cube // (n * n)
    for (i0, j0, k0, di, dj, dk, val) in blocks:
        sel = ((ci >= i0) & (ci < i0 + di) & (cj >= j0) & (cj < j0 + dj)
               & (ck >= k0) & (ck < k0 + dk))
        sig[sel] = val
    return sig


def _seeded_block(rng, n, n_air, di, dj, dk):
    ke = n - n_air
    i0 = int(rng.integers(2, n - 2 - di + 1))
    j0 = int(rng.integers(2, n - 2 - dj + 1))
    # top of block at least one layer below the surface, at least 2 above bottom
    k_top_max = ke - 1
    k0 = int(rng.integers(2, k_top_max - dk + 1))
    return i0, j0, k0


def make_config(idx, m=None, n=None):
    """Configurations C1..C4 (idx 1..4) of the synthetic workloads.  For idx 4
    a smaller n keeps its structure (32 loops, 128 receivers, 10 poles) on a
    smaller box, for profiling captures."""
    rng = np.random.default_rng(19951 + idx)
    if idx == 1:
        n, h = 8, 50.0
    elif idx == 2:
        n, h = 20, 25.0
    elif idx == 3:
        n, h = 40, 12.5
    elif idx == 4:
        n = 46 if n is None else int(n)
        h = (100.0 / 9.0) * 46.0 / n
    else:
        raise ValueError(idx)
    n_air = (3 * n) // 8
    xyz, tets = kuhn_box(n, h, n_air)
    earth = _earth_mask(n, n_air)
    sig = np.full(tets.shape[0], SIGMA_AIR)
    sig[earth] = 0.01
    if idx == 1:
        loops = [square_loop(n, n_air, n // 2 - 1, n // 2 - 1, 2)]
        rx = np.array([[0.0, 0.0, 0.0]])
        K, mm = 16, 8
    elif idx == 2:
        i0, j0, k0 = _seeded_block(rng, n, n_air, 4, 4, 3)
        sig = _block_sigma(n, n_air, sig, [(i0, j0, k0, 4, 4, 3, 0.1)])
        loops = []
        for cy in (-75.0, 75.0):
            for cx in (-75.0, 75.0):
                ic, jc = _grid_index(n, h, cx), _grid_index(n, h, cy)
                loops.append(square_loop(n, n_air, ic - 2, jc - 2, 4))
        rx = _surface_rx(n, h, np.arange(-175.0, 176.0, 50.0), [-75.0, -25.0, 25.0, 75.0])
        K, mm = 24, 8
    elif idx == 3:
        ke = n - n_air
        white = rng.standard_normal((n, n, ke))
        from scipy.ndimage import gaussian_filter
        z = gaussian_filter(white, sigma=5.0, mode="nearest")
        z = (z - z.mean()) / z.std()
        cube = _cube_of_tet(n)
        ci, cj, ck = cube % n, (cube // n) % n, cube // (n * n)
        e = earth
        sig[e] = 10.0 ** (-2.0 + 0.5 * z[ci[e], cj[e], ck[e]])
        loops = []
        for cy in (-50.0, 50.0):
            for cx in (-150.0, -50.0, 50.0, 150.0):
                ic, jc = _grid_index(n, h, cx), _grid_index(n, h, cy)
                loops.append(square_loop(n, n_air, ic - 4, jc - 4, 8))
        v = np.arange(-175.0, 176.0, 50.0)
        rx = _surface_rx(n, h, v, v)
        K, mm = 32, 8
    else:  # idx == 4
        blocks = []
        for val in (0.1, 0.3):
            i0, j0, k0 = _seeded_block(rng, n, n_air, 6, 6, 4)
            blocks.append((i0, j0, k0, 6, 6, 4, val))
        sig = _block_sigma(n, n_air, sig, blocks)
        loops = []
        side = max(2, (9 * n) // 46)
        xs_ = np.linspace(3, n - 3 - side, 8).round().astype(int)
        ys_ = np.linspace(3, n - 3 - side, 4).round().astype(int)
        for jy in ys_:
            for ix in xs_:
                loops.append(square_loop(n, n_air, int(ix), int(jy), side))
        ks = n - n_air
        ia = np.linspace(3, n - 3, 16).round().astype(int)
        jb = np.linspace(4, n - 4, 8).round().astype(int)
        rx = np.array([[xyz[vertex_id(n, int(a), int(b), ks), 0],
                        xyz[vertex_id(n, int(a), int(b), ks), 1], 0.0]
                       for b in jb for a in ia])
        K, mm = 40, 10
    start = np.full(tets.shape[0], SIGMA_AIR)
    start[earth] = 0.01
    return Survey(name=f"C{idx}", n=n, h=h, n_air=n_air, xyz=xyz, tets=tets,
                  sigma=sig, is_param=earth.astype(np.uint8), loops=loops, rx=rx,
                  times=times_log(K), m=m if m is not None else mm,
                  sigma_start=start)


def make_c5_model(i, n=None, n_models=48):
    """Model i of the uneven batch C5: n seeded uniform in 12..28 cubes per side
    (a 500 m box), its own C3-style log-normal conductivity (log10 sigma = -2 +
    0.5 z, z a Gaussian-filtered seeded field, 5-cell correlation), 2..8
    square loops at seeded surface positions, 16 receivers on a 4 x 4
    surface lattice, 24 times, 8 pole pairs.  n overrides the size (small
    boxes for tests)."""
    rng = np.random.default_rng(19951 + 5)
    sizes = rng.integers(12, 29, size=n_models)
    nloops = rng.integers(2, 9, size=n_models)
    rng_i = np.random.default_rng(19951 + 5 * 1000 + i)
    n = int(sizes[i]) if n is None else int(n)
    h = 500.0 / n
    n_air = (3 * n) // 8
    xyz, tets = kuhn_box(n, h, n_air)
    earth = _earth_mask(n, n_air)
    ke = n - n_air
    from scipy.ndimage import gaussian_filter
    z = gaussian_filter(rng_i.standard_normal((n, n, ke)), sigma=5.0, mode="nearest")
    z = (z - z.mean()) / max(z.std(), 1e-12)
    cube = _cube_of_tet(n)
    ci, cj, ck = cube % n, (cube // n) % n, cube // (n * n)
    sig = np.full(tets.shape[0], SIGMA_AIR)
    sig[earth] = 10.0 ** (-2.0 + 0.5 * z[ci[earth], cj[earth], ck[earth]])
    side = max(2, n // 6)
    loops = []
    for _ in range(int(nloops[i])):
        i0 = int(rng_i.integers(1, n - side))
        j0 = int(rng_i.integers(1, n - side))
        loops.append(square_loop(n, n_air, i0, j0, side))
    lat = np.linspace(2, n - 2, 4).round().astype(int)
    rx = np.array([[xyz[vertex_id(n, int(a), int(b), ke), 0], xyz[vertex_id(n, int(a), int(b), ke), 1], 0.0]
                   for b in lat for a in lat])
    start = np.full(tets.shape[0], SIGMA_AIR)
    start[earth] = 0.01
    return Survey(name=f"C5[{i}]", n=n, h=h, n_air=n_air, xyz=xyz, tets=tets, sigma=sig,
                  is_param=earth.astype(np.uint8), loops=loops, rx=rx, times=times_log(24), m=8,
                  sigma_start=start)


def tiny_box(n=2, h=100.0, n_air=1, sigma_earth=0.01, sigma_air=SIGMA_AIR):
    """A very small box (2^3 .. 4^3 cubes) for brute-force checks."""
    xyz, tets = kuhn_box(n, h, n_air)
    earth = _earth_mask(n, n_air)
    sig = np.full(tets.shape[0], sigma_air)
    sig[earth] = sigma_earth
    return xyz, tets, sig, earth.astype(np.uint8)


def seeded_vectors(seed, *shapes):
    """Seeded standard-normal test vectors (e.g. delta log sigma, delta d)."""
    rng = np.random.default_rng(seed)
    return [rng.standard_normal(s) for s in shapes]
