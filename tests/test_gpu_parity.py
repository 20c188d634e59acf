"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (per data entry, floored at 1e-4 of the largest |value| of the
same transmitter-receiver pair over time):  FP64 path 1e-9, FP32 factors with
FP64 refinement 1e-6.  J^T w: relative 2-norm 1e-9 / 1e-6.  J v of the FP64
path: 1e-8, ten times the spread between two FP64 runs of the oracle that
differ only in their elimination ordering (9.9e-10 on the 20^3 box): the
residue sum of J v cancels more than that of the response.  J v of the
refined FP32 path: 1e-6, like the data.  The shifted matrices are
ill-conditioned on the air's gradient fields, which is why the comparison is
made on the data, never on the solution vectors themselves.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.inversion import gn_operator, gn_rhs, lsqr, regulariser
from oracle.tem import Oracle
from paper_2605_19951_gb300 import inputs

TOL = {"fp64": 1e-9, "fp32r": 1e-6}
TOL_JV = {"fp64": 1e-8, "fp32r": 1e-6}


def _tem():
    from paper_2605_19951_gb300 import build, tem
    import os
    if not os.path.exists(tem.LIB_PATH):
        build.build()
    return tem


def floored_err(a, ref, floor=1e-4):
    a, ref = np.asarray(a), np.asarray(ref)
    peak = np.abs(ref).max(axis=2, keepdims=True)
    return np.abs(a - ref) / np.maximum(np.abs(ref), floor * peak)


def _model(s, xi, al, prec, leaf=0):
    tem = _tem()
    p = tem.TEM_FP64 if prec == "fp64" else tem.TEM_FP32_REFINED
    return tem.Model(s.xyz, s.tets, s.sigma, s.is_param, s.loops, s.rx, xi, al, precision=p, leaf_max=leaf)


def _cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


class Case:
    def __init__(self, idx, seed):
        self.s = inputs.make_config(idx)
        self.xi, self.al = inputs.load_rational(self.s.m, self.s.times)
        rng = np.random.default_rng(seed)
        self.m0 = self.s.log_sigma() + 0.2 * rng.standard_normal(self.s.n_param)
        self.o = Oracle(self.s.xyz, self.s.tets, self.s.sigma, self.s.is_param, self.s.loops, self.s.rx,
                        self.xi, self.al)
        self.o.set_model(self.m0)
        self.d = self.o.forward()
        self.v = rng.standard_normal(self.s.n_param)
        self.w = rng.standard_normal(self.d.shape)
        self.jv = self.o.jvp(self.v)
        self.jtw = self.o.jtvp(self.w)


@pytest.fixture(scope="module")
def c1():
    return Case(1, 101)


@pytest.fixture(scope="module")
def c2():
    return Case(2, 202)


def _prod_launches(mdl):
    info = mdl.info()
    return info["tc_prod_launches"], info["simt_prod_launches"]


def _assert_product_path(mdl, before, prec, tensor_cores):
    """The FP32 solves ran their front products on the kernel asked for:
    k_tc_kint (tcgen05) with tensor cores on, k_prod_simt otherwise."""
    tc, simt = _prod_launches(mdl)
    if prec == "fp64":
        return
    if tensor_cores:
        assert tc > before[0] and simt == before[1], (before, tc, simt)
    else:
        assert simt > before[1] and tc == before[0], (before, tc, simt)


def _check_case(case, prec, leaf=0, tensor_cores=True):
    mdl = _model(case.s, case.xi, case.al, prec, leaf)
    try:
        if not tensor_cores:
            _tem().tem_set_tensor_cores(mdl.ctx, 0)
        before = _prod_launches(mdl)
        mdl.factor(_cuda(case.m0))
        d = mdl.forward().cpu().numpy()
        assert floored_err(d, case.d).max() <= TOL[prec]
        jv = mdl.jvp(_cuda(case.v)).cpu().numpy()
        assert floored_err(jv, case.jv).max() <= TOL_JV[prec]
        jtw = mdl.jtvp(_cuda(case.w)).cpu().numpy()
        assert np.linalg.norm(jtw - case.jtw) <= TOL[prec] * np.linalg.norm(case.jtw)
        info = mdl.info()
        assert info["last_pivot_front"] == -1 and info["min_pivot_abs"] > 0
        _assert_product_path(mdl, before, prec, tensor_cores)
    finally:
        mdl.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32r"])
def test_c1(c1, prec):
    _check_case(c1, prec)


@pytest.mark.parametrize("prec,tensor_cores", [("fp64", False), ("fp32r", True), ("fp32r", False)])
@pytest.mark.parametrize("leaf", [8, 33, 300])
def test_c1_leaf_sizes(c1, leaf, prec, tensor_cores):
    """Different dissection leaves give ragged fronts (k not a multiple of
    the 32-wide pivot block or the 64-row product tiles, single-front trees),
    on the tensor-core products and on the FP32-pipe products.  C1 has one
    transmitter: the solves carry it with a zero right-hand side as padding."""
    _check_case(c1, prec, leaf, tensor_cores)


def test_c1_fp32_simt_products(c1):
    """FP32 mode with the front products on the FP32 pipes instead of the
    tensor cores."""
    _check_case(c1, "fp32r", tensor_cores=False)


@pytest.mark.parametrize("prec", ["fp64", "fp32r"])
def test_c2(c2, prec):
    _check_case(c2, prec)


def test_assembly_matches_oracle(c1):
    """K and M(sigma) of the library equal the oracle's, entry by entry, after
    mapping unknowns through their edge end points."""
    tem = _tem()
    mdl = _model(c1.s, c1.xi, c1.al, "fp64")
    try:
        mdl.factor(_cuda(c1.m0))
        rp, ci, kv, mv = tem.tem_export_pattern(mdl.ctx, with_m=True)
        ev = tem.tem_export_dofs(mdl.ctx)
    finally:
        mdl.close()
    fe = c1.o.fe
    nv = fe.xyz.shape[0]
    okey = fe.edges[:, 0] * nv + fe.edges[:, 1]
    lkey = ev[:, 0] * nv + ev[:, 1]
    e = np.searchsorted(okey, lkey)
    assert np.array_equal(okey[e], lkey)
    odof = fe.dof[e]
    assert np.all(odof >= 0)
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    K = c1.o.fe.K.tocsr()
    M = c1.o.M.tocsr()
    ko = np.asarray(K[odof[rows], odof[ci]]).ravel()
    mo = np.asarray(M[odof[rows], odof[ci]]).ravel()
    assert np.abs(kv - ko).max() <= 1e-12 * np.abs(ko).max()
    assert np.abs(mv - mo).max() <= 1e-12 * np.abs(mo).max()
    assert K.nnz == len(kv)


def test_adjoint_gpu(c1):
    mdl = _model(c1.s, c1.xi, c1.al, "fp64")
    try:
        mdl.factor(_cuda(c1.m0))
        mdl.forward()
        rng = np.random.default_rng(9)
        for _ in range(3):
            v = rng.standard_normal(c1.s.n_param)
            w = rng.standard_normal(c1.d.shape)
            a = float(np.sum(mdl.jvp(_cuda(v)).cpu().numpy() * w))
            b = float(np.sum(v * mdl.jtvp(_cuda(w)).cpu().numpy()))
            assert abs(a - b) <= 1e-11 * max(abs(a), abs(b))
    finally:
        mdl.close()


@pytest.mark.parametrize("n_tx", [37, 70])
def test_many_transmitters(n_tx):
    """More than 32 right-hand sides: 37 (odd, padded to 38: two RHS chunks,
    the second ragged) and 70 (three chunks), on both product kernels."""
    s = inputs.make_config(1)
    n, na = s.n, s.n_air
    squares = [(i0, j0, side) for side in (1, 2, 3, 4) for i0 in range(1, n - side) for j0 in range(1, n - side)]
    pick = np.random.default_rng(n_tx).permutation(len(squares))[:n_tx]   # distinct squares off the PEC walls
    loops = [inputs.square_loop(n, na, *squares[q]) for q in pick]
    s.loops = loops
    xi, al = inputs.load_rational(8, s.times)
    rng = np.random.default_rng(n_tx)
    m0 = s.log_sigma() + 0.1 * rng.standard_normal(s.n_param)
    o = Oracle(s.xyz, s.tets, s.sigma, s.is_param, loops, s.rx, xi, al)
    o.set_model(m0)
    v = rng.standard_normal(s.n_param)
    w = rng.standard_normal((n_tx, 1, len(s.times)))
    ref_d, ref_jv, ref_jtw = o.forward(), o.jvp(v), o.jtvp(w)
    for prec, tc in (("fp64", False), ("fp32r", True), ("fp32r", False)):
        mdl = _model(s, xi, al, prec)
        try:
            if not tc:
                _tem().tem_set_tensor_cores(mdl.ctx, 0)
            before = _prod_launches(mdl)
            mdl.factor(_cuda(m0))
            d = mdl.forward().cpu().numpy()
            assert floored_err(d, ref_d).max() <= TOL[prec]
            jv = mdl.jvp(_cuda(v)).cpu().numpy()
            assert floored_err(jv, ref_jv).max() <= TOL_JV[prec]
            jtw = mdl.jtvp(_cuda(w)).cpu().numpy()
            assert np.linalg.norm(jtw - ref_jtw) <= TOL[prec] * np.linalg.norm(ref_jtw)
            _assert_product_path(mdl, before, prec, tc)
        finally:
            mdl.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32r"])
def test_lsqr_matches_oracle(c2, prec):
    """Device LSQR (FP64 scalars on the GPU) against the oracle's LSQR on the
    same Gauss-Newton system of the 20^3 box, Section 3.3, for 1..30
    iterations.  Two correct LSQR runs whose rounding differs at 1e-14
    diverge by ~8x per iteration once the Krylov basis loses orthogonality
    (measured, FP64: iterates 3e-10 apart at 12, 1.2e-9 at 13, 4e-3 at 20;
    refined FP32, whose J v is 1e-7-accurate: 2.6e-11 at 5, 2.1e-8 at 10).
    So the FP64 iterates are compared at 1e-9 through iteration 12 and the
    objective ||A x_k - b|| through 14; the refined ones at 1e-8 through 8 and
    10.  Every one of the 30 iterates must decrease the objective
    monotonically and stay within 2% of the oracle's (max measured 0.6%),
    both evaluated with the oracle's operator."""
    s = c2.s
    W = regulariser(s.xyz, s.tets, s.is_param)
    d_obs = c2.d * (1 + 0.03 * np.random.default_rng(3).standard_normal(c2.d.shape))
    wd = 1.0 / (0.03 * np.abs(d_obs) + 1e-4 * np.abs(d_obs).max())
    m_ref = s.log_sigma()
    lam = 10.0
    mv, rmv = gn_operator(c2.o, W, wd.ravel(), lam)
    b = gn_rhs(c2.d, d_obs, wd.ravel(), W, c2.m0, m_ref, lam)
    _, its = lsqr(mv, rmv, b, 30)
    tol_x, k_x, k_r = (1e-9, 12, 14) if prec == "fp64" else (1e-8, 8, 10)
    mdl = _model(s, c2.xi, c2.al, prec)
    try:
        mdl.factor(_cuda(c2.m0))
        mdl.forward()
        prev = np.inf
        for k in list(range(1, 15)) + [20, 25, 30]:
            dm = mdl.lsqr(_cuda(d_obs), _cuda(wd), _cuda(m_ref), lam, k).cpu().numpy()
            ref = its[k - 1]
            rg, ro = np.linalg.norm(mv(dm) - b), np.linalg.norm(mv(ref) - b)
            if k <= k_x:
                assert np.linalg.norm(dm - ref) <= tol_x * np.linalg.norm(ref), k
            if k <= k_r:
                assert abs(rg - ro) <= tol_x * ro, k
            assert rg <= prev * (1 + 1e-12) and abs(rg - ro) <= 2e-2 * ro, (k, rg, ro)
            prev = rg
    finally:
        mdl.close()


def test_autograd_function(c1):
    tem = _tem()
    mdl = _model(c1.s, c1.xi, c1.al, "fp64")
    try:
        m = _cuda(c1.m0).requires_grad_(True)
        d = tem.TemForward.apply(mdl, m)
        loss = (d * _cuda(c1.w)).sum()
        loss.backward()
        g = m.grad.cpu().numpy()
        assert np.linalg.norm(g - c1.jtw) <= 1e-9 * np.linalg.norm(c1.jtw)
    finally:
        mdl.close()


def test_errors_are_statuses(c1):
    tem = _tem()
    mdl = _model(c1.s, c1.xi, c1.al, "fp64")
    try:
        with pytest.raises(tem.TemError) as e:
            mdl.jvp(_cuda(c1.v))
        assert e.value.code == -6                      # TEM_ERR_STATE
        with pytest.raises(tem.TemError) as e:
            tem.tem_set_refine(mdl.ctx, 99, 1e-4, 0.0)
        assert e.value.code == -1
    finally:
        mdl.close()
    ctx = tem.tem_create(tem.TEM_FP64)
    try:
        tem.tem_mesh(ctx, c1.s.xyz, c1.s.tets, c1.s.sigma, c1.s.is_param)
        with pytest.raises(tem.TemError) as e:
            tem.tem_poles(ctx, np.array([1.0 + 1j]), np.ones((1, 4)))   # Re xi >= 0 refused
        assert e.value.code == -1
        bad = [np.array([0, 1, 2], dtype=np.int32)]                     # not a closed mesh path
        tem.tem_poles(ctx, c1.xi, c1.al)
        with pytest.raises(tem.TemError) as e:
            tem.tem_sources(ctx, bad, c1.s.rx)
        assert e.value.code == -7
    finally:
        tem.tem_destroy(ctx)


def _oracle_residuals(s, xi, mdl, m0):
    """||(K - xi_i M) g_i - f_x|| / ||f_x|| for every pole and transmitter, with
    the library's forward solutions g mapped to the oracle's unknowns and the
    oracle's own assembly of K, M(sigma) and f (FP64 SpMV)."""
    from oracle.fem import FEModel
    from oracle.survey import loop_source
    tem = _tem()
    g = tem.tem_export_forward(mdl.ctx)
    ev = tem.tem_export_dofs(mdl.ctx)
    fe = FEModel(s.xyz, s.tets)
    nv = fe.xyz.shape[0]
    okey = fe.edges[:, 0] * nv + fe.edges[:, 1]
    e = np.searchsorted(okey, ev[:, 0] * nv + ev[:, 1])
    odof = fe.dof[e]
    sig = s.sigma.copy()
    sig[s.is_param.astype(bool)] = np.exp(m0)
    M = fe.mass(sig)
    F = np.stack([loop_source(fe, lp) for lp in s.loops], axis=1)
    go = np.zeros((g.shape[0], fe.N, g.shape[2]), dtype=complex)
    go[:, odof, :] = g
    res = np.array([[np.linalg.norm(r) for r in ((fe.K - x * M) @ go[i] - F).T] for i, x in enumerate(xi)])
    return res / np.linalg.norm(F, axis=0)[None, :]


def _check_refined_vs_fp64(cfg, n=None):
    """Refined FP32 against the FP64 GPU path on a full-size configuration
    (the oracle cannot factor these in a test's time): data and J v per channel
    within 1e-6 (floored at 1e-4 of the channel's peak), J^T w within 1e-6;
    the FP64 path's adjoint identity <J v, w> = <v, J^T w>; and the residual of
    both paths' forward solutions against the oracle's own K, M and f."""
    s = inputs.make_config(cfg, n=n) if cfg == 4 else inputs.make_config(cfg)
    xi, al = inputs.load_rational(s.m, s.times)
    rng = np.random.default_rng(300 + cfg)
    m0 = s.log_sigma() + 0.1 * rng.standard_normal(s.n_param)
    v = rng.standard_normal(s.n_param)
    w = rng.standard_normal((len(s.loops), len(s.rx), len(s.times)))
    out = {}
    for prec in ("fp64", "fp32r"):
        mdl = _model(s, xi, al, prec)
        try:
            before = _prod_launches(mdl)
            mdl.factor(_cuda(m0))
            out[prec] = (mdl.forward().cpu().numpy(), mdl.jvp(_cuda(v)).cpu().numpy(),
                         mdl.jtvp(_cuda(w)).cpu().numpy())
            out[prec + "_res"] = _oracle_residuals(s, xi, mdl, m0).max()
            _assert_product_path(mdl, before, prec, True)
        finally:
            mdl.close()
    d64, jv64, jt64 = out["fp64"]
    d32, jv32, jt32 = out["fp32r"]
    assert abs(np.sum(jv64 * w) - np.sum(v * jt64)) <= 1e-11 * abs(np.sum(v * jt64))
    assert floored_err(d32, d64).max() <= TOL["fp32r"]
    assert floored_err(jv32, jv64).max() <= TOL_JV["fp32r"]
    assert np.linalg.norm(jt32 - jt64) <= TOL["fp32r"] * np.linalg.norm(jt64)
    # backward errors: the FP64 factor's solutions sit at ~1e-14 (C3, C4: <= 8.5e-15), the refined
    # pairs at <= 3.4e-11 (low poles; the floored gradient fields carry most of what is left)
    assert out["fp64_res"] <= 1e-13 and out["fp32r_res"] <= 1e-9, (out["fp64_res"], out["fp32r_res"])
    return out


def test_c3_refined_vs_fp64():
    """C3: 40^3 box, log-normal conductivity, 8 loops, 64 receivers, 32 times."""
    _check_refined_vs_fp64(3)


def test_c4_refined_vs_fp64():
    """C4, the benchmark's workload: 46^3 box (662,446 unknowns), two blocks,
    32 loops, 128 receivers, 40 times, 10 pole pairs, in the launch
    configuration bench.py times (default refinement, tensor-core products)."""
    _check_refined_vs_fp64(4)


@pytest.mark.parametrize("prec", ["fp64", "fp32r"])
def test_pivot_failure_is_a_status(c1, prec):
    """A NaN conductivity makes a pivot non-finite: tem_factor returns
    TEM_ERR_PIVOT (from the device status word, no fault), the context refuses
    solves until a good factorisation, and a good one restores parity."""
    tem = _tem()
    mdl = _model(c1.s, c1.xi, c1.al, prec)
    try:
        bad = c1.m0.copy()
        bad[len(bad) // 2] = np.nan
        with pytest.raises(tem.TemError) as e:
            mdl.factor(_cuda(bad))
        assert e.value.code == -3                      # TEM_ERR_PIVOT
        assert mdl.info()["last_pivot_front"] >= 0
        with pytest.raises(tem.TemError) as e:
            mdl.forward()
        assert e.value.code == -6                      # TEM_ERR_STATE: not factored
        mdl.factor(_cuda(c1.m0))
        assert mdl.info()["last_pivot_front"] == -1
        assert floored_err(mdl.forward().cpu().numpy(), c1.d).max() <= TOL[prec]
    finally:
        mdl.close()


def test_timeout_is_a_status(c1):
    """Bounded waits of the tensor-core solve kernel: with the wait limit cut
    to one poll the pipeline waits run out on purpose, the kernel drains its
    loads and MMAs and returns, and the call fails with TEM_ERR_TIMEOUT; with
    the default limit restored the same context solves correctly again."""
    tem = _tem()
    mdl = _model(c1.s, c1.xi, c1.al, "fp32r")
    try:
        mdl.factor(_cuda(c1.m0))
        tem.tem_set_wait_limit(mdl.ctx, 1, 1e-6)
        try:
            with pytest.raises(tem.TemError) as e:
                mdl.forward()
            assert e.value.code == -4                  # TEM_ERR_TIMEOUT
        finally:
            tem.tem_set_wait_limit(mdl.ctx, 1 << 26, 1.0)
        d = mdl.forward().cpu().numpy()
        assert floored_err(d, c1.d).max() <= TOL["fp32r"]
        jv = mdl.jvp(_cuda(c1.v)).cpu().numpy()
        assert floored_err(jv, c1.jv).max() <= TOL_JV["fp32r"]
    finally:
        mdl.close()


def test_c2_fronts_on_tensor_cores_or_fp32_pipes(c2):
    """The FP32 factorisation with its trailing updates as rank-128 tcgen05
    products (the default) and as rank-32 SIMT updates: both refine to the
    oracle's data, J v and J^T w at the refined tolerance, and the default
    factorisation launches the tensor-core kernel."""
    tem = _tem()
    for tcf in (1, 0):
        mdl = _model(c2.s, c2.xi, c2.al, "fp32r")
        try:
            tem.tem_set_tc_fronts(mdl.ctx, tcf)
            before = mdl.info()["tc_update_launches"]
            mdl.factor(_cuda(c2.m0))
            launched = mdl.info()["tc_update_launches"] - before
            assert (launched > 0) == bool(tcf), (tcf, launched)
            assert floored_err(mdl.forward().cpu().numpy(), c2.d).max() <= TOL["fp32r"]
            assert floored_err(mdl.jvp(_cuda(c2.v)).cpu().numpy(), c2.jv).max() <= TOL_JV["fp32r"]
            jtw = mdl.jtvp(_cuda(c2.w)).cpu().numpy()
            assert np.linalg.norm(jtw - c2.jtw) <= TOL["fp32r"] * np.linalg.norm(c2.jtw)
        finally:
            mdl.close()


def test_async_calls_capture_into_a_cuda_graph(c1):
    """Asynchronous mode: tem_forward and a 3-iteration tem_lsqr (all poles x
    transmitters, refinement and gradient-space corrections included) are
    captured on the context's stream into one CUDA graph; two replays give the
    synchronous results (the FWD21 atomics may reorder sums: 1e-9), and
    tem_status reports a clean device status after each."""
    tem = _tem()
    s = c1.s
    stream = torch.cuda.Stream()
    mdl = tem.Model(s.xyz, s.tets, s.sigma, s.is_param, s.loops, s.rx, c1.xi, c1.al,
                    precision=tem.TEM_FP32_REFINED, stream=stream.cuda_stream)
    try:
        d_obs = _cuda(c1.d * (1 + 0.03 * np.random.default_rng(3).standard_normal(c1.d.shape)))
        wd = 1.0 / (0.03 * d_obs.abs() + 1e-4 * d_obs.abs().max())
        m_ref = _cuda(s.log_sigma())
        m0 = _cuda(c1.m0)
        torch.cuda.synchronize()   # inputs made on the default stream, used on the context's
        with torch.cuda.stream(stream):
            mdl.factor(m0)
            d_ref = mdl.forward()
            dm_ref = mdl.lsqr(d_obs, wd, m_ref, 10.0, 3)
        stream.synchronize()
        assert floored_err(d_ref.cpu().numpy(), c1.d).max() <= TOL["fp32r"]
        tem.tem_set_async(mdl.ctx, 1)
        d_g = torch.full(mdl.shape, np.nan, dtype=torch.float64, device="cuda")
        dm_g = torch.full((mdl.P,), np.nan, dtype=torch.float64, device="cuda")
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            tem.tem_forward(mdl.ctx, d_g)
            tem.tem_lsqr(mdl.ctx, d_obs, wd, m_ref, 10.0, 3, dm_g)
        for _ in range(2):
            d_g.fill_(np.nan)
            dm_g.fill_(np.nan)
            graph.replay()
            tem.tem_status(mdl.ctx)
            d, dm = d_g.cpu().numpy(), dm_g.cpu().numpy()
            assert floored_err(d, d_ref.cpu().numpy()).max() <= 1e-9
            assert np.linalg.norm(dm - dm_ref.cpu().numpy()) <= 1e-9 * np.linalg.norm(dm_ref.cpu().numpy())
        tem.tem_set_async(mdl.ctx, 0)
    finally:
        mdl.close()


def _gn_inputs(c1):
    s = c1.s
    m_ref = s.log_sigma()
    # far from the start model; lambda 1 and 4 LSQR iterations keep the GN directions well
    # determined (two oracle runs whose data differ by 1e-13 stay 1e-13 apart), and lambda cools
    m_true = m_ref + 3.0 + 0.5 * np.random.default_rng(9).standard_normal(m_ref.shape)
    from oracle.tem import Oracle
    o = Oracle(s.xyz, s.tets, s.sigma, s.is_param, s.loops, s.rx, c1.xi, c1.al)
    o.set_model(m_true)
    d_true = o.forward()
    d_obs = d_true * (1 + 0.03 * np.random.default_rng(5).standard_normal(d_true.shape))
    wd = 1.0 / (0.03 * np.abs(d_obs) + 1e-4 * np.abs(d_obs).max())
    return o, m_ref, d_obs, wd


def test_gauss_newton_matches_oracle(c1):
    """Four Gauss-Newton iterations (Section 3.3: LSQR direction, Armijo line
    search, lambda cooling) on the library's calls (FP64: tem_factor,
    tem_forward, tem_lsqr, tem_gn_eval, tem_model_step) against the oracle's
    own GN loop on the same data: objective, misfit, step lengths, trial
    counts and lambda per iteration, and the final model.  The line-search
    branches themselves are pinned on the CPU (tests/test_gn_logic.py)."""
    from oracle.gn import gauss_newton
    from paper_2605_19951_gb300.gn import GaussNewton
    o, m_ref, d_obs, wd = _gn_inputs(c1)
    W = regulariser(c1.s.xyz, c1.s.tets, c1.s.is_param)
    m_o, hist_o = gauss_newton(o, W, d_obs, wd, m_ref, m_ref, lam=1.0, n_lsqr=4, n_iter=4, conv_tol=0.4)
    mdl = _model(c1.s, c1.xi, c1.al, "fp64")
    try:
        gn = GaussNewton(mdl, _cuda(d_obs), _cuda(wd), _cuda(m_ref), _cuda(m_ref), lam=1.0, n_lsqr=4,
                         conv_tol=0.4)
        hist = gn.run(4)
        m_g = gn.m.cpu().numpy()
    finally:
        mdl.close()
    assert len(hist) == len(hist_o) == 4
    assert hist_o[-1]["lam"] < hist_o[0]["lam"]                          # lambda cooled
    assert min(abs(x) for h in hist_o for x in h["margins"]) > 1e-3     # no Armijo test near its bound
    for a, b in zip(hist, hist_o):
        assert a["trials"] == b["trials"] and a["lam"] == b["lam"], (a, b)
        for k in ("phi0", "phi", "chi2", "eta"):
            assert abs(a[k] - b[k]) <= 1e-8 * abs(b[k]), (k, a[k], b[k])
    assert hist[-1]["phi"] < hist[0]["phi0"]
    assert np.linalg.norm(m_g - m_o) <= 1e-8 * np.linalg.norm(m_o)


def test_gauss_newton_checkpoint_resume(c1, tmp_path):
    """The GN state written after every iteration restarts a run: two
    iterations in one run equal one iteration, a checkpoint, and one more
    iteration resumed from it in a fresh context."""
    from paper_2605_19951_gb300.gn import GaussNewton
    _, m_ref, d_obs, wd = _gn_inputs(c1)
    args = (_cuda(d_obs), _cuda(wd), _cuda(m_ref))
    mdl = _model(c1.s, c1.xi, c1.al, "fp64")
    try:
        gn = GaussNewton(mdl, *args, _cuda(m_ref), lam=1.0, n_lsqr=4, conv_tol=0.4)
        gn.run(2)
        m_straight = gn.m.cpu().numpy()
    finally:
        mdl.close()
    ck = str(tmp_path / "gn_state.npz")
    mdl = _model(c1.s, c1.xi, c1.al, "fp64")
    try:
        GaussNewton(mdl, *args, _cuda(m_ref), lam=1.0, n_lsqr=4, conv_tol=0.4, checkpoint=ck).run(1)
    finally:
        mdl.close()
    mdl = _model(c1.s, c1.xi, c1.al, "fp64")
    try:
        gn = GaussNewton.resume(ck, mdl, *args, n_lsqr=4, conv_tol=0.4)
        assert gn.it == 1 and len(gn.history) == 1
        gn.run(1)
        assert gn.it == 2
        m_resumed = gn.m.cpu().numpy()
    finally:
        mdl.close()
    assert np.linalg.norm(m_resumed - m_straight) <= 1e-10 * np.linalg.norm(m_straight)


def test_uneven_batch_in_one_graph():
    """Configuration C5 at small sizes: five uneven models (6^3 .. 12^3 cubes,
    their own log-normal conductivity and 2-8 loops) through one tem_batch call
    and through one CUDA graph whose branches are the models' streams; both
    equal each model computed alone (forward and J^T w), which the single-model
    tests pin to the oracle; one model is also checked against the oracle."""
    tem = _tem()
    from paper_2605_19951_gb300.batch import Batch
    sizes = [6, 10, 8, 12, 7]
    surveys = [inputs.make_c5_model(i, n=n) for i, n in enumerate(sizes)]
    xi, al = inputs.load_rational(8, surveys[0].times)
    rng = np.random.default_rng(55)
    ms = [_cuda(s.log_sigma()) for s in surveys]
    ws = [_cuda(rng.standard_normal((len(s.loops), len(s.rx), len(s.times)))) for s in surveys]
    refs = []
    for s, m, w in zip(surveys, ms, ws):
        mdl = _model(s, xi, al, "fp32r")
        try:
            mdl.factor(m)
            refs.append((mdl.forward().cpu().numpy(), mdl.jtvp(w).cpu().numpy()))
        finally:
            mdl.close()
    o = Oracle(surveys[1].xyz, surveys[1].tets, surveys[1].sigma, surveys[1].is_param, surveys[1].loops,
               surveys[1].rx, xi, al)
    o.set_model(surveys[1].log_sigma())
    assert floored_err(refs[1][0], o.forward()).max() <= TOL["fp32r"]
    jt_o = o.jtvp(ws[1].cpu().numpy())
    assert np.linalg.norm(refs[1][1] - jt_o) <= TOL["fp32r"] * np.linalg.norm(jt_o)
    b = Batch(surveys, xi, al)
    try:
        for d, jtw in [b.run(ms, ws), b.capture(ms, ws), b.replay(), b.replay()]:
            for (dr, jr), dd, jj in zip(refs, d, jtw):
                assert floored_err(dd.cpu().numpy(), dr).max() <= 1e-8
                assert np.linalg.norm(jj.cpu().numpy() - jr) <= 1e-8 * np.linalg.norm(jr)
    finally:
        b.close()
