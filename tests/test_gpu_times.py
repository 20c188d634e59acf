"""New observation times on the device (tem_times, Section 2.3): the residues
alpha_i^[j] of the fixed poles are fitted on the GPU, and the response at the
new times comes from the factors of the old ones (the poles, hence the
shifted matrices, do not depend on the times).

Residue tolerance: both sides solve the same penalised least-squares problem
in FP64 with backward-stable methods (the device by Householder QR, the
oracle by LAPACK's SVD-based lstsq).  First-order perturbation theory of
least squares bounds the normwise relative gap of two such solutions, per
time, by cond(B) eps (2 + cond(B) |r| / (|B| |alpha|)); the test evaluates
that bound on the oracle's own matrix and residual (8 poles: ~1e-9, 10 poles:
~4e-8; a CPU Householder solve differs from lstsq by 2e-12 / 7e-11).
The data at new times: the tolerances of the parity tests (FP64 1e-9,
refined FP32 1e-6, floored per channel at 1e-4 of its peak over time).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import rational
from oracle.tem import Oracle
from paper_2605_19951_gb300 import inputs

TOL = {"fp64": 1e-9, "fp32r": 1e-6}
EPS = 2.0 ** -52


def _tem():
    from paper_2605_19951_gb300 import build, tem
    import os
    if not os.path.exists(tem.LIB_PATH):
        build.build()
    return tem


def _cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def floored_err(a, ref, floor=1e-4):
    peak = np.abs(ref).max(axis=2, keepdims=True)
    return np.abs(a - ref) / np.maximum(np.abs(ref), floor * peak)


def _model(s, xi, al, prec):
    tem = _tem()
    p = tem.TEM_FP64 if prec == "fp64" else tem.TEM_FP32_REFINED
    return tem.Model(s.xyz, s.tets, s.sigma, s.is_param, s.loops, s.rx, xi, al, precision=p)


def _ls_bound(xi, times, z, mu):
    """Per time: cond(B) eps (2 + cond(B) |r| / (|B| |x|)) for the oracle's
    penalised least-squares system."""
    Ba, Ea = rational._augmented(z, xi, np.exp(-np.outer(z, times)), mu)
    x, *_ = np.linalg.lstsq(Ba, Ea, rcond=None)
    sv = np.linalg.svd(Ba, compute_uv=False)
    cond, nb = sv[0] / sv[-1], sv[0]
    r = np.linalg.norm(Ba @ x - Ea, axis=0)
    return cond * EPS * (2.0 + cond * r / (nb * np.linalg.norm(x, axis=0)))


TIME_SETS = {
    "log40": inputs.times_log(40),
    "rand7": np.sort(np.random.default_rng(7).uniform(1e-5, 1e-2, 7)),
    "wide300": np.logspace(-6, -1, 300),
}


@pytest.mark.parametrize("m", [8, 10])
@pytest.mark.parametrize("tset", sorted(TIME_SETS))
def test_residue_fit_matches_oracle(m, tset):
    """Device residues equal the oracle's penalised least-squares fit within
    the perturbation bound, for the default sample set and another one."""
    s = inputs.make_config(1, m=m)
    xi, al = inputs.load_rational(m, s.times)
    t = TIME_SETS[tset]
    mdl = _model(s, xi, al, "fp64")
    try:
        for fit in ({}, {"n_z": 500, "z_min": 1e-1, "z_max": 1e8, "mu": 1e-3}):
            a_dev = mdl.set_times(t, **fit)
            z = rational.sample_points(fit.get("n_z", 2200), fit.get("z_min", 1e-2), fit.get("z_max", 1e9))
            mu = fit.get("mu", rational.MU)
            a_ref = rational.fit_alpha(xi, t, z=z, mu=mu)
            bound = _ls_bound(xi, t, z, mu)
            gap = np.linalg.norm(a_dev - a_ref, axis=0) / np.linalg.norm(a_ref, axis=0)
            assert a_dev.shape == (m, len(t))
            assert np.all(gap <= bound), (tset, fit, gap.max(), bound.min())
            assert mdl.info()["n_times"] == len(t)
    finally:
        mdl.close()


def test_stored_table_is_reproduced():
    """The stored tables were written by the oracle's fit with the default
    sample set: the device fit of the same times returns them."""
    s = inputs.make_config(1, m=10)
    xi, al = inputs.load_rational(10, inputs.times_log(40))
    mdl = _model(s, xi, inputs.load_rational(10, s.times)[1], "fp64")
    try:
        a_dev = mdl.set_times(inputs.times_log(40))
        bound = _ls_bound(xi, inputs.times_log(40), rational.sample_points(), rational.MU)
        gap = np.linalg.norm(a_dev - al, axis=0) / np.linalg.norm(al, axis=0)
        assert np.all(gap <= bound), gap.max()
    finally:
        mdl.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32r"])
def test_new_times_reuse_the_factors(prec):
    """Factor once with 16 times, switch to 40 other times: forward, J v,
    J^T w and LSQR at the new times equal the oracle's with its own residues
    for those times.  No tem_factor runs after the switch: the forward at
    the new times succeeds on the factors of the old ones (Section 2.3: the
    shifted matrices do not depend on the times)."""
    tem = _tem()
    s = inputs.make_config(1)
    xi, al = inputs.load_rational(s.m, s.times)
    rng = np.random.default_rng(11)
    m0 = s.log_sigma() + 0.2 * rng.standard_normal(s.n_param)
    t2 = np.logspace(-4.5, -2.5, 40)
    al2 = rational.fit_alpha(xi, t2)
    o = Oracle(s.xyz, s.tets, s.sigma, s.is_param, s.loops, s.rx, xi, al2)
    o.set_model(m0)
    d_ref = o.forward()
    v = rng.standard_normal(s.n_param)
    w = rng.standard_normal(d_ref.shape)
    mdl = _model(s, xi, al, prec)
    try:
        mdl.factor(_cuda(m0))
        mdl.forward()
        mdl.set_times(t2)
        with pytest.raises(tem.TemError, match="TEM_ERR_STATE"):
            mdl.jvp(_cuda(v))
        d = mdl.forward().cpu().numpy()
        assert d.shape == d_ref.shape
        assert floored_err(d, d_ref).max() <= TOL[prec]
        jv = mdl.jvp(_cuda(v)).cpu().numpy()
        assert floored_err(jv, o.jvp(v)).max() <= TOL[prec] * (10 if prec == "fp64" else 1)
        jtw_ref = o.jtvp(w)
        jtw = mdl.jtvp(_cuda(w)).cpu().numpy()
        assert np.linalg.norm(jtw - jtw_ref) <= TOL[prec] * np.linalg.norm(jtw_ref)
        # the LSQR work vectors follow the new data size
        wd = 1.0 / (0.03 * np.abs(d_ref) + 1e-4 * np.abs(d_ref).max())
        dm = mdl.lsqr(_cuda(d_ref * 1.01), _cuda(wd), _cuda(s.log_sigma()), 10.0, 3).cpu().numpy()
        assert dm.shape == (s.n_param,) and np.all(np.isfinite(dm))
    finally:
        mdl.close()


def test_times_arguments_are_checked():
    tem = _tem()
    s = inputs.make_config(1)
    xi, al = inputs.load_rational(s.m, s.times)
    mdl = _model(s, xi, al, "fp64")
    try:
        for bad in ([1e-3, -1e-3], [0.0], []):
            with pytest.raises(tem.TemError, match="TEM_ERR_ARG"):
                mdl.set_times(np.array(bad, dtype=np.float64))
        with pytest.raises(tem.TemError, match="TEM_ERR_ARG"):
            mdl.set_times(inputs.times_log(8), z_min=1e3, z_max=1e2)
        with pytest.raises(tem.TemError, match="too large"):   # refused before anything is allocated
            mdl.set_times(inputs.times_log(4096), n_z=1 << 20)
        assert mdl.info()["n_times"] == 16   # a refused call changes nothing
    finally:
        mdl.close()


@pytest.mark.parametrize("m", [8, 10])
def test_pole_fit_matches_the_stored_fit(m):
    """Poles fitted on the device by variable projection (tem_fit_poles) from
    the oracle fit's starting poles, on the same 40 times, sample set and
    penalty as the stored tables (which the oracle's fit wrote: scipy's
    trust-region least squares on the same objective).  A nonlinear fit has no
    unique answer, so the test compares what the method fixes: the device's
    objective is the oracle's objective evaluated at the device's poles, it is
    no worse than the stored poles' (within 0.1%), the approximant's max error
    against exp on the check grid is within 10% of the stored one's, the
    poles stay in Re < 0 < Im, and their imaginary parts (sorted) agree with
    the stored poles' within 1%."""
    tem = _tem()
    t = inputs.times_log(40)
    xs, _ = inputs.load_rational(m, t)
    xi, (f0, f1, steps) = tem.tem_fit_poles(rational.seed_poles(m), t, max_iter=400)
    f_ref = rational.vp_objective(xs, t)
    assert f1 < f0 and steps > 0
    assert abs(f1 - rational.vp_objective(xi, t)) <= 1e-8 * f1
    assert f1 <= 1.001 * f_ref, (f1, f_ref)
    e_dev = rational.max_error(xi, rational.fit_alpha(xi, t), t).max()
    e_ref = rational.max_error(xs, rational.fit_alpha(xs, t), t).max()
    assert e_dev <= 1.1 * e_ref, (e_dev, e_ref)
    assert np.all(xi.real < 0) and np.all(xi.imag > 0)
    im_dev, im_ref = np.sort(xi.imag), np.sort(xs.imag)
    assert np.all(np.abs(im_dev - im_ref) <= 1e-2 * im_ref), (im_dev, im_ref)


def test_pole_fit_arguments_are_checked():
    tem = _tem()
    t = inputs.times_log(8)
    for bad in (np.array([1.0 + 1.0j]), np.array([-1.0 - 1.0j])):   # Re >= 0, Im <= 0
        with pytest.raises(tem.TemError, match="TEM_ERR_ARG"):
            tem.tem_fit_poles(bad, t)
    with pytest.raises(tem.TemError, match="TEM_ERR_ARG"):
        tem.tem_fit_poles(rational.seed_poles(4), np.array([-1.0]))
    with pytest.raises(tem.TemError, match="too large"):
        tem.tem_fit_poles(rational.seed_poles(8), inputs.times_log(200), n_z=1 << 20)
