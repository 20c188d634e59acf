"""Control logic of the Gauss-Newton driver (Section 3.3) on the CPU.

The library's driver (paper_2605_19951_gb300.gn) and the oracle's loop
(oracle.gn) run on one small analytic nonlinear problem, d(m) = B exp(m),
whose products both drivers see identically: the driver through a stand-in
for the library calls it makes (factor, forward, LSQR, tem_gn_eval,
tem_model_step), the oracle through its own interface.  The problem starts far
from the truth with little regularisation, so the line search backtracks,
takes quadratic-model steps, hits the eta lower bound, and lambda cools; the
two histories and models must agree, and a run resumed from a checkpoint must
continue the same trajectory."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.gn import gauss_newton
from oracle.inversion import lsqr as oracle_lsqr
from paper_2605_19951_gb300 import gn as gn_mod

rng = np.random.default_rng(4)
P, ND = 6, 12
B = rng.uniform(0.5, 1.5, (ND, P))
W = np.diff(np.eye(P), axis=0)                  # first differences (a chain regulariser)
M_TRUE = np.log(np.array([3.0, 0.2, 5.0, 1.0, 0.05, 2.0]))
D_OBS = (B @ np.exp(M_TRUE)).reshape(1, 3, 4)


def _d_obs(scale):
    return (B @ np.exp(scale * M_TRUE)).reshape(1, 3, 4)
WD = np.full(D_OBS.shape, 10.0)
M_REF = np.zeros(P)


class Problem:
    """Forward, J v, J^T w of d(m) = B exp(m) at the current model."""

    forward_shape = D_OBS.shape

    def set_model(self, m):
        self.m = np.array(m, dtype=np.float64)

    def forward(self):
        return (B @ np.exp(self.m)).reshape(D_OBS.shape)

    def jvp(self, v):
        return (B @ (np.exp(self.m) * v)).reshape(D_OBS.shape)

    def jtvp(self, w):
        return np.exp(self.m) * (B.T @ np.asarray(w).ravel())


class FakeModel:
    """What the driver calls on a tem.Model, on the analytic problem."""

    ctx = "fake"

    def __init__(self):
        self.p = Problem()

    def factor(self, m):
        self.p.set_model(m.numpy())

    def forward(self):
        return torch.as_tensor(self.p.forward())

    def lsqr(self, d_obs, wd, m_ref, lam, n_iter):
        from oracle.inversion import gn_operator, gn_rhs
        w = wd.numpy().ravel()
        mv, rmv = gn_operator(self.p, W, w, lam)
        b = gn_rhs(self.p.forward(), d_obs.numpy(), w, W, self.p.m, m_ref.numpy(), lam)
        return torch.as_tensor(oracle_lsqr(mv, rmv, b, n_iter)[0])


@pytest.fixture
def fake_calls(monkeypatch):
    model = FakeModel()

    def gn_eval(ctx, d_obs, wd, m_ref, lam, dm=None, grad=None):
        p = model.p
        r = (wd.numpy() * (p.forward() - d_obs.numpy())).ravel()
        wv = W @ (p.m - m_ref.numpy())
        out = np.array([0.5 * r @ r + lam * 0.5 * wv @ wv, 0.5 * r @ r, 0.5 * wv @ wv, r @ r / r.size, 0.0])
        if grad is not None:
            g = p.jtvp(wd.numpy().ravel() * r) + lam * (W.T @ wv)
            grad.copy_(torch.as_tensor(g))
            if dm is not None:
                out[4] = g @ dm.numpy()
        return out

    def model_step(ctx, m, dm, eta, out):
        out.copy_(m + eta * dm)

    monkeypatch.setattr(gn_mod.tem, "tem_gn_eval", gn_eval)
    monkeypatch.setattr(gn_mod.tem, "tem_model_step", model_step)
    return model


def _args(scale=1.0):
    return torch.as_tensor(_d_obs(scale)), torch.as_tensor(WD), torch.as_tensor(M_REF)


@pytest.mark.parametrize("scale", [2.0, 3.0])
def test_driver_matches_oracle_loop(fake_calls, scale):
    """scale 2: a chain of halvings, then a quadratic-model step; scale 3: the
    eta lower bound after four halvings, then lambda cooling."""
    kw = dict(lam=1e-4, n_lsqr=6, conv_tol=0.3)
    m_o, hist_o = gauss_newton(Problem(), W, _d_obs(scale), WD, M_REF, M_REF, n_iter=6, **kw)
    gn = gn_mod.GaussNewton(fake_calls, *_args(scale), torch.as_tensor(M_REF), **kw)
    hist = gn.run(6)
    trials = [h["trials"] for h in hist_o]
    etas = [h["eta"] for h in hist_o]
    assert max(trials) >= 4                                        # backtracked several times
    if scale == 2.0:
        assert any(e not in (1.0, 0.5, 0.25, 0.125, 1.0 / 16) for e in etas)   # a quadratic-model step
    else:
        assert any(e == 1.0 / 16 for e in etas)                    # the eta lower bound
        assert hist_o[-1]["lam"] < hist_o[0]["lam"]                # lambda cooled
    assert len(hist) == len(hist_o)
    for a, b in zip(hist, hist_o):
        assert a["trials"] == b["trials"] and a["lam"] == b["lam"] and a["eta"] == pytest.approx(b["eta"], rel=1e-12)
        assert a["phi"] == pytest.approx(b["phi"], rel=1e-12) and a["chi2"] == pytest.approx(b["chi2"], rel=1e-12)
    assert np.allclose(gn.m.numpy(), m_o, rtol=1e-12, atol=1e-14)
    assert hist[-1]["phi"] < hist[0]["phi0"]


def test_resume_continues_the_trajectory(fake_calls, tmp_path):
    kw = dict(lam=1e-4, n_lsqr=6, conv_tol=0.3)
    straight = gn_mod.GaussNewton(fake_calls, *_args(3.0), torch.as_tensor(M_REF), **kw)
    straight.run(4)
    ck = str(tmp_path / "state.npz")
    first = gn_mod.GaussNewton(fake_calls, *_args(3.0), torch.as_tensor(M_REF), checkpoint=ck, **kw)
    first.run(2)
    resumed = gn_mod.GaussNewton.resume(ck, fake_calls, *_args(3.0), n_lsqr=6, conv_tol=0.3)
    assert resumed.it == 2 and resumed.lam == first.lam
    resumed.run(2)
    assert [h["phi"] for h in resumed.history] == pytest.approx([h["phi"] for h in straight.history], rel=1e-12)
    assert np.allclose(resumed.m.numpy(), straight.m.numpy(), rtol=1e-12, atol=1e-14)
