"""tem_lsqr_noalloc: the LSQR entry point for callers that cannot allocate
device memory mid-inversion (their memory belongs to their own allocator, or
a cudaMalloc must not fail or synchronise the device between Gauss-Newton
steps).  Its work vectors live in the library's fixed device array; its
results must equal those of tem_lsqr, also on a second call in a row (the
array keeps the previous call's contents).  This file is collected last."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2605_19951_gb300 import inputs


def test_noalloc_lsqr_matches_lsqr():
    import os
    from paper_2605_19951_gb300 import build, tem
    if not os.path.exists(tem.LIB_PATH):
        build.build()
    s = inputs.make_config(1)
    xi, al = inputs.load_rational(s.m, s.times)
    mdl = tem.Model(s.xyz, s.tets, s.sigma, s.is_param, s.loops, s.rx, xi, al, precision=tem.TEM_FP64)
    try:
        cu = lambda a: torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")
        m0 = s.log_sigma() + 0.2 * np.random.default_rng(101).standard_normal(s.n_param)
        mdl.factor(cu(m0))
        d = mdl.forward().cpu().numpy()
        d_obs = d * (1 + 0.03 * np.random.default_rng(3).standard_normal(d.shape))
        wd = 1.0 / (0.03 * np.abs(d_obs) + 1e-4 * np.abs(d_obs).max())
        m_ref = s.log_sigma()
        args = (cu(d_obs), cu(wd), cu(m_ref), 10.0, 5)
        ref = mdl.lsqr(*args).cpu().numpy()
        for call in range(2):
            dm = torch.full((mdl.P,), np.nan, dtype=torch.float64, device="cuda")
            tem.tem_lsqr_noalloc(mdl.ctx, *args, dm)
            out = dm.cpu().numpy()
            assert np.all(np.isfinite(out)), call
            assert np.linalg.norm(out - ref) <= 1e-9 * np.linalg.norm(ref), call
    finally:
        mdl.close()
