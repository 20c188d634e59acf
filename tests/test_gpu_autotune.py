"""The assembly-tree autotuner on the GPU: it measures every candidate tree of
a mesh with the library's own factor and solves, picks the cheapest by the
Gauss-Newton cost model, and a batch built on the tuned trees gives the same
data and J^T w as per-model runs on the default trees (refined FP32 within
1e-6 per channel, floored at 1e-4 of the channel's peak; J^T w relative
2-norm 1e-6: two trees differ only in rounding order)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2605_19951_gb300 import inputs


def _cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def floored_err(a, ref, floor=1e-4):
    peak = np.abs(ref).max(axis=2, keepdims=True)
    return np.abs(a - ref) / np.maximum(np.abs(ref), floor * peak)


def test_autotuned_trees_in_a_batch(tmp_path):
    from paper_2605_19951_gb300 import autotune, batch, build, tem
    import os
    if not os.path.exists(tem.LIB_PATH):
        build.build()
    surveys = [inputs.make_c5_model(i, n=n) for i, n in enumerate((12, 13, 12))]
    xi, al = inputs.load_rational(8, inputs.times_log(24))
    cands = ((128, 32), (64, 0), (300, 48))
    cache = str(tmp_path / "trees.json")
    trees, tables = batch.tune_trees(surveys, xi, al, cache=cache, candidates=cands)
    assert sorted(tables) == [12, 13]
    for n, table in tables.items():
        assert len(table) == len(cands)
        for r in table:
            assert r["factor_ms"] > 0 and r["pair_ms"] > 0 and r["nnz_l"] > 0
        best = min(table, key=lambda r: r["gn_ms"])
        assert (best["leaf_max"], best["amalgamation"]) == trees[[s.n for s in surveys].index(n)]
    # the cache answers without measuring
    again, _ = batch.tune_trees(surveys, xi, al, cache=cache, candidates=cands)
    assert again == trees

    rng = np.random.default_rng(5)
    logs = [_cuda(s.log_sigma()) for s in surveys]
    ws = [_cuda(rng.standard_normal((len(s.loops), len(s.rx), len(s.times)))) for s in surveys]
    ref = []
    for s, lg, w in zip(surveys, logs, ws):
        mdl = tem.Model(s.xyz, s.tets, s.sigma, s.is_param, s.loops, s.rx, xi, al)
        try:
            mdl.factor(lg)
            ref.append((mdl.forward().cpu().numpy(), mdl.jtvp(w).cpu().numpy()))
        finally:
            mdl.close()
    b = batch.Batch(surveys, xi, al, trees=trees)
    try:
        d, jtw = b.capture(logs, ws)
        d, jtw = b.replay()
        for (d0, j0), d1, j1 in zip(ref, d, jtw):
            assert floored_err(d1.cpu().numpy(), d0).max() <= 1e-6
            j1 = j1.cpu().numpy()
            assert np.linalg.norm(j1 - j0) <= 1e-6 * np.linalg.norm(j0)
    finally:
        b.close()
