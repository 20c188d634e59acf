"""Host logic of the assembly-tree autotuner (no GPU): the choice minimises
the measured Gauss-Newton cost (factor + forward + 30 pairs), results are
cached per mesh signature, and the signature separates different meshes and
source counts.  The measurements are scripted."""
import json

import numpy as np

from paper_2605_19951_gb300 import autotune, inputs, tem


def _fake(times):
    calls = []

    def run(leaf, am):
        calls.append((leaf, am))
        f, fw, p = times[(leaf, am)]
        return {"leaf_max": leaf, "amalgamation": am, "factor_ms": f, "forward_ms": fw, "pair_ms": p,
                "nnz_l": 0, "gn_ms": autotune.gn_cost(f, fw, p)}
    return run, calls


def test_choice_minimises_gauss_newton_cost(tmp_path):
    s = inputs.make_config(1)
    xi, al = inputs.load_rational(s.m, s.times)
    # (128, 0) has the fastest factor, (64, 32) the fastest pair: 30 pairs outweigh the factor
    times = {(128, 32): (100.0, 10.0, 20.0), (128, 0): (80.0, 10.0, 21.0), (64, 32): (140.0, 10.0, 18.0)}
    run, calls = _fake(times)
    cache = str(tmp_path / "trees.json")
    best, table = autotune.tune(s, xi, al, candidates=list(times), cache=cache, measure_fn=run)
    assert best == (64, 32) and len(calls) == 3
    assert [r["gn_ms"] for r in table] == [100 + 10 + 600, 80 + 10 + 630, 140 + 10 + 540]
    # cached: no second measurement, same answer
    run2, calls2 = _fake(times)
    assert autotune.tune(s, xi, al, candidates=list(times), cache=cache, measure_fn=run2)[0] == (64, 32)
    assert calls2 == []
    stored = json.load(open(cache))
    assert list(stored.values())[0]["best"] == [64, 32]


def test_signature_separates_meshes_and_sources():
    a, b = inputs.make_config(1), inputs.make_config(2, n=6)
    p = tem.TEM_FP32_REFINED
    assert autotune.signature(a, p, 8) == autotune.signature(inputs.make_config(1), p, 8)
    assert autotune.signature(a, p, 8) != autotune.signature(b, p, 8)
    assert autotune.signature(a, p, 8) != autotune.signature(a, tem.TEM_FP64, 8)
    assert autotune.signature(a, p, 8) != autotune.signature(a, p, 10)
    c = inputs.make_config(1)
    c.loops = c.loops + c.loops
    assert autotune.signature(a, p, 8) != autotune.signature(c, p, 8)


def test_batch_tunes_once_per_mesh_size(tmp_path):
    from paper_2605_19951_gb300 import autotune as at, batch
    surveys = [inputs.make_c5_model(i, n=n) for i, n in enumerate((12, 14, 12, 14, 12))]
    xi, al = inputs.load_rational(8, inputs.times_log(24))
    seen = []

    def fake_tune(s, xi_, al_, precision, cache=None, candidates=at.CANDIDATES):
        seen.append(s.n)
        return ((128, 32) if s.n == 12 else (64, 32)), []
    orig = at.tune
    at.tune = fake_tune
    try:
        trees, _ = batch.tune_trees(surveys, xi, al)
    finally:
        at.tune = orig
    assert sorted(seen) == [12, 14]
    assert trees == [(128, 32), (64, 32), (128, 32), (64, 32), (128, 32)]
    assert np.all([t in at.CANDIDATES for t in trees])
