"""Autotuner of the assembly tree (supernode sizes) of a mesh.

The tree decides how the dense front work is tiled on the device: the
dissection's leaf size sets the leaf fronts (k up to the limit), and the
amalgamation threshold merges small separators into their parents.  Both
trade explicit zeros (more factor entries to stream) against fronts that
fill only part of the 128-lane tensor-core tiles; which side wins depends on
the mesh.  The tuner measures instead of modelling: for each candidate it
builds the context, factors, and times one forward and J.v + J^T.w pairs
with CUDA events, and scores a Gauss-Newton iteration by the paper's linear
cost model (factor + forward + n_lsqr pairs, Section 4, Fig. 10).  Results
are cached per mesh signature in a JSON file, so a mesh is tuned once.
"""
from __future__ import annotations

import hashlib
import json
import os
import statistics

import numpy as np

from . import tem

# (leaf_max, amalgamation threshold); the first entry is the library default
CANDIDATES = ((128, 32), (128, 0), (64, 32), (256, 32), (300, 48))


def signature(survey, precision, m):
    """Key of a tuning result: mesh, parameter cells, sources and precision."""
    h = hashlib.sha1()
    for a in (survey.xyz, survey.tets, survey.is_param):
        h.update(np.ascontiguousarray(a).tobytes())
    h.update(f"{len(survey.loops)}:{len(survey.rx)}:{precision}:{m}".encode())
    return h.hexdigest()[:20]


def gn_cost(factor_ms, forward_ms, pair_ms, n_lsqr=30):
    """One Gauss-Newton iteration by the linear cost model (ms)."""
    return factor_ms + forward_ms + n_lsqr * pair_ms


def _events(torch, fn, reps):
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def measure(survey, xi, alpha, leaf_max, amalg, precision=tem.TEM_FP32_REFINED, reps=2):
    """Factor, forward and pair times (ms) of one candidate tree, and its
    factor entries per pole."""
    import torch
    mdl = tem.Model(survey.xyz, survey.tets, survey.sigma, survey.is_param, survey.loops, survey.rx, xi, alpha,
                    precision=precision, leaf_max=leaf_max, amalgamation=amalg)
    try:
        m0 = torch.as_tensor(survey.log_sigma(), device="cuda")
        mdl.factor(m0)                       # first call allocates
        mdl.forward()
        gen = torch.Generator(device="cuda").manual_seed(7)
        v = torch.randn(mdl.P, dtype=torch.float64, device="cuda", generator=gen)
        w = torch.randn(*mdl.shape, dtype=torch.float64, device="cuda", generator=gen)
        mdl.jvp(v), mdl.jtvp(w)              # warm-up
        fac = _events(torch, lambda: mdl.factor(m0), reps)
        fwd = _events(torch, lambda: mdl.forward(), reps)
        pair = _events(torch, lambda: (mdl.jvp(v), mdl.jtvp(w)), reps)
        nnz = mdl.info()["nnz_l"]
    finally:
        mdl.close()
    return {"leaf_max": leaf_max, "amalgamation": amalg, "factor_ms": fac, "forward_ms": fwd, "pair_ms": pair,
            "nnz_l": nnz, "gn_ms": gn_cost(fac, fwd, pair)}


def tune(survey, xi, alpha, precision=tem.TEM_FP32_REFINED, candidates=CANDIDATES, cache=None,
         measure_fn=None):
    """Best (leaf_max, amalgamation) of the candidates for this survey by the
    measured Gauss-Newton cost; returns (best, table).  With `cache` (a JSON
    path) a survey already tuned is not measured again."""
    key = signature(survey, precision, len(xi))
    store = {}
    if cache and os.path.exists(cache):
        with open(cache) as fh:
            store = json.load(fh)
        if key in store:
            ent = store[key]
            return (ent["best"][0], ent["best"][1]), ent["table"]
    run = measure_fn or (lambda leaf, am: measure(survey, xi, alpha, leaf, am, precision))
    table = [run(leaf, am) for leaf, am in candidates]
    best = min(table, key=lambda r: r["gn_ms"])
    choice = (best["leaf_max"], best["amalgamation"])
    if cache:
        store[key] = {"best": list(choice), "table": table}
        tmp = cache + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(store, fh, indent=1)
        os.replace(tmp, cache)
    return choice, table
