"""Uneven batches of independent surveys (configuration C5) in one CUDA graph.

Every model is a tem.Model on its own CUDA stream.  One tem_batch call issues
the requested operations of all models (factor, forward, J^T w) on their
streams without synchronising in between; Batch.capture records that call
into one CUDA graph whose branches are the models' streams (forked from and
joined into the capturing stream), so that a replay runs the models
concurrently, small and large alike, in one graph launch.
"""
from __future__ import annotations

from . import tem


class Batch:
    def __init__(self, surveys, xi, alpha, precision=tem.TEM_FP32_REFINED, trees=None):
        """trees: per survey (leaf_max, amalgamation) of its assembly tree, or
        None for the library defaults (see tune_trees)."""
        import torch
        self.torch = torch
        self.streams = [torch.cuda.Stream() for _ in surveys]
        trees = trees or [(0, None)] * len(surveys)
        self.models = [tem.Model(s.xyz, s.tets, s.sigma, s.is_param, s.loops, s.rx, xi, alpha,
                                 precision=precision, stream=st.cuda_stream, leaf_max=tr[0], amalgamation=tr[1])
                       for s, st, tr in zip(surveys, self.streams, trees)]
        self.graph = None

    def close(self):
        for m in self.models:
            m.close()

    @property
    def ctxs(self):
        return [m.ctx for m in self.models]

    def _outputs(self):
        t = self.torch
        d = [t.empty(m.shape, dtype=t.float64, device="cuda") for m in self.models]
        jtw = [t.empty(m.P, dtype=t.float64, device="cuda") for m in self.models]
        return d, jtw

    def run(self, log_sigma, w, ops=tem.TEM_BATCH_FACTOR | tem.TEM_BATCH_FORWARD | tem.TEM_BATCH_JTVP):
        """One synchronous tem_batch call; returns (data, J^T w) per model."""
        self.torch.cuda.synchronize()   # inputs made on other streams
        d, jtw = self._outputs()
        tem.tem_batch(self.ctxs, ops, log_sigma, d, w, jtw)
        return d, jtw

    def capture(self, log_sigma, w, ops=tem.TEM_BATCH_FACTOR | tem.TEM_BATCH_FORWARD | tem.TEM_BATCH_JTVP):
        """Record the batch into one CUDA graph (after one eager run for the
        allocations); the outputs are written by every replay."""
        t = self.torch
        self.run(log_sigma, w, ops)
        self.d, self.jtw = self._outputs()
        self._args = (log_sigma, w)
        for c in self.ctxs:
            tem.tem_set_async(c, 1)
        main = t.cuda.Stream()
        self.graph = t.cuda.CUDAGraph()
        with t.cuda.graph(self.graph, stream=main):
            fork = t.cuda.Event()
            fork.record(main)
            for st in self.streams:
                st.wait_event(fork)
            tem.tem_batch(self.ctxs, ops, log_sigma, self.d, w, self.jtw)
            for st in self.streams:
                done = t.cuda.Event()
                done.record(st)
                main.wait_event(done)
        return self.d, self.jtw

    def replay(self):
        self.graph.replay()
        for c in self.ctxs:
            tem.tem_status(c)
        return self.d, self.jtw


def tune_trees(surveys, xi, alpha, precision=tem.TEM_FP32_REFINED, cache=None, candidates=None):
    """Assembly tree of every survey chosen by the autotuner: one measured
    tuning per mesh size (surveys with the same number of cubes per side share
    the choice: the tree depends on the mesh, not on the conductivities or the
    loops).  Returns the per-survey (leaf_max, amalgamation) and the tables."""
    from . import autotune
    chosen, tables = {}, {}
    for s in surveys:
        if s.n in chosen:
            continue
        kw = {"cache": cache} if candidates is None else {"cache": cache, "candidates": candidates}
        chosen[s.n], tables[s.n] = autotune.tune(s, xi, alpha, precision, **kw)
    return [chosen[s.n] for s in surveys], tables
