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
    def __init__(self, surveys, xi, alpha, precision=tem.TEM_FP32_REFINED):
        import torch
        self.torch = torch
        self.streams = [torch.cuda.Stream() for _ in surveys]
        self.models = [tem.Model(s.xyz, s.tets, s.sigma, s.is_param, s.loops, s.rx, xi, alpha,
                                 precision=precision, stream=st.cuda_stream)
                       for s, st in zip(surveys, self.streams)]
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
