"""Pole sharding with the library on the GPU (Algorithm 1: every pole's
shifted system is independent).  Two ranks, spawned as processes on this
GPU, each build a context with their own poles and residue rows; forward,
J v and J^T w are each the rank's partial sum plus one all-reduce (gloo, on
the host: the ranks' kernels never wait on one another).  The assembled
results equal a single context over all poles up to rounding: the pole sums
are taken in another order, and the sweeps' atomic updates make every run's
rounding differ, which the residue sums amplify.  So the parity tests'
tolerances apply: data and J^T w 1e-9 (FP64) / 1e-6 (refined FP32), J v
1e-8 / 1e-6 (per channel floored at 1e-4 of the peak for the data and J v,
relative 2-norm for J^T w)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2605_19951_gb300 import inputs

TOL = {"fp64": 1e-9, "fp32r": 1e-6}
TOL_JV = {"fp64": 1e-8, "fp32r": 1e-6}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _inputs(seed=21):
    s = inputs.make_config(2)
    xi, al = inputs.load_rational(s.m, s.times)
    rng = np.random.default_rng(seed)
    m0 = s.log_sigma() + 0.2 * rng.standard_normal(s.n_param)
    v = rng.standard_normal(s.n_param)
    w = rng.standard_normal((len(s.loops), len(s.rx), len(s.times)))
    return s, xi, al, m0, v, w


def _products(mdl, m0, v, w):
    cu = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    mdl.factor(cu(m0))
    return mdl.forward(), mdl.jvp(cu(v)), mdl.jtvp(cu(w))


def _rank_main(rank, world, port, prec, out):
    import torch.distributed as dist
    from paper_2605_19951_gb300 import tem
    from paper_2605_19951_gb300.shard import ShardedOperator, local_poles
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        s, xi, al, m0, v, w = _inputs()
        xl, al_l = local_poles(xi, al, rank, world)
        p = tem.TEM_FP64 if prec == "fp64" else tem.TEM_FP32_REFINED
        mdl = tem.Model(s.xyz, s.tets, s.sigma, s.is_param, s.loops, s.rx, xl, al_l, precision=p)
        try:
            cu = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
            mdl.factor(cu(m0))
            op = ShardedOperator(mdl, dist, device="cpu")   # gloo reduces host tensors
            d, jv, jtw = (x.numpy() for x in (op.forward(), op.jvp(cu(v)), op.jtvp(cu(w))))
        finally:
            mdl.close()
        if rank == 0:
            np.savez(out, d=d, jv=jv, jtw=jtw)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("prec", ["fp64", "fp32r"])
def test_pole_sharded_library_matches_one_context(prec, tmp_path):
    import torch.multiprocessing as mp
    from paper_2605_19951_gb300 import build, tem
    if not os.path.exists(tem.LIB_PATH):
        build.build()
    out = str(tmp_path / "sharded.npz")
    mp.start_processes(_rank_main, args=(2, _free_port(), prec, out), nprocs=2, join=True, start_method="spawn")
    got = np.load(out)
    s, xi, al, m0, v, w = _inputs()
    p = tem.TEM_FP64 if prec == "fp64" else tem.TEM_FP32_REFINED
    mdl = tem.Model(s.xyz, s.tets, s.sigma, s.is_param, s.loops, s.rx, xi, al, precision=p)
    try:
        d, jv, jtw = (x.cpu().numpy() for x in _products(mdl, m0, v, w))
    finally:
        mdl.close()

    def floored(a, ref):
        peak = np.abs(ref).max(axis=2, keepdims=True)
        return (np.abs(a - ref) / np.maximum(np.abs(ref), 1e-4 * peak)).max()
    assert floored(got["d"], d) <= TOL[prec]
    assert floored(got["jv"], jv) <= TOL_JV[prec]
    assert np.linalg.norm(got["jtw"] - jtw) <= TOL[prec] * np.linalg.norm(jtw)
