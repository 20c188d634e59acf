"""Pole sharding on CPU ranks (gloo, world size 2 and 3): each rank runs the
oracle's shifted solves for its own poles only, and one all-reduce per
product assembles forward, J v and J^T w; the results must equal the
single-process oracle over all poles (only the order of the pole sums
differs).  Section 2.3 (independent shifted systems), Algorithm 1."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2605_19951_gb300 import inputs
from paper_2605_19951_gb300.shard import local_poles, pole_partition


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle.tem import Oracle
        from paper_2605_19951_gb300.shard import ShardedOperator
        s = inputs.make_config(1)
        xi, al = inputs.load_rational(s.m, s.times)
        xl, al_l = local_poles(xi, al, rank, world)
        o = Oracle(s.xyz, s.tets, s.sigma, s.is_param, s.loops, s.rx, xl, al_l, threads=1)
        rng = np.random.default_rng(11)
        m0 = s.log_sigma() + 0.2 * rng.standard_normal(s.n_param)
        o.set_model(m0)
        v = rng.standard_normal(s.n_param)
        w = rng.standard_normal(o.forward_shape)
        op = ShardedOperator(o, dist)
        d, jv, jtw = op.forward().numpy(), op.jvp(v).numpy(), op.jtvp(w).numpy()
        np.savez(os.path.join(out_dir, f"r{rank}.npz"), d=d, jv=jv, jtw=jtw)
    finally:
        dist.destroy_process_group()


def test_pole_partition():
    assert pole_partition(10, 3) == [[0, 1, 2], [3, 4, 5, 6], [7, 8, 9]]
    for m in range(1, 13):
        for world in range(1, m + 1):
            parts = pole_partition(m, world)
            assert sorted(sum(parts, [])) == list(range(m))
            assert max(map(len, parts)) - min(map(len, parts)) <= 1
    with pytest.raises(ValueError):
        pole_partition(2, 3)


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_products_equal_single_process(tmp_path, world):
    from oracle.tem import Oracle
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    s = inputs.make_config(1)
    xi, al = inputs.load_rational(s.m, s.times)
    o = Oracle(s.xyz, s.tets, s.sigma, s.is_param, s.loops, s.rx, xi, al)
    rng = np.random.default_rng(11)
    o.set_model(s.log_sigma() + 0.2 * rng.standard_normal(s.n_param))
    v = rng.standard_normal(s.n_param)
    w = rng.standard_normal(o.forward_shape)
    ref = {"d": o.forward(), "jv": o.jvp(v), "jtw": o.jtvp(w)}
    for r in range(world):
        got = np.load(tmp_path / f"r{r}.npz")
        for k in ("d", "jv", "jtw"):
            # the pole sums cancel (residue sums), so summation order shows at ~1e-12 of the terms
            scale = np.abs(ref[k]).max()
            assert np.abs(got[k] - ref[k]).max() <= 1e-12 * scale, (r, k)
