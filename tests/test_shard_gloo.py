"""The multi-rank split on CPU (gloo, world size 2): views dealt over the
ranks cover every view once, each rank's FP64 oracle gradient of its own
views summed by all-reduce equals the oracle gradient of all views, and the
step time is the slowest rank's."""

import os

import numpy as np
import pytest

import synth
from tests import helpers as H

torch = pytest.importorskip("torch")


def _scene():
    views = [synth.scenes.pinhole((0.4, 0.3, -3.2), 64, 48), synth.scenes.pinhole((-2.6, -0.5, -1.8), 40, 56),
             synth.scenes.pinhole((2.0, 1.2, 2.5), 32, 24), synth.scenes.pinhole((0.1, 2.9, 1.0), 48, 48)]
    return synth.make_scene([(24, 24, 0, 0, 0)], (24, 24), 0.6, views, sh_degree=1, seed=31, log_scale=(-3.0, 0.5))


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    import oracle as orc
    from paper_2602_23040_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sc = _scene()
    mine = shard.shard_views(sc.views, rank, world)
    sub = synth.scenes.Scene(**{**sc.__dict__, "views": [sc.views[i] for i in mine]})
    w = np.random.default_rng(7).standard_normal(3 * sc.pixels)
    off = np.concatenate([[0], np.cumsum([3 * v.width * v.height for v in sc.views])])
    w_sub = np.concatenate([w[off[i]:off[i + 1]] for i in mine]) if mine else np.zeros(0)
    o = orc.forward(sub)
    g = torch.from_numpy(orc.backward(sub, o, w_sub)["grad_soa"].copy())
    shard.allreduce_texel_grads(g)
    t = shard.max_over_ranks(float(rank + 1))
    np.save(os.path.join(out_dir, f"g{rank}.npy"), g.numpy())
    np.save(os.path.join(out_dir, f"v{rank}.npy"), np.array(mine + [-1]))
    np.save(os.path.join(out_dir, f"t{rank}.npy"), np.array([t]))
    dist.destroy_process_group()


def test_shard_views_partition():
    from paper_2602_23040_gb300 import shard
    sc = synth.config_scene(3)
    for world in (1, 2, 3, 8):
        parts = [shard.shard_views(sc.views, r, world) for r in range(world)]
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sc.views)))
        px = [sum(sc.views[i].width * sc.views[i].height for i in p) for p in parts]
        assert max(px) - min(px) <= max(v.width * v.height for v in sc.views)


def test_gradient_allreduce_over_two_gloo_ranks(orc, tmp_path):
    mp = torch.multiprocessing.get_context("spawn")
    port = 29500 + (os.getpid() % 1000)
    procs = [mp.Process(target=_worker, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    sc = _scene()
    w = np.random.default_rng(7).standard_normal(3 * sc.pixels)
    o = orc.forward(sc)
    full = orc.backward(sc, o, w)["grad_soa"]
    for r in range(2):
        g = np.load(tmp_path / f"g{r}.npy")
        assert H.rel_err(g, full) < 1e-12
        assert float(np.load(tmp_path / f"t{r}.npy")[0]) == 2.0
    v0, v1 = (set(np.load(tmp_path / f"v{r}.npy").tolist()) - {-1} for r in range(2))
    assert v0.isdisjoint(v1) and v0 | v1 == set(range(len(sc.views)))
