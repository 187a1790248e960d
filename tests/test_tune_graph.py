"""Autotuner cache logic (CPU) and on the GPU: the sweep picks a measured
option and records it; the capturable batched entry point replayed from a
CUDA graph with new iso-values equals the synchronous batched call."""
import json

import pytest
import torch

from paper_2004_08475_b300 import tune


def test_best_options_default_and_nearest(tmp_path):
    p = str(tmp_path / "c.json")
    assert tune.best_options(1 << 20, 4, gpu="G", path=p) == tune.DEFAULT
    cache = {tune.bucket_key(1 << 20, 4, "G"): {"best": {"log2_brick": 2, "load_factor": 0.25, "block_size": 128}}}
    with open(p, "w") as f:
        json.dump(cache, f)
    assert tune.best_options(1 << 20, 4, gpu="G", path=p)["log2_brick"] == 2
    assert tune.best_options(1 << 22, 4, gpu="G", path=p)["block_size"] == 128   # nearest bucket
    assert tune.best_options(1 << 20, 3, gpu="G", path=p) == tune.DEFAULT       # other level count


@pytest.mark.gpu
def test_tune_sweep_records(tmp_path):
    from paper_2004_08475_b300 import synth
    x, l, s, iso, info = synth.octree_gaussians(seed=41, roots=5, root_level=4, device="cuda")
    p = str(tmp_path / "c.json")
    r = tune.tune(x, l, s, iso, space={"log2_brick": (2, 3), "load_factor": (0.5,), "block_size": (256,)},
                  reps=1, path=p)
    assert r["best"]["log2_brick"] in (2, 3) and r["best_ms"] > 0 and len(r["table"]) == 2
    assert tune.best_options(info["n"], int(l.max()) + 1, path=p) == r["best"]


@pytest.mark.gpu
def test_graph_replay_equals_sync_batch():
    from paper_2004_08475_b300 import amriso, synth
    from tests.parity import canonical
    x, l, s, iso, info = synth.octree_gaussians(seed=42, roots=5, root_level=4, device="cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = amriso.AmrContext(0, stream)
        ctx.upload(x, l, s)
        ctx.build_locator()
        ctx.dual_cells()
        out = torch.empty((1 << 20, 3, 3), dtype=torch.float32, device="cuda")
        d_iso = torch.empty(4, dtype=torch.float32, device="cuda")
        d_off = torch.zeros(5, dtype=torch.int64, device="cuda")
        d_iso.copy_(torch.tensor([iso, iso * 0.8, iso * 1.1, iso * 0.6]))
        ctx.iso_batch_async(d_iso, out, d_off)
        stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            ctx.iso_batch_async(d_iso, out, d_off)
        for isos in ([iso * 0.7, iso, iso * 1.2, iso * 0.9], [iso * 0.5, iso * 0.55, iso * 0.6, iso * 0.65]):
            d_iso.copy_(torch.tensor(isos))
            g.replay()
            stream.synchronize()
            offs = d_off.cpu().tolist()
            ref, roffs = ctx.iso_batch(isos)
            assert offs == roffs.tolist()
            for k in range(4):
                a = out[offs[k]:offs[k + 1]].cpu().numpy()
                b = ref[roffs[k]:roffs[k + 1]].cpu().numpy()
                assert (canonical(a) == canonical(b)).all()
