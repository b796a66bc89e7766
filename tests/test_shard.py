"""Host logic of the multi-rank path (CPU, gloo): sample ranges per rank and the
one FP64 all-reduce that combines per-field results (Eqs. 18, 23)."""
import os
import socket

import numpy as np
import pytest

from paper_1612_09517_gb300 import shard

torch = pytest.importorskip("torch")


def _stats(phi_s, phi_t, surv):
    """Per-field block as rp_yields reports it: means, SE with M - 1, mean survival."""
    M = phi_s.shape[1]
    se = lambda x: np.std(x, axis=1, ddof=1) / np.sqrt(M)
    return np.stack([phi_s.mean(1), phi_t.mean(1), se(phi_s), se(phi_t), surv.mean(1)], axis=1)


def _samples(n_fields=7, M=53, seed=1234):
    rng = np.random.default_rng(seed)
    phi_s = rng.uniform(0.2, 0.8, (n_fields, M))
    surv = rng.uniform(0.0, 0.1, (n_fields, M))
    phi_t = 1.0 - surv - phi_s
    return phi_s, phi_t, surv


def test_sample_ranges_partition_the_samples():
    for M in range(0, 40):
        for world in range(1, 6):
            got = [shard.sample_range(M, world, r) for r in range(world)]
            idx = np.concatenate([np.arange(o, o + c) for o, c in got]) if M else np.array([])
            assert np.array_equal(idx, np.arange(M))
            counts = [c for _, c in got]
            assert max(counts) - min(counts) <= 1
    with pytest.raises(ValueError):
        shard.sample_range(10, 2, 2)


@pytest.mark.parametrize("world", [1, 2, 3, 5])
def test_combined_shards_equal_the_single_run(world):
    phi_s, phi_t, surv = _samples()
    M = phi_s.shape[1]
    total = np.zeros((phi_s.shape[0], 5))
    for r in range(world):
        o, c = shard.sample_range(M, world, r)
        sl = slice(o, o + c)
        total += shard.field_sums(_stats(phi_s[:, sl], phi_t[:, sl], surv[:, sl]), c)
    got = shard.combine(total, M)
    assert np.allclose(got, _stats(phi_s, phi_t, surv), rtol=1e-12, atol=1e-15)


def test_field_sums_need_two_samples():
    with pytest.raises(ValueError):
        shard.field_sums(np.zeros((1, 5)), 1)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        phi_s, phi_t, surv = _samples()
        M = phi_s.shape[1]
        o, c = shard.sample_range(M, world, rank)
        sl = slice(o, o + c)
        out_g, M_g = shard.allreduce_yields(_stats(phi_s[:, sl], phi_t[:, sl], surv[:, sl]), c)
        t = shard.max_over_ranks([1.0 + rank, 5.0 - rank])
        np.savez(os.path.join(outdir, f"rank{rank}.npz"), out=out_g, M=M_g, t=t)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_combine_like_one(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    ref = _stats(*_samples())
    for r in range(world):
        d = np.load(tmp_path / f"rank{r}.npz")
        assert int(d["M"]) == 53
        assert np.allclose(d["out"], ref, rtol=1e-12, atol=1e-15)
        assert np.array_equal(d["t"], [2.0, 5.0])
