"""Host-side plumbing of the multi-GPU path: LPT partition of the haloes and
the final gather, run as two gloo ranks on the CPU.  Each rank computes its
share with the oracle in place of its GPU; the gathered catalogue must be
the one a single process computes."""
import os
import socket

import numpy as np
import pytest

from oracle import ahf_oracle as O
from paper_0904_3662_gb300 import shard, synth

REC = np.dtype([("n_bound", "<i8"), ("n_iter", "<i4"), ("m_vir", "<f8"), ("r_vir", "<f8")])


def _oracle_compute(pop):
    def compute(idx):
        out = O.unbind_population(pop, O.Params(), halos=[int(h) for h in idx])
        rec = np.zeros(len(idx), dtype=REC)
        bound = []
        for k, h in enumerate(idx):
            o = out[int(h)]
            rec[k] = (len(o["order"]), o["n_iter"], o["m_vir"], o["r_vir"])
            bound.append(np.asarray(o["bound_idx"], dtype=np.int64))
        return rec, bound
    return compute


def test_lpt_partition_properties():
    rng = np.random.default_rng(3)
    counts = synth.powerlaw_counts(rng, 500, 100, 100_000)
    for n in (1, 2, 3, 8):
        parts = shard.lpt_partition(counts, n)
        allh = np.sort(np.concatenate(parts))
        np.testing.assert_array_equal(allh, np.arange(len(counts)))
        ld = shard.loads(counts, parts)
        # Graham's bound for greedy list scheduling
        assert max(ld) <= counts.sum() / n + counts.max()
        assert shard.lpt_partition(counts, n)[0].tolist() == parts[0].tolist()
    # a dominant halo is alone on its rank
    counts2 = np.array([10_000_000] + [1000] * 50)
    parts = shard.lpt_partition(counts2, 4)
    owner = [r for r, p in enumerate(parts) if 0 in p][0]
    assert parts[owner].tolist() == [0]
    with pytest.raises(ValueError):
        shard.lpt_partition(counts, 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, result_path):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        pop = synth.halo_batch(seed=61, n_halos=9, n_lo=100, n_hi=3_000)
        got = shard.run_sharded(pop.n_halos, pop.count, _oracle_compute(pop), rank, world)
        if rank == 0:
            rec, bound = got
            np.save(result_path + ".rec.npy", rec)
            np.save(result_path + ".len.npy", np.array([len(b) for b in bound]))
            np.save(result_path + ".flat.npy", np.concatenate(bound))
        else:
            assert got is None
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_gather_the_single_process_catalogue(tmp_path):
    import torch.multiprocessing as mp
    path = str(tmp_path / "cat")
    mp.start_processes(_rank_main, args=(2, _free_port(), path), nprocs=2, join=True, start_method="spawn")
    rec = np.load(path + ".rec.npy")
    lens = np.load(path + ".len.npy")
    flat = np.load(path + ".flat.npy")
    pop = synth.halo_batch(seed=61, n_halos=9, n_lo=100, n_hi=3_000)
    ref_rec, ref_bound = shard.run_sharded(pop.n_halos, pop.count, _oracle_compute(pop), 0, 1)
    np.testing.assert_array_equal(rec, ref_rec)
    np.testing.assert_array_equal(lens, [len(b) for b in ref_bound])
    np.testing.assert_array_equal(flat, np.concatenate(ref_bound))
