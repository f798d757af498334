"""Multi-rank split of one realization (Section II.B): scatterer shards per rank and one
sum-reduce of the spectra, run as 2 and 3 CPU ranks over gloo (the oracle computes each rank's
partial spectra, so no GPU is needed)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_shard_range_covers_disjoint_aligned():
    from paper_2408_11472_gb300.sharding import block_scatterers, shard_range
    a = block_scatterers()
    assert a > 0 and a % 32 == 0
    for n in (0, 1, a - 1, a, 5 * a + 17, 4194304):
        for world in (1, 2, 3, 8):
            spans = [shard_range(n, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            for (s0, e0), (s1, e1) in zip(spans, spans[1:]):
                assert e0 == s1 and s0 <= e0
            for s, e in spans:
                assert (s % a == 0 or s == n) and (e % a == 0 or e == n)
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)


def _rank_main(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    import oracle
    import scenegen as sg
    from paper_2408_11472_gb300.sharding import sharded_spectra

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        c = sg.config(1)
        rd, pf, fp = c["radar"], c["platform"], c["fast"]
        sc = sg.sea_surface(80, 13)
        orc = oracle.Oracle(threads=2)

        def partial(start, stop):
            part = {k: (v[start:stop] if isinstance(v, np.ndarray) else v) for k, v in sc.items()}
            T = orc.doppler_spectra(rd, pf, part, 31, 3, fp.n_fast, fp.n_doppler)
            return torch.from_numpy(np.ascontiguousarray(T))

        T = sharded_spectra(partial, sc["x"].size, world, rank)
        if rank == 0:
            np.save(out_path, T.numpy())
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_tile_split_equals_single_realization(tmp_path):
    import oracle
    import scenegen as sg

    out = str(tmp_path / "T.npy")
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    T2 = np.load(out)
    c = sg.config(1)
    sc = sg.sea_surface(80, 13)
    T1 = oracle.Oracle().doppler_spectra(c["radar"], c["platform"], sc, 31, 3, c["fast"].n_fast,
                                         c["fast"].n_doppler)
    assert np.abs(T1).max() > 0
    np.testing.assert_allclose(T2, T1, rtol=0, atol=1e-12 * np.abs(T1).max())


def test_three_rank_ragged_split_equals_single_realization(tmp_path):
    """6400 scatterers are 6.25 blocks: three ranks get 3, 2 and 1.25 blocks (a ragged
    last shard); the all-reduced spectra still equal the single-rank ones."""
    import oracle
    import scenegen as sg
    from paper_2408_11472_gb300.sharding import shard_range

    n = 80 * 80
    spans = [shard_range(n, 3, r) for r in range(3)]
    assert len({e - s for s, e in spans}) == 3               # three different shard sizes
    out = str(tmp_path / "T3.npy")
    mp.start_processes(_rank_main, args=(3, _free_port(), out), nprocs=3, join=True,
                       start_method="spawn")
    T3 = np.load(out)
    c = sg.config(1)
    T1 = oracle.Oracle().doppler_spectra(c["radar"], c["platform"], sg.sea_surface(80, 13), 31, 3,
                                         c["fast"].n_fast, c["fast"].n_doppler)
    np.testing.assert_allclose(T3, T1, rtol=0, atol=1e-12 * np.abs(T1).max())
