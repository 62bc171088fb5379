"""Host logic of the chunked scan (no GPU): the log-sum-exp merge of partial accumulators, the
checkpoint file, and the merge across two gloo ranks on CPU."""
import os

import numpy as np
import pytest
import scipy.special

from paper_1609_06634_gb300 import driver


def _partial(x):
    """(M, S) of a set of ln L values per image: M = max, S = sum exp(x - M)."""
    M = x.max(axis=1)
    return np.stack([M, np.exp(x - M[:, None]).sum(axis=1)], axis=1)


def test_merge_equals_logsumexp_of_the_union():
    rng = np.random.default_rng(1)
    x = -3000.0 + 40.0 * rng.standard_normal((5, 900))
    parts = [_partial(x[:, a:b]) for a, b in [(0, 100), (100, 101), (101, 640), (640, 900)]]
    acc = parts[0]
    for p in parts[1:]:
        acc = driver.merge_partials(acc, p)
    np.testing.assert_allclose(acc[:, 0] + np.log(acc[:, 1]), scipy.special.logsumexp(x, axis=1), rtol=1e-14)
    # order does not matter
    acc2 = parts[3]
    for p in parts[2::-1]:
        acc2 = driver.merge_partials(acc2, p)
    np.testing.assert_allclose(acc2[:, 0] + np.log(acc2[:, 1]), acc[:, 0] + np.log(acc[:, 1]), rtol=1e-14)


def test_merge_with_an_empty_part_is_the_identity():
    rng = np.random.default_rng(2)
    a = _partial(rng.standard_normal((4, 10)))
    empty = np.tile([-np.inf, 0.0], (4, 1))
    np.testing.assert_array_equal(driver.merge_partials(a, empty), a)
    np.testing.assert_array_equal(driver.merge_partials(empty, a), a)


def test_checkpoint_roundtrip_and_fingerprint(tmp_path):
    q = np.random.default_rng(3).standard_normal((20, 4)).astype(np.float32)
    ctfs = [(1e4, 0.1, 0.0, 300.0), (2e4, 0.1, 50.0, 300.0)]
    fp = driver.fingerprint(q, ctfs, 4, 32, 2.0, 16, 8)
    assert fp == driver.fingerprint(q.copy(), ctfs, 4, 32, 2.0, 16, 8)
    assert fp != driver.fingerprint(q, ctfs, 3, 32, 2.0, 16, 8)
    assert fp != driver.fingerprint(q, ctfs, 4, 32, 2.0, 16, 4)
    path = str(tmp_path / "scan.npz")
    acc = np.random.default_rng(4).standard_normal((16, 2))
    driver.save_checkpoint(path, acc, 2, fp)
    assert not os.path.exists(path + ".tmp")
    got, nxt = driver.load_checkpoint(path, fp)
    np.testing.assert_array_equal(got, acc)
    assert nxt == 2
    with pytest.raises(ValueError):
        driver.load_checkpoint(path, driver.fingerprint(q, ctfs, 4, 32, 2.0, 17, 8))
    assert driver.load_checkpoint(str(tmp_path / "none.npz"), fp) is None


def _rank(rank, world, port, x, out_path):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # each rank holds the accumulators of its own shard of the grid
    n = x.shape[1]
    lo, hi = rank * n // world, (rank + 1) * n // world
    acc = torch.from_numpy(_partial(x[:, lo:hi]))
    merged = driver.allreduce_partials(acc)
    np.save(out_path + f".{rank}.npy", merged.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_allreduce_partials_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    x = -500.0 + 10.0 * np.random.default_rng(5).standard_normal((6, 301))
    out = str(tmp_path / "merged")
    port = 29500 + (os.getpid() % 2000)
    mp.spawn(_rank, args=(2, port, x, out), nprocs=2, join=True)
    ref = scipy.special.logsumexp(x, axis=1)
    for r in range(2):
        m = np.load(out + f".{r}.npy")
        np.testing.assert_allclose(m[:, 0] + np.log(m[:, 1]), ref, rtol=1e-14)
