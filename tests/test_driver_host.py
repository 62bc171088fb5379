"""Host logic of the chunked scan (no GPU): the log-sum-exp merge operator of partial accumulators
(a host restatement here, the reference the library's bioem_acc_merge is tested against on the GPU),
the checkpoint file, and the merge across two gloo ranks on CPU."""
import os

import numpy as np
import pytest
import scipy.special

from paper_1609_06634_gb300 import driver


def _partial(x):
    """(M, S) of a set of ln L values per image: M = max, S = sum exp(x - M)."""
    M = x.max(axis=1)
    return np.stack([M, np.exp(x - M[:, None]).sum(axis=1)], axis=1)


def host_merge(parts):
    """(M, S) + (M', S') = (m, S e^{M - m} + S' e^{M' - m}), m = max(M, M'), folded over parts
    [k, n, 2] in order; a part with M = -inf is empty (test-side reference of bioem_acc_merge)."""
    parts = np.asarray(parts, dtype=np.float64)
    M = np.max(parts[:, :, 0], axis=0)
    with np.errstate(invalid="ignore"):
        terms = np.where(np.isfinite(parts[:, :, 0]), parts[:, :, 1] * np.exp(parts[:, :, 0] - M[None]), 0.0)
    return np.stack([M, terms.sum(axis=0)], axis=1)


def _merge_torch(stacked):
    import torch
    return torch.from_numpy(host_merge(stacked.numpy()))


def test_merge_equals_logsumexp_of_the_union():
    rng = np.random.default_rng(1)
    x = -3000.0 + 40.0 * rng.standard_normal((5, 900))
    parts = [_partial(x[:, a:b]) for a, b in [(0, 100), (100, 101), (101, 640), (640, 900)]]
    acc = host_merge(parts)
    np.testing.assert_allclose(acc[:, 0] + np.log(acc[:, 1]), scipy.special.logsumexp(x, axis=1), rtol=1e-14)
    acc2 = host_merge(parts[::-1])   # order does not matter
    np.testing.assert_allclose(acc2[:, 0] + np.log(acc2[:, 1]), acc[:, 0] + np.log(acc[:, 1]), rtol=1e-14)


def test_merge_with_an_empty_part_is_the_identity():
    rng = np.random.default_rng(2)
    a = _partial(rng.standard_normal((4, 10)))
    empty = np.tile([-np.inf, 0.0], (4, 1))
    np.testing.assert_array_equal(host_merge([a, empty]), a)
    np.testing.assert_array_equal(host_merge([empty, a]), a)


def test_driver_modules_do_no_likelihood_arithmetic():
    """driver.py and proposal.py sequence library calls; no exp / log / max over likelihood values."""
    import re
    root = os.path.dirname(driver.__file__)
    for name in ("driver.py", "proposal.py"):
        src = open(os.path.join(root, name)).read()
        code = re.sub(r'""".*?"""', "", src, flags=re.S)
        code = "\n".join(line.split("#")[0] for line in code.splitlines())
        for pat in (r"np\.exp\(", r"np\.log\(", r"np\.maximum\(", r"\.max\(axis", r"(?<!group_)logsumexp\("):
            assert not re.search(pat, code), (name, pat)


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
    merged = driver.allreduce_partials(acc, merge=_merge_torch)
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
