"""GPU: 96 / 192 px parity against the oracle; the batched (graph-captured, multi-segment) launch
against the oracle and against per-segment bioem_score; the autotuner's choice and cache file,
including a corrupted cache."""
import os

import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu
TOL = 1e-3


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1609_06634_gb300 as bioem
    from paper_1609_06634_gb300 import build
    build.build()
    return bioem, bioem.Context(0)


def _dev(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda:0")


def _stack_images(wl, k, n=None):
    """Oracle-synthesised images of stack k (each from its seeded model)."""
    st = wl["stacks"][k]
    cfg = st["config"]
    out = []
    for i in range(len(st["truth"]) if n is None else n):
        t = st["truth"][i]
        atoms = wl["atoms"][st["models"][i]]
        img1 = oracle.apply_psf(oracle.project(atoms, t["quat"], cfg.sigma_A, cfg.npix, cfg.pixel_A),
                                (t["defocus_A"], t["amp_contrast"], t["bfactor"], t["voltage_kV"]), cfg.pixel_A)
        out.append(oracle.synthesize_image(img1, t["dx"], t["dy"], t["norm"], t["offset"], st["noise"][i], cfg.snr))
    return np.asarray(out, dtype=np.float32)


@pytest.mark.parametrize("k", [1, 3])   # 96 px (+-12) and 192 px (+-24)
def test_large_sizes_match_oracle(env, k):
    bioem, ctx = env
    wl = workloads.batched_workload(workloads.BatchedConfig(n_models=2))
    st = wl["stacks"][k]
    cfg = st["config"]
    imgs = _stack_images(wl, k, n=2)
    quats = st["quats"][::97][:6]
    ctfs = st["ctfs"][:2]
    atoms = wl["atoms"][0]
    ref = oracle.score(imgs, atoms, quats, ctfs, cfg.sigma_A, cfg.pixel_A, cfg.max_shift)
    im = bioem.prepare_images(ctx, _dev(imgs), cfg.pixel_A)
    ps = bioem.project_model(ctx, _dev(atoms), cfg.sigma_A, _dev(quats), ctfs, cfg.npix, cfg.pixel_A)
    out = bioem.score_all(ctx, im, ps, cfg.max_shift, per_orient=True, best=True)
    assert ctx.status() == 0
    np.testing.assert_allclose(out["logP"].cpu().numpy(), ref["logP"], rtol=0, atol=TOL)
    np.testing.assert_allclose(out["logP_orient"].cpu().numpy(), ref["logP_orient"], rtol=0, atol=TOL)
    np.testing.assert_allclose(out["best_logL"].cpu().numpy(), [b[4] for b in ref["best"]], rtol=0, atol=TOL)


@pytest.fixture(scope="module")
def batch_case(env):
    bioem, ctx = env
    cfg = workloads.BatchedConfig(n_models=3, stacks=(workloads.StackSpec(64, 6, 0, 2), workloads.StackSpec(96, 5, 0, 2),
                                                      workloads.StackSpec(128, 4, 0, 2), workloads.StackSpec(192, 3, 0, 2)))
    wl = workloads.batched_workload(cfg)
    stacks, projsets = [], []
    for k, st in enumerate(wl["stacks"]):
        sc = st["config"]
        stacks.append(bioem.prepare_images(ctx, _dev(_stack_images(wl, k)), sc.pixel_A))
    for m in range(cfg.n_models):
        row = []
        for k, st in enumerate(wl["stacks"]):
            sc = st["config"]
            row.append(bioem.project_model(ctx, _dev(wl["atoms"][m]), sc.sigma_A, _dev(st["quats"]), st["ctfs"], sc.npix,
                                           sc.pixel_A))
        projsets.append(row)
    shifts = [st["config"].max_shift for st in wl["stacks"]]
    return cfg, wl, stacks, projsets, shifts


def test_batch_matches_single_launches(env, batch_case):
    bioem, ctx = env
    cfg, wl, stacks, projsets, shifts = batch_case
    batch = bioem.Batch(ctx, stacks, projsets, shifts)
    assert batch.evals == sum(cfg.n_models * im.n_img * projsets[0][k].n_ps for k, im in enumerate(stacks))
    out1 = batch.run().cpu().numpy().copy()
    out2 = batch.run().cpu().numpy()
    assert ctx.status() == 0
    np.testing.assert_array_equal(out1, out2)   # graph replays are deterministic
    col = 0
    for k, im in enumerate(stacks):
        for m in range(cfg.n_models):
            want = bioem.score(ctx, im, projsets[m][k], shifts[k]).cpu().numpy()
            got = out1[m, col:col + im.n_img]
            # float32 output: allow its rounding on top of the parity tolerance
            np.testing.assert_allclose(got, want, rtol=3e-7, atol=TOL)
        col += im.n_img
    batch.close()


def test_batch_matches_oracle(env, batch_case):
    """The batched log P matrix (one persistent launch over every (model, stack) segment, each item
    running its size instance: 64 / 96 / 128 / 192 px) against the FP64 oracle, element by element.
    Each stack's grid holds 288 parameter sets, so every segment ends in a ragged chunk (the
    default chunks are 256 sets, 64 at 192 px).  Tolerance: 1e-3 plus the float32 output's rounding."""
    bioem, ctx = env
    cfg, wl, stacks, projsets, shifts = batch_case
    batch = bioem.Batch(ctx, stacks, projsets, shifts)
    got = batch.run().cpu().numpy().copy()
    assert ctx.status() == 0
    batch.close()
    col = 0
    for k, im in enumerate(stacks):
        st = wl["stacks"][k]
        sc = st["config"]
        assert len(st["quats"]) * len(st["ctfs"]) % 64 != 0   # ragged last chunk
        imgs = _stack_images(wl, k)
        for m in range(cfg.n_models):
            ref = oracle.score(imgs, wl["atoms"][m], st["quats"], st["ctfs"], sc.sigma_A, sc.pixel_A, sc.max_shift)
            np.testing.assert_allclose(got[m, col:col + im.n_img], ref["logP"], rtol=3e-7, atol=TOL,
                                       err_msg=f"model {m}, stack {k} ({sc.npix} px)")
        col += im.n_img


def test_autotune_and_cache(env, batch_case, tmp_path):
    bioem, ctx = env
    cfg, wl, stacks, projsets, shifts = batch_case
    path = str(tmp_path / "tune.txt")
    chunk = bioem.autotune(ctx, stacks[2], projsets[0][2], shifts[2], path)
    pb = 7   # pairs per batch of the batched 128 px instance
    assert chunk in (pb * 2, pb * 8, pb * 32, pb * 64, pb * 128)
    lines = open(path).read().split()
    assert lines[:3] == ["128", str(shifts[2]), str(chunk)]
    assert bioem.autotune(ctx, stacks[2], projsets[0][2], shifts[2], path) == chunk   # served from the cache
    batch = bioem.Batch(ctx, stacks, projsets, shifts)
    out = batch.run().cpu().numpy()
    assert np.all(np.isfinite(out))
    os.remove(path)
    # a corrupted cache: the invalid entry for this case is skipped, the case is tuned afresh and
    # the file is rewritten with valid lines only
    with open(path, "w") as f:
        f.write(f"128 {shifts[2]} 5\n999 4 64\nnot a number\n")
    chunk2 = bioem.autotune(ctx, stacks[2], projsets[0][2], shifts[2], path)
    assert chunk2 in (pb * 2, pb * 8, pb * 32, pb * 64, pb * 128)
    taken, skipped = bioem.autotune_load(path)
    assert skipped == 0 and taken >= 1
    assert f"128 {shifts[2]} {chunk2}" in open(path).read()
    os.remove(path)
