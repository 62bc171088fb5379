"""Learned-proposal path: train the network on forward-model projections, propose coarse cells,
score each image only on the fine parameter sets of its proposed cells.

Orchestration of library calls; every computation runs in the CUDA kernels behind the C ABI
(synthetic maps, network training / inference / top-k, projection, gathered scoring).  The host
side builds index lists (which fine parameter sets belong to which proposed cells) and composes
the synthetic training images from the library's noiseless maps with seeded shifts, scales,
offsets and noise.
"""
from __future__ import annotations

import concurrent.futures
import math
import time

import numpy as np

from . import (CNN, Context, acc_logP, group_logsumexp, prepare_images, project_model, score_gathered,
               score_gathered_pairs, synthetic_maps)


def _torch():
    import torch
    return torch


def compose(ctx: Context, atoms_dev: list, d: dict, cfg, gen, out=None):
    """Images N I1(r + d) - mu + lambda z for the parameter draws d (device float32 [n, N, N])."""
    torch = _torch()
    n = len(d["quat"])
    N = cfg.npix
    dev = ctx.device
    if out is None:
        out = torch.empty((n, N, N), dtype=torch.float32, device=dev)
    yy = torch.arange(N, device=dev).view(1, N, 1)
    xx = torch.arange(N, device=dev).view(1, 1, N)
    chunk = 4096
    for m in range(len(atoms_dev)):
        idx_all = np.nonzero(d["model"] == m)[0]
        for c0 in range(0, len(idx_all), chunk):
            idx = idx_all[c0:c0 + chunk]
            q = torch.from_numpy(np.ascontiguousarray(d["quat"][idx])).to(dev)
            rows = [(d["defocus_A"][i], cfg.amp_contrast, d["bfactor"][i], cfg.voltage_kV) for i in idx]
            maps = synthetic_maps(ctx, atoms_dev[m], cfg.sigma_A, q, rows, N, cfg.pixel_A)
            it = torch.from_numpy(idx).to(dev)
            dy = torch.from_numpy(d["dy"][idx]).to(dev).view(-1, 1, 1)
            dx = torch.from_numpy(d["dx"][idx]).to(dev).view(-1, 1, 1)
            b = torch.arange(len(idx), device=dev).view(-1, 1, 1)
            sig = maps[b, (yy + dy) % N, (xx + dx) % N] * torch.from_numpy(d["norm"][idx]).float().to(dev).view(-1, 1, 1)
            lam = torch.sqrt(sig.double().var(dim=(1, 2), unbiased=False) / cfg.snr).float().view(-1, 1, 1)
            z = torch.randn(sig.shape, generator=gen, device=dev)
            out[it] = sig - torch.from_numpy(d["offset"][idx]).float().to(dev).view(-1, 1, 1) + lam * z
    return out


def train(net: CNN, images, yq, yd, epochs: int, batch: int, lr: float, gen) -> list:
    """Adam epochs over shuffled mini-batches; mean loss per epoch."""
    torch = _torch()
    n = images.shape[0]
    losses = []
    for ep in range(epochs):
        perm = torch.randperm(n, generator=gen, device=images.device)
        tot = torch.zeros((), dtype=torch.float64, device=images.device)
        steps = 0
        for b0 in range(0, n - batch + 1, batch):
            sel = perm[b0:b0 + batch]
            loss = net.train_step(images[sel].contiguous(), yq[sel].contiguous(), yd[sel].contiguous(), lr)
            tot += loss.double().mean()
            steps += 1
        losses.append(float(tot.item()) / max(1, steps))
    return losses


def redraw_nuisance(d: dict, cfg, rng) -> dict:
    """The same projections (model, orientation, defocus, B) with new displacements, normalisations
    and offsets; compose() then adds new noise.  Training on a fresh draw every epoch keeps the
    network from memorising the noise of a fixed set of training images."""
    n = len(d["quat"])
    s = cfg.max_shift
    e = dict(d)
    e["dx"] = rng.integers(-s, s + 1, n)
    e["dy"] = rng.integers(-s, s + 1, n)
    e["norm"] = rng.uniform(0.5, 2.0, n)
    e["offset"] = rng.uniform(-1.0, 1.0, n)
    return e


def train_redrawn(ctx: Context, net: CNN, atoms_dev: list, d: dict, cfg, epochs: int, batch: int, lr: float, gen,
                  rng, images=None) -> list:
    """Adam epochs, each over the training projections composed with a fresh draw of displacement,
    normalisation, offset and noise (the first epoch uses `images` if given)."""
    torch = _torch()
    yq = torch.from_numpy(d["label_q"]).to(ctx.device)
    yd = torch.from_numpy(d["label_d"]).to(ctx.device)
    losses = []
    for ep in range(epochs):
        if images is None or ep > 0:
            images = compose(ctx, atoms_dev, redraw_nuisance(d, cfg, rng) if ep > 0 else d, cfg, gen, out=images)
        losses += train(net, images, yq, yd, epochs=1, batch=batch, lr=lr, gen=gen)
    return losses


def _cell_lists(bins: np.ndarray, pos: np.ndarray, n_defocus: int, n_b: int, kids: int, cells=None):
    """Per-image parameter-set lists (CSR) of the joint bins whose cells are in the current wave:
    bin (cell, defocus d) -> sets ((pos[cell] * kids + j) * n_ctf + d * n_b + b) for its kids child
    orientations j and every B index b, in image-major, bin-major order.  Returns (mask [n, K] of
    the bins in this wave, offsets [n + 1] int64, flat set indices int32).  `cells` = bins //
    n_defocus may be passed in when the same bins are listed for many waves."""
    bins = np.asarray(bins)
    if cells is None:
        cells = bins // n_defocus
    pc = pos[cells]
    mask = pc >= 0
    nctf = n_defocus * n_b
    # set index = pos * kids * nctf + d * n_b  +  (j * nctf + b): one int32 head per selected bin plus
    # the bin's kids * n_b fixed offsets, built by one broadcast add
    head = (pc[mask].astype(np.int32) * np.int32(kids * nctf)
            + (bins[mask] % n_defocus).astype(np.int32) * np.int32(n_b))
    tail = (np.arange(kids, dtype=np.int32)[:, None] * np.int32(nctf)
            + np.arange(n_b, dtype=np.int32)[None, :]).reshape(-1)
    flat = (head[:, None] + tail[None, :]).reshape(-1)
    counts = mask.sum(axis=1).astype(np.int64) * (kids * n_b)
    off = np.zeros(len(counts) + 1, dtype=np.int64)
    np.cumsum(counts, out=off[1:])
    return mask, off, flat


def _wave_lists(bins: np.ndarray, n_coarse: int, n_defocus: int, n_b: int, kids: int, wave: int):
    """The lists of _cell_lists for every wave of the used cells (sorted cell ids, `wave` cells per
    wave), without a pass over all bins per wave: the bins are grouped by wave once (a stable radix
    sort of their wave numbers keeps each wave's bins in image-major, bin-major order), then each
    wave's lists are built from its own bins only.  Yields (cells of the wave, flattened indices
    into bins of the wave's bins, offsets [n + 1] int64, flat set indices int32)."""
    bins = np.asarray(bins)
    n, K = bins.shape
    cells = (bins // n_defocus).ravel()
    used = np.unique(cells)
    rank = np.full(n_coarse, -1, dtype=np.int64)
    rank[used] = np.arange(len(used))
    r = rank[cells]
    n_waves = (len(used) + wave - 1) // wave
    w = (r // wave).astype(np.int16 if n_waves < 32768 else np.int32)
    order = np.argsort(w, kind="stable")
    bounds = np.zeros(n_waves + 1, dtype=np.int64)
    np.cumsum(np.bincount(w, minlength=n_waves), out=bounds[1:])
    nctf = n_defocus * n_b
    tail = (np.arange(kids, dtype=np.int32)[:, None] * np.int32(nctf)
            + np.arange(n_b, dtype=np.int32)[None, :]).reshape(-1)
    flat_bins = bins.ravel()
    for t in range(n_waves):
        idx = order[bounds[t]:bounds[t + 1]]
        pos = (r[idx] - t * wave).astype(np.int32)
        head = pos * np.int32(kids * nctf) + (flat_bins[idx] % n_defocus).astype(np.int32) * np.int32(n_b)
        flat = (head[:, None] + tail[None, :]).reshape(-1)
        counts = np.bincount(idx // K, minlength=n).astype(np.int64) * (kids * n_b)
        off = np.zeros(n + 1, dtype=np.int64)
        np.cumsum(counts, out=off[1:])
        yield used[t * wave:(t + 1) * wave], idx, off, flat


def score_cells(ctx: Context, images, atoms_dev, bins: np.ndarray, cfg, wave: int = 256) -> dict:
    """ln P of every image over the union of its joint cells bins[i] (coarse cell * n_defocus + defocus
    bin), each cell expanded to its fine orientations x the cell's defocus x every B.  ln P is
    normalised by the FULL fine grid (n_fine x n_defocus x n_B x S), so cells not scored count as
    zero likelihood: it equals the full-grid posterior when the cells hold all its mass."""
    import workloads
    torch = _torch()
    dev = ctx.device
    n_img = bins.shape[0]
    nd, nb = cfg.n_defocus, len(cfg.bfactors)
    nctf = nd * nb
    fine_q = workloads.hopf_grid(cfg.fine_level).astype(np.float32)
    kids = cfg.children
    S = (2 * cfg.max_shift + 1) ** 2
    log_norm = math.log(len(fine_q) * nctf * S)
    bins = np.asarray(bins, dtype=np.int64)
    n_cells = 0
    acc = torch.empty((n_img, 2), dtype=torch.float64, device=dev)
    first = True
    evals = 0
    t0 = time.perf_counter()
    rows = cfg.ctf_rows()
    for wc, _, off, flat in _wave_lists(bins, cfg.n_coarse, nd, nb, kids, wave):
        n_cells += len(wc)
        child = workloads.hopf_children(cfg.coarse_level, cfg.fine_level, wc).ravel()
        q = torch.from_numpy(np.ascontiguousarray(fine_q[child])).to(dev)
        ps = project_model(ctx, atoms_dev, cfg.sigma_A, q, rows, cfg.npix, cfg.pixel_A)
        counts = np.diff(off)
        evals += int(counts.sum())
        score_gathered(ctx, images, ps, cfg.max_shift, torch.from_numpy(off.astype(np.int32)).to(dev),
                       torch.from_numpy(flat).to(dev), max(1, int(counts.max())), acc, first)
        first = False
        ps.close()
    logp = acc_logP(ctx, acc, log_norm)
    torch.cuda.synchronize()
    return {"logP": logp.cpu().numpy(), "evals": evals, "seconds": time.perf_counter() - t0,
            "cells": int(n_cells)}


def rerank_coarse(ctx: Context, images, atoms_dev, bins: np.ndarray, cfg, keep: int, wave: int = 128,
                  level: int | None = None) -> dict:
    """Exact re-ranking of proposed joint bins: bin (coarse cell, defocus) is scored at the cell's
    orientations of Hopf level `level` (default: the coarse level itself, one orientation per cell;
    one level finer: the cell's 8 children) x its defocus x every B, as ln sum over them and over the
    displacements of L (the closed-form likelihood of the scoring path, summed by the library); per
    image the `keep` best bins are returned, best first.  The cells are projected in waves of `wave`
    orientations: 128 x 8 PSFs = 68 MB of projection spectra stay in L2 while every image scores its
    share of them (K1 = 8192 at level 3, 2000 images: 4.5e7 evals/s against 3.5e7 with waves of
    2304 orientations; 32 orientations per wave lose more to per-wave launches than they gain)."""
    import workloads
    torch = _torch()
    dev = ctx.device
    nd, nb = cfg.n_defocus, len(cfg.bfactors)
    level = cfg.coarse_level if level is None else level
    kids = 8 ** (level - cfg.coarse_level)
    grid_q = workloads.hopf_grid(level).astype(np.float32)
    bins = np.asarray(bins, dtype=np.int64)
    scores = np.full(bins.shape, -np.inf)
    flat_scores = scores.reshape(-1)
    evals = 0
    t0 = time.perf_counter()
    # the host builds the next wave's lists while the GPU scores the current one
    gen = _wave_lists(bins, cfg.n_coarse, nd, nb, kids, max(1, wave // kids))
    with concurrent.futures.ThreadPoolExecutor(max_workers=1) as pool:
        pending = pool.submit(next, gen, None)
        while True:
            item = pending.result()
            if item is None:
                break
            pending = pool.submit(next, gen, None)
            wc, idx, off, flat = item
            child = workloads.hopf_children(cfg.coarse_level, level, wc).ravel() if kids > 1 else wc
            ps = project_model(ctx, atoms_dev, cfg.sigma_A,
                               torch.from_numpy(np.ascontiguousarray(grid_q[child])).to(dev), cfg.ctf_rows(),
                               cfg.npix, cfg.pixel_A)
            counts = np.diff(off)
            v = score_gathered_pairs(ctx, images, ps, cfg.max_shift, torch.from_numpy(off.astype(np.int32)).to(dev),
                                     torch.from_numpy(flat).to(dev), max(1, int(counts.max())))
            # ln sum over each bin's children and B-factors (the library's log-sum-exp; the host orders bins)
            flat_scores[idx] = group_logsumexp(ctx, v, kids * nb).cpu().numpy()
            evals += int(counts.sum())
            ps.close()
    order = np.argsort(-scores, axis=1, kind="stable")[:, :keep]
    return {"bins": np.take_along_axis(bins, order, axis=1), "evals": evals,
            "seconds": time.perf_counter() - t0}


def all_bins(n_img: int, cfg) -> np.ndarray:
    """Every joint bin for every image (the full grid)."""
    return np.tile(np.arange(cfg.n_coarse * cfg.n_defocus, dtype=np.int64), (n_img, 1))
