"""Chunked, resumable scan over an orientation grid, and the merge of partial posteriors.

A grid whose projection spectra do not fit device memory at once (294,912 orientations x 8 PSFs at
128 px is 157 GB) is projected and scored chunk by chunk.  Each chunk folds into per-image float64
accumulators (M, S) with ln sum_{p,d} L = M + ln S (the state of Eq. 9's sum over the parameter sets
scored so far).  After every chunk the accumulators and the index of the next chunk are written to
a checkpoint file (atomically: a temporary file, then a rename), together with a fingerprint of the
inputs; a scan started again with the same inputs and checkpoint continues where it stopped.

Partial accumulators of disjoint parts of the grid (chunks, or the shards of several processes)
combine with the log-sum-exp operator (M, S) + (M', S') = (m, S e^{M - m} + S' e^{M' - m}),
m = max(M, M'); `merge_partials` applies it on the device through the library (bioem_acc_merge)
and `allreduce_partials` across the ranks of a torch.distributed group (one all-gather: the single
exchange step a sharded grid needs, then the library's merge in rank order).

All scoring arithmetic runs in the library's kernels; this module only sequences calls and files.
"""
from __future__ import annotations

import hashlib
import math
import os

import numpy as np

from . import acc_logP, acc_merge, project_model, score_accumulate


def _torch():
    import torch
    return torch


def fingerprint(quats: np.ndarray, ctfs, max_shift: int, npix: int, pixel_A: float, n_img: int, chunk: int) -> str:
    """Identity of a scan's inputs (grid, PSFs, window, image size and count, chunking)."""
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(quats, dtype=np.float32).tobytes())
    h.update(np.asarray(ctfs, dtype=np.float64).tobytes())
    h.update(np.asarray([max_shift, npix, n_img, chunk], dtype=np.int64).tobytes())
    h.update(np.asarray([pixel_A], dtype=np.float64).tobytes())
    return h.hexdigest()


def save_checkpoint(path: str, acc: np.ndarray, next_chunk: int, fp: str) -> None:
    """Write (accumulators, next chunk, fingerprint) atomically."""
    tmp = path + ".tmp"
    with open(tmp, "wb") as f:
        np.savez(f, acc=np.asarray(acc, dtype=np.float64), next_chunk=np.int64(next_chunk), fingerprint=np.str_(fp))
    os.replace(tmp, path)


def load_checkpoint(path: str, fp: str):
    """(accumulators, next chunk) of a checkpoint written for the same inputs, else None."""
    if not os.path.exists(path):
        return None
    with np.load(path) as z:
        if str(z["fingerprint"]) != fp:
            raise ValueError(f"checkpoint {path} belongs to a different scan")
        return z["acc"].copy(), int(z["next_chunk"])


def merge_partials(ctx, *parts):
    """(M, S) accumulators [n, 2] (float64 device tensors) of the union of disjoint grid parts,
    merged by the library in argument order."""
    torch = _torch()
    return acc_merge(ctx, torch.stack([p.contiguous() for p in parts]))


def allreduce_partials(acc, group=None, ctx=None, merge=None):
    """Merge every rank's [n, 2] (M, S) accumulators (a torch tensor) with one all-gather; each rank
    gets the merged result.  The gathered parts [world, n, 2] are merged in rank order by
    ``merge(parts)`` when given, else by the library on ``ctx``'s device (bioem_acc_merge).
    Works with any torch.distributed backend (NCCL on GPUs; gloo on CPU, where the caller supplies
    ``merge`` because the library runs on GPUs only)."""
    torch = _torch()
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [torch.empty_like(acc) for _ in range(world)]
    dist.all_gather(parts, acc.contiguous(), group=group)
    stacked = torch.stack(parts)
    if merge is not None:
        return merge(stacked)
    if ctx is None:
        raise ValueError("allreduce_partials: pass the library context (or a merge function)")
    return acc_merge(ctx, stacked.to(ctx.device))


class OrientationScan:
    """ln P of prepared images over quats x ctfs, projected and scored `chunk` orientations at a time.

    run(max_chunks) scores up to max_chunks further chunks (all by default) and returns True when the
    grid is complete; with `checkpoint` set, the state is saved after every chunk and a new scan of
    the same inputs resumes from it.  log_p() returns ln P once complete (bioem_score's value)."""

    def __init__(self, ctx, images, atoms, sigma_A: float, quats: np.ndarray, ctfs, npix: int, pixel_A: float,
                 max_shift: int, chunk: int, checkpoint: str | None = None):
        torch = _torch()
        self.ctx, self.images, self.atoms = ctx, images, atoms
        self.sigma_A, self.npix, self.pixel_A, self.max_shift = sigma_A, npix, pixel_A, max_shift
        self.quats = np.ascontiguousarray(quats, dtype=np.float32)
        self.ctfs = [tuple(c) for c in ctfs]
        self.chunk = int(chunk)
        self.n_chunks = (len(self.quats) + self.chunk - 1) // self.chunk
        self.checkpoint = checkpoint
        self.fp = fingerprint(self.quats, self.ctfs, max_shift, npix, pixel_A, images.n_img, self.chunk)
        self.acc = torch.empty((images.n_img, 2), dtype=torch.float64, device=ctx.device)
        self.next_chunk = 0
        if checkpoint:
            st = load_checkpoint(checkpoint, self.fp)
            if st is not None:
                self.acc.copy_(torch.from_numpy(st[0]))
                self.next_chunk = st[1]

    @property
    def done(self) -> bool:
        return self.next_chunk >= self.n_chunks

    def run(self, max_chunks: int | None = None) -> bool:
        torch = _torch()
        todo = self.n_chunks - self.next_chunk if max_chunks is None else max_chunks
        for _ in range(max(0, todo)):
            if self.done:
                break
            c0 = self.next_chunk * self.chunk
            q = torch.from_numpy(self.quats[c0:c0 + self.chunk]).to(self.ctx.device)
            ps = project_model(self.ctx, self.atoms, self.sigma_A, q, self.ctfs, self.npix, self.pixel_A)
            score_accumulate(self.ctx, self.images, ps, self.max_shift, self.acc, first=self.next_chunk == 0)
            ps.close()
            self.next_chunk += 1
            if self.checkpoint:
                save_checkpoint(self.checkpoint, self.acc.cpu().numpy(), self.next_chunk, self.fp)
        return self.done

    def log_p(self):
        if not self.done:
            raise RuntimeError(f"scan incomplete: {self.next_chunk} of {self.n_chunks} chunks")
        S = (2 * self.max_shift + 1) ** 2
        return acc_logP(self.ctx, self.acc, math.log(len(self.quats) * len(self.ctfs) * S))
