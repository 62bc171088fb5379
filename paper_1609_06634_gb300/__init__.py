"""Python binding of the BioEM sm_103a scoring library (argument marshalling only).

Every computation runs in the CUDA kernels behind the C ABI of ``include/bioem.h``; this module
only checks tensor dtypes/devices, passes raw device pointers and the caller's CUDA stream, and
wraps the library-owned handles.  PyTorch provides device memory and streams.  There is no CPU
path: if the library is missing or no GPU is present the calls raise.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native
from ._native import CTF

__all__ = ["BioEMError", "Context", "Images", "ProjSet", "prepare_images", "project_model", "score", "score_all",
           "best_params", "score_pairs", "score_noalloc", "Batch", "autotune", "autotune_load", "CNN", "score_gathered", "acc_logP",
           "acc_merge", "group_logsumexp", "ln1m", "fma_peak", "synthetic_maps", "ctf_array", "lib"]

OK = 0
ERR_INVALID_ARG, ERR_UNSUPPORTED_SIZE, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_NUMERIC = -1, -2, -3, -4, -5, -6


def lib():
    return _native.load()


class BioEMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{msg} (status {code})")
        self.code = code


def _torch():
    import torch
    return torch


def _check(ctx, code: int, what: str):
    if code != OK:
        detail = lib().bioem_last_error(ctx._h).decode() if ctx is not None and ctx._h else ""
        raise BioEMError(code, f"{what}: {lib().bioem_status_string(code).decode()} {detail}".strip())


def _dev_tensor(t, dtype, device, name, ndim=None, last=None):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or t.device != device:
        raise BioEMError(ERR_INVALID_ARG, f"{name} must be a tensor on {device}")
    if t.dtype != dtype:
        raise BioEMError(ERR_INVALID_ARG, f"{name} must be {dtype}")
    if ndim is not None and t.dim() != ndim:
        raise BioEMError(ERR_INVALID_ARG, f"{name} must have {ndim} dimensions")
    if last is not None and t.shape[-1] != last:
        raise BioEMError(ERR_INVALID_ARG, f"{name} last dimension must be {last}")
    return t.contiguous()


def ctf_array(ctfs) -> ctypes.Array:
    """Host array of bioem_ctf from rows (defocus_A, amp_contrast, bfactor_A2, voltage_kV)."""
    rows = np.asarray(ctfs, dtype=np.float64).reshape(-1, 4)
    arr = (CTF * len(rows))()
    for i, r in enumerate(rows):
        arr[i] = CTF(*[float(v) for v in r])
    return arr


class Context:
    """A library context on one CUDA device, enqueueing on a CUDA stream.

    The stream defaults to torch's current stream at creation.  Every call enqueues on it, reading
    its input tensors and writing its output tensors (allocated on torch's current stream) there.
    While that is torch's current stream, ordinary stream order makes this safe.  When it is not,
    the caller orders it: ``ctx.stream.wait_stream(torch.cuda.current_stream())`` before a call
    whose inputs were just produced, and the reverse before reading results or freeing inputs.
    """

    def __init__(self, device=0, stream=None):
        torch = _torch()
        self.device = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        self._h = None
        code = lib().bioem_create(ctypes.byref(h), self.device.index or 0, ctypes.c_void_p(self.stream.cuda_stream))
        if code != OK:
            raise BioEMError(code, "bioem_create failed")
        self._h = h

    def set_scratch_limit(self, nbytes: int):
        _check(self, lib().bioem_set_scratch_limit(self._h, int(nbytes)), "set_scratch_limit")

    PRECISIONS = {"fp32": 0, "bf16x2": 1, "fp16x2": 2, "bf16x2_real": 3, "fp16x2_real": 4, "fp16x2_fft": 5}

    def set_precision(self, mode):
        """Arithmetic of the correlation step for score/score_all/best_params/score_pairs: "fp32"
        (FFT form on the CUDA cores), "bf16x2" or "fp16x2" (two-term split-precision GEMM on the
        tensor cores over the half spectrum), "bf16x2_real" / "fp16x2_real" (the same GEMM over
        real-space pixels), "fp16x2_fft" (the FFT form with its column transforms as split-FP16
        tensor-core products; 128 px, max_shift <= 16), or the C constant."""
        m = self.PRECISIONS[mode] if isinstance(mode, str) else int(mode)
        _check(self, lib().bioem_set_precision(self._h, m), "set_precision")

    @property
    def precision(self) -> str:
        m = int(lib().bioem_get_precision(self._h))
        return {v: k for k, v in self.PRECISIONS.items()}[m]

    def set_wait_test(self, skip_chunk: int, wait_ns: int = 5_000_000):
        """bioem_set_wait_test: the next tensor-core scoring launch leaves K chunk skip_chunk unfed, so a
        bounded barrier wait (wait_ns) expires and the launch ends with BIOEM_ERR_TIMEOUT in the status."""
        _check(self, lib().bioem_set_wait_test(self._h, int(skip_chunk), int(wait_ns)), "set_wait_test")

    def set_kernel_timing(self, on: bool = True):
        """Record CUDA events on this context's stream around every library kernel launch."""
        _check(self, lib().bioem_set_kernel_timing(self._h, 1 if on else 0), "set_kernel_timing")

    def kernel_time(self, name: str) -> tuple[float, int]:
        """(summed device ms, launches) of one library kernel since the last reset (synchronises)."""
        ms = ctypes.c_double(0.0)
        n = ctypes.c_ulonglong(0)
        _check(self, lib().bioem_kernel_time(self._h, name.encode(), ctypes.byref(ms), ctypes.byref(n)), "kernel_time")
        return ms.value, n.value

    def reset_kernel_stats(self):
        _check(self, lib().bioem_reset_kernel_stats(self._h), "reset_kernel_stats")

    def launch_count(self) -> int:
        """Kernels launched by the library with this context since creation or the last reset."""
        return int(lib().bioem_launch_count(self._h))

    def status(self) -> int:
        """Synchronise the stream and read (and clear) the device status word."""
        out = ctypes.c_int(0)
        _check(self, lib().bioem_get_status(self._h, ctypes.byref(out)), "get_status")
        return out.value

    def close(self):
        if self._h:
            lib().bioem_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _Handle:
    _free = None

    def __init__(self, ctx: Context, h, **meta):
        self.ctx = ctx
        self._h = h
        self.__dict__.update(meta)

    def close(self):
        if self._h:
            getattr(lib(), self._free)(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Images(_Handle):
    _free = "bioem_free_images"


class ProjSet(_Handle):
    _free = "bioem_free_projset"


def prepare_images(ctx: Context, images, pixel_A: float) -> Images:
    """bioem_prepare_images on a [n, ny, nx] float32 device tensor."""
    torch = _torch()
    t = _dev_tensor(images, torch.float32, ctx.device, "images", ndim=3)
    h = ctypes.c_void_p()
    n, ny, nx = t.shape
    _check(ctx, lib().bioem_prepare_images(ctx._h, ctypes.c_void_p(t.data_ptr()), n, nx, ny, float(pixel_A),
                                           ctypes.byref(h)), "prepare_images")
    return Images(ctx, h, n_img=n, npix=nx, pixel_A=float(pixel_A))


def project_model(ctx: Context, atoms, sigma_A: float, quats, ctfs, npix: int, pixel_A: float) -> ProjSet:
    """bioem_project_model: atoms [n, 4] and quats [nq, 4] float32 device tensors, ctfs host rows."""
    torch = _torch()
    a = _dev_tensor(atoms, torch.float32, ctx.device, "atoms", ndim=2, last=4)
    q = _dev_tensor(quats, torch.float32, ctx.device, "quats", ndim=2, last=4)
    c = ctf_array(ctfs)
    h = ctypes.c_void_p()
    _check(ctx, lib().bioem_project_model(ctx._h, ctypes.c_void_p(a.data_ptr()), a.shape[0], float(sigma_A),
                                          ctypes.c_void_p(q.data_ptr()), q.shape[0], c, len(c), npix, npix,
                                          float(pixel_A), ctypes.byref(h)), "project_model")
    return ProjSet(ctx, h, nq=q.shape[0], nctf=len(c), n_ps=q.shape[0] * len(c), npix=npix, pixel_A=float(pixel_A))


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def score_all(ctx: Context, images: Images, projset: ProjSet, max_shift: int, per_orient: bool = False,
              best: bool = False) -> dict:
    """One pass over the grid: log P per image, optionally per orientation and maximising parameters."""
    torch = _torch()
    n = images.n_img
    dev = ctx.device
    out = {"logP": torch.empty(n, dtype=torch.float64, device=dev)}
    if per_orient:
        out["logP_orient"] = torch.empty((n, projset.nq), dtype=torch.float64, device=dev)
    if best:
        for k in ("best_q", "best_ctf", "best_dx", "best_dy"):
            out[k] = torch.empty(n, dtype=torch.int32, device=dev)
        out["best_logL"] = torch.empty(n, dtype=torch.float64, device=dev)
    g = out.get
    _check(ctx, lib().bioem_score_all(ctx._h, images._h, projset._h, int(max_shift), _ptr(g("logP")),
                                      _ptr(g("logP_orient")), _ptr(g("best_q")), _ptr(g("best_ctf")),
                                      _ptr(g("best_dx")), _ptr(g("best_dy")), _ptr(g("best_logL"))), "score_all")
    return out


def score(ctx: Context, images: Images, projset: ProjSet, max_shift: int, out=None):
    """bioem_score: [n_img] float64 log P(image | model) on the device."""
    torch = _torch()
    if out is None:
        out = torch.empty(images.n_img, dtype=torch.float64, device=ctx.device)
    _check(ctx, lib().bioem_score(ctx._h, images._h, projset._h, int(max_shift), _ptr(out), ctypes.c_void_p(0)),
           "score")
    return out


def score_noalloc(ctx: Context, images: Images, projset: ProjSet, max_shift: int, out):
    """bioem_score_noalloc: log P into the caller's [n_img] float64 device tensor ``out``.

    The library allocates no device memory in this call (its scratch is a fixed 16 MiB array
    reserved when the library is loaded), for callers that must not allocate while scoring.
    """
    torch = _torch()
    t = _dev_tensor(out, torch.float64, ctx.device, "out", ndim=1)
    if t.data_ptr() != out.data_ptr() or t.shape[0] != images.n_img:
        raise BioEMError(ERR_INVALID_ARG, "out must be a contiguous [n_img] float64 tensor")
    _check(ctx, lib().bioem_score_noalloc(ctx._h, images._h, projset._h, int(max_shift), _ptr(out)), "score_noalloc")
    return out


def best_params(ctx: Context, images: Images, projset: ProjSet, max_shift: int) -> dict:
    torch = _torch()
    n = images.n_img
    out = {k: torch.empty(n, dtype=torch.int32, device=ctx.device) for k in ("q", "ctf", "dx", "dy")}
    out["logL"] = torch.empty(n, dtype=torch.float64, device=ctx.device)
    _check(ctx, lib().bioem_best_params(ctx._h, images._h, projset._h, int(max_shift), _ptr(out["q"]), _ptr(out["ctf"]),
                                        _ptr(out["dx"]), _ptr(out["dy"]), _ptr(out["logL"])), "best_params")
    return out


def score_pairs(ctx: Context, images: Images, projset: ProjSet, max_shift: int, ps_begin: int = 0,
                ps_count: int | None = None):
    """Per-pair max_d ln L and ln sum_d L, [n_img, ps_count] float64."""
    torch = _torch()
    if ps_count is None:
        ps_count = projset.n_ps - ps_begin
    pmax = torch.empty((images.n_img, ps_count), dtype=torch.float64, device=ctx.device)
    plse = torch.empty_like(pmax)
    _check(ctx, lib().bioem_score_pairs(ctx._h, images._h, projset._h, int(max_shift), int(ps_begin), int(ps_count),
                                        _ptr(pmax), _ptr(plse)), "score_pairs")
    return pmax, plse


class Batch:
    """bioem_batch: models x image stacks of mixed sizes scored by one graph-captured persistent launch.

    ``stacks``: list of Images (64/96/128/192 px); ``projsets[m][k]``: model m projected for stack k;
    ``max_shift[k]``: shift window of stack k.  ``out`` is the [n_models, n_images_total] float32 log P
    matrix written by every ``run()``.
    """

    def __init__(self, ctx: Context, stacks, projsets, max_shift):
        torch = _torch()
        self.ctx = ctx
        self._h = None
        self.stacks, self.projsets = list(stacks), [list(r) for r in projsets]
        n_models, n_stacks = len(self.projsets), len(self.stacks)
        n_cols = sum(im.n_img for im in self.stacks)
        self.out = torch.empty((n_models, n_cols), dtype=torch.float32, device=ctx.device)
        st = (ctypes.c_void_p * n_stacks)(*[im._h for im in self.stacks])
        ps = (ctypes.c_void_p * (n_models * n_stacks))(*[p._h for row in self.projsets for p in row])
        sh = (ctypes.c_int * n_stacks)(*[int(v) for v in max_shift])
        h = ctypes.c_void_p()
        _check(ctx, lib().bioem_batch_create(ctx._h, n_models, n_stacks, st, ps, sh, _ptr(self.out), ctypes.byref(h)),
               "batch_create")
        self._h = h

    @property
    def evals(self) -> int:
        return int(lib().bioem_batch_evals(self._h))

    def run(self):
        _check(self.ctx, lib().bioem_batch_run(self._h), "batch_run")
        return self.out

    def close(self):
        if self._h:
            lib().bioem_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def autotune(ctx: Context, images: Images, projset: ProjSet, max_shift: int, cache_path: str | None = None) -> int:
    """bioem_autotune: chunk size chosen for (image size, max_shift); cached in cache_path if given."""
    out = ctypes.c_int(0)
    _check(ctx, lib().bioem_autotune(ctx._h, images._h, projset._h, int(max_shift),
                                     cache_path.encode() if cache_path else None, ctypes.byref(out)), "autotune")
    return out.value


def autotune_load(cache_path: str) -> tuple[int, int]:
    """bioem_autotune_load: (entries taken, lines skipped) of an autotune cache file (no GPU work)."""
    taken, skipped = ctypes.c_int(0), ctypes.c_int(0)
    code = lib().bioem_autotune_load(cache_path.encode(), ctypes.byref(taken), ctypes.byref(skipped))
    if code != OK:
        raise BioEMError(code, f"autotune_load: cannot read {cache_path}")
    return taken.value, skipped.value


class CNN:
    """bioem_cnn: the learned orientation / defocus proposal network (own CUDA kernels)."""

    def __init__(self, ctx: Context, image_px: int = 128, downsample: int = 2, channels: int = 32,
                 n_qbins: int = 4608, n_dbins: int = 4, max_batch: int = 256, seed: int = 0):
        self.ctx = ctx
        self._h = None
        h = ctypes.c_void_p()
        _check(ctx, lib().bioem_cnn_create(ctx._h, image_px, downsample, channels, n_qbins, n_dbins, max_batch,
                                           int(seed), ctypes.byref(h)), "cnn_create")
        self._h = h
        self.image_px, self.n_qbins, self.n_dbins, self.max_batch = image_px, n_qbins, n_dbins, max_batch
        self.n_params = int(lib().bioem_cnn_num_params(h))

    def _imgs(self, images):
        torch = _torch()
        t = _dev_tensor(images, torch.float32, self.ctx.device, "images", ndim=3)
        if t.shape[1] != self.image_px or t.shape[2] != self.image_px:
            raise BioEMError(ERR_INVALID_ARG, "image size does not match the network")
        return t

    def _labels(self, y):
        torch = _torch()
        return _dev_tensor(y, torch.int32, self.ctx.device, "labels", ndim=1)

    def set_params(self, theta):
        torch = _torch()
        t = _dev_tensor(theta, torch.float32, self.ctx.device, "params", ndim=1)
        _check(self.ctx, lib().bioem_cnn_set_params(self._h, _ptr(t)), "cnn_set_params")

    def get_params(self):
        torch = _torch()
        out = torch.empty(self.n_params, dtype=torch.float32, device=self.ctx.device)
        _check(self.ctx, lib().bioem_cnn_get_params(self._h, _ptr(out)), "cnn_get_params")
        return out

    def forward(self, images):
        torch = _torch()
        t = self._imgs(images)
        lq = torch.empty((t.shape[0], self.n_qbins), dtype=torch.float32, device=self.ctx.device)
        ld = torch.empty((t.shape[0], self.n_dbins), dtype=torch.float32, device=self.ctx.device)
        _check(self.ctx, lib().bioem_cnn_forward(self._h, _ptr(t), t.shape[0], _ptr(lq), _ptr(ld)), "cnn_forward")
        return lq, ld

    def gradients(self, images, yq, yd):
        torch = _torch()
        t = self._imgs(images)
        g = torch.empty(self.n_params, dtype=torch.float32, device=self.ctx.device)
        loss = torch.empty(t.shape[0], dtype=torch.float32, device=self.ctx.device)
        _check(self.ctx, lib().bioem_cnn_gradients(self._h, _ptr(t), _ptr(self._labels(yq)), _ptr(self._labels(yd)),
                                                   t.shape[0], _ptr(g), _ptr(loss)), "cnn_gradients")
        return g, loss

    def train_step(self, images, yq, yd, lr: float, loss_out=None):
        torch = _torch()
        t = self._imgs(images)
        if loss_out is None:
            loss_out = torch.empty(t.shape[0], dtype=torch.float32, device=self.ctx.device)
        _check(self.ctx, lib().bioem_cnn_train_step(self._h, _ptr(t), _ptr(self._labels(yq)), _ptr(self._labels(yd)),
                                                    t.shape[0], float(lr), _ptr(loss_out)), "cnn_train_step")
        return loss_out

    def propose(self, images, k: int):
        torch = _torch()
        t = self._imgs(images)
        bins = torch.empty((t.shape[0], k), dtype=torch.int32, device=self.ctx.device)
        scores = torch.empty((t.shape[0], k), dtype=torch.float32, device=self.ctx.device)
        _check(self.ctx, lib().bioem_propose(self._h, _ptr(t), t.shape[0], int(k), _ptr(bins), _ptr(scores)), "propose")
        return bins, scores

    def close(self):
        if self._h:
            lib().bioem_cnn_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def score_gathered(ctx: Context, images: Images, projset: ProjSet, max_shift: int, offsets, ps_idx,
                   max_per_image: int, acc, first: bool):
    """bioem_score_gathered: fold image w's scores over projset sets ps_idx[offsets[w]:offsets[w+1]] into acc."""
    torch = _torch()
    o = _dev_tensor(offsets, torch.int32, ctx.device, "offsets", ndim=1)
    p = _dev_tensor(ps_idx, torch.int32, ctx.device, "ps_idx", ndim=1)
    a = _dev_tensor(acc, torch.float64, ctx.device, "acc", ndim=2, last=2)
    if a.data_ptr() != acc.data_ptr():
        raise BioEMError(ERR_INVALID_ARG, "acc must be contiguous")
    _check(ctx, lib().bioem_score_gathered(ctx._h, images._h, projset._h, int(max_shift), _ptr(o), _ptr(p), p.shape[0],
                                           int(max_per_image), _ptr(a), 1 if first else 0), "score_gathered")
    return acc


def score_gathered_pairs(ctx: Context, images: Images, projset: ProjSet, max_shift: int, offsets, ps_idx,
                         max_per_image: int):
    """bioem_score_gathered_pairs: ln sum_d L for every listed (image, parameter set), [nnz] float64."""
    torch = _torch()
    o = _dev_tensor(offsets, torch.int32, ctx.device, "offsets", ndim=1)
    p = _dev_tensor(ps_idx, torch.int32, ctx.device, "ps_idx", ndim=1)
    out = torch.empty(p.shape[0], dtype=torch.float64, device=ctx.device)
    _check(ctx, lib().bioem_score_gathered_pairs(ctx._h, images._h, projset._h, int(max_shift), _ptr(o), _ptr(p),
                                                 p.shape[0], int(max_per_image), _ptr(out)), "score_gathered_pairs")
    return out


def acc_logP(ctx: Context, acc, log_norm: float):
    torch = _torch()
    a = _dev_tensor(acc, torch.float64, ctx.device, "acc", ndim=2, last=2)
    out = torch.empty(a.shape[0], dtype=torch.float64, device=ctx.device)
    _check(ctx, lib().bioem_acc_logP(ctx._h, _ptr(a), a.shape[0], float(log_norm), _ptr(out)), "acc_logP")
    return out


def acc_merge(ctx: Context, parts, out=None):
    """bioem_acc_merge: the (M, S) accumulators of the union of disjoint grid parts.

    ``parts``: [n_parts, n, 2] (or [n, 2] for a single part) float64 device tensor; returns [n, 2]."""
    torch = _torch()
    p = _dev_tensor(parts, torch.float64, ctx.device, "parts")
    if p.dim() == 2:
        p = p.unsqueeze(0)
    if p.dim() != 3 or p.shape[2] != 2:
        raise BioEMError(ERR_INVALID_ARG, "parts must be [n_parts, n, 2]")
    if out is None:
        out = torch.empty((p.shape[1], 2), dtype=torch.float64, device=ctx.device)
    o = _dev_tensor(out, torch.float64, ctx.device, "out", ndim=2, last=2)
    if o.data_ptr() != out.data_ptr() or o.shape[0] != p.shape[1]:
        raise BioEMError(ERR_INVALID_ARG, "out must be a contiguous [n, 2] float64 tensor")
    _check(ctx, lib().bioem_acc_merge(ctx._h, _ptr(p), p.shape[0], p.shape[1], _ptr(out)), "acc_merge")
    return out


def group_logsumexp(ctx: Context, values, group_len: int):
    """bioem_group_logsumexp: ln sum exp over consecutive groups of ``group_len`` float64 values."""
    torch = _torch()
    v = _dev_tensor(values, torch.float64, ctx.device, "values").reshape(-1)
    if v.numel() % group_len:
        raise BioEMError(ERR_INVALID_ARG, "values must hold whole groups")
    n_groups = v.numel() // group_len
    out = torch.empty(n_groups, dtype=torch.float64, device=ctx.device)
    _check(ctx, lib().bioem_group_logsumexp(ctx._h, _ptr(v), n_groups, int(group_len), _ptr(out)), "group_logsumexp")
    return out


def ln1m(ctx: Context, x):
    """bioem_ln1m: ln(1 - x) for float32 x = rho^2 as the scoring kernels evaluate it (test hook)."""
    torch = _torch()
    v = _dev_tensor(x, torch.float32, ctx.device, "x").reshape(-1)
    out = torch.empty_like(v)
    _check(ctx, lib().bioem_ln1m(ctx._h, _ptr(v), v.numel(), _ptr(out)), "ln1m")
    return out


def fma_peak(ctx: Context, kind: str = "fp32", reps: int = 5) -> float:
    """bioem_fma_peak: measured CUDA-core multiply-add throughput, flop/s ("fp32", "fp32x2", "fp64")."""
    k = {"fp32": 0, "fp32x2": 1, "fp64": 2}[kind]
    out = ctypes.c_double(0.0)
    _check(ctx, lib().bioem_fma_peak(ctx._h, k, int(reps), ctypes.byref(out)), "fma_peak")
    return out.value


def score_accumulate(ctx: Context, images: Images, projset: ProjSet, max_shift: int, acc, first: bool):
    """Fold every parameter set of `projset` into acc [n_img, 2] float64 (max, sum) accumulators."""
    torch = _torch()
    a = _dev_tensor(acc, torch.float64, ctx.device, "acc", ndim=2, last=2)
    if a.data_ptr() != acc.data_ptr():
        raise BioEMError(ERR_INVALID_ARG, "acc must be contiguous")
    _check(ctx, lib().bioem_score_accumulate(ctx._h, images._h, projset._h, int(max_shift), _ptr(acc), 1 if first else 0),
           "score_accumulate")
    return acc


def ensemble(ctx: Context, logP, weights=None, n_iter: int = 0) -> dict:
    """Ensemble posterior of Eq. 10 from a [n_models, n_img] device tensor of ln P (float32 or
    float64): {"log_post": ln P(M | Omega) at the final weights, "weights": [n_models] float64,
    "model_log_post": [n_models] sum over images of ln P of each model alone}."""
    torch = _torch()
    t = _dev_tensor(logP, logP.dtype if logP.dtype in (torch.float32, torch.float64) else torch.float64,
                    ctx.device, "logP", ndim=2)
    M, n = t.shape
    w = torch.full((M,), 1.0 / M, dtype=torch.float64, device=ctx.device) if weights is None else \
        _dev_tensor(weights, torch.float64, ctx.device, "weights", ndim=1).clone()
    out = torch.empty(M + 1, dtype=torch.float64, device=ctx.device)
    _check(ctx, lib().bioem_ensemble(ctx._h, _ptr(t), t.element_size(), int(M), int(n), _ptr(w), int(n_iter),
                                     _ptr(out)), "ensemble")
    return {"log_post": out[0], "weights": w, "model_log_post": out[1:]}


def synthetic_maps(ctx: Context, atoms, sigma_A: float, quats, ctfs, npix: int, pixel_A: float):
    """bioem_synthetic_maps: I1 for pairs (quats[i], ctfs[i]) as a [n, npix, npix] float32 device tensor."""
    torch = _torch()
    a = _dev_tensor(atoms, torch.float32, ctx.device, "atoms", ndim=2, last=4)
    q = _dev_tensor(quats, torch.float32, ctx.device, "quats", ndim=2, last=4)
    c = ctf_array(ctfs)
    if len(c) != q.shape[0]:
        raise BioEMError(ERR_INVALID_ARG, "one CTF row per quaternion")
    out = torch.empty((q.shape[0], npix, npix), dtype=torch.float32, device=ctx.device)
    _check(ctx, lib().bioem_synthetic_maps(ctx._h, ctypes.c_void_p(a.data_ptr()), a.shape[0], float(sigma_A),
                                           ctypes.c_void_p(q.data_ptr()), c, q.shape[0], npix, npix, float(pixel_A),
                                           _ptr(out)), "synthetic_maps")
    return out
