"""ctypes loader of the in-tree CUDA library ``libbioem_gb300.so`` (no torch types cross it)."""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libbioem_gb300.so")

c_int, c_double, c_void_p, c_char_p, c_ull = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_char_p, ctypes.c_ulonglong


class CTF(ctypes.Structure):
    """Mirror of ``bioem_ctf``."""
    _fields_ = [("defocus_A", c_double), ("amp_contrast", c_double), ("bfactor_A2", c_double),
                ("voltage_kV", c_double)]


# name -> (restype, argtypes); every symbol declared in include/bioem.h
SIGNATURES = {
    "bioem_create": (c_int, [ctypes.POINTER(c_void_p), c_int, c_void_p]),
    "bioem_set_stream": (c_int, [c_void_p, c_void_p]),
    "bioem_set_scratch_limit": (c_int, [c_void_p, c_ull]),
    "bioem_set_precision": (c_int, [c_void_p, c_int]),
    "bioem_get_precision": (c_int, [c_void_p]),
    "bioem_set_wait_test": (c_int, [c_void_p, ctypes.c_longlong, c_ull]),
    "bioem_destroy": (None, [c_void_p]),
    "bioem_get_status": (c_int, [c_void_p, ctypes.POINTER(c_int)]),
    "bioem_last_error": (c_char_p, [c_void_p]),
    "bioem_status_string": (c_char_p, [c_int]),
    "bioem_prepare_images": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_double, ctypes.POINTER(c_void_p)]),
    "bioem_project_model": (c_int, [c_void_p, c_void_p, c_int, c_double, c_void_p, c_int, ctypes.POINTER(CTF), c_int,
                                    c_int, c_int, c_double, ctypes.POINTER(c_void_p)]),
    "bioem_score": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p]),
    "bioem_best_params": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p,
                                  c_void_p]),
    "bioem_score_all": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_void_p,
                                c_void_p, c_void_p, c_void_p]),
    "bioem_score_noalloc": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p]),
    "bioem_score_pairs": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, c_void_p, c_void_p]),
    "bioem_synthetic_maps": (c_int, [c_void_p, c_void_p, c_int, c_double, c_void_p, ctypes.POINTER(CTF), c_int, c_int,
                                     c_int, c_double, c_void_p]),
    "bioem_set_kernel_timing": (c_int, [c_void_p, c_int]),
    "bioem_kernel_time": (c_int, [c_void_p, c_char_p, ctypes.POINTER(c_double), ctypes.POINTER(c_ull)]),
    "bioem_reset_kernel_stats": (c_int, [c_void_p]),
    "bioem_launch_count": (c_ull, [c_void_p]),
    "bioem_batch_create": (c_int, [c_void_p, c_int, c_int, ctypes.POINTER(c_void_p), ctypes.POINTER(c_void_p),
                                   ctypes.POINTER(c_int), c_void_p, ctypes.POINTER(c_void_p)]),
    "bioem_batch_run": (c_int, [c_void_p]),
    "bioem_batch_evals": (ctypes.c_longlong, [c_void_p]),
    "bioem_batch_free": (None, [c_void_p]),
    "bioem_autotune": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_char_p, ctypes.POINTER(c_int)]),
    "bioem_autotune_load": (c_int, [c_char_p, ctypes.POINTER(c_int), ctypes.POINTER(c_int)]),
    "bioem_score_gathered": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_int, c_int, c_void_p,
                                     c_int]),
    "bioem_acc_logP": (c_int, [c_void_p, c_void_p, c_int, c_double, c_void_p]),
    "bioem_acc_merge": (c_int, [c_void_p, c_void_p, c_int, c_int, c_void_p]),
    "bioem_group_logsumexp": (c_int, [c_void_p, c_void_p, ctypes.c_longlong, c_int, c_void_p]),
    "bioem_ln1m": (c_int, [c_void_p, c_void_p, ctypes.c_longlong, c_void_p]),
    "bioem_fma_peak": (c_int, [c_void_p, c_int, c_int, ctypes.POINTER(c_double)]),
    "bioem_score_gathered_pairs": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_int, c_int,
                                           c_void_p]),
    "bioem_score_accumulate": (c_int, [c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_int]),
    "bioem_ensemble": (c_int, [c_void_p, c_void_p, c_int, c_int, c_int, c_void_p, c_int, c_void_p]),
    "bioem_cnn_create": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_int, c_int, c_ull, ctypes.POINTER(c_void_p)]),
    "bioem_cnn_num_params": (ctypes.c_longlong, [c_void_p]),
    "bioem_cnn_set_params": (c_int, [c_void_p, c_void_p]),
    "bioem_cnn_get_params": (c_int, [c_void_p, c_void_p]),
    "bioem_cnn_forward": (c_int, [c_void_p, c_void_p, c_int, c_void_p, c_void_p]),
    "bioem_cnn_gradients": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, c_void_p, c_void_p]),
    "bioem_cnn_train_step": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_int, ctypes.c_float, c_void_p]),
    "bioem_propose": (c_int, [c_void_p, c_void_p, c_int, c_int, c_void_p, c_void_p]),
    "bioem_cnn_free": (None, [c_void_p]),
    "bioem_images_count": (c_int, [c_void_p]),
    "bioem_projset_count": (c_int, [c_void_p]),
    "bioem_free_images": (None, [c_void_p]),
    "bioem_free_projset": (None, [c_void_p]),
}

_LIB = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load the library once; raise if it has not been built (there is no fallback path)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError(f"BioEM CUDA library not built: {path} is missing "
                           "(run `python -c \"import __graft_entry__ as g; g.build()\"`)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib
