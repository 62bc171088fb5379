"""Write the stored FP64 oracle values the GPU tests compare with:

  tiny_logP.txt            log P of the 16 tiny-workload images
  precision64_subset.txt   per image of the 64-image precision subsets (full 6912-set grid, +-4 px):
  precision128_subset.txt  log P, best ln L, best (q, ctf, dy, dx), best minus runner-up pair max

Calls only ``oracle`` and ``workloads`` (seeded draws).  Run from the repository root:
    python tests/golden/make_golden.py [tiny|precision64|precision128 ...]
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads  # noqa: E402


def precision_subset(name):
    cfg = workloads.get_config(name)
    wl = workloads.workload(cfg)
    imgs = oracle.synthesize_images(wl)
    r = oracle.score(imgs, wl["atoms"], wl["quats"], wl["ctfs"], cfg.sigma_A, cfg.pixel_A, cfg.max_shift)
    rows = []
    for w in range(len(imgs)):
        top2 = np.sort(r["pair_max"][w])[-2:]
        q, c, dy, dx, ll = r["best"][w]
        rows.append([r["logP"][w], ll, q, c, dy, dx, top2[1] - top2[0]])
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"{name}_subset.txt")
    header = (f"FP64 oracle values for the {len(imgs)} images of the {name} workload ({cfg.npix}x{cfg.npix} @ "
              f"{cfg.pixel_A} A, {len(wl['quats']) * len(wl['ctfs'])} parameter sets, shifts +-{cfg.max_shift}); "
              "columns: log P, best ln L, best q, best ctf, best dy, best dx, best minus runner-up pair max; "
              "written by tests/golden/make_golden.py")
    np.savetxt(out, np.asarray(rows), fmt="%.15e", header=header)


def tiny():
    cfg = workloads.get_config("tiny")
    wl = workloads.workload(cfg)
    imgs = oracle.synthesize_images(wl)
    r = oracle.score(imgs, wl["atoms"], wl["quats"], wl["ctfs"], cfg.sigma_A, cfg.pixel_A, cfg.max_shift)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_logP.txt")
    header = ("FP64 oracle log P(image | model) of the 16 images of the tiny workload "
              "(32x32 @ 2 A, 6912 parameter sets, shifts +-4); written by tests/golden/make_golden.py")
    np.savetxt(out, r["logP"], fmt="%.15e", header=header)


def main(names):
    for n in names:
        tiny() if n == "tiny" else precision_subset(n)


if __name__ == "__main__":
    main(sys.argv[1:] or ["tiny", "precision64", "precision128"])
