"""Write tests/golden/tiny_logP.txt: the FP64 oracle's log P of the 16 tiny-workload images.

Calls only ``oracle`` and ``workloads`` (seeded draws).  Run from the repository root:
    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import workloads  # noqa: E402


def main():
    cfg = workloads.get_config("tiny")
    wl = workloads.workload(cfg)
    imgs = oracle.synthesize_images(wl)
    r = oracle.score(imgs, wl["atoms"], wl["quats"], wl["ctfs"], cfg.sigma_A, cfg.pixel_A, cfg.max_shift)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_logP.txt")
    header = ("FP64 oracle log P(image | model) of the 16 images of the tiny workload "
              "(32x32 @ 2 A, 6912 parameter sets, shifts +-4); written by tests/golden/make_golden.py")
    np.savetxt(out, r["logP"], fmt="%.15e", header=header)


if __name__ == "__main__":
    main()
