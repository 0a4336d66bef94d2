"""Fill the launch-variant cache (fsp_autotune) for the benchmark geometries on this GPU.

    python -m paper_2103_08531_gb300.tune [--out PATH] [--mode 1|2]

Each geometry's forward passes are timed in every launch variant the library
offers for them (column-tile engine and values per thread, the radix split of
the transforms at 128, 256 and 512 points, CTAs per SM, the middle-pass kernel
for 1024- to 8192-point lines); the fastest variant per
(pass, padded length) is written to PATH, keyed by GPU architecture.  Mode 1
keeps entries already in the file, mode 2 re-times everything.  Solves read the
file through Plan.autotune(PATH, 0) or FSP_AUTOTUNE=cached FSP_TUNE_CACHE=PATH.
"""
from __future__ import annotations

import argparse
import os

import torch

from . import solver

HERE = os.path.dirname(os.path.abspath(__file__))
TUNE_CACHE = os.path.join(HERE, "tune_cache.json")

# the geometries of the benchmark workloads: the 256^3 cube, the 4096^2 square,
# the 128^3 training grid and the five beam-bunch shapes (spacings do not
# change the passes)
GEOMETRIES = [((256, 256, 256), (2 / 256,) * 3), ((4096, 4096), (2 / 4096,) * 2), ((128, 128, 128), (2 / 128,) * 3),
              ((64, 64, 64), (0.01,) * 3), ((96, 96, 96), (0.01,) * 3), ((64, 64, 256), (0.01,) * 3),
              ((128, 128, 512), (0.01,) * 3)]


def tune(path: str = TUNE_CACHE, mode: int = 1, geometries=GEOMETRIES) -> str:
    for shape, h in geometries:
        plan = solver.Plan(shape, h, "vgf")
        plan.autotune(path, mode)
        plan.close()
        torch.cuda.empty_cache()
    return path


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--out", default=TUNE_CACHE)
    ap.add_argument("--mode", type=int, default=1, choices=[1, 2])
    args = ap.parse_args()
    print(tune(args.out, args.mode))


if __name__ == "__main__":
    main()
