"""FEC's serial point-wise scheme against the exact components, on seeded workloads.

TEST INFRASTRUCTURE ONLY (it runs the oracle).  Prints one Markdown table row
per workload: cluster counts of the serial loop and of the exact components
(same size bounds), exact components the serial loop splits, and the points in
them.  Run from the repository root:

    python -m oracle.serial_report
"""
from __future__ import annotations

import time

from paper_2208_07678_gb300 import synth

from .paper_fec import compare_with_exact


def workloads():
    c = synth.blobs_20k()
    yield "blobs_20k", c.xyz, c.d, c.min_size, c.max_size
    c = synth.frame_120k()
    yield "frame_120k", c.xyz, c.d, c.min_size, c.max_size
    for sigma in (0.0, 0.2):
        xyz = synth.voxel_clusters(7, 1000, 100, sigma=sigma)
        yield f"voxel_clusters 1000 x 100, sigma {sigma}", xyz, 0.5, 1, (1 << 63) - 1


def main():
    print("| workload | n | exact clusters | serial clusters | exact components split | points in them | s |")
    print("|---|---|---|---|---|---|---|")
    for name, xyz, d, lo, hi in workloads():
        t0 = time.perf_counter()
        r = compare_with_exact(xyz, d, lo, hi)
        dt = time.perf_counter() - t0
        print(f"| {name} | {r['n']:,} | {r['k_exact']:,} | {r['k_serial']:,} | "
              f"{r['components_split']:,} | {r['points_in_split_components']:,} | {dt:.1f} |")


if __name__ == "__main__":
    main()
