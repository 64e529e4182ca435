"""Runs N frames of a workload through the C ABI, untimed (for profilers).

  python -m paper_2307_15412_gb300.run_case [--workload full|tiny] [--frames N]
         [--scenes S] [--no-flush]

Each frame: build_bvh, trace_frame, synth_if (plain FP32), range_doppler on
one of S resident seeded scenes; L2 is flushed (256 MiB write) before each
frame unless --no-flush, as in the benchmark.
"""
from __future__ import annotations

import argparse
import os
import sys


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="full", choices=["full", "tiny"])
    ap.add_argument("--frames", type=int, default=4)
    ap.add_argument("--scenes", type=int, default=2)
    ap.add_argument("--no-flush", action="store_true")
    args = ap.parse_args()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch

    from paper_2307_15412_gb300 import inputs as I
    from paper_2307_15412_gb300 import rr

    if args.workload == "full":
        radar, grid, nt = I.workload_full_frame()
        scenes = [I.hand_scene(k, nt, range_m=I.FULL_FRAME_RANGE, speed=I.FULL_FRAME_SPEED)
                  for k in range(args.scenes)]
    else:
        radar, grid, nt = I.workload_tiny()
        scenes = [I.hand_scene(k, nt) for k in range(args.scenes)]
    ctx = rr.Context(0)
    for k, s in enumerate(scenes):
        ctx.scene_upload(k, s.V, s.F, s.vel)
    if_out = torch.empty((radar.n_rx, radar.n_chirps, radar.n_samples, 2), dtype=torch.float32, device="cuda:0")
    rd_out = torch.empty_like(if_out)
    flush = None if args.no_flush else torch.empty(256 << 20, dtype=torch.uint8, device="cuda:0")
    for i in range(args.frames):
        if flush is not None:
            flush.zero_()
        ctx.run_frame(i % len(scenes), radar, grid, if_out=if_out, rd_out=rd_out)
    ctx.sync()
    torch.cuda.synchronize()
    ctx.close()
    print("ran %d frames" % args.frames)


if __name__ == "__main__":
    main()
