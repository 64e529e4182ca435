"""Runs N steps of a workload through the C ABI, untimed (for profilers).

  python -m paper_2307_15412_gb300.run_case [--workload full|tiny] [--steps N]
         [--scenes S] [--batch] [--variant 0|1|2] [--no-flush]
  python -m paper_2307_15412_gb300.run_case --mlp [--steps N] [--mlp-batch B]

Each step runs every one of the S resident seeded scenes: one rr_run_frame
per scene, or with --batch one rr_batch_run over all of them.  --variant
selects the synthesis (0 FP32, 1 tensor-core BF16x3, 2 tensor-core TF32).
L2 is flushed (256 MiB write) before each step unless --no-flush, as in the
benchmark.  --mlp instead runs the learned surrogate (32-1024-1024-1024-6144,
seeded parameters): per step one training step and one inference on a
batch of B seeded inputs.
"""
from __future__ import annotations

import argparse
import os
import sys


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="full", choices=["full", "tiny"])
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--scenes", type=int, default=2)
    ap.add_argument("--batch", action="store_true")
    ap.add_argument("--variant", type=int, default=0, choices=[0, 1, 2])
    ap.add_argument("--no-flush", action="store_true")
    ap.add_argument("--mlp", action="store_true")
    ap.add_argument("--mlp-batch", type=int, default=4096)
    args = ap.parse_args()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch

    from paper_2307_15412_gb300 import inputs as I
    from paper_2307_15412_gb300 import rr

    if args.mlp:
        return run_mlp(args, torch, I, rr)
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
    S = len(scenes)
    if_out = torch.empty((S, radar.n_rx, radar.n_chirps, radar.n_samples, 2), dtype=torch.float32, device="cuda:0")
    rd_out = torch.empty_like(if_out)
    flush = None if args.no_flush else torch.empty(256 << 20, dtype=torch.uint8, device="cuda:0")
    for i in range(args.steps):
        if flush is not None:
            flush.zero_()
        if args.batch:
            ctx.batch_run([(k, grid) for k in range(S)], radar, if_out=if_out, rd_out=rd_out, variant=args.variant)
        else:
            for k in range(S):
                ctx.run_frame(k, radar, grid, if_out=if_out[k], rd_out=rd_out[k], variant=args.variant)
    ctx.sync()
    torch.cuda.synchronize()
    ctx.close()
    print("ran %d steps of %d scenes" % (args.steps, S))


def run_mlp(args, torch, I, rr):
    dims = (32, 1024, 1024, 1024, 6144)
    ctx = rr.Context(0)
    ctx.surrogate_create(dims)
    ctx.surrogate_set_params(I.surrogate_init_params(dims, 0))
    B = args.mlp_batch
    x = torch.from_numpy(I.surrogate_features(I.surrogate_inputs(0, B))).cuda()
    t = torch.randn((B, dims[-1]), generator=torch.Generator().manual_seed(0)).cuda()
    y = torch.empty((B, dims[-1]), dtype=torch.float32, device="cuda:0")
    for i in range(args.steps):
        ctx.surrogate_train_step(x, t, lr=1e-4)
        ctx.surrogate_forward(x, y)
    ctx.sync()
    torch.cuda.synchronize()
    ctx.close()
    print("ran %d surrogate steps at batch %d" % (args.steps, B))


if __name__ == "__main__":
    main()
