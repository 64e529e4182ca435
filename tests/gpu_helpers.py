"""Shared helpers of the GPU parity tests (no method arithmetic)."""
import numpy as np


def to_complex(t):
    """torch float32 [..., 2] (CUDA or CPU) -> numpy complex128."""
    a = t.detach().double().cpu().numpy()
    return a[..., 0] + 1j * a[..., 1]


def rel_l2(got, ref):
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(got - ref) / (den if den > 0 else 1.0))


def gpu_hits(ctx, scene, n_rx, K):
    """Copies the scene's hit list (K hits) to host numpy arrays."""
    import torch
    dev = "cuda:%d" % ctx.device
    ray = torch.empty(max(K, 1), dtype=torch.int32, device=dev)
    tri = torch.empty_like(ray)
    t = torch.empty(max(K, 1), dtype=torch.float32, device=dev)
    d = torch.empty((n_rx, max(K, 1)), dtype=torch.float32, device=dev)
    a = torch.empty_like(d)
    dd = torch.empty_like(d)
    if K > 0:
        ctx.get_hits(scene, K, ray, tri, t, d, a, dd)
    ctx.sync()
    return dict(ray=ray[:K].cpu().numpy(), tri=tri[:K].cpu().numpy(), t=t[:K].cpu().numpy(),
                d=d[:, :K].cpu().numpy(), a=a[:, :K].cpu().numpy(), dd=dd[:, :K].cpu().numpy(),
                d_dev=d[:, :K].contiguous(), a_dev=a[:, :K].contiguous(), dd_dev=dd[:, :K].contiguous())


def trace_scene(ctx, scene_id, scene, radar, grid, cap=0):
    ctx.scene_upload(scene_id, scene.V, scene.F, scene.vel)
    ctx.build_bvh(scene_id)
    cnt = ctx.trace_frame(scene_id, radar, grid, hit_capacity=cap)
    ctx.sync()
    return gpu_hits(ctx, scene_id, radar.n_rx, cnt[0])


def per_ray(n_rays, hits):
    tri = np.full(n_rays, -1, np.int64)
    t = np.zeros(n_rays)
    tri[hits["ray"]] = hits["tri"]
    t[hits["ray"]] = hits["t"]
    return tri, t
