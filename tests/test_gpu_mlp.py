"""GPU: the learned surrogate's BF16 tensor-core kernels through the C ABI
against the FP64 oracle (oracle/mlp.py).

Tolerances:
  * one layer (a single GEMM + bias) on BF16-rounded operands against the
    FP64 product of the same rounded values: rel-L2 <= 1e-5 (FP32
    accumulation of exactly representable products);
  * the whole network against the FP64 oracle on unrounded values:
    rel-L2 <= 3e-2 for outputs and each layer's gradients (every layer's
    input is rounded to BF16, 2^-9 relative, and the rounding errors of
    four layers add up; near-zero pre-activations may also take the other
    side of the ReLU);
  * the whole network against the oracle evaluated with the kernels'
    storage points (weights, input, hidden activations and gradients
    rounded to BF16; ReLU decided on the stored activation): rel-L2 <= 2e-3
    (left: FP32 against FP64 accumulation, and the odd BF16 rounding that
    lands on the other side of a tie);
  * AdamW on the GPU's own gradients against the oracle's update of the same
    FP32 values: |diff| <= 1e-6 (1 + |p|).
"""
import numpy as np
import pytest

from oracle import mlp as omlp

from gpu_helpers import rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    from paper_2307_15412_gb300 import rr
    c = rr.Context(0)
    yield c
    c.close()


def bf16(a):
    """Round-to-nearest-even to bfloat16, returned as float64 (test-side
    definition of the operand rounding the kernels apply)."""
    f = np.ascontiguousarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def pack(params):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params]).astype(np.float32)


def unpack(flat, dims):
    out, off = [], 0
    for i in range(len(dims) - 1):
        n_in, n_out = dims[i], dims[i + 1]
        W = flat[off:off + n_in * n_out].reshape(n_out, n_in)
        off += n_in * n_out
        b = flat[off:off + n_out]
        off += n_out
        out.append((W, b))
    return out


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


@pytest.mark.parametrize("B,K,N", [(8, 32, 8), (128, 64, 128), (136, 40, 200), (256, 1024, 1024),
                                   (4096, 32, 1024), (512, 1024, 6144), (24, 8, 264)])
def test_single_layer_gemm(ctx, B, K, N):
    """y = x W^T + b: tiles with ragged M, N and K (TMA zero fill)."""
    rng = np.random.default_rng(B + K + N)
    W = rng.normal(size=(N, K)) / np.sqrt(K)
    b = rng.normal(size=N)
    x = rng.uniform(-1, 1, size=(B, K))
    ctx.surrogate_create([K, N])
    ctx.surrogate_set_params(pack([(W, b)]))
    y = torch.empty((B, N), dtype=torch.float32, device="cuda:0")
    ctx.surrogate_forward(dev(x), y)
    ctx.sync()
    ref = bf16(x) @ bf16(W).T + np.float32(b).astype(np.float64)
    assert rel_l2(y.cpu().numpy().astype(np.float64), ref) <= 1e-5


ARCH = [32, 1024, 1024, 1024, 6144]


def test_forward_matches_oracle_full_architecture(ctx):
    params = omlp.init_params(ARCH, 11)
    params = [(W, np.random.default_rng(3).normal(0, 0.05, size=b.shape)) for W, b in params]
    x = np.random.default_rng(5).uniform(-1, 1, size=(64, 32))
    ctx.surrogate_create(ARCH)
    assert ctx.surrogate_num_params() == sum(W.size + b.size for W, b in params)
    ctx.surrogate_set_params(pack(params))
    y = torch.empty((64, 6144), dtype=torch.float32, device="cuda:0")
    ctx.surrogate_forward(dev(x), y)
    ctx.sync()
    ref, _ = omlp.forward(params, x)
    assert rel_l2(y.cpu().numpy().astype(np.float64), ref) <= 3e-2


def _grads(ctx, params, dims, x, t):
    ctx.surrogate_create(dims)
    ctx.surrogate_set_params(pack(params))
    n = ctx.surrogate_num_params()
    g = torch.empty(n, dtype=torch.float32, device="cuda:0")
    loss = torch.empty(1, dtype=torch.float32, device="cuda:0")
    ctx.surrogate_gradients(dev(x), dev(t), g, loss)
    ctx.sync()
    return loss.item(), unpack(g.cpu().numpy().astype(np.float64), dims)


@pytest.mark.parametrize("dims,B", [([32, 64, 64, 48], 16), ([32, 256, 256, 512], 128), ([32, 1024, 1024, 1024, 6144], 64)])
def test_gradients_match_oracle_with_bf16_storage(ctx, dims, B):
    params = omlp.init_params(dims, 21)
    params = [(W, np.random.default_rng(4).normal(0, 0.05, size=b.shape)) for W, b in params]
    rng = np.random.default_rng(9)
    x = rng.uniform(-1, 1, size=(B, dims[0]))
    t = rng.normal(size=(B, dims[-1]))
    loss, got = _grads(ctx, params, dims, x, t)
    ref_loss, ref_g = omlp.backward(params, x, t, store=bf16)
    assert loss / (B * dims[-1]) == pytest.approx(ref_loss, rel=2e-3)
    for l, ((gW, gb), (rW, rb)) in enumerate(zip(got, ref_g)):
        assert rel_l2(gW, rW) <= 2e-3, (l, rel_l2(gW, rW))
        assert rel_l2(gb, rb) <= 2e-3, (l, rel_l2(gb, rb))


@pytest.mark.parametrize("dims,B", [([32, 256, 256, 512], 128), ([32, 1024, 1024, 1024, 6144], 256)])
def test_gradients_match_oracle(ctx, dims, B):
    params = omlp.init_params(dims, 21)
    params = [(W, np.random.default_rng(4).normal(0, 0.05, size=b.shape)) for W, b in params]
    rng = np.random.default_rng(9)
    x = rng.uniform(-1, 1, size=(B, dims[0]))
    t = rng.normal(size=(B, dims[-1]))
    ctx.surrogate_create(dims)
    ctx.surrogate_set_params(pack(params))
    n = ctx.surrogate_num_params()
    g = torch.empty(n, dtype=torch.float32, device="cuda:0")
    loss = torch.empty(1, dtype=torch.float32, device="cuda:0")
    ctx.surrogate_gradients(dev(x), dev(t), g, loss)
    ctx.sync()
    ref_loss, ref_g = omlp.backward(params, x, t)
    got = unpack(g.cpu().numpy().astype(np.float64), dims)
    assert loss.item() / (B * dims[-1]) == pytest.approx(ref_loss, rel=3e-2)
    for l, ((gW, gb), (rW, rb)) in enumerate(zip(got, ref_g)):
        assert rel_l2(gW, rW) <= 3e-2, (l, rel_l2(gW, rW))
        assert rel_l2(gb, rb) <= 3e-2, (l, rel_l2(gb, rb))


def test_adamw_step_matches_oracle(ctx):
    dims = [32, 64, 48]
    params = omlp.init_params(dims, 2)
    rng = np.random.default_rng(1)
    x = rng.uniform(-1, 1, size=(32, 32))
    t = rng.normal(size=(32, 48))
    ctx.surrogate_create(dims)
    p0 = pack(params)
    ctx.surrogate_set_params(p0)
    n = ctx.surrogate_num_params()
    g = torch.empty(n, dtype=torch.float32, device="cuda:0")
    ctx.surrogate_gradients(dev(x), dev(t), g)
    lr, wd = 1e-2, 0.05
    ctx.surrogate_train_step(dev(x), dev(t), lr=lr, weight_decay=wd)
    p1 = torch.empty(n, dtype=torch.float32, device="cuda:0")
    ctx.surrogate_get_params(p1)
    ctx.sync()
    gg = g.cpu().numpy().astype(np.float64)
    decay = np.concatenate([np.concatenate([np.ones(W.size), np.zeros(b.size)]) for W, b in params])
    ref = np.empty(n)
    for mask_val in (0.0, 1.0):
        sel = decay == mask_val
        pr, _, _ = omlp.adamw_step(p0.astype(np.float64)[sel], gg[sel], np.zeros(sel.sum()), np.zeros(sel.sum()), 1,
                                   lr, wd=wd * mask_val)
        ref[sel] = pr
    got = p1.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= 1e-6 * (1 + np.abs(ref)))


def test_training_fits_a_teacher_network(ctx):
    """A student of the same shape trained by the GPU kernels on a teacher's
    outputs: the epoch loss keeps falling, by 5x or more in 40 epochs."""
    dims = [32, 256, 256, 256]
    teacher = omlp.init_params(dims, 40)
    rng = np.random.default_rng(41)
    X = rng.uniform(-1, 1, size=(8192, 32))
    T, _ = omlp.forward(teacher, X)
    ctx.surrogate_create(dims)
    ctx.surrogate_set_params(pack(omlp.init_params(dims, 42)))
    losses = ctx.surrogate_train(dev(X), dev(T), epochs=40, batch=256, seed=3, lr=2e-3)
    assert all(np.isfinite(losses))
    assert losses[-1] <= 0.2 * losses[0], losses
    assert losses[-1] < min(losses[:20]), losses


def test_infer_flags_rows_outside_the_training_box(ctx):
    dims = [32, 64, 16]
    ctx.surrogate_create(dims)
    ctx.surrogate_set_params(pack(omlp.init_params(dims, 1)))
    x = np.random.default_rng(0).uniform(-1, 1, size=(21, 32)).astype(np.float32)  # ragged count
    x[3, 5] = 1.5
    x[20, 0] = -1.01
    y = torch.empty((21, 16), dtype=torch.float32, device="cuda:0")
    fb = torch.empty(21, dtype=torch.uint8, device="cuda:0")
    ctx.surrogate_infer(dev(x), y, fb)
    ctx.sync()
    flags = fb.cpu().numpy()
    assert list(np.nonzero(flags)[0]) == [3, 20]
    ref, _ = omlp.forward(omlp.init_params(dims, 1), x.astype(np.float64))
    assert rel_l2(y.cpu().numpy().astype(np.float64), ref) <= 3e-2
