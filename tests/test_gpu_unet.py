"""The convolutional warm start (lbms_unet_* of include/lbms_net.h) against a
plain PyTorch FP32 reference of the same network on the CPU (Conv3d,
max_pool3d, ConvTranspose3d, concatenation), with BF16 roundings at the
points where the device stores BF16: weights, activations after each
ReLU / transposed convolution, and the gradients at those points.

Checks: the forward pass; the loss and every parameter gradient; the
first Adam step; training; parameter layout round trips; and the warm
start of a porous anode whose extents are not multiples of 4.
"""
import numpy as np
import pytest

from workloads import cases

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
F = torch.nn.functional


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_01600_gb300 import lbms
    lbms.load()
    return lbms


def _bf(t):
    return t.to(torch.bfloat16).to(torch.float32)


class _GradBF16(torch.autograd.Function):
    """Identity forward; the incoming gradient rounded to BF16 (the device
    stores the head's output gradient as BF16)."""

    @staticmethod
    def forward(ctx, x):
        return x.view_as(x)

    @staticmethod
    def backward(ctx, g):
        return _bf(g)


def _reference(params, x):
    """The network as PyTorch functional ops; params in lbms_unet_get order."""
    p = [torch.tensor(a, requires_grad=True) for a in params]
    # straight-through BF16 weights: the value is rounded, the gradient is not
    W = [w + (_bf(w) - w).detach() for w in p[0::2]]
    b = p[1::2]

    def conv(h, i):
        return _bf(F.relu(F.conv3d(h, W[i], b[i], padding=1)))

    x0 = _bf(torch.tensor(x))
    e1 = conv(conv(x0, 0), 1)
    e2 = conv(conv(F.max_pool3d(e1, 2), 2), 3)
    e3 = conv(conv(F.max_pool3d(e2, 2), 4), 5)
    u2 = _bf(F.conv_transpose3d(e3, W[6], b[6], stride=2))
    d2 = conv(conv(torch.cat([u2, e2], 1), 7), 8)
    u1 = _bf(F.conv_transpose3d(d2, W[9], b[9], stride=2))
    d1 = conv(conv(torch.cat([u1, e1], 1), 10), 11)
    y = _GradBF16.apply(F.conv3d(d1, W[12], b[12]))
    return p, y


def _loss(y, t, m):
    return (((y - t) * m) ** 2).sum() / (3.0 * m.sum())


def _random_params(net, seed, head_scale=0.3):
    rng = np.random.default_rng(seed)
    out = []
    for sh in net.shapes():
        if len(sh) == 1:
            out.append((0.05 * rng.standard_normal(sh)).astype(np.float32))
        else:
            fan = int(np.prod(sh[1:])) if sh[2] == 3 or sh[2] == 1 else sh[0]
            a = np.sqrt(6.0 / fan) * (head_scale if sh[2] == 1 else 1.0)
            out.append(rng.uniform(-a, a, sh).astype(np.float32))
    return out


def _volumes(B, Z, Y, X, seed, porosity=0.6):
    """Inputs like the anode volumes: 16 feature channels in [0, 1] on fluid
    voxels (zero on solid ones), channel 16 the fluid mask."""
    rng = np.random.default_rng(seed)
    m = (rng.random((B, 1, Z, Y, X)) < porosity).astype(np.float32)
    f = rng.random((B, 16, Z, Y, X)).astype(np.float32) * m
    return np.concatenate([f, m], axis=1)


def _targets(x):
    """A smooth function of the inputs (learnable), zero on solid voxels."""
    m = x[:, 16:17]
    box = F.avg_pool3d(torch.tensor(x[:, 0:3]), 3, stride=1, padding=1).numpy()
    return (4.0 * box + x[:, 3:6] * x[:, 6:7] - 1.0) * m


SHAPES = [(2, 8, 12, 16), (1, 4, 8, 20), (3, 4, 4, 12)]   # B, Z, Y, X (the last two pad levels 1 and 2)


@pytest.mark.parametrize("B,Z,Y,X", SHAPES)
def test_forward_matches_reference(L, B, Z, Y, X):
    net = L.UNet(width=28, max_voxels=4096, seed=1)
    params = _random_params(net, 21)
    net.set(params)
    x = _volumes(B, Z, Y, X, 22)
    out = net.forward(x)
    _, y = _reference(params, x)
    y = y.detach().numpy()
    assert out.shape == y.shape
    scale = np.abs(y).max()
    assert scale > 0.1
    assert np.linalg.norm(out - y) <= 1e-2 * np.linalg.norm(y)
    assert np.all(np.abs(out - y) <= 3e-2 * np.abs(y) + 1e-2 * scale)
    assert net.gemm_calls() == 13 + 0          # one product per layer, all on tcgen05
    net.close()


@pytest.mark.parametrize("B,Z,Y,X", SHAPES[:2])
def test_loss_and_gradients_match_reference(L, B, Z, Y, X):
    net = L.UNet(width=28, max_voxels=4096, seed=2)
    params = _random_params(net, 31)
    net.set(params)
    x = _volumes(B, Z, Y, X, 32)
    t = _targets(x).astype(np.float32)
    loss = net.train_batch(x, t, lr=0.0)
    p, y = _reference(params, x)
    lref = _loss(y, torch.tensor(t), torch.tensor(x[:, 16:17]))
    lref.backward()
    assert loss == pytest.approx(float(lref.detach()), rel=1e-2)
    grads = net.get(1)
    assert [g.shape for g in grads] == [tuple(q.shape) for q in p]
    # Element bound: 5 % of the entry + 5 % of the layer's largest.  The
    # bottom level of the (1, 4, 8, 20) batch holds 10 voxels, where one BF16
    # rounding or ReLU-mask flip between the two summation orders moves one
    # channel's entries by up to 3.3 % of the layer maximum (measured: 3 of
    # 169,344 entries of e3a, one channel); in norm every layer stays within
    # 2.8 % of the reference.
    for i, (g, q) in enumerate(zip(grads, p)):
        r = q.grad.numpy()
        gmax = np.abs(r).max()
        assert gmax > 0, f"parameter {i}: zero reference gradient"
        assert np.linalg.norm(g - r) <= 3e-2 * np.linalg.norm(r), f"parameter {i}"
        assert np.all(np.abs(g - r) <= 5e-2 * np.abs(r) + 5e-2 * gmax), f"parameter {i}"
    # the parameters did not move at lr = 0
    for a, b in zip(net.get(0), params):
        assert np.array_equal(a, b)
    net.close()


def test_parameter_layout_round_trip(L):
    net = L.UNet(width=12, max_voxels=1024, seed=3)
    n, _ = net.info()
    shapes = net.shapes()
    assert n == sum(int(np.prod(s)) for s in shapes)
    params = _random_params(net, 41)
    net.set(params)
    for a, b in zip(net.get(0), params):
        assert np.array_equal(a, b)
    # the parameter count of the comparison network (width 28)
    w = L.UNet(width=28, max_voxels=1024, seed=0)
    assert w.info()[0] == 1050031
    w.close()
    net.close()


def test_fresh_network_starts_at_the_profile(L):
    """He-uniform convolutions but a zero head: the first output is zero."""
    net = L.UNet(width=28, max_voxels=4096, seed=4)
    out = net.forward(_volumes(1, 8, 8, 16, 5))
    assert np.all(out == 0.0)
    net.close()


def test_first_adam_step_moves_every_weight_by_lr(L):
    net = L.UNet(width=16, max_voxels=4096, seed=5)
    params = _random_params(net, 51)
    net.set(params)
    x = _volumes(2, 8, 8, 16, 52)
    t = _targets(x).astype(np.float32)
    net.train_batch(x, t, lr=0.0)
    g = net.get(1)
    net.train_batch(x, t, lr=1e-3)
    moved = 0
    for W1, W0, gW in zip(net.get(0), params, g):
        m = np.abs(gW) > 1e-4
        moved += int(m.sum())
        assert np.allclose((W1 - W0)[m], -1e-3 * np.sign(gW[m]), rtol=1e-3, atol=1e-7)
    assert moved > 0.25 * sum(p.size for p in params)
    net.close()


def test_training_reduces_the_loss(L):
    """300 Adam steps on one batch: the same network in plain PyTorch FP32
    (same data, zero head, lr 2e-3) goes from 0.246 to 0.098 and levels off
    near 0.07 by 600 steps, so a halving is the bar."""
    net = L.UNet(width=16, max_voxels=4096, seed=6)
    x = _volumes(2, 8, 12, 16, 61)
    t = _targets(x).astype(np.float32)
    first = net.train_batch(x, t, lr=2e-3)
    for _ in range(300):
        last = net.train_batch(x, t, lr=2e-3)
    assert last < 0.5 * first
    net.close()


def test_bad_volumes_are_rejected(L):
    net = L.UNet(width=8, max_voxels=1024, seed=7)
    with pytest.raises(L.LbmsError):
        net.forward(_volumes(1, 4, 4, 6, 1))          # extent not a multiple of 4
    with pytest.raises(L.LbmsError):
        net.forward(_volumes(1, 8, 8, 32, 1))         # 2048 voxels > max_voxels
    with pytest.raises(L.LbmsError):
        net.train(10)                                 # no training volumes
    net.close()


def _anodes(seeds, shape=(14, 16, 38)):
    out = []
    for k, sd in enumerate(seeds):
        out.append(cases.porous(shape, radius=2, porosity=0.45 + 0.02 * (k % 3), seed=sd,
                                current_A_cm2=0.5 + 0.25 * (k % 4)))
    return out


def test_warm_start_predicts_better_than_the_profile_and_converges_to_the_same_state(L):
    """Trained on 8 steady anodes of 38 x 16 x 14 cells (placed in 40 x 16 x
    16 volumes), the U-Net's start of a held-out anode is closer to its
    steady state than the Section 4.1 profile, and the LBM from it reaches
    the same steady state."""
    train = _anodes([401, 402, 403, 404, 405, 406, 407, 408])
    test = _anodes([499])[0].with_(current_A_cm2=1.0)
    b = L.Batch.from_cases(train, precision="fp32", extrapolate_every=5000)
    for k, c in enumerate(train):
        b.set_bc(c.x_in, c.current_A_cm2, case=k)
    b.run_to_residual(1e-9, 2_000_000)
    net = L.UNet(width=16, max_voxels=8 * 40 * 16 * 16, seed=8)
    for k in range(len(train)):
        net.add_sample(b, k)
    assert net.info()[1] == len(train)
    net.train(400, max_batch=8, lr=2e-3)

    ref = L.Solver.from_case(test, precision="fp64")
    ref.set_bc(test.x_in, test.current_A_cm2)
    ref.run_to_residual(1e-12, 3_000_000)
    Xs = ref.fields()
    prof = L.Solver.from_case(test, precision="fp64", init_mode="profile1d")
    prof.set_bc(test.x_in, test.current_A_cm2)
    Xp = prof.fields()
    warm = L.Solver.from_case(test, precision="fp64")
    warm.set_bc(test.x_in, test.current_A_cm2)
    Xw = net.warm_start(warm)
    f = ~test.solid
    assert np.allclose(Xw[:, f].sum(axis=0), 1.0, atol=1e-12)
    assert np.array_equal(warm.fields()[:, f], Xw[:, f])
    assert np.all(Xw[:, ~f] == 0.0)
    rms_w = np.sqrt(((Xw - Xs)[:, f] ** 2).mean())
    rms_p = np.sqrt(((Xp - Xs)[:, f] ** 2).mean())
    assert rms_w < rms_p
    warm.run_to_residual(1e-12, 3_000_000)
    assert np.abs(warm.fields() - Xs)[:, f].max() < 1e-7
    net.close()


def test_training_on_added_volumes_of_two_grids(L):
    """Training volumes of two grids (two batch layouts sharing the buffers,
    which grow for the larger one): the loss of the training loop falls, and
    afterwards the forward pass on the first grid still matches the PyTorch
    reference with the trained parameters (no halo row left dirty by the
    other layout)."""
    net = L.UNet(width=12, max_voxels=4 * 16 * 16 * 24, seed=9)
    a = _volumes(3, 8, 8, 16, 91)
    b = _volumes(2, 16, 16, 24, 92)
    for x in list(a) + list(b):
        net.add_volume(x, _targets(x[None])[0].astype(np.float32))
    assert net.info()[1] == 5
    first = net.train(2, max_batch=4, lr=2e-3)
    last = net.train(200, max_batch=4, lr=2e-3)
    params = net.get(0)
    out = net.forward(a)
    _, y = _reference(params, a)
    y = y.detach().numpy()
    assert np.linalg.norm(out - y) <= 1e-2 * np.linalg.norm(y)
    # 100 cosine-decayed steps per grid at width 12: measured 0.240 -> 0.185
    assert last < 0.85 * first
    net.close()
