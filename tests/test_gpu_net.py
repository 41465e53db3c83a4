"""The warm-start network (include/lbms_net.h) against a plain PyTorch FP32
reference of the same computation on the CPU: the forward pass, the loss,
the gradients and one Adam step; then training and the warm start itself on
small porous anodes, where the LBM from the predicted start must reach the
same steady state as from the uniform start."""
import numpy as np
import pytest

import closed_forms as cf
from workloads import cases

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def L():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_01600_gb300 import lbms
    lbms.load()
    return lbms


def _bf(t):
    return t.to(torch.bfloat16).to(torch.float32)


def _random_net(L, width, depth, seed):
    net = L.Net(width=width, depth=depth, seed=seed)
    rng = np.random.default_rng(seed)
    layers = []
    for W, b in net.get(0):
        fan = W.shape[1] if W.shape[1] != L.Net.FEATURES else 16
        layers.append(((rng.standard_normal(W.shape) * np.sqrt(2.0 / fan)).astype(np.float32),
                       (0.1 * rng.standard_normal(b.shape)).astype(np.float32)))
    net.set(layers)
    return net, layers


def _features(L, rows, seed):
    rng = np.random.default_rng(seed)
    f = np.zeros((rows, L.Net.FEATURES), dtype=np.float32)
    f[:, :16] = rng.uniform(-1.0, 1.0, (rows, 16))
    return L.to_bf16_bits(f), L.from_bf16_bits(L.to_bf16_bits(f)).reshape(rows, -1)


def _reference(layers, x, targets=None):
    """FP32 reference with the network's BF16 roundings: weights, the input
    rows and every hidden activation are rounded to BF16."""
    ts = [(torch.tensor(W, requires_grad=True), torch.tensor(b, requires_grad=True)) for W, b in layers]
    h = torch.tensor(x)
    for l, (W, b) in enumerate(ts):
        z = h @ _bf(W).T + b
        h = _bf(torch.relu(z)) if l < len(ts) - 1 else z
    if targets is None:
        return h.detach().numpy(), None, None
    loss = ((h - torch.tensor(targets)) ** 2).mean()
    loss.backward()
    return h.detach().numpy(), float(loss.detach()), [(W.grad.numpy(), b.grad.numpy()) for W, b in ts]


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


GEMMS = ["tcgen05", "mma_sync"]


def _used_only(net, kind):
    tc, ms = net.gemm_calls()
    return (tc > 0 and ms == 0) if kind == "tcgen05" else (ms > 0 and tc == 0)


@pytest.mark.parametrize("gemm", GEMMS)
@pytest.mark.parametrize("width,rows", [(128, 256), (704, 192)])
def test_forward_matches_reference(L, gemm, width, rows):
    """Forward pass on the tcgen05 (TMA + TMEM) and the mma.sync products;
    width 704 and 192 rows leave partial 128-row tiles (zero-filled by TMA)."""
    net, layers = _random_net(L, width, 2, 5)
    net.set_gemm(gemm)
    bits, x = _features(L, rows, 6)
    out = net.forward(bits)
    ref, _, _ = _reference(layers, x)
    assert out.shape == (rows, 3)
    assert _rel(out, ref) < 5e-3
    assert np.all(np.abs(out - ref) <= 2e-2 * np.abs(ref) + 1e-2 * np.abs(ref).max())
    assert _used_only(net, gemm)


@pytest.mark.parametrize("gemm", GEMMS)
def test_gradients_and_loss_match_reference(L, gemm):
    net, layers = _random_net(L, 128, 2, 7)
    net.set_gemm(gemm)
    bits, x = _features(L, 512, 8)
    t = np.random.default_rng(9).standard_normal((512, 3)).astype(np.float32)
    loss = net.train_batch(bits, t, lr=0.0)
    assert _used_only(net, gemm)
    _, ref_loss, ref_grads = _reference(layers, x, t)
    assert loss == pytest.approx(ref_loss, rel=1e-4)
    got = net.get(1)
    for (gW, gb), (rW, rb) in zip(got, ref_grads):
        assert _rel(gW, rW) < 3e-2
        assert _rel(gb, rb) < 3e-2
        # element by element: the device rounds the output and hidden-layer
        # gradients to BF16 (2^-8 relative) before the weight-gradient
        # products, so each entry is within a few per cent of its own size
        # plus a few per cent of the layer's largest entry
        for g, r in ((gW, rW), (gb, rb)):
            assert np.all(np.abs(g - r) <= 3e-2 * np.abs(r) + 2e-2 * np.abs(r).max())
    # lr = 0 leaves the parameters as they were
    for (W, b), (W0, b0) in zip(net.get(0), layers):
        assert np.array_equal(W, W0) and np.array_equal(b, b0)


def test_first_adam_step_moves_every_weight_by_lr(L):
    """At step 1 Adam's bias-corrected update is lr * g / |g| (Kingma & Ba)."""
    net, layers = _random_net(L, 64, 1, 11)
    bits, x = _features(L, 128, 12)
    t = np.random.default_rng(13).standard_normal((128, 3)).astype(np.float32)
    net.train_batch(bits, t, lr=0.0)
    g = net.get(1)
    net.train_batch(bits, t, lr=1e-3)
    for (W1, _), (W0, _), (gW, _) in zip(net.get(0), layers, g):
        m = np.abs(gW) > 1e-4
        assert np.allclose((W1 - W0)[m], -1e-3 * np.sign(gW[m]), rtol=1e-3, atol=1e-7)


def test_training_reduces_the_loss(L):
    net = L.Net(width=128, depth=2, seed=17)
    bits, x = _features(L, 1024, 18)
    t = np.stack([np.sin(2 * x[:, 0]) + x[:, 1] * x[:, 2], x[:, 3] ** 2, np.cos(x[:, 4])], axis=1).astype(np.float32)
    first = net.train_batch(bits, t, lr=3e-3)
    for _ in range(300):
        last = net.train_batch(bits, t, lr=3e-3)
    assert last < 0.1 * first


def _anodes(seeds, shape=(16, 16, 40)):
    out = []
    for k, sd in enumerate(seeds):
        c = cases.porous(shape, radius=2, porosity=0.45 + 0.02 * (k % 3), seed=sd,
                         current_A_cm2=0.5 + 0.25 * (k % 4))
        out.append(c)
    return out


def test_warm_start_predicts_better_than_the_profile_and_converges_to_the_same_state(L):
    train = _anodes([301, 302, 303, 304, 305, 306, 307, 308])
    test = _anodes([399])[0].with_(current_A_cm2=1.0)
    b = L.Batch.from_cases(train, precision="fp32", extrapolate_every=5000)
    for k, c in enumerate(train):
        b.set_bc(c.x_in, c.current_A_cm2, case=k)
    b.run_to_residual(1e-9, 2_000_000)
    net = L.Net(width=256, depth=3, seed=19)
    for k in range(len(train)):
        net.add_sample(b, k)
    assert net.info()[1] == sum(c.n_fluid for c in train)
    net.train(600, batch=4096, lr=2e-3)

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
    err_w = np.abs(Xw - Xs)[:, f].max()
    err_p = np.abs(Xp - Xs)[:, f].max()
    assert err_w < err_p
    # the LBM, not the network, decides the result
    warm.run_to_residual(1e-12, 3_000_000)
    assert np.abs(warm.fields() - Xs)[:, f].max() < 1e-7


def _reference_features(case):
    """The feature rows of lbms_net_features computed independently in
    numpy: the closed-form 1-D profile (Eq. 19 with the outlet fluxes of
    Eq. 39 held across the anode, closed_forms) at each cell's x, box-filter
    fluid fractions, the plane porosity and the cumulative resistance."""
    solid = case.solid
    nz, ny, nx = solid.shape
    m = (~solid).astype(np.float64)
    g = case.gas
    xs = np.arange(nx) * case.length_x / (nx - 1)
    prof = cf.anode_1d(xs, case.x_in, case.current_A_cm2, g.T, g.p, g.pore_diameter, g.eps_over_tau)
    boxes = []
    for h in (1, 3, 7):
        sx = np.zeros_like(m)
        cx = np.zeros(nx)
        for d in range(-h, h + 1):
            lo, hi = max(0, -d), min(nx, nx - d)          # x + d stays inside [0, nx)
            sx[:, :, lo:hi] += m[:, :, lo + d:hi + d]
            cx[lo:hi] += 1
        sy = sum(np.roll(sx, -d, axis=1) for d in range(-h, h + 1))
        hz = h if nz > 1 else 0
        sz = sum(np.roll(sy, -d, axis=0) for d in range(-hz, hz + 1))
        boxes.append(sz / (cx[None, None, :] * (2 * h + 1) * (2 * hz + 1)))
    phi = np.maximum(m.sum(axis=(0, 1)) / (ny * nz), 1.0 / (ny * nz))
    res = np.concatenate([[0.0], np.cumsum(0.5 * (1.0 / phi[:-1] + 1.0 / phi[1:]))])
    fl = np.flatnonzero(~solid.reshape(-1))
    x = fl % nx
    F = np.zeros((fl.size, 64))
    F[:, 0:3] = prof[:, x].T
    F[:, 3] = x / (nx - 1)
    for q in range(3):
        F[:, 4 + q] = boxes[q].reshape(-1)[fl]
    F[:, 7] = 0.5 * case.current_A_cm2
    F[:, 8:11] = np.array(case.x_in)[None, :]
    F[:, 11] = F[:, 3] * F[:, 7]
    F[:, 12] = phi[x]
    F[:, 13] = res[x] / res[-1]
    F[:, 14] = 0.25 / phi[x]
    F[:, 15] = 1.0
    return F


@pytest.mark.parametrize("gemm", GEMMS)
def test_full_width_network_products(L, gemm):
    """The products of the network as the warm start trains it (width 704,
    batch 8192): forward 8192 x 704 x 64, 8192 x 704 x 704 and 8192 x 64 x 704;
    weight gradients 704 x 704 x 8192 with the K = 8192 reduction split in 16
    (704 = 5.5 tiles of 128 rows); input gradients.  Output, loss and every
    gradient against the FP32 reference, element by element."""
    net, layers = _random_net(L, 704, 2, 23)
    net.set_gemm(gemm)
    bits, x = _features(L, 8192, 24)
    t = np.random.default_rng(25).standard_normal((8192, 3)).astype(np.float32)
    out = net.forward(bits)
    loss = net.train_batch(bits, t, lr=0.0)
    ref_out, ref_loss, ref_grads = _reference(layers, x, t)
    assert np.all(np.abs(out - ref_out) <= 2e-2 * np.abs(ref_out) + 1e-2 * np.abs(ref_out).max())
    assert loss == pytest.approx(ref_loss, rel=1e-3)
    for (gW, gb), (rW, rb) in zip(net.get(1), ref_grads):
        for g, r in ((gW, rW), (gb, rb)):
            assert _rel(g, r) < 3e-2
            assert np.all(np.abs(g - r) <= 3e-2 * np.abs(r) + 2e-2 * np.abs(r).max())
    assert _used_only(net, gemm)
    net.close()


@pytest.mark.parametrize("shape", [(12, 10, 30), (24, 50)])
def test_feature_rows_match_an_independent_build(L, shape):
    """Every entry of the GPU-built feature rows (box filters, per-x table,
    assembly) against the numpy build above, to one BF16 rounding."""
    case = cases.porous(shape, radius=2, porosity=0.5, seed=91, current_A_cm2=1.25,
                        x_in=(0.6, 0.15, 0.25))
    s = L.Solver.from_case(case, precision="fp32")
    s.set_bc(case.x_in, case.current_A_cm2)
    net = L.Net(width=64, depth=1, seed=3)
    got = net.features(s, case.n_fluid)
    ref = _reference_features(case)
    want = L.from_bf16_bits(L.to_bf16_bits(ref.astype(np.float32))).reshape(ref.shape)
    assert got.shape == ref.shape
    assert np.all(np.abs(got - want) <= 2.0 ** -7 * np.abs(want) + 1e-30), \
        np.argwhere(np.abs(got - want) > 2.0 ** -7 * np.abs(want))[:5]
    assert np.all(got[:, 16:] == 0.0)
    net.close()
    s.close()
