"""Pins of the G_theta CPU oracle: finite-difference gradients, delta responses, padding."""
import numpy as np
import pytest

from oracle import gtheta_oracle as g


def small_net(seed=3):
    W, b = g.init_params(seed, scale_last=1.0)
    rng = np.random.default_rng(seed + 1)
    for l in range(6):
        b[l] = 0.1 * rng.standard_normal(b[l].shape)
    return W, b


def test_conv_of_delta_reproduces_flipped_taps():
    H = 7
    x = np.zeros((H, H, 1))
    x[3, 3, 0] = 1.0
    w = np.arange(9, dtype=float).reshape(3, 3, 1, 1)
    y = g.conv3(x, w, np.zeros(1))[..., 0]
    # y[i, j] = w[i - 3 + 1, j - 3 + 1] for the taps that reach the delta: y[3-(dy-1), 3-(dx-1)] = w[dy, dx]
    for dy in range(3):
        for dx in range(3):
            assert y[3 - (dy - 1), 3 - (dx - 1)] == w[dy, dx, 0, 0]
    assert np.count_nonzero(y) == 8  # w[0,0] = 0


def test_zero_padding_matches_embedded_field():
    """A field convolved with zero padding equals the same field embedded in a larger zero field."""
    rng = np.random.default_rng(0)
    x = rng.standard_normal((6, 5, 2))
    w = rng.standard_normal((3, 3, 4, 2))
    big = np.zeros((10, 9, 2))
    big[2:8, 2:7] = x
    y = g.conv3(x, w, np.zeros(4))
    yb = g.conv3(big, w, np.zeros(4))
    assert np.allclose(y, yb[2:8, 2:7])


@pytest.mark.parametrize("relative", [False, True])
@pytest.mark.parametrize("layer", [0, 2, 5])
def test_gradients_match_central_differences(layer, relative):
    rng = np.random.default_rng(7)
    H = 9
    u = 0.7 * rng.standard_normal((H, H))
    target = 0.1 * rng.standard_normal((H, H))
    W, b = small_net()

    def loss_of(W_, b_):
        gu, acts = g.forward(u, W_, b_)
        return g.mse_crop_loss(acts[-1][..., 0], target, 1, relative)[0]

    gu, acts = g.forward(u, W, b)
    _, dr = g.mse_crop_loss(acts[-1][..., 0], target, 1, relative)
    gW, gb = g.backward(acts, W, dr)
    hstep = 1e-6
    for idx in [(0, 1, 0, 0), (1, 2, 0, 0), (2, 0, 0, 0)]:
        i = (idx[0], idx[1], idx[2] % W[layer].shape[2], idx[3] % W[layer].shape[3])
        Wp = [w.copy() for w in W]
        Wm = [w.copy() for w in W]
        Wp[layer][i] += hstep
        Wm[layer][i] -= hstep
        fd = (loss_of(Wp, b) - loss_of(Wm, b)) / (2 * hstep)
        assert abs(fd - gW[layer][i]) <= 1e-6 * max(1.0, abs(fd)), (layer, i, fd, gW[layer][i])
    bp = [x.copy() for x in b]
    bm = [x.copy() for x in b]
    bp[layer][0] += hstep
    bm[layer][0] -= hstep
    fd = (loss_of(W, bp) - loss_of(W, bm)) / (2 * hstep)
    assert abs(fd - gb[layer][0]) <= 1e-6 * max(1.0, abs(fd))


def test_forward_is_residual_and_local():
    """G(U) = U + R(U) and R has a 13 x 13 receptive field (six 3 x 3 layers)."""
    W, b = small_net()
    rng = np.random.default_rng(1)
    u = rng.standard_normal((20, 20))
    gu, acts = g.forward(u, W, b)
    assert np.allclose(gu, u + acts[-1][..., 0])
    u2 = u.copy()
    u2[0, 0] += 1.0
    gu2, _ = g.forward(u2, W, b)
    changed = np.argwhere(np.abs(gu2 - gu) > 0)
    assert changed[:, 0].max() <= 6 and changed[:, 1].max() <= 6


def test_adam_step_matches_definition_on_a_scalar():
    p = np.array([1.0])
    m = np.zeros(1)
    v = np.zeros(1)
    g.adam_step(p, np.array([0.5]), m, v, t=1, lr=0.1)
    # first step: mh = g, vh = g^2 -> p -= lr * g / (|g| + eps)
    assert abs(p[0] - (1.0 - 0.1 * 0.5 / (0.5 + 1e-8))) < 1e-15


def test_bf16_round_matches_torch_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    x = np.concatenate([rng.standard_normal(4000) * 10.0 ** rng.integers(-8, 8, 4000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.0078125, 3.0e38, -1.5e-40]])
    # values exactly halfway between two BF16 neighbours: ties go to the even pattern
    half = (np.arange(1, 200, dtype=np.uint32) << 16 | 0x8000).view(np.float32).astype(np.float64)
    x = np.concatenate([x, half, -half])
    want = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(g.bf16_round(x), want)


def test_bf16_storage_model_is_close_to_fp64():
    W, b = small_net(5)
    rng = np.random.default_rng(2)
    u = 0.5 * rng.standard_normal((12, 12))
    gu, acts = g.forward(u, W, b)
    gq, aq = g.forward(u, W, b, bf16=True)
    r, rq = acts[-1][..., 0], aq[-1][..., 0]
    assert np.abs(rq - r).max() <= 3e-2 * np.abs(r).max()
    assert np.abs(rq - r).max() > 0.0
    # every stored hidden activation is a BF16 value
    for a in aq[1:6]:
        assert np.array_equal(g.bf16_round(a), a)


def test_bf16_backward_matches_fp64_backward_to_bf16_accuracy():
    W, b = small_net(9)
    rng = np.random.default_rng(4)
    u = 0.6 * rng.standard_normal((10, 10))
    t = 0.05 * rng.standard_normal((10, 10))
    _, a = g.forward(u, W, b)
    _, dr = g.mse_crop_loss(a[-1][..., 0], t, 2)
    gW, gb = g.backward(a, W, dr)
    _, aq = g.forward(u, W, b, bf16=True)
    _, drq = g.mse_crop_loss(aq[-1][..., 0], t, 2)
    gWq, gbq = g.backward(aq, W, drq, bf16=True)
    for l in range(6):
        rel = np.linalg.norm(gWq[l] - gW[l]) / np.linalg.norm(gW[l])
        assert rel < 5e-2, (l, rel)


def test_relative_crop_loss_is_the_relative_squared_error():
    """Relative loss of one crop: r = (1 + c) t on the window gives c^2 (up to the 1e-12 floor),
    whatever the scale of t; outside the window nothing counts."""
    rng = np.random.default_rng(3)
    for scale in (1e-3, 1.0, 50.0):
        t = scale * rng.standard_normal((10, 10))
        r = 1.25 * t
        r[0, :] += 7.0  # outside the window (margin 2)
        loss, dr = g.mse_crop_loss(r, t, 2, relative=True)
        et = float((t[2:8, 2:8] ** 2).sum())
        assert abs(loss - 0.0625 * et / (et + 1e-12 * 36)) <= 1e-12
        assert np.all(dr[:2] == 0) and np.all(dr[:, :2] == 0)
        # the gradient of the relative loss is the absolute one scaled by count / E
        _, dra = g.mse_crop_loss(r, t, 2)
        e = float((t[2:8, 2:8] ** 2).sum()) + 1e-12 * 36
        assert np.allclose(dr, dra * 36 / e, rtol=1e-12, atol=0)
