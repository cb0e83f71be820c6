"""Pins of the CNN oracle: cross-correlation closed forms and central finite
differences of the whole network's loss (no GPU)."""
import numpy as np

from oracle import cnn


def test_identity_kernel_copies_input():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 3, 5, 6))
    w = np.zeros((3, 3, 3, 3))
    for c in range(3):
        w[c, c, 1, 1] = 1.0
    y = cnn.conv3x3(x, w, np.zeros(3))
    assert np.array_equal(y, x)


def test_delta_input_gives_flipped_kernel():
    # cross-correlation: a unit impulse at (r, c) produces w[o, 0, 1-di, 1-dj]
    # at (r+di, c+dj), i.e. the kernel rotated by 180 degrees around it
    rng = np.random.default_rng(1)
    w = rng.standard_normal((2, 1, 3, 3))
    x = np.zeros((1, 1, 7, 7))
    x[0, 0, 3, 3] = 1.0
    y = cnn.conv3x3(x, w, np.zeros(2))
    for o in range(2):
        assert np.array_equal(y[0, o, 2:5, 2:5], w[o, 0, ::-1, ::-1])


def test_zero_padding_at_borders():
    x = np.ones((1, 1, 4, 4))
    w = np.ones((1, 1, 3, 3))
    y = cnn.conv3x3(x, w, np.zeros(1))
    assert y[0, 0, 0, 0] == 4.0 and y[0, 0, 0, 1] == 6.0 and y[0, 0, 1, 1] == 9.0


def test_uniform_logits_loss_is_log_classes():
    logits = np.zeros((1, 5, 3, 3))
    labels = np.zeros((1, 3, 3), dtype=int)
    loss, d = cnn.loss_and_dlogits(logits, labels)
    assert abs(loss - np.log(5.0)) < 1e-15
    assert np.allclose(d.sum(axis=1), 0.0)


def test_gradients_match_central_differences():
    rng = np.random.default_rng(2)
    params = cnn.init_params(rng, cin=4, ch=5, ncls=5)
    params = [p + 0.1 * rng.standard_normal(p.shape) for p in params]
    x = rng.standard_normal((2, 4, 5, 4))
    labels = rng.integers(0, 5, size=(2, 5, 4))

    def loss_of(ps):
        logits, _ = cnn.forward(ps, x)
        return cnn.loss_and_dlogits(logits, labels)[0]

    logits, cache = cnn.forward(params, x)
    _, dl = cnn.loss_and_dlogits(logits, labels)
    grads = cnn.backward(params, cache, dl)
    h = 1e-6
    for pi, (p, g) in enumerate(zip(params, grads)):
        flat = p.reshape(-1)
        idx = rng.choice(flat.size, size=min(12, flat.size), replace=False)
        for k in idx:
            old = flat[k]
            flat[k] = old + h
            lp = loss_of(params)
            flat[k] = old - h
            lm = loss_of(params)
            flat[k] = old
            num = (lp - lm) / (2 * h)
            assert abs(num - g.reshape(-1)[k]) <= 1e-7 + 1e-5 * abs(num), (pi, k, num, g.reshape(-1)[k])


def _torch_bf16(a):
    import torch
    return torch.as_tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def test_bf16_rounding_is_the_library_conversion():
    # the oracle's bit-level rounding against torch's float32 -> bfloat16
    # conversion (round to nearest, ties to even), over many binades, signs,
    # subnormals and exact ties
    rng = np.random.default_rng(5)
    a = rng.standard_normal(20000) * np.exp2(rng.integers(-130, 120, 20000))
    ties = (1.0 + (2 * rng.integers(0, 128, 200) + 1) * 2.0 ** -8) * np.exp2(rng.integers(-20, 20, 200))
    for v in (a, ties, -ties, np.array([0.0, -0.0, 1.0, 2.0 ** -140, 3.0e38])):
        assert np.array_equal(cnn.bf16(v), _torch_bf16(v))


def test_bf16_ties_go_to_even():
    # halfway between two bf16 neighbours (spacing 2^-7 above 1): the one
    # with an even last significand bit wins
    assert cnn.bf16(1.0 + 2.0 ** -8) == 1.0
    assert cnn.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert cnn.bf16(-(1.0 + 2.0 ** -8)) == -1.0
    assert cnn.bf16(1.0 + 2.0 ** -8 + 2.0 ** -20) == 1.0 + 2.0 ** -7


def test_bf16_network_on_one_pixel_rounds_each_hidden_operand():
    # on a 1x1 image every 3x3 convolution reduces to its centre tap, so the
    # network is a chain of scalar products that can be followed by hand;
    # the values are chosen so that every BF16 rounding changes its operand
    a, w2c, c0 = 1.0 + 2.0 ** -9 + 2.0 ** -12, 1.5 + 2.0 ** -10, 0.0625
    w1 = np.zeros((1, 1, 3, 3)); w1[0, 0, 1, 1] = a
    w2 = np.zeros((1, 1, 3, 3)); w2[0, 0, 1, 1] = w2c
    w3 = np.zeros((2, 1, 3, 3)); w3[0, 0, 1, 1] = c0
    params = [w1, np.zeros(1), w2, np.zeros(1), w3, np.zeros(2)]
    x = np.ones((1, 1, 1, 1))
    labels = np.zeros((1, 1, 1), dtype=int)
    logits, cache = cnn.forward(params, x, cnn.bf16)
    _, z1, a1, z2, a2 = cache
    assert a1[0, 0, 0, 0] == 1.0                       # a rounds to 1
    assert a2[0, 0, 0, 0] == 1.5                       # w2c * 1 rounds to 1.5
    assert logits[0, 0, 0, 0] == c0 * 1.5 and logits[0, 1, 0, 0] == 0.0
    _, dl = cnn.loss_and_dlogits(logits, labels)
    g = cnn.backward(params, cache, dl, cnn.bf16)
    # two-class softmax: p0 = logistic(z0 - z1); label 0
    p0 = 1.0 / (1.0 + np.exp(-c0 * 1.5))
    d0, d1 = _torch_bf16(p0 - 1.0), _torch_bf16(1.0 - p0)
    assert d0 != p0 - 1.0                              # the loss gradient is rounded
    assert np.array_equal(g[5], [d0, d1])              # db3
    assert np.array_equal(g[4][:, 0, 1, 1], [1.5 * d0, 1.5 * d1])   # dw3 = a2 * dl
    dz2 = _torch_bf16(c0 * d0)                         # da2 = w3^T dl, masked, rounded
    assert g[3][0] == dz2 and g[2][0, 0, 1, 1] == 1.0 * dz2
    dz1 = _torch_bf16(w2c * dz2)                       # da1 = w2 dz2, masked, rounded
    assert dz1 != w2c * dz2
    assert g[1][0] == dz1 and g[0][0, 0, 1, 1] == dz1
    # every other tap sees the zero padding: no gradient
    for k, gi in enumerate((g[0], g[2], g[4])):
        m = np.ones(gi.shape, bool); m[:, :, 1, 1] = False
        assert np.all(gi[m] == 0.0), k


def test_bf16_network_equals_plain_network_on_bf16_exact_values():
    # when every hidden value is already a BF16 number (small dyadic
    # weights, inputs and biases), the rounded network is the plain one
    rng = np.random.default_rng(6)
    params = [rng.integers(-2, 3, (5, 4, 3, 3)) / 8.0, rng.integers(-2, 3, 5) / 8.0,
              rng.integers(-2, 3, (5, 5, 3, 3)) / 8.0, rng.integers(-2, 3, 5) / 8.0,
              rng.integers(-2, 3, (5, 5, 3, 3)) / 8.0, rng.integers(-2, 3, 5) / 8.0]
    x = rng.integers(-2, 3, (2, 4, 5, 6)) / 4.0
    l0, c0 = cnn.forward(params, x)
    l1, c1 = cnn.forward(params, x, cnn.bf16)
    assert np.array_equal(l0, l1)
    for a, b in zip(c0, c1):
        assert np.array_equal(a, b)
