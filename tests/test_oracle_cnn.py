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
