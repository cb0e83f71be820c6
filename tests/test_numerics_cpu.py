"""Error bounds of the numerical shortcuts the float64 kernels take where
the FP64 pipe is the bottleneck, restated in numpy (no GPU needed):

- friction's inverse cube root: a float seed within 2^-21 relative, then
  one Newton step r <- r + r (1 - h r^3) / 3, is within about 2^-41;
- the CFL bound formed once per step: dx / max(s) equals the smallest of
  the per-leaf quotients dx / s (a correctly rounded division is monotone
  in its divisor)."""
import numpy as np


def _newton_rcbrt(h, r):
    # the kernel fuses the last two operations of each line (FMA); separate
    # roundings here only widen the error by a few units of 2^-53
    r3 = (r * r) * r
    d = 1.0 - h * r3
    return r * d * (1.0 / 3.0) + r


def test_one_newton_step_squares_the_seed_error():
    rng = np.random.default_rng(7)
    h = np.exp(rng.uniform(np.log(1e-6), np.log(1e4), 200000))
    exact = h ** (-1.0 / 3.0)
    for rel in (2.0 ** -21, -(2.0 ** -21), 2.0 ** -23):
        seed = exact * (1.0 + rel)
        r = _newton_rcbrt(h, seed)
        err = np.abs(r / exact - 1.0)
        # 2 rel^2 from the iteration, a few units of 2^-53 from rounding
        assert err.max() <= 2.0 * rel * rel + 8 * 2.0 ** -53
    # the bound the kernel's comment states for its seed
    assert 2.0 * (2.0 ** -21) ** 2 + 8 * 2.0 ** -53 < 2.0 ** -40


def test_cfl_bound_from_the_largest_speed():
    rng = np.random.default_rng(11)
    for _ in range(200):
        dx = rng.uniform(0.1, 10.0)
        s = rng.uniform(0.01, 50.0, rng.integers(1, 64))
        assert dx / s.max() == np.min(dx / s)
