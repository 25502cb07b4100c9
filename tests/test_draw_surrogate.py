"""The detail draw's float32 surrogate key (CPU, no GPU): -ln(u) is taken as
-log(u) for u <= 1/2 and as -log1p(-(1 - u)) above, with 1 - u formed from
the integer 2^53 - (2m + 1), so each branch's argument is one rounding from
exact and -ln is well conditioned on both sides.  Evaluated here in numpy
float32 against FP64 over u from the whole range (both ends included), the
relative error stays far inside the 2^-16 bound the draw's candidate filter
assumes; the one-branch form -log(float(u)) does not near u = 1, where the
selected keys are."""
import numpy as np


def _surrogate(a, g):
    # a = 2m + 1 (odd, below 2^53), u = a 2^-53
    lo = a <= (1 << 52)
    u = (a.astype(np.float32) * np.float32(2.0 ** -53))
    v = ((np.uint64(1 << 53) - a).astype(np.float32) * np.float32(2.0 ** -53))
    with np.errstate(divide="ignore"):  # both branches are evaluated; each is used only on its side
        L = np.where(lo, -np.log(u), -np.log1p(-v)).astype(np.float32)
    return (L / g).astype(np.float32)


def _exact(a, g):
    u = a.astype(np.float64) * 2.0 ** -53
    return -np.log(u) / g.astype(np.float64)


def test_surrogate_key_within_bound():
    rng = np.random.default_rng(11)
    m = rng.integers(0, 1 << 52, size=1_000_000, dtype=np.uint64)
    # both ends of u: the largest and the smallest m
    m[:1000] = np.uint64((1 << 52) - 1) - np.arange(1000, dtype=np.uint64)
    m[1000:2000] = np.arange(1000, dtype=np.uint64)
    a = 2 * m + np.uint64(1)
    g = rng.uniform(1e-4, 10.0, size=a.size).astype(np.float32)
    rel = np.abs(_surrogate(a, g).astype(np.float64) - _exact(a, g)) / _exact(a, g)
    assert rel.max() < 2.0 ** -20
    # the one-branch form loses the keys near u = 1 (the smallest keys)
    naive = (-np.log((a.astype(np.float32) * np.float32(2.0 ** -53))) / g).astype(np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        rel_naive = np.abs(naive[:1000] - _exact(a[:1000], g[:1000])) / _exact(a[:1000], g[:1000])
    assert np.nanmax(rel_naive) > 2.0 ** -16
