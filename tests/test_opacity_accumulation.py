"""The opacity kernel's accumulation, emulated in FP32: each point's partial
sum over 4 chunks of 32 lines is a plain FP32 sum, and every 128 lines it is
folded into a compensated (hi, lo) pair by TwoSum (Knuth's error-free
addition: s = hi + a, b' = s - hi, lo += (hi - (s - b')) + (a - b'), hi = s).
The result hi + lo then carries about one FP32 rounding however many lines
reach the point, where a plain FP32 sum over all lines drifts with their
number."""
import numpy as np

F = np.float32


def _folded(terms, chunk=128):
    hi, lo = F(0), F(0)
    for c0 in range(0, len(terms), chunk):
        acc = F(0)
        for t in terms[c0:c0 + chunk]:
            acc = F(acc + t)
        s = F(hi + acc)
        bp = F(s - hi)
        lo = F(lo + F(F(hi - F(s - bp)) + F(acc - bp)))
        hi = s
    return F(hi + lo)


def _plain(terms):
    acc = F(0)
    for t in terms:
        acc = F(acc + t)
    return acc


def test_compensated_fold_keeps_one_rounding():
    rng = np.random.default_rng(11)
    for n in (300, 20000):
        terms = (10 ** rng.uniform(-4, 0, n)).astype(np.float32)      # positive line terms
        exact = float(np.sum(terms.astype(np.float64)))
        folded = abs(float(_folded(terms)) - exact) / exact
        assert folded <= 2.0 ** -23
        if n == 20000:
            assert abs(float(_plain(terms)) - exact) / exact > 10 * folded
