"""Host check of the arithmetic argument behind the tensor-core double-float
kernels (exact split products, Ozaki's scheme): a scaled double-float value
in (-1, 1) written as six bf16 slices on the grids 2^(-7-8k), each slice
with at most 8 significant bits, the slices summing to the value within
2^-47, and the sums of slice products with s + t = u staying below 2^24
units of their common grid for the K of each kernel.  The steps are replayed
in IEEE FP32 with NumPy (round to nearest), one value at a time; this file
checks the scheme's claims, it is not the oracle of any result."""
import numpy as np

F = np.float32
CS = [F(1.5 * 2.0 ** (16 - 8 * k)) for k in range(6)]


def split6(h, l):
    """The kernels' split of h + l (FP32 hi and lo parts), step by step."""
    h, l = F(h), F(l)
    s = []
    r = h
    for k in range(6):
        sk = F(F(r + CS[k]) - CS[k])
        s.append(sk)
        if k < 5:
            r = F(r - sk)
        if k == 2:
            r = F(r + l)
    return s


def sig_bits(x):
    """Significant bits of a finite float (0 for zero)."""
    if x == 0.0:
        return 0
    m, _ = np.frexp(abs(float(x)))
    n = 0
    while m != int(m):
        m *= 2
        n += 1
    return n


def _df(x):
    h = F(x)
    return h, F(x - float(h))


def test_slices_are_bf16_exact_and_sum_to_the_value():
    rng = np.random.default_rng(5)
    vals = np.concatenate([rng.uniform(-1, 1, 4000),
                           rng.uniform(-1, 1, 2000) * 2.0 ** rng.integers(-30, 0, 2000),
                           [0.0, 1 - 2.0 ** -40, -(1 - 2.0 ** -40), 2.0 ** -60]])
    worst = 0.0
    for x in vals:
        h, l = _df(x)
        s = split6(h, l)
        for k, sk in enumerate(s):
            v = float(sk)
            # on the grid 2^(-7-8k), at most 8 significant bits (bf16), bounded
            q = v / 2.0 ** (-7 - 8 * k)
            assert q == int(q), (x, k, v)
            assert abs(q) <= (192 if k == 3 else 128), (x, k, q)
            assert sig_bits(v) <= 8, (x, k, v)
        worst = max(worst, abs(sum(float(v) for v in s) - (float(h) + float(l))))
    assert worst <= 2.0 ** -47, worst


def test_products_with_equal_slice_sum_fit_24_bits():
    """For every u, sum over K terms of sum_{s+t=u} |a_s b_t| in units of
    2^(-14-8u) stays below 2^24 for K = 96 (stencil), 32 (update), 64 (Gram
    tile) and up to the stated limit K = 146, with every slice at its largest
    magnitude."""
    # largest slice magnitudes in grid units: 128, and 192 for slice 3
    smax = [128.0, 128.0, 128.0, 192.0, 128.0, 128.0]
    for K in (96, 32, 64, 146):
        for u in range(6):
            bound = K * sum(smax[s] * smax[u - s] for s in range(u + 1))
            assert bound < 2.0 ** 24, (K, u, bound)


def test_split_product_matches_double_product():
    """sum over s + t <= 5 of a_s b_t reproduces a b to about 2^-45."""
    rng = np.random.default_rng(6)
    worst = 0.0
    for _ in range(3000):
        a, b = rng.uniform(-1, 1, 2)
        ah, al = _df(a)
        bh, bl = _df(b)
        sa, sb = split6(ah, al), split6(bh, bl)
        p = sum(float(sa[s]) * float(sb[t]) for s in range(6) for t in range(6) if s + t <= 5)
        worst = max(worst, abs(p - (float(ah) + float(al)) * (float(bh) + float(bl))))
    assert worst <= 2.0 ** -45, worst
