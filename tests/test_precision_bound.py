"""The precision form's rounding bound (BL_XPREC_BF16), checked on the CPU with
an emulation of what the BF16 z pass computes: each FP32 value rounded to BF16
(nearest, ties to even, from its bit pattern), then FP32 accumulation in the
pass's order (two chains per lane over 16-byte chunks of 8 values, their sum,
then a 32-lane butterfly).  The bound
    |z_bf16 - x'r| <= (2^-8 + (1 + 2^-8) gamma_m) ||x|| ||r||,
m = chunks per lane * 4 + 1 + 5, must hold on every column."""
import numpy as np


def bf16_rne(x32: np.ndarray) -> np.ndarray:
    """FP32 -> BF16 (kept as FP32 with the low 16 bits zero), round to nearest even."""
    b = x32.astype(np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    b = (b + 0x7FFF + lsb) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def zpass_bf16_emulated(x32: np.ndarray, r32: np.ndarray) -> np.float32:
    n = x32.size
    nch = (n + 7) // 8
    rpl = (nch + 31) // 32
    xb = np.zeros(nch * 8, np.float32)
    xb[:n] = bf16_rne(x32)
    rr = np.zeros(nch * 8, np.float32)
    rr[:n] = r32
    lane_sums = np.zeros(32, np.float32)
    for lane in range(32):
        a0 = np.float32(0)
        a1 = np.float32(0)
        for q in range(rpl):
            ch = lane + 32 * q
            if ch >= nch:
                continue
            for v in range(0, 8, 2):
                a0 = np.float32(a0 + np.float32(xb[ch * 8 + v] * rr[ch * 8 + v]))
                a1 = np.float32(a1 + np.float32(xb[ch * 8 + v + 1] * rr[ch * 8 + v + 1]))
        lane_sums[lane] = np.float32(a0 + a1)
    s = lane_sums.copy()
    for off in (16, 8, 4, 2, 1):  # butterfly: every lane ends with the same sum
        s = (s + s[np.arange(32) ^ off]).astype(np.float32)
    return s[0]


def bound(x32, r32):
    n = x32.size
    rpl = ((n + 7) // 8 + 31) // 32
    m = rpl * 4 + 1 + 5
    u = 2.0 ** -24
    gam = m * u / (1 - m * u) + 8 * u  # as zpass_reg_gamma (the 8u covers the FP32 products)
    return (2.0 ** -8 + (1 + 2.0 ** -8) * gam) * np.linalg.norm(x32.astype(np.float64)) * \
        np.linalg.norm(r32.astype(np.float64))


def test_bf16_bound_holds_on_random_and_adversarial_columns():
    rng = np.random.default_rng(31)
    worst = 0.0
    for trial in range(300):
        n = int(rng.integers(1, 1025))
        kind = trial % 4
        if kind == 0:
            x = rng.standard_normal(n)
        elif kind == 1:      # values just above a BF16 rounding midpoint, same sign as r
            x = (1.0 + (2 * rng.integers(0, 64, n) + 1) * 2.0 ** -8 + 2.0 ** -20) * rng.choice([-1, 1], n)
        elif kind == 2:      # wide dynamic range
            x = rng.standard_normal(n) * 10.0 ** rng.uniform(-6, 6, n)
        else:                # a constant column offset (raw, uncentred values)
            x = 50.0 + rng.standard_normal(n)
        r = rng.standard_normal(n)
        if kind == 1:
            r = np.abs(r) * np.sign(x)
        x32, r32 = x.astype(np.float32), r.astype(np.float32)
        exact = float(np.dot(x32.astype(np.float64), r32.astype(np.float64)))
        got = float(zpass_bf16_emulated(x32, r32))
        b = bound(x32, r32)
        assert abs(got - exact) <= b, (trial, n, got, exact, b)
        worst = max(worst, abs(got - exact) / b)
    assert worst > 0.05       # the bound is not vacuous: some columns use a good part of it


def test_bf16_rounding_is_nearest_even_and_within_half_an_ulp():
    rng = np.random.default_rng(32)
    x = (rng.standard_normal(20000) * 10.0 ** rng.uniform(-30, 30, 20000)).astype(np.float32)
    xb = bf16_rne(x)
    rel = np.abs(xb.astype(np.float64) - x) / np.abs(x.astype(np.float64))
    assert np.all(rel <= 2.0 ** -8)
    # ties go to the even BF16 pattern
    t = np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8], np.float32)
    assert bf16_rne(t)[0] == np.float32(1.0) and bf16_rne(t)[1] == np.float32(1.0 + 2 * 2.0 ** -7)
