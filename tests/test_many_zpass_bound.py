"""The rounding bound of the persistent many-problem kernel's z pass (bl_many.cu,
many_zpass), checked on the CPU with an emulation of its accumulation order: G
lanes (a power of two, the smallest with G * U >= n/4, at most 32) share a
column; lane li takes the 16-byte chunks li, li + G, ... in rounds of U, each
chunk's four products fused into its FP32 chain; the group's first lane adds
the n mod 4 tail rows; the G lanes are combined by a butterfly.  The KKT test
relies on
    |fl(x'r) - x'r| <= gamma_m ||x|| ||r||,  m = 4 ceil((n/4) / G) + 3 + log2 G,
with gamma_m = m u / (1 - m u) + 8u as the kernel forms it."""
import numpy as np

F32 = np.float32
U32 = 2.0 ** -24


def group_size(n, U):
    nfull = n // 4
    G, LG = 1, 0
    while G * U < nfull and G < 32:
        G <<= 1
        LG += 1
    return G, LG


def fma32(a, b, c):
    # the product of two floats is exact in FP64; one more rounding to FP32
    return F32(np.float64(a) * np.float64(b) + np.float64(c))


def zpass_emulated(x, r, U):
    n = x.size
    nfull = n // 4
    G, _ = group_size(n, U)
    acc = np.zeros(G, F32)
    for li in range(G):
        a = F32(0)
        for q0 in range(li, nfull, G * U):
            for u in range(U):
                q = q0 + G * u
                if q < nfull:
                    for k in range(4):
                        a = fma32(x[4 * q + k], r[4 * q + k], a)
        if li == 0:
            for i in range(nfull * 4, n):
                a = fma32(x[i], r[i], a)
        acc[li] = a
    o = G >> 1
    while o > 0:
        acc = (acc + acc[np.arange(G) ^ o]).astype(F32)
        o >>= 1
    return acc[0]


def gamma(n, U):
    G, LG = group_size(n, U)
    m = 4 * ((n // 4 + G - 1) // G) + 3 + LG
    return m * U32 / (1.0 - m * U32) + 8.0 * U32


def exact(x, r):
    return float(np.sum(x.astype(np.longdouble) * r.astype(np.longdouble)))


def test_bound_holds_on_random_and_adversarial_columns():
    rng = np.random.default_rng(17)
    worst = 0.0
    for trial in range(240):
        U = 8 if trial % 2 else 16
        n = int(rng.integers(1, 2049))
        kind = trial % 4
        if kind == 0:
            x, r = rng.standard_normal(n), rng.standard_normal(n)
        elif kind == 1:   # one sign: no cancellation, the largest accumulated error
            x, r = np.abs(rng.standard_normal(n)) + 1.0, np.abs(rng.standard_normal(n)) + 1.0
        elif kind == 2:   # wide dynamic range
            x = rng.standard_normal(n) * 10.0 ** rng.uniform(-6, 6, n)
            r = rng.standard_normal(n)
        else:             # values just above powers of two (products round at each step)
            x = (1.0 + rng.integers(1, 4, n) * 2.0 ** -22) * 2.0 ** rng.integers(-3, 4, n)
            r = (1.0 + rng.integers(1, 4, n) * 2.0 ** -21)
        x, r = x.astype(F32), r.astype(F32)
        err = abs(float(zpass_emulated(x, r, U)) - exact(x, r))
        b = gamma(n, U) * float(np.linalg.norm(x.astype(np.float64)) * np.linalg.norm(r.astype(np.float64)))
        assert err <= b, (n, U, kind, err, b)
        worst = max(worst, err / b)
    assert worst > 1e-3   # the bound is not vacuous on these columns


def test_group_sizes_match_the_kernel_rule():
    # n <= 2048 and U = 8: one round of at most U chunks per lane unless G is capped at 32
    for n, U, G in [(7, 8, 1), (32, 8, 1), (33, 8, 1), (36, 8, 2), (133, 8, 8), (1024, 8, 32), (1820, 8, 32), (2048, 16, 32)]:
        assert group_size(n, U)[0] == G
