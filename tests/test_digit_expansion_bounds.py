"""The exactness argument of the FP64-accurate tensor-core GEMM, checked on the host with
plain integer arithmetic (a restatement of the expansion from its definition, independent of
the CUDA code): every FP64 value x with |x| < 2^e is the integer G = round(|x| 2^(61-e))
written as a top digit d_0 in [0, 64] and eleven balanced base-32 digits in [-15, 16]
(x ~ sign(x) 2^(e-61) G, |x - value| <= 2^(e-62)); all values are exact in BF16 (integers of
at most 8 significant bits); and the sums that one significance level L = s + t collects
over a pass of 3584 real K terms stay below 2^24 even at the digit extremes, so the FP32
accumulation is exact."""
import numpy as np

SLICES, KPASS = 12, 3584


def digits(x: float, e: int):
    m, ex = np.frexp(abs(x))                       # |x| = m 2^ex, m in [0.5, 1)
    M, sh = int(m * 2.0 ** 53), int(ex) - 53 + 61 - e   # |x| 2^(61-e) = M 2^sh, M < 2^53
    G = M << sh if sh >= 0 else (M + (1 << (-sh - 1))) >> -sh   # rounded half up
    d = [0] * SLICES
    for s in range(SLICES - 1, 0, -1):
        r = G % 32
        if r > 16:
            r -= 32
        d[s] = r
        G = (G - r) // 32
    d[0] = G
    return [(-v if x < 0 else v) for v in d]


def test_digit_ranges_and_reconstruction():
    rng = np.random.default_rng(0)
    for _ in range(20000):
        e = int(rng.integers(-30, 30))
        x = float(rng.uniform(-1, 1)) * 2.0 ** e
        d = digits(x, e)
        assert 0 <= abs(d[0]) <= 64 and all(-16 <= v <= 16 for v in d[1:])
        val = sum(v * 2 ** (5 * (SLICES - 1 - s)) for s, v in enumerate(d))   # integer
        assert abs(abs(val) * 2.0 ** (e - 61) - abs(x)) <= 2.0 ** (e - 62)


def test_extreme_digits_are_exact_in_bf16():
    # integers up to 256 in magnitude have at most 8 significant bits: exact in BF16
    for v in range(-64, 65):
        assert float(np.float32(v)) == v and (abs(v) < 256)


def test_level_sums_stay_below_2_pow_24():
    worst = []
    for L in range(SLICES):
        pairs = [(s, L - s) for s in range(L + 1) if L - s < SLICES]
        per_term = sum((64 if s == 0 else 16) * (64 if t == 0 else 16) for s, t in pairs)
        worst.append(per_term)
    assert worst[0] == 64 * 64 and max(worst) == 2 * 64 * 16 + (SLICES - 2) * 256
    assert KPASS % 16 == 0 and max(worst) * KPASS < 2 ** 24
