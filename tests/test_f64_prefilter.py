"""CPU check of the FP32 pre-filter of the FP64 comparison.

The FP64 test accepts trial word w against alpha iff RN64(u T) < alpha with
u = w 2^-32 (exact).  GB300 runs FP64 arithmetic at a small fraction of its
FP32 rate, so the kernels first decide the test in FP32 with proven margins
and run the FP64 product only for trials that land within a relative 2^-17
band of the threshold (and for bounds or propensities outside FP32's normal
range):

  p_f = RN32(RN32(w) * Tq),  Tq = RN32(T) 2^-32        (|p_f / uT - 1| < 2^-22)
  a_f = alpha truncated to FP32 from its bits           (0 <= 1 - a_f / alpha < 2^-23)
  accept  if p_f < RN32(a_f (1 - 2^-18))   (then uT < alpha (1 - 2^-19))
  reject  if p_f > RN32(a_f (1 + 2^-18))   (then uT > alpha)
  alpha = +-0: reject;  otherwise (negative, tiny, huge, inf, NaN) the FP64 test.

This model restates that arithmetic with NumPy's IEEE float32/float64
operations and must agree with the FP64 test on every input, including
propensities a few ulps from RN64(uT), at the band's edges, zero,
subnormal, huge, infinite and NaN.  The kernels' own agreement with the
oracle is checked bit for bit by the GPU parity tests."""
import numpy as np

F32 = np.float32
LO, HI = F32(1.0 - 2.0 ** -18), F32(1.0 + 2.0 ** -18)


def exact(w, T, a):
    u = np.float64(w) * 2.0 ** -32          # exact: w < 2^32
    return bool(u * T < a)


def fast_bound(T):
    """The pre-filter's precomputation per bound (None: FP64 test only)."""
    e = int(np.float64(T).view(np.uint64)) >> 52       # with the sign bit
    if not (1023 - 94 <= e <= 1023 + 126):
        return None
    return F32(F32(T) * F32(2.0 ** -32))


def model(w, T, a, Tq):
    if Tq is not None:
        bits = int(np.float64(a).view(np.uint64))
        hi, lo = bits >> 32, bits & 0xffffffff
        e = hi >> 20                        # with the sign bit: negatives fail the range
        if (e - 898) & 0xffffffff <= 252:   # positive, exponent in [-125, 127]
            af = np.uint32(((e - 896) << 23) | ((hi & 0xfffff) << 3) | (lo >> 29)).view(F32)
            pf = F32(F32(w) * Tq)
            if pf < F32(af * LO):
                return True, "fast"
            if pf > F32(af * HI):
                return False, "fast"
        elif ((hi & 0x7fffffff) | lo) == 0:
            return False, "zero"
    return exact(w, T, a), "exact"


def model_f32(w, T, a32, Tq):
    """The same filter for FP32 propensities (a_f = alpha exactly)."""
    if Tq is not None:
        e = int(np.float32(a32).view(np.uint32)) >> 23   # with the sign bit
        if 2 <= e <= 254:
            pf = F32(F32(w) * Tq)
            if pf < F32(a32 * LO):
                return True, "fast"
            if pf > F32(a32 * HI):
                return False, "fast"
        elif (int(np.float32(a32).view(np.uint32)) & 0x7fffffff) == 0:
            return False, "zero"
    return exact(w, T, np.float64(a32)), "exact"


def _cases(rng, n):
    """(w, T, alpha) with alpha near the threshold RN64(u T) or anywhere."""
    out = []
    for _ in range(n):
        w = int(rng.integers(0, 2 ** 32))
        if rng.random() < 0.05:
            w = int(rng.choice([0, 1, 2, 255, 256, 2 ** 24 - 1, 2 ** 24 + 1, 2 ** 32 - 1]))
        T = float(2.0 ** rng.uniform(-94, 126.99)) if rng.random() < 0.9 else \
            float(rng.choice([2.0 ** -94, 2.0 ** 126, 1.0, 3.0, 2.0 ** -95, 2.0 ** 127, 1e-300, 1e300]))
        r = np.float64(w) * 2.0 ** -32 * T
        k = rng.random()
        if k < 0.35:     # a few ulps around the threshold
            a = r
            for _ in range(int(rng.integers(0, 4))):
                a = np.nextafter(a, np.inf if rng.random() < 0.5 else -np.inf)
        elif k < 0.6:    # around the band's edges
            a = r / (1.0 + float(rng.choice([-1, 1])) * 2.0 ** -18 * float(rng.uniform(0.5, 2.0)))
        elif k < 0.9:    # anywhere within a few decades
            a = r * 10.0 ** rng.uniform(-3, 3) if r > 0 else float(2.0 ** rng.uniform(-100, 100))
        else:            # special values
            a = float(rng.choice([0.0, -0.0, 5e-324, 2.0 ** -1022, 2.0 ** -126, 2.0 ** -125,
                                  2.0 ** -127, 2.0 ** 127, 2.0 ** 128, 1.7e308, np.inf, np.nan,
                                  -1.0, -5e-324, -np.inf, float(-r) if r > 0 else -2.0]))
        out.append((w, T, float(a)))
    return out


def test_prefilter_equals_fp64_test():
    rng = np.random.default_rng(12345)
    kinds = {"fast": 0, "zero": 0, "exact": 0}
    for w, T, a in _cases(rng, 200_000):
        got, kind = model(w, T, a, fast_bound(T))
        kinds[kind] += 1
        assert got == exact(w, T, a), (w, T, a, kind)
    # even on these inputs, most of them built to sit inside the band, a
    # large share of the decisions is made in FP32
    assert kinds["fast"] > 0.4 * sum(kinds.values()), kinds


def test_prefilter_f32_propensities_equal_fp64_test():
    rng = np.random.default_rng(54321)
    with np.errstate(over="ignore"):   # huge values overflow FP32 (skipped, or +inf margins)
        for w, T, a in _cases(rng, 100_000):
            if not np.isfinite(np.float32(a)) and np.isfinite(a):
                continue   # FP32 data cannot hold it
            a32 = np.float32(a)
            got, _ = model_f32(w, T, a32, fast_bound(T))
            assert got == exact(w, T, np.float64(a32)), (w, T, float(a32))


def test_prefilter_takes_fp64_rarely_on_random_trials():
    """On ordinary trials (random w, alpha from the propensity law) the FP64
    product is needed for about one trial in 10^5."""
    rng = np.random.default_rng(7)
    alpha = rng.exponential(1.0, 4096)
    T = float(alpha.max())
    Tq = fast_bound(T)
    n, slow = 200_000, 0
    for _ in range(n):
        w, a = int(rng.integers(0, 2 ** 32)), float(alpha[rng.integers(0, alpha.size)])
        got, kind = model(w, T, a, Tq)
        assert got == exact(w, T, a)
        slow += kind == "exact"
    assert slow <= n * 1e-4, slow
