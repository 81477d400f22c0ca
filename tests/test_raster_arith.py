"""The integer and float arguments the coverage kernel's exactness rests on,
checked on the CPU with Python integers (no GPU; these restate the kernel's
arithmetic, the GPU parity tests check the kernel itself).

- Fast-form masks: C' clamped to +-(4080 S + 1), the value at sample 15 of a
  pixel, stepped down to sample 0 with the two n-rooks increments, gives every
  sample the sign of the unclamped edge function, and every value stays in int32
  for S = |A| + |B| < 2^18.
- Row search: the two rounds of three loads find the last row whose span prefix
  is at most the item index, as a plain binary search does.
- Row spans: the union of the two edge groups' extents with saturating
  float-to-int conversions gives the same pixel range as clamping to +-1e9
  first."""
import math
import random

I32 = 2 ** 31


def _signs_direct(c_true, a, b, cx, cy):
    return [c_true + a * (cx + 16 * k) + b * (cy + 16 * ((5 * k) % 16)) >= 0 for k in range(16)]


def _signs_stepped(c_true, a, b, cx, cy):
    s = abs(a) + abs(b)
    lim = 4080 * s + 1
    c = max(min(c_true, lim), -lim)
    v = c + 240 * a + 176 * b + a * cx + b * cy  # sample 15
    i1 = 16 * a + 80 * b
    i2 = i1 - 256 * b
    out = [None] * 16
    for k in range(15, -1, -1):
        assert -I32 <= v < I32
        out[k] = v >= 0
        if k > 0:
            v -= i1 if ((5 * (k - 1)) & 15) <= 10 else i2
    return out


def test_fast_mask_stepping_keeps_every_sign_in_int32():
    rng = random.Random(7)
    smax = 2 ** 18 - 1
    for _ in range(20000):
        a = rng.randint(-smax, smax)
        rest = smax - abs(a)
        b = rng.randint(-rest, rest)
        if rng.random() < 0.3:  # the largest edges
            b = rng.choice([-1, 1]) * rest
        s = abs(a) + abs(b)
        c_true = rng.choice([rng.randint(-2 ** 40, 2 ** 40), rng.randint(-300 * s - 9, 300 * s + 9)])
        cx, cy = 256 * rng.randint(0, 15), 256 * rng.randint(0, 15)
        assert _signs_stepped(c_true, a, b, cx, cy) == _signs_direct(c_true, a, b, cx, cy)


def _binary(rp, li):
    k = 0
    for st in (8, 4, 2, 1):
        if rp[k + st] <= li:
            k += st
    return k, rp[k]


def _two_rounds(rp, li):
    r4, r8, r12 = rp[4], rp[8], rp[12]
    k = 8 if r8 <= li else 0
    rk0 = r8 if k else 0
    rk4 = r12 if k else r4
    s4 = rk4 <= li
    k += 4 if s4 else 0
    rb = rk4 if s4 else rk0
    q1, q2, q3 = rp[k + 1], rp[k + 2], rp[k + 3]
    s2 = q2 <= li
    rodd = q3 if s2 else q1
    s1 = rodd <= li
    pre = rodd if s1 else (q2 if s2 else rb)
    k += (2 if s2 else 0) + (1 if s1 else 0)
    return k, pre


def test_row_search_two_rounds_match_binary_search():
    rng = random.Random(11)
    for _ in range(50000):
        nrow = rng.randint(1, 16)
        widths = [rng.choice([0, 0, 1, 1, 2, 3, 5, 16]) for _ in range(nrow)]
        rp = [0]
        for w in widths:
            rp.append(rp[-1] + w)
        if rp[-1] == 0:
            continue
        rp += [0xFFFF] * (17 - len(rp))  # rows past the last
        li = rng.randrange(rp[nrow])
        k, pre = _two_rounds(rp, li)
        assert (k, pre) == _binary(rp, li)
        assert k == max(j for j in range(nrow) if rp[j] <= li) and pre == rp[k]


def _sat_int(x, up):
    """cvt.rpi / cvt.rmi to s32: saturating, NaN to 0."""
    if math.isnan(x):
        return 0
    if x == math.inf:
        return I32 - 1
    if x == -math.inf:
        return -I32
    v = math.ceil(x) if up else math.floor(x)
    return max(-I32, min(I32 - 1, v))


def test_span_union_with_saturating_conversions():
    rng = random.Random(13)
    # L and M are maxima of finite fma results or -inf (a side no edge bounds)
    vals = [-math.inf, -3e9, 3e9, -1e9, 1e9]
    for _ in range(50000):
        pick = lambda: rng.choice(vals) if rng.random() < 0.2 else rng.uniform(-5000.0, 9000.0)
        L0, M0, L1, M1 = pick(), pick(), pick(), pick()
        two = rng.random() < 0.6
        tw = rng.randint(1, 16)
        hi0, hi1 = -M0, -M1
        ok0, ok1 = L0 <= hi0, two and L1 <= hi1
        # the clamp-based form
        lo = (min(L0, L1) if ok1 else L0) if ok0 else L1
        hi = (max(hi0, hi1) if ok1 else hi0) if ok0 else hi1
        ref = (0, 0)
        if ok0 or ok1:
            lo, hi = max(lo, -1e9), min(hi, 1e9)
            pa = max(0, math.ceil((lo - 240.0) / 256.0))
            pb = min(tw - 1, math.floor(hi / 256.0))
            if pb >= pa:
                ref = (pa, pb - pa + 1)
        # the branch-free form
        lo2 = min(L0 if ok0 else math.inf, L1 if ok1 else math.inf)
        hi2 = max(hi0 if ok0 else -math.inf, hi1 if ok1 else -math.inf)
        pa2 = max(0, _sat_int((lo2 - 240.0) / 256.0, True))
        pb2 = min(tw - 1, _sat_int(hi2 / 256.0, False))
        new = (pa2, pb2 - pa2 + 1) if pb2 >= pa2 else (0, 0)
        assert new == ref, (L0, M0, L1, M1, two, tw)
