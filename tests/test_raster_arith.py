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
  first.
- Binning words: the box word's fields and the direct rounds' tile indices name
  the candidate tiles of the quad's box, up to the largest canvas accepted."""
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


def test_bin_words_and_direct_rounds_give_the_candidate_tiles():
    """The binning passes' per-quad words and direct rounds, restated: candidate i
    of a box of ntx x nty tiles from (tx0, ty0) is tile (tx0 + i % ntx, ty0 + i //
    ntx); the box word holds the first candidate's index in 26 bits, ntx - 1 in 5
    and the tall flag in bit 31; a box of two tiles is binned directly in tbase and
    tbase + 1 (two columns) or tbase + tiles_x (two rows); a hit mask of at most
    two bits names the same tiles as the enumeration.  Checked against brute force
    on random boxes up to the largest canvas the call accepts (2^26 tiles)."""
    rng = random.Random(7)
    for _ in range(20000):
        tiles_x = rng.choice([1, 2, 3, 16, 128, 1 << 13])
        tiles_y = max(1, min((1 << 26) // tiles_x, rng.choice([1, 2, 5, 128, 1 << 13])))
        ntx = rng.randint(1, min(tiles_x, 31))
        nty = rng.randint(1, min(tiles_y, 31 // ntx))
        tx0 = rng.randrange(tiles_x - ntx + 1)
        ty0 = rng.randrange(tiles_y - nty + 1)
        n = ntx * nty
        assert 1 <= n <= 31
        cand = [(ty0 + dy) * tiles_x + tx0 + dx for dy in range(nty) for dx in range(ntx)]
        tbase = ty0 * tiles_x + tx0
        assert tbase < (1 << 26)
        tall = rng.randrange(2)
        box = tbase | (ntx - 1) << 26 | tall << 31
        assert box < (1 << 32)
        d_tbase, d_ntx, d_tall = box & 0x3ffffff, ((box >> 26) & 31) + 1, box >> 31
        assert (d_tbase, d_ntx, d_tall) == (tbase, ntx, tall)
        for i in range(n):
            assert d_tbase + (i // d_ntx) * tiles_x + i % d_ntx == cand[i]
        if n == 2:
            assert [tbase, tbase + (1 if ntx == 2 else tiles_x)] == cand
        # a mask of at most two hits: the set bits' tiles, lowest first
        bits = sorted(rng.sample(range(n), rng.randint(1, min(2, n))))
        h = sum(1 << b for b in bits)
        i0 = (h & -h).bit_length() - 1
        got = [d_tbase + (i0 // d_ntx) * tiles_x + i0 % d_ntx]
        h2 = h & (h - 1)
        if h2:
            i1 = (h2 & -h2).bit_length() - 1
            got.append(d_tbase + (i1 // d_ntx) * tiles_x + i1 % d_ntx)
        assert got == [cand[b] for b in bits]
        # the one-tile word: the tile index below the tall flag in bit 30
        direct = 0x80000000 | tall << 30 | cand[0]
        assert direct != 0xffffffff and (direct & 0x3fffffff) == cand[0]
