"""Pins for the oracle's random draws: Philox4x32-10 against its published
known-answer vectors, and the derived root / IC coin / LT draw against the
distributions they must have."""
import os

import numpy as np
import pytest
from scipy import stats

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLD):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        w = [int(x, 16) for x in line.split()]
        rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


def test_philox_known_answers():
    kats = _kat()
    assert len(kats) == 3
    for ctr, key, want in kats:
        got = oracle.philox4x32_10(ctr, key)
        assert [int(x) for x in got] == want


def test_philox_words_uniform():
    # 24-bit draws (the part the method uses) are uniform: chi^2 over 256 bins
    words = []
    for i in range(4096):
        words.extend(int(x) for x in oracle.philox4x32_10([i, 0, 7, 2], [12345, 0]))
    u24 = np.array(words, dtype=np.uint64) >> 8
    hist = np.bincount((u24 >> 16).astype(np.int64), minlength=256)
    assert stats.chisquare(hist).pvalue > 1e-4


def test_root_uniform_over_vertices():
    # Sec. II-B: the BFS start vertex is uniform over V
    n = 97
    roots = np.array([oracle.root(3, s, n) for s in range(97 * 400)])
    assert roots.min() >= 0 and roots.max() < n
    assert stats.chisquare(np.bincount(roots, minlength=n)).pvalue > 1e-4


def test_root_multiply_shift_extremes():
    # root = floor(x * n / 2^64) lies in [0, n) for every n, including n = 2^32 - 1
    for n in (2, 3, 1000, 2**31 + 11, 2**32 - 1):
        for s in range(50):
            r = oracle.root(9, s, n)
            assert 0 <= r < n


@pytest.mark.parametrize("p", [0.0, 1.0, 0.05, 0.3333333, 1e-7, 0.999999])
def test_ic_threshold_exact(p):
    # thr = ceil(p * 2^24) evaluated exactly (p * 2^24 is exact in fp32)
    f = np.float32(p)
    from fractions import Fraction
    want = -(-Fraction(float(f)) * (1 << 24) // 1)
    assert oracle.ic_threshold(float(f)) == int(want)


def test_ic_coin_frequency_matches_threshold():
    # Sec. II-A (IC): edge live with probability p; here P(live) = thr / 2^24
    thr = oracle.ic_threshold(0.3)
    trials = 40000
    live = sum(oracle.ic_live(5, s, e, thr) for s in range(trials // 8) for e in range(8))
    p = thr / 2**24
    sd = np.sqrt(trials * p * (1 - p))
    assert abs(live - trials * p) < 5 * sd


def test_ic_coin_edge_cases():
    for s in range(200):
        for e in range(6):
            assert oracle.ic_live(1, s, e, 1 << 24)       # p = 1: always live
            assert not oracle.ic_live(1, s, e, 0)         # p = 0: never live


def test_lt_draw_uniform():
    r = np.array([oracle.lt_draw(11, s, v) for s in range(200) for v in range(64)])
    assert r.max() < (1 << 24)
    assert stats.chisquare(np.bincount(r >> 18, minlength=64)).pvalue > 1e-4


# ---- exact conventions (statistics cannot see an off-by-one of 2^-24) ----

def _words(seed, set_id, c2, tag):
    return [int(x) for x in oracle.philox4x32_10(
        [set_id & 0xFFFFFFFF, set_id >> 32, c2, tag], [seed & 0xFFFFFFFF, seed >> 32])]


def test_root_counter_layout_and_multiply_shift():
    # root of set s = floor(((w1 << 32) | w0) * n / 2^64), words of
    # Philox(ctr = (s_lo, s_hi, 0, 1), key = (seed_lo, seed_hi))
    for (seed, s, n) in [(1, 0, 4096), (2**40 + 3, 2**33 + 5, 1 << 20), (7, 123, 1000003)]:
        w = _words(seed, s, 0, 1)
        x = (w[1] << 32) | w[0]
        assert oracle.root(seed, s, n) == (x * n) >> 64


def test_ic_coin_counter_layout_and_strict_compare():
    # coin of in-edge e = word (e & 3) of Philox(ctr = (s_lo, s_hi, e >> 2, 2));
    # live iff (word >> 8) < thr, strictly
    for (seed, s, e) in [(1, 0, 0), (5, 77, 6), (2**35 + 1, 2**32 + 9, 1023), (9, 4, 4097)]:
        r = _words(seed, s, e >> 2, 2)[e & 3] >> 8
        assert not oracle.ic_live(seed, s, e, r)
        assert oracle.ic_live(seed, s, e, r + 1)


def test_lt_draw_counter_layout():
    # LT draw at vertex v = word 0 of Philox(ctr = (s_lo, s_hi, v, 3)) >> 8
    for (seed, s, v) in [(3, 0, 0), (3, 8, 4000000), (2**33, 2**32 + 1, 17)]:
        assert oracle.lt_draw(seed, s, v) == _words(seed, s, v, 3)[0] >> 8


def test_lt_cumulative_thresholds_exact():
    # cthr_j = min(ceil(2^24 * sum_{i<=j} w_i), 2^24) with the fp32 weights summed
    # exactly (Fractions); the oracle's fp64 running sum is exact for these
    from fractions import Fraction
    import numpy as np
    w = np.array([0.1, 0.2, 0.3, 0.05, 0.35], dtype=np.float32)
    n = 6
    row = np.array([0, 5, 5, 5, 5, 5, 5], dtype=np.uint64)
    src = np.array([1, 2, 3, 4, 5], dtype=np.uint32)
    o = oracle.Oracle(n, row, src, w, oracle.LT)
    acc = Fraction(0)
    want = []
    for x in w:
        acc += Fraction(float(x))
        want.append(min(-(-acc * (1 << 24) // 1), 1 << 24))
    assert o.thresholds().tolist() == want
