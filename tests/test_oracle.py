"""Pins for the CPU oracle against things other than itself.

* the definition of a stable sort (numpy's stable argsort, Python's sorted);
* brute force over every short array on an extreme 4-letter alphabet;
* invariants (permutation, order, stability) and textbook special cases;
* closed forms and exact rational arithmetic for the statistics (Alg. 1);
* the published SplitMix64 sequence and the closed form of the learned map on
  an evenly spaced sample.
"""
import itertools
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2605_14419_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
ALPHABET = [0, 1, 2 ** 63, 2 ** 64 - 1]


def stable_reference(keys):
    """Stable sort by definition: order of the tuples (key, input position)."""
    idx = np.argsort(keys, kind="stable")
    return keys[idx], idx.astype(np.uint32)


def check_sorted_pairs(k_in, v_in, k_out, v_out):
    # permutation of the input pairs
    a = np.lexsort((v_in, k_in))
    b = np.lexsort((v_out, k_out))
    assert np.array_equal(k_in[a], k_out[b]) and np.array_equal(v_in[a], v_out[b])
    # non-decreasing keys
    assert np.all(k_out[:-1] <= k_out[1:])


@pytest.mark.parametrize("family", ["uniform", "normal", "zipf", "nearly_sorted", "descending"])
@pytest.mark.parametrize("n", [0, 1, 2, 97, 1000, 20011])
def test_matches_stable_argsort(family, n):
    keys = inputs.FAMILIES[family](n, seed=7 + n)
    vals = inputs.index_payload(n)
    k, v = oracle.zsort_pairs(keys, vals)
    rk, rv = stable_reference(keys)
    assert np.array_equal(k, rk)
    assert np.array_equal(v, rv)


@pytest.mark.parametrize("gen", [inputs.lognormal, inputs.gaussian_mixture, inputs.dense_interval_u64])
def test_matches_stable_argsort_skewed(gen):
    keys = gen(50_000, seed=3)
    vals = inputs.index_payload(keys.size)
    k, v = oracle.zsort_pairs(keys, vals)
    rk, rv = stable_reference(keys)
    assert np.array_equal(k, rk) and np.array_equal(v, rv)


def test_random_payload_travels_with_key():
    rng = np.random.default_rng(1)
    keys = rng.integers(0, 50, 5000).astype(np.uint64)  # many ties
    vals = rng.integers(0, 2 ** 32, 5000, dtype=np.uint64).astype(np.uint32)
    k, v = oracle.zsort_pairs(keys, vals)
    idx = np.argsort(keys, kind="stable")
    assert np.array_equal(k, keys[idx]) and np.array_equal(v, vals[idx])


@pytest.mark.parametrize("leaf,count_range", [(96, 65000), (1, 0)])
def test_brute_force_short_arrays(leaf, count_range):
    """Every array of length <= 6 over {0, 1, 2^63, 2^64-1} (5461 arrays),
    against Python's sorted() on (key, position).  leaf=1, count_range=0 turn
    off the insertion and counting shortcuts so every level partitions."""
    for n in range(0, 7):
        for combo in itertools.product(ALPHABET, repeat=n):
            keys = np.array(combo, dtype=np.uint64)
            vals = np.arange(n, dtype=np.uint32)
            k, v = oracle.zsort_pairs(keys, vals, leaf=leaf, count_range=count_range)
            order = sorted(range(n), key=lambda i: (combo[i], i))
            assert [int(x) for x in v] == order, combo
            assert [int(x) for x in k] == [combo[i] for i in order], combo


def test_brute_force_length8_sampled():
    rng = np.random.default_rng(0)
    for _ in range(3000):
        combo = [ALPHABET[i] for i in rng.integers(0, 4, 8)]
        keys = np.array(combo, dtype=np.uint64)
        k, v = oracle.zsort_pairs(keys, np.arange(8, dtype=np.uint32), leaf=1, count_range=0)
        order = sorted(range(8), key=lambda i: (combo[i], i))
        assert [int(x) for x in v] == order


def test_special_cases():
    n = 5000
    # all equal: identity (R2 early exit)
    k, v, tr = oracle.zsort_pairs(np.full(n, 12345, np.uint64), inputs.index_payload(n), with_trace=True)
    assert np.array_equal(v, np.arange(n)) and tr.equal_exits == 1 and tr.partitions == 0
    # strictly descending distinct keys: reversal
    d = inputs.descending(n)
    k, v = oracle.zsort_pairs(d, inputs.index_payload(n))
    assert np.array_equal(v, np.arange(n)[::-1]) and np.array_equal(k, d[::-1])
    # n = 1
    k, v = oracle.zsort_pairs(np.array([7], np.uint64), np.array([3], np.uint32))
    assert k[0] == 7 and v[0] == 3
    # two distinct values far apart: stable two-way split
    rng = np.random.default_rng(5)
    two = np.where(rng.random(n) < 0.3, np.uint64(2 ** 64 - 1), np.uint64(0))
    k, v = oracle.zsort_pairs(two, inputs.index_payload(n))
    lo = np.nonzero(two == 0)[0]
    hi = np.nonzero(two != 0)[0]
    assert np.array_equal(v, np.concatenate([lo, hi]))
    # keys that collide in binary64: 2^63 and 2^63 + 1 (R1 keeps them apart)
    near = (np.uint64(2 ** 63) + rng.integers(0, 2, n).astype(np.uint64))
    k, v = oracle.zsort_pairs(near, inputs.index_payload(n), count_range=0, leaf=1)
    rk, rv = stable_reference(near)
    assert np.array_equal(v, rv)


def test_counting_sort_branch_taken_for_small_range():
    keys = (np.uint64(2 ** 50) + np.random.default_rng(2).integers(0, 60000, 30000).astype(np.uint64))
    k, v, tr = oracle.zsort_pairs(keys, inputs.index_payload(keys.size), with_trace=True)
    assert tr.counting_sorts == 1 and tr.partitions == 0
    rk, rv = stable_reference(keys)
    assert np.array_equal(v, rv)


def test_geometric_keys_need_the_progress_guard():
    """Keys 2^i (i = 0..63) repeated: the z-score map with meanEst puts all
    of a cluster into one bucket at some level; the guard must still end."""
    rng = np.random.default_rng(9)
    keys = (np.uint64(1) << rng.integers(0, 64, 20000).astype(np.uint64))
    k, v, tr = oracle.zsort_pairs(keys, inputs.index_payload(keys.size), leaf=1, count_range=0,
                                  with_trace=True)
    rk, rv = stable_reference(keys)
    assert np.array_equal(v, rv)
    assert tr.max_depth < 100


def test_cluster_count_and_scale():
    """k = max(2, floor(0.6 sqrt(n))), scale = k/4 (R5)."""
    for n, k_expected in [(10 ** 5, 189), (10 ** 6, 600), (65536, 153), (3, 2)]:
        _, _, tr = oracle.zsort_pairs(inputs.uniform(n, 1), inputs.index_payload(n), with_trace=True)
        assert tr.k == k_expected
        assert tr.scale == k_expected / 4


@pytest.mark.parametrize("gen", [inputs.uniform, inputs.normal, inputs.lognormal, inputs.gaussian_mixture,
                                 inputs.zipf, inputs.descending])
def test_level1_partition_invariant(gen):
    """max(C_j) <= min(C_{j+1}) for the level-1 clusters of Eq. 1 (section
    "Proposed Work": every key of a cluster is at most every key of the next
    one), checked over the oracle's own cluster of every key: in key order
    the cluster index never decreases, and every non-empty cluster's largest
    key is at most the next non-empty cluster's smallest."""
    keys = gen(40_000, 11)
    for k in (7, 120, 1024):
        b = oracle.level1_buckets(keys, k).astype(np.int64)
        assert b.min() >= 0 and b.max() <= k - 1
        order = np.argsort(keys, kind="stable")
        assert np.all(np.diff(b[order]) >= 0)
        used = np.unique(b)
        lo = np.array([keys[b == j].min() for j in used], dtype=np.uint64)
        hi = np.array([keys[b == j].max() for j in used], dtype=np.uint64)
        assert np.all(hi[:-1] <= lo[1:])


def test_level1_partition_invariant_catches_a_non_monotone_map():
    """The check above fails for a map that is not monotone (a dropped
    absolute value in Zmin folds the keys below the mean back up)."""
    keys = inputs.normal(5000, 3)
    mn, _mx, mean, sd = oracle.stats(keys)
    d = (keys - np.uint64(mn)).astype(np.float64)
    k = 64
    h = ((d - mean) / sd - mean / sd) * (k / 4)  # Zmin with the wrong sign
    b = np.clip(np.floor(np.abs(h)), 0, k - 1).astype(np.int64)
    order = np.argsort(keys, kind="stable")
    assert not np.all(np.diff(b[order]) >= 0)


def test_meanest_closed_form_on_arithmetic_progression():
    """R9 (zsortRec): a sub-problem takes mean = meanEst = ((j + 0.5)/scale -
    Zmin) * sd + mean of its parent, moved into its own frame, and computes
    its sd about that mean.  On keys base + i*step (i = 0..N-1) every quantity
    has a closed form: the parent's sd = step*sqrt((N^2-1)/12), Zmin = mean/sd,
    so meanEst = (j + 0.5) * sd / scale; cluster j holds the i with
    floor(i*step*scale/sd) = j; the child's sd about m = meanEst - i_lo*step is
    sqrt(sum_{t<c} (t*step - m)^2 / c).  Computed here in 40-digit decimals."""
    from decimal import Decimal, getcontext

    getcontext().prec = 40
    N, step, base = 20000, 7, 2 ** 40
    keys = np.uint64(base) + np.random.default_rng(0).permutation(N).astype(np.uint64) * np.uint64(step)
    k_out, v_out, tr, recs = oracle.zsort_pairs_records(keys, inputs.index_payload(N), count_range=0)
    assert np.all(k_out[:-1] <= k_out[1:])
    k = int(np.floor(0.6 * np.sqrt(N)))
    assert tr.k == k
    D = Decimal
    scale = D(k) / 4
    sd_p = D(step) * ((D(N) * N - 1) / 12).sqrt()
    depth1 = [r for r in recs if r.depth == 1]
    # every child of the top level with more than 96 keys is recursed once
    assert len(depth1) >= 60
    seen = set()
    for r in depth1:
        j = r.parent_bucket
        seen.add(j)
        est = (D(j) + D("0.5")) * sd_p / scale
        assert abs(D(r.est_parent_d) - est) <= D("1e-9") * est
        # the child's keys: i in [i_lo, i_lo + c), all in cluster j of Eq. 1
        i_lo = (r.min - base) // step
        assert r.parent_min == base and (r.min - base) % step == 0
        c = r.size
        for i in (i_lo, i_lo + c - 1):
            h = D(i * step) * scale / sd_p
            # not within rounding distance of an edge (except the key 0 itself)
            assert int(h) == j and (i == 0 or h - int(h) > D("1e-9")) and int(h) + 1 - h > D("1e-9")
        if i_lo > 0:
            assert int(D((i_lo - 1) * step) * scale / sd_p) == j - 1
        m = est - D(i_lo * step)
        assert abs(D(r.mean) - m) <= D("1e-9") * abs(m)
        s1 = D(c) * (c - 1) / 2
        s2 = D(c - 1) * c * (2 * c - 1) / 6
        var = (D(step) * step * s2 - 2 * m * step * s1 + c * m * m) / c
        assert abs(D(r.sd) - var.sqrt()) <= D("1e-9") * var.sqrt()
        assert abs(D(r.zmin) - abs(m) / var.sqrt()) <= D("1e-9") * (abs(m) / var.sqrt() + 1)
    assert len(seen) == len(depth1)


def _f32(x):
    """Round a positive Fraction to the nearest binary32 (ties to even);
    normal range only."""
    from fractions import Fraction

    assert x > 0
    e = x.numerator.bit_length() - x.denominator.bit_length()
    if Fraction(2) ** e > x:
        e -= 1
    ulp = Fraction(2) ** (e - 23)
    q, rem = divmod(x, ulp)
    if rem * 2 > ulp or (rem * 2 == ulp and q % 2 == 1):
        q += 1
    return q * ulp


def test_pwl_stored_slope_reading():
    """R11: inside piece s the learned map takes frac = fl32(fl32(u - q_s) *
    r_s) with the stored slope r_s = fl32(1 / (q_{s+1} - q_s)), not the
    quotient fl32((u - q_s) / width).  The case below has a piece of width
    82 * 2^-24 and a key exactly in its middle: the quotient is 1/2 exactly
    (bucket 2s + 1 with K = 2), while the rounded slope is below 1/82 * 2^24,
    so the product falls just short of 1/2 (bucket 2s).  Expected values are
    computed here in exact rational arithmetic."""
    from fractions import Fraction

    two24 = 1 << 24
    P, k = 4, 8  # K = k / P = 2 sub-buckets per piece
    qi = [0, 100, 182, 1000, two24 - 1]  # breakpoints in units of 2^-24; piece 1 is 82 wide
    q = np.array([x / two24 for x in qi], dtype=np.float32)
    mn, mx = 0, two24 - 1  # E = 24: u = key * 2^-24 exactly
    key = 100 + 41
    width = Fraction(82, two24)
    slope = _f32(1 / width)
    assert slope < two24 / Fraction(82)
    frac = _f32(Fraction(41, two24) * slope)
    assert frac < Fraction(1, 2)
    expect = 1 * 2 + int(frac * 2)
    quotient_bucket = 1 * 2 + int(Fraction(41, two24) / width * 2)
    assert (expect, quotient_bucket) == (2, 3)
    assert oracle.pwl_buckets(np.array([key], dtype=np.uint64), mn, mx, q, k, P=P)[0] == expect
    # the neighbours on either side land where both readings agree
    b = oracle.pwl_buckets(np.array([100, 140, 142, 181, 182], dtype=np.uint64), mn, mx, q, k, P=P)
    assert list(b) == [2, 2, 3, 3, 4]


def _exact_stats(keys):
    mn = int(keys.min())
    d = [int(x) - mn for x in keys]
    n = len(d)
    mean = Fraction(sum(d), n)
    var = sum((Fraction(x) - mean) ** 2 for x in d) / n
    return mn, int(keys.max()), mean, var


@pytest.mark.parametrize("gen,n", [(inputs.uniform, 4000), (inputs.lognormal, 4000),
                                   (inputs.gaussian_mixture, 4000), (inputs.zipf, 4000)])
def test_stats_against_exact_rationals(gen, n):
    keys = gen(n, 21)
    mn, mx, mean, sd = oracle.stats(keys)
    emn, emx, emean, evar = _exact_stats(keys)
    assert mn == emn and mx == emx
    assert abs(mean - float(emean)) <= 1e-12 * max(1.0, float(emean))
    assert abs(sd * sd - float(evar)) <= 1e-12 * float(evar)


def test_stats_closed_forms():
    # d = 0..N-1: mean (N-1)/2, var (N^2 - 1)/12
    N = 100_001
    keys = np.uint64(2 ** 63 + 5) + np.arange(N, dtype=np.uint64)
    mn, mx, mean, sd = oracle.stats(keys)
    assert mn == 2 ** 63 + 5 and mx == 2 ** 63 + 5 + N - 1
    assert mean == (N - 1) / 2
    assert abs(sd ** 2 - (N * N - 1) / 12) <= 1e-12 * (N * N - 1) / 12
    # two values 2^63, 2^63+1 in equal number: sd = 1/2 exactly
    keys = np.array([2 ** 63, 2 ** 63 + 1] * 500, dtype=np.uint64)
    assert oracle.stats(keys)[3] == 0.5
    # uniform over [0, R): sd ~ R / sqrt(12)
    keys = inputs.uniform(200_000, 4)
    sd = oracle.stats(keys)[3]
    assert abs(sd / (2.0 ** 64 / np.sqrt(12)) - 1) < 0.01


def test_key_encoding_int64():
    x = np.array([np.iinfo(np.int64).min, -5, -1, 0, 1, 7, np.iinfo(np.int64).max], dtype=np.int64)
    u = oracle.key_from_i64(x)
    assert np.all(u[:-1] < u[1:])
    assert np.array_equal(oracle.key_to_i64(u), x)
    rnd = inputs.dense_interval_i64(10000, 2)
    u = oracle.key_from_i64(rnd)
    assert np.array_equal(np.argsort(u, kind="stable"), np.argsort(rnd, kind="stable"))


def test_key_encoding_float64_total_order():
    x = np.array([-np.inf, -1e300, -1.0, -5e-324, -0.0, 0.0, 5e-324, 1.0, 1e300, np.inf])
    u = oracle.key_from_f64(x)
    assert np.all(u[:-1] < u[1:])  # strict, and -0.0 < +0.0
    back = oracle.key_to_f64(u)
    assert np.array_equal(back.view(np.uint64), x.view(np.uint64))
    rnd = inputs.normal_f64_specials(20000, 3)
    u = oracle.key_from_f64(rnd)
    order = np.argsort(u, kind="stable")
    s = rnd[order]
    assert np.all(s[:-1] <= s[1:])  # IEEE order agrees except the zero signs
    zeros = s[s == 0.0]
    assert np.all(np.signbit(zeros[: np.count_nonzero(np.signbit(zeros))]))


def test_splitmix64_published_sequence():
    with open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) as f:
        want = [int(line, 16) for line in f if line.strip() and not line.startswith("#")]
    gamma = 0x9E3779B97F4A7C15
    got = [oracle.splitmix64((i * gamma) % 2 ** 64) for i in range(len(want))]
    assert got == want


def test_sample_positions_stratified():
    for length, m in [(65536, 65536), (10 ** 6, 4096), (123457, 1000)]:
        pos = oracle.sample_positions(99, length, m)
        lo = (np.arange(m, dtype=object) * length) // m
        hi = (np.arange(1, m + 1, dtype=object) * length) // m
        p = pos.astype(object)
        assert all(lo[i] <= p[i] < hi[i] for i in range(m))
    assert np.array_equal(oracle.sample_positions(1, 4096, 4096), np.arange(4096))


def test_pwl_closed_form_on_even_sample():
    """Sample = 0..m-1 (m = 2^16), min 0, max m-1: u = d / 2^16 exactly, the
    breakpoints are q_j = j/256, and outside the last piece the bucket is
    floor(d * k / m)."""
    m, k = 65536, 1024
    sample = np.arange(m, dtype=np.uint64)
    q = oracle.pwl_train(sample, 0, m - 1)
    assert q[0] == 0.0 and q[256] == np.float32((m - 1) / m)
    assert np.array_equal(q[:256], np.arange(256, dtype=np.float32) / 256)
    d = np.arange(0, 255 * 256, 37, dtype=np.uint64)
    b = oracle.pwl_buckets(d, 0, m - 1, q, k)
    assert np.array_equal(b, (d * np.uint64(k) // np.uint64(m)).astype(np.uint32))


def test_pwl_balanced_on_its_sample_and_monotone():
    keys = inputs.lognormal(300_000, 5)
    mn, mx, q, sample = oracle.learned_map(keys, seed=17, m=8192, k=1024)
    assert np.all(q[:-1] <= q[1:])
    b = oracle.pwl_buckets(sample, mn, mx, q, 1024)
    piece = b // 4
    counts = np.bincount(piece, minlength=256)
    # distinct sample values: every piece holds exactly m / 256 of them
    if np.unique(sample).size == sample.size:
        assert np.all(counts == 8192 // 256)
    # monotone over sorted probes that include every breakpoint's neighbours
    probes = np.unique(np.concatenate([np.sort(sample), [mn, mx], np.sort(sample) + np.uint64(1)]))
    probes = probes[probes <= mx]
    pb = oracle.pwl_buckets(probes, mn, mx, q, 1024)
    assert np.all(pb[:-1] <= pb[1:])
    assert pb[0] == 0 and pb[-1] <= 1023


def test_split_map_closed_form_on_even_sample():
    """Exact-key map on a sample of keys base + i*step (i < m): the
    breakpoints are the keys at ranks j m / P and every piece has the same
    width, so the bucket of base + d (d < (P-1) m / P * step) is
    floor(d * k / (m * step)) -- the same closed form as the normalised map,
    here at 2^62 + ..., where binary32 normalisation would round."""
    m, k, step, base = 65536, 512, 3, 2 ** 62 + 12345
    sample = np.uint64(base) + np.arange(m, dtype=np.uint64) * np.uint64(step)
    b, r = oracle.split_train(sample, base, base + (m - 1) * step)
    assert np.array_equal(b[:256], (np.uint64(base) + np.arange(256, dtype=np.uint64) * np.uint64(256 * step)))
    d = np.arange(0, 255 * 256 * step, 97, dtype=np.uint64)
    got = oracle.split_buckets(np.uint64(base) + d, b, r, k)
    assert np.array_equal(got, (d * np.uint64(k) // np.uint64(m * step)).astype(np.uint32))


def test_split_map_resolves_a_dense_interval_that_fp32_collapses():
    """90% of the keys in [2^63 - 2^19, 2^63 + 2^19) (the int64 law of the
    adversarial workload, encoded): normalised to binary32 the interval is one
    value and the map piles it into one bucket; with exact-key breakpoints
    the sample's largest bucket stays within 4x the mean load, and the map is
    monotone over the keys and over probes around every breakpoint."""
    keys = inputs.dense_interval_i64(400_000, 4).view(np.uint64) ^ np.uint64(2 ** 63)
    mn, mx = int(keys.min()), int(keys.max())
    m, k = 65536, 512
    pos = oracle.sample_positions(17, keys.size, m).astype(np.int64)
    sample = keys[pos]
    q = oracle.pwl_train(sample, mn, mx)
    pwl = oracle.pwl_buckets(sample, mn, mx, q, k)
    assert np.bincount(pwl.astype(np.int64), minlength=k).max() > 0.5 * m
    b, r = oracle.split_train(sample, mn, mx)
    sb = oracle.split_buckets(sample, b, r, k)
    assert np.bincount(sb.astype(np.int64), minlength=k).max() <= 4 * m / k
    order = np.argsort(keys, kind="stable")
    kb = oracle.split_buckets(keys[order], b, r, k)
    assert np.all(np.diff(kb.astype(np.int64)) >= 0) and kb[0] == 0
    probes = np.unique(np.concatenate([b, b[1:] - np.uint64(1), b[:-1] + np.uint64(1)]))
    pb = oracle.split_buckets(probes, b, r, k)
    assert np.all(np.diff(pb.astype(np.int64)) >= 0)


def test_segmented_oracle():
    keys, vals, off, _ = inputs.segmented(40, 3, lo=2, hi=5000)
    k, v = oracle.zsort_segmented(keys, vals, off)
    for i in range(40):
        a, b = int(off[i]), int(off[i + 1])
        idx = np.argsort(keys[a:b], kind="stable")
        assert np.array_equal(k[a:b], keys[a:b][idx])
        assert np.array_equal(v[a:b], vals[a:b][idx])


@pytest.mark.parametrize("k", [2, 7, 189, 1024])
def test_level1_map_closed_form(k):
    """Eq. 1 with Zmin = |(min - mean)/sd|: the mean cancels, so on an
    arithmetic progression d_i = i * step the cluster is
    min(k-1, floor(i * step * (k/4) / sd)) with sd = step * sqrt((N^2-1)/12)."""
    N, step = 10_000, 3
    keys = np.uint64(2 ** 62) + np.arange(N, dtype=np.uint64) * np.uint64(step)
    b = oracle.level1_buckets(keys, k)
    sd = step * np.sqrt((N * N - 1) / 12.0)
    i = np.arange(N, dtype=np.float64)
    expect = np.minimum(k - 1, np.floor(i * step * (k / 4.0) / sd)).astype(np.uint64)
    # the two sides round differently; allow disagreement only on the few
    # keys that sit within 1e-9 of a bucket edge
    h = i * step * (k / 4.0) / sd
    edge = np.abs(h - np.round(h)) < 1e-9
    assert np.array_equal(b[~edge], expect[~edge])
    assert b[0] == 0 and np.all(b[:-1] <= b[1:])
    # the map covers [min, min + 4 sd): the first key past it is in bucket k-1
    first_clip = int(np.ceil(4 * sd / step))
    if first_clip < N:
        assert b[first_clip] == k - 1 and b[first_clip - 2] < k - 1 or k == 2


def test_level1_map_uniform_fractions():
    """Uniform keys: sd = R/sqrt(12), so 4 sd = 1.1547 R and bucket j holds
    about 1.1547/k of the keys for j < k-1 (closed form of Eq. 1)."""
    keys = inputs.uniform(400_000, 12)
    k = 64
    b = oracle.level1_buckets(keys, k)
    frac = np.bincount(b.astype(np.int64), minlength=k) / keys.size
    assert np.allclose(frac[: int(k / 1.1547) - 1], 4.0 / np.sqrt(12) / k, rtol=0.05)
    assert frac[k - 1] < 1.0 / k


# ---------------------------------------------------------------- MLP map
def mlp_knot_loss(params, q):
    return sum((oracle.mlp_eval(params, float(q[j])) - j / 256) ** 2 for j in range(257))


def test_mlp_start_is_the_piecewise_interpolation():
    """With no training step, unit h is the ramp from knot 8h to knot 8h + 8
    with weight 1/32: f(q[8h]) = h/32 (up to the rounding of sqrt(1/32)^2),
    linear in between."""
    keys = inputs.gaussian_mixture(200_000, 3)
    mn, mx, q, _ = oracle.learned_map(keys, seed=5, m=65536, k=512)
    p = oracle.mlp_train(q, 0)
    for h in range(33):
        assert abs(oracle.mlp_eval(p, float(q[8 * h])) - h / 32) < 1e-5, h
    # midway between two knots of one ramp (distinct knots): half a step more
    for h in range(32):
        lo, hi = float(q[8 * h]), float(q[8 * h + 8])
        if hi > lo:
            mid = np.float32((lo + hi) / 2)
            assert abs(oracle.mlp_eval(p, float(mid)) - (h + 0.5) / 32) < 1e-4


def test_mlp_identity_knots_give_the_uniform_map():
    """Knots q_j = j/256 (an evenly spread sample): the start state is
    f(u) = u, so the bucket of u = d / 2^16 is floor(d * k / 2^16) below the
    top knot."""
    m, k = 65536, 1024
    q = oracle.pwl_train(np.arange(m, dtype=np.uint64), 0, m - 1)
    p = oracle.mlp_train(q, 0)
    d = np.arange(0, 255 * 256, 41, dtype=np.uint64)
    b = oracle.mlp_buckets(d, 0, m - 1, p, k)
    want = (d * np.uint64(k) // np.uint64(m)).astype(np.int64)
    assert np.max(np.abs(b.astype(np.int64) - want)) <= 1  # f0, inv rescale by f(u_max)


@pytest.mark.parametrize("gen", [inputs.lognormal, inputs.gaussian_mixture, inputs.uniform,
                                 inputs.normal, inputs.dense_interval_u64])
def test_mlp_training_lowers_the_error_and_stays_monotone(gen):
    keys = gen(300_000, 9)
    mn, mx, q, sample = oracle.learned_map(keys, seed=11, m=65536, k=512)
    p0, p = oracle.mlp_train(q, 0), oracle.mlp_train(q, 128)
    assert mlp_knot_loss(p, q) < mlp_knot_loss(p0, q)
    assert np.all(np.isfinite(p))
    # positive weights by construction: w = omega^2, a = alpha^2
    probes = np.unique(np.concatenate([np.sort(sample), [mn, mx], np.sort(sample) + np.uint64(1)]))
    probes = probes[probes <= mx]
    b = oracle.mlp_buckets(probes, mn, mx, p, 512)
    assert np.all(b[:-1] <= b[1:])
    assert b[0] == 0 and b[-1] <= 511
    # a dense grid of u: f non-decreasing
    us = np.linspace(0.0, float(q[-1]), 5001, dtype=np.float32)
    fs = [oracle.mlp_eval(p, float(u)) for u in us]
    assert all(a <= b for a, b in zip(fs, fs[1:]))


def test_mlp_balance_on_uniform_keys():
    keys = inputs.uniform(400_000, 12)
    mn, mx, q, sample = oracle.learned_map(keys, seed=13, m=65536, k=512)
    b = oracle.mlp_buckets(sample, mn, mx, oracle.mlp_train(q, 128), 512)
    assert np.bincount(b, minlength=512).max() <= 2 * 65536 // 512


# ---------------------------------------------------------------- CPU comparison sorts
@pytest.mark.parametrize("gen", [inputs.uniform, inputs.zipf, inputs.descending])
def test_stdsort_comparator_is_the_stable_sort(gen):
    keys = gen(30_000, 5)
    vals = inputs.index_payload(keys.size)
    k, v = oracle.stdsort_pairs(keys, vals)
    rk, rv = stable_reference(keys)
    assert np.array_equal(k, rk) and np.array_equal(v, rv)


def test_threaded_segmented_oracle_matches_sequential():
    keys, vals, off, _ = inputs.segmented(120, 8, lo=2, hi=20_000)
    k1, v1 = oracle.zsort_segmented(keys, vals, off)
    k2, v2, t = oracle.zsort_segmented_mt(keys, vals, off, threads=4)
    assert t == 4 and np.array_equal(k1, k2) and np.array_equal(v1, v2)
    _, _, tall = oracle.zsort_segmented_mt(keys, vals, off)
    assert tall >= 1
