"""The synthetic input recipe: the generators draw what their docstrings state
(background composition, substitution and indel model, workload shapes, seeding).
They hold none of the method's arithmetic; these checks keep the workloads the
benchmark and the parity tests run on the ones described."""
import math

import numpy as np
import pytest

from paper_0905_1744_gb300 import datagen


def test_background_composition():
    rng = datagen.rng_for(0, 123)
    x = datagen.background(rng, 2_000_000)
    assert x.dtype == np.uint8 and x.max() < 20
    freq = np.bincount(x, minlength=20) / x.size
    # 16-bit quantised CDF plus sampling noise (std < 2.1e-4 at this size)
    np.testing.assert_allclose(freq, datagen.BACKGROUND, atol=1.2e-3)


def test_substitutions_only(monkeypatch):
    """Without indels every member keeps the ancestor's length and differs from it
    at a fraction near its own rate r ~ U[0.20, 0.40]; no substitution keeps the
    original residue."""
    monkeypatch.setattr(datagen, "INDEL_RATE", 0.0)
    rng = datagen.rng_for(0, 7)
    anc = datagen.background(rng, 20000)
    codes, lens = datagen.mutate_family(rng, anc, 64)
    assert (lens == 20000).all()
    members = codes.reshape(64, 20000)
    frac = (members != anc[None, :]).mean(axis=1)
    assert frac.min() > 0.20 - 0.015 and frac.max() < 0.40 + 0.015
    assert frac.std() > 0.03               # rates differ between members (U[0.2, 0.4]: 0.058)


def test_indels_only(monkeypatch):
    """Without substitutions the members are the ancestor with indels. Insertions
    and deletions have equal odds and the same length law, so the length change
    per member is small on average; it leans positive because overlapping
    deletions merge (about +11 residues here, for about 275 inserted and 275
    deleted). Its spread follows the 0.02 per-position event rate."""
    monkeypatch.setattr(datagen, "SUB_RATE", (0.0, 0.0))
    rng = datagen.rng_for(0, 8)
    anc = datagen.background(rng, 5000)
    codes, lens = datagen.mutate_family(rng, anc, 400)
    d = lens - 5000
    # 100 events a member of mean length 5.5, +-: std of the sum about 60
    assert 0 <= d.mean() < 25 and 25 < d.std() < 110
    assert lens.min() >= datagen.MIN_LEN
    assert codes.size == lens.sum() and codes.max() < 20


def test_short_members_keep_their_deletions_out():
    rng = datagen.rng_for(0, 9)
    anc = datagen.background(rng, datagen.MIN_LEN)
    codes, lens = datagen.mutate_family(rng, anc, 2000)
    assert lens.min() >= datagen.MIN_LEN


def test_workload_shapes():
    c1 = datagen.config1()
    assert c1.n == 200 and c1.p == 4
    assert c1.lengths.min() >= 100 and c1.lengths.max() <= 400
    c2 = datagen.config2()
    assert c2.n == 20000 and c2.p == 16 and c2.codes.max() < 20
    assert 250 < c2.lengths.mean() < 350                        # ancestors N(300, 100)
    assert c2.offsets.dtype == np.int64 and c2.codes.dtype == np.uint8
    for i in (0, 7, 31):
        s = datagen.batch_set(i)
        assert 50 <= s.n <= 5000 and s.p == max(1, math.ceil(s.n / 500))
    s = datagen.serving_set(3)
    assert 100 <= s.n <= 20000 and s.p == 16


def test_seeding_is_deterministic_and_seed_dependent():
    a, b = datagen.config1(seed=0), datagen.config1(seed=0)
    np.testing.assert_array_equal(a.codes, b.codes)
    np.testing.assert_array_equal(a.offsets, b.offsets)
    c = datagen.config1(seed=1)
    assert a.codes.size != c.codes.size or (a.codes != c.codes).any()
    # each set of a many-set workload has its own stream: the same set alone or in a list
    s3 = datagen.batch_set(3)
    np.testing.assert_array_equal(datagen.many_sets("batch", [2, 3], workers=1)[1].codes,
                                  s3.codes)


def test_poisson_arrivals():
    t = datagen.poisson_arrivals(20000, rate_per_s=200.0)
    assert (np.diff(t) > 0).all()
    assert t[-1] == pytest.approx(100.0, rel=0.03)              # 20000 arrivals at 200/s


def test_random_keys_ties():
    hi, lo = datagen.random_keys(1000, seed=1, distinct=7)
    assert len(set(zip(hi.tolist(), lo.tolist()))) <= 7
    hi, lo = datagen.random_keys(1000, seed=1)
    assert hi.dtype == np.uint64 and lo.dtype == np.uint64
