"""The seeded workload generator: deterministic, subset-invariant, shaped as
stated (CPU only)."""
import numpy as np

from paper_1910_09020_gb300 import synth


def test_fixed_deterministic_and_subset_invariant():
    a, b = synth.pairs_fixed(7, 0, 1000, 100, synth.SHORT_POISSON, threads=3)
    c, d = synth.pairs_fixed(7, 0, 1000, 100, synth.SHORT_POISSON, threads=1)
    assert (a == c).all() and (b == d).all()
    e, f = synth.pairs_fixed(7, 400, 50, 100, synth.SHORT_POISSON)
    assert (e == a[400:450]).all() and (f == b[400:450]).all()
    assert set(np.unique(a)) <= set(b"ACGT")
    assert set(np.unique(b)) <= set(b"ACGT")


def test_poisson_halves():
    reads, refs = synth.pairs_fixed(3, 0, 4000, 100, synth.SHORT_POISSON)
    ham = (reads != refs).sum(axis=1)
    # odd pairs: independent sequences, ~75 % mismatching positions
    assert 65 < ham[1::2].mean() < 85
    # even pairs: Poisson(3) edits -> mostly similar
    assert np.median(ham[0::2]) < 40
    assert (ham[0::2] == 0).mean() > 0.03  # P(k = 0) = e^-3 ~ 5 %


def test_uniform_k_edit_counts():
    reads, refs = synth.pairs_fixed(5, 0, 3000, 100, synth.SHORT_UNIFORM_K)
    ham = (reads != refs).sum(axis=1)
    assert (ham == 0).mean() > 0.05  # k = 0 w.p. 1/11


def test_varlen_and_log_uniform():
    L = synth.log_uniform(9, 0, 5000, 64, 10000)
    assert L.min() >= 64 and L.max() <= 10000
    # log-uniform: median near sqrt(64 * 10000) = 800
    assert 600 < np.median(L) < 1050
    reads, refs, off = synth.pairs_varlen(9, 0, L[:200], synth.rate_recipe(0.1))
    assert off[-1] == L[:200].sum() == len(reads) == len(refs)
    r2, f2, off2 = synth.pairs_varlen(9, 0, L[:200], synth.rate_recipe(0.1),
                                      threads=1)
    assert (r2 == reads).all() and (f2 == refs).all()


def test_thresholds_floor():
    L = np.array([100, 150, 250, 99, 0, 100000], np.int32)
    assert list(synth.thresholds(L, 5)) == [5, 7, 12, 4, 0, 5000]
    assert list(synth.thresholds(L, 1)) == [1, 1, 2, 0, 0, 1000]
    assert list(synth.thresholds(L, 10)) == [10, 15, 25, 9, 0, 10000]


def test_poisson_arrivals_rate():
    t = synth.poisson_arrivals(1, 20000, 100.0)
    assert np.all(np.diff(t) > 0)
    assert abs(t[-1] / 20000 - 0.01) < 0.001
