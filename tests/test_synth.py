"""The seeded input generators: deterministic, with the shapes and value ranges of the workloads."""
import numpy as np

from paper_2307_10479_gb300 import synth


def test_uniform_deterministic_and_prefix_stable():
    a = synth.uniform(100, 8, 0)
    assert a.dtype == np.float32 and a.shape == (100, 8)
    assert np.array_equal(a, synth.uniform(100, 8, 0))
    assert np.array_equal(a[:50], synth.uniform(50, 8, 0))
    assert (a >= 0).all() and (a < 1).all()


def test_mixture_u8_is_integer_valued_and_prefix_stable():
    w = synth.scaled(synth.WORKLOADS["sift-1m-d128"], 70_000, 20)
    x = w.base()
    assert x.shape == (70_000, 128) and x.dtype == np.float32
    assert np.array_equal(x, np.rint(x)) and x.min() >= 0 and x.max() <= 255
    assert np.array_equal(x[:1000], synth.scaled(w, 1000, 20).base())
    q = w.queries()
    assert q.shape == (20, 128) and not np.array_equal(q, x[:20])


def test_vmf_rows_are_unit_and_concentrated():
    w = synth.scaled(synth.WORKLOADS["glove-1.2m-d100"], 2000, 10)
    x = w.base()
    np.testing.assert_allclose(np.linalg.norm(x, axis=1), 1.0, rtol=1e-5)
    # kappa = 50 in 100-D: the mean cosine to the own direction is about kappa / (m - 1 + ...) ~ 0.4
    dirs = synth.vmf_directions(2000, 100, 7)
    best = (x @ dirs.T).max(1)
    assert 0.25 < best.mean() < 0.7


def test_distinct_ids():
    ids = synth.distinct_ids(1000, 300, 2)
    assert len(set(ids.tolist())) == 300 and ids.min() >= 0 and ids.max() < 1000
