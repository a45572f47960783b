"""Shared comparison rules for the GPU-vs-oracle parity tests.

The bar (float32 GPU search vs the FP64 oracle): result ids identical on at least 99.9% of the
queries; on the others the two lists may differ only where distances tie within 1e-5 relative;
recall@k of the two within 0.001; returned distances within 1e-5 relative of the oracle's."""
import numpy as np

REL = 1e-5


def eps32(eps):
    """The eps a search of the library ran with: the C ABI takes eps as a float32."""
    return float(np.float32(eps))


def recall(ids, gt):
    k = ids.shape[1]
    return float(np.mean([len(set(a.tolist()) & set(b.tolist())) / k for a, b in zip(ids, gt[:, :k])]))


def compare_lists(g_ids, g_d, o_ids, o_d, min_identical=0.999, rel=REL):
    """Returns (fraction identical, indices of differing queries). Asserts the tie rule."""
    g_ids, o_ids = np.asarray(g_ids), np.asarray(o_ids)
    g_d, o_d = np.asarray(g_d, np.float64), np.asarray(o_d, np.float64)
    same = np.all(g_ids == o_ids, axis=1)
    diff = np.flatnonzero(~same)
    for q in diff:
        # every position: the two distances agree within rel (a different id at the same rank is
        # a tie or a near-tie broken by float32 rounding)
        a, b = g_d[q], o_d[q]
        fin = np.isfinite(b)
        assert np.array_equal(np.isfinite(a), fin), f"query {q}: result sizes differ"
        np.testing.assert_allclose(a[fin], b[fin], rtol=rel, atol=0, err_msg=f"query {q}: not a tie")
    fin = np.isfinite(o_d[same])
    np.testing.assert_allclose(g_d[same][fin], o_d[same][fin], rtol=rel, atol=1e-6)
    frac = float(same.mean()) if len(same) else 1.0
    assert frac >= min_identical, f"only {frac:.4f} of queries identical ({len(diff)} differ)"
    return frac, diff
