"""Host logic of bench.py that decides reported numbers: the eps grid and its bisection, the
algorithmic-byte count of a search, and when a recorded ncu traffic figure may be reported."""
import numpy as np
import pytest

import bench


def test_eps_grid_is_increasing_from_zero_with_the_documented_steps():
    g = np.array(bench.EPS_GRID)
    assert g[0] == 0.0 and np.all(np.diff(g) > 0)
    steps = np.round(np.diff(g), 6)
    assert set(steps[g[1:] <= 0.01]) <= {0.001}
    assert set(steps[(g[1:] > 0.01) & (g[1:] <= 0.1)]) <= {0.005}
    assert set(steps[g[1:] > 0.1]) <= {0.02}


@pytest.mark.parametrize("cut", [0.1043, 0.1001, 0.1199, 0.1200, 0.003])
def test_bisection_finds_the_smallest_reaching_eps_to_a_thousandth(cut):
    calls = []

    def reaches(e):
        calls.append(e)
        return e >= cut

    lo = max([e for e in bench.EPS_GRID if e < cut], default=0.0)
    hi = min(e for e in bench.EPS_GRID if e >= cut)
    got = bench.bisect_eps(lo, hi, reaches)
    assert got >= cut and got - cut <= 0.0011
    assert len(calls) <= 6                                    # 0.02 / 2^5 < 0.001


def test_algorithmic_bytes_per_query_terms():
    # B_q = 4 dim + 4 d H + row_bytes E + 8 k, summed over queries
    trace = np.array([[3, 40, 0, 0], [5, 70, 0, 0]], np.int32)
    got = bench.algorithmic_bytes(trace, dim=128, degree=30, k=10, row_bytes=132)
    want = sum(4 * 128 + 4 * 30 * h + 132 * e + 8 * 10 for h, e in ((3, 40), (5, 70)))
    assert got == want


def _traffic_file(path, digest, eps_fp8, eps_plain):
    path.write_text("# comment: with a colon\n"
                    f"source_digest: {digest}\nworkload: {bench.WORKLOAD}\n"
                    f"eps_fp8: {eps_fp8}\neps_plain: {eps_plain}\n"
                    "dram_bytes_per_launch_fp8: 906472960\ndram_bytes_per_launch_plain: 20666544640\n")


def test_recorded_traffic_only_for_the_same_sources_and_eps(tmp_path, monkeypatch):
    f = tmp_path / "traffic.txt"
    monkeypatch.setattr(bench, "TRAFFIC", str(f))
    _traffic_file(f, bench.source_digest(), 0.003, 0.08)
    assert bench.recorded_traffic("fp8", 0.003) == 906472960
    assert bench.recorded_traffic("plain", 0.08) == 20666544640
    assert bench.recorded_traffic("fp8", 0.004) is None      # captured at another eps
    _traffic_file(f, "0" * 16, 0.003, 0.08)
    assert bench.recorded_traffic("fp8", 0.003) is None      # kernels changed since the capture
    f.unlink()
    assert bench.recorded_traffic("fp8", 0.003) is None      # no capture



def test_row_bytes_match_the_stored_layouts():
    # float32 rows padded to 4 floats, bf16 to 8 values, FP8 codes to 16 bytes plus a float32 scale
    assert [bench.row_bytes(p, 128) for p in ("f32", "bf16", "fp8")] == [512, 256, 132]
    assert [bench.row_bytes(p, 100) for p in ("f32", "bf16", "fp8")] == [400, 208, 116]
    assert [bench.row_bytes(p, 960) for p in ("f32", "bf16", "fp8")] == [3840, 1920, 964]


def test_default_forms_are_the_headline_forms():
    f = bench.make_forms()
    assert list(f) == ["plain float32, fixed entry", "float32, pivot entry", "bf16 + re-rank 32, pivot entry",
                       "fp8 + re-rank 32, pivot entry"]
    assert f["fp8 + re-rank 32, pivot entry"] == dict(precision="fp8", rerank=32, entry="pivot")
    assert "fp8 + re-rank 64, pivot entry" in bench.make_forms(64)
