"""The synthetic workloads against the values the paper prints (fixtures in tests/golden/, each
citing its table): their build parameters are the rows of Table 2 they stand in for, and their
shapes those of Table 1's datasets."""
import os

import pytest

from paper_2307_10479_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

# workload -> the dataset row it stands in for (the 1M x 960 precision stress follows Enron's
# build row: same degree and extension settings for a high-dimensional set)
STAND_INS = {"sift-1m-d128": "SIFT1M", "glove-1.2m-d100": "GloVe", "mix-1m-d960": "Enron"}


def _table(name):
    rows = {}
    for line in open(os.path.join(GOLDEN, name)):
        if line.strip() and not line.startswith("#"):
            f = line.split()
            rows[f[0]] = [float(x) for x in f[1:]]
    return rows


@pytest.mark.parametrize("workload", sorted(STAND_INS))
def test_build_parameters_are_table_2(workload):
    d, k_ext, eps_ext, k_opt, eps_opt, i_opt = _table("table2_deg_parameters.txt")[STAND_INS[workload]]
    w = synth.WORKLOADS[workload]
    assert (w.degree, w.k_ext, w.k_opt, w.i_opt) == (d, k_ext, k_opt, i_opt)
    assert w.eps_ext == pytest.approx(eps_ext) and w.eps_opt == pytest.approx(eps_opt)


@pytest.mark.parametrize("workload", ["sift-1m-d128", "glove-1.2m-d100"])
def test_shapes_are_table_1(workload):
    m, base, queries, topk, lid = _table("table1_datasets.txt")[STAND_INS[workload]]
    w = synth.WORKLOADS[workload]
    assert w.dim == m and w.nq == queries
    assert abs(w.n - base) / base < 0.02                      # GloVe's 1,183,514 rounded to 1.2M
