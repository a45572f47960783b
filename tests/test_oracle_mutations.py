"""The oracle's pins catch plausible mistakes. Each case copies the oracle's sources to a temporary
directory, plants one mistake (a flipped comparison, a dropped update, a dropped term), builds
that copy, and runs the pin tests against it in a subprocess (DEG_ORACLE_LIB points the oracle
at the copy): at least one pin must fail. The repository's sources are never modified."""
import os
import shutil
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRCS = ["oracle_search.cpp", "oracle_build.cpp", "oracle_quant.cpp", "oracle_mlp.cpp"]

# name: (source, text, planted text, pin file[, sites]); every site of the text is replaced, and
# the number of sites is checked (1 unless given)
MUTATIONS = {
    "stop test not strict": ("oracle_search.cpp", "if (s.d > r * (1.0 + eps)) break;",
                             "if (s.d >= r * (1.0 + eps)) break;", "test_oracle_search.py"),
    "admission not inclusive": ("oracle_search.cpp", "if (dn <= r * (1.0 + eps)) {",
                                "if (dn < r * (1.0 + eps)) {", "test_oracle_search.py"),
    "result insertion not inclusive": ("oracle_search.cpp", "if (dn <= r) {", "if (dn < r) {",
                                       "test_oracle_search.py"),
    "radius not updated on a trim": ("oracle_search.cpp",
                                     "                        R.erase(std::prev(R.end()));\n"
                                     "                        r = std::prev(R.end())->d;",
                                     "                        R.erase(std::prev(R.end()));", "test_oracle_search.py"),
    "trim drops the smallest": ("oracle_search.cpp",
                                "                        R.erase(std::prev(R.end()));\n"
                                "                        r = std::prev(R.end())->d;",
                                "                        R.erase(R.begin());\n"
                                "                        r = std::prev(R.end())->d;", "test_oracle_search.py"),
    "seeds not checked": ("oracle_search.cpp", "if (!C.insert(s).second) continue;", "if (C.count(s)) continue;",
                          "test_oracle_search.py"),
    "seed not counted as an evaluation": ("oracle_search.cpp", "        const double ds = dist_to_q(s);\n        ++evals;",
                                          "        const double ds = dist_to_q(s);", "test_oracle_search.py"),
    "no float32 re-rank": ("oracle_quant.cpp",
                           "for (Cand& c : R) c.d = distance(base + (int64_t)c.id * dim, qv, dim);",
                           "(void)base;", "test_oracle_search.py"),
    "first ReLU dropped": ("oracle_mlp.cpp", "            h1[j] = a > 0 ? a : 0;", "            h1[j] = a;",
                           "test_oracle_mlp.py", 2),                 # the loss and the prediction paths
    "backward pass ignores the second ReLU": ("oracle_mlp.cpp", "            d2[i] = h2[i] > 0 ? g : 0;",
                                              "            d2[i] = g;", "test_oracle_mlp.py"),
    "first-layer weight gradient transposed": ("oracle_mlp.cpp",
                                               "grad[OW1 + j * IN + i] += d1[j] * (double)xs[i];",
                                               "grad[OW1 + (i * H + j) % (H * IN)] += d1[j] * (double)xs[i];",
                                               "test_oracle_mlp.py"),
    "squared distance": ("oracle_search.cpp", "        s += t * t;\n    }\n    return std::sqrt(s);",
                         "        s += t * t;\n    }\n    return s;", "test_oracle_search.py"),
    "upper median": ("oracle_search.cpp", "med[j] = col[(n - 1) / 2];", "med[j] = col[n / 2];",
                     "test_oracle_search.py"),
    "median vertex ties to the higher id": ("oracle_search.cpp", "if (d < best_d) { best_d = d; best = (int32_t)i; }",
                                            "if (d <= best_d) { best_d = d; best = (int32_t)i; }", "test_oracle_search.py"),
    "FP8 scale for the wrong maximum": ("oracle_quant.cpp", "m > 0.f ? m / 448.0f : 1.0f", "m > 0.f ? m / 240.0f : 1.0f",
                                        "test_oracle_quant.py"),
    "bf16 truncates": ("oracle_quant.cpp", "    u += 0x7fffu + lsb;", "    u += 0u * lsb;", "test_oracle_quant.py"),
    "E4M3 subnormal boundary": ("oracle_quant.cpp", "e < -6 ? std::ldexp(1.0, -9)", "e < -7 ? std::ldexp(1.0, -9)",
                                "test_oracle_quant.py"),
    "checkMRNG against the shorter edge": ("oracle_build.cpp", "if (w12 > std::max(weight(v1, u), weight(v2, u))) return false;",
                                           "if (w12 > std::min(weight(v1, u), weight(v2, u))) return false;",
                                           "test_oracle_build.py"),
    "edge swap gain with the wrong sign": ("oracle_build.cpp", "const double g2 = gain - delta(s, v2) + weight(s, nb);",
                                           "const double g2 = gain + delta(s, v2) - weight(s, nb);", "test_oracle_build.py"),
    "insertion skips the RNG check": ("oracle_build.cpp", "if (!skip_rng && !check_mrng_tentative(v, b, U)) continue;",
                                      "if (false) continue;", "test_capi_host.py"),
    "case b tests S1 twice": ("oracle_build.cpp", "for (const Cand& c : S4) path |= (c.id == v4);",
                              "for (const Cand& c : S1) path |= (c.id == v1);", "test_capi_host.py"),
    "longest edge ties to the higher id": ("oracle_build.cpp", "(w == wn && c < n)", "(w == wn && c > n)",
                                           "test_capi_host.py"),
    "one edge-swap iteration too many": ("oracle_build.cpp", "for (int it = 0; it < i_opt; ++it)",
                                         "for (int it = 0; it <= i_opt; ++it)", "test_capi_host.py"),
}
# Not listed: case a accepting a zero gain (">= 0" for "> 0") changes nothing unless the gain, a sum
# of square-root distances, is exactly zero, which non-degenerate data never gives.


@pytest.fixture(scope="module")
def objects(tmp_path_factory):
    """The unmodified sources compiled once; a mutant recompiles only the file it changes."""
    d = tmp_path_factory.mktemp("oracle_objs")
    for f in os.listdir(os.path.dirname(oracle.__file__)):
        if f.endswith((".cpp", ".h")):
            shutil.copy(os.path.join(os.path.dirname(oracle.__file__), f), d / f)
    for s in SRCS:
        subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-c", str(d / s), "-o", str(d / (s + ".o"))], check=True)
    return d


def _link(objects, out, replaced=None):
    objs = [str(replaced if replaced and s == replaced.name[:-2] else objects / (s + ".o")) for s in SRCS]
    subprocess.run(["g++", "-shared", "-o", str(out), *objs, "-lpthread"], check=True)


def _run_pins(lib_path, pin_file):
    env = dict(os.environ, DEG_ORACLE_LIB=str(lib_path))
    return subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", pin_file), "-x", "-q",
                           "-p", "no:cacheprovider", "-m", "not gpu"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)


def test_unmodified_copy_passes_the_pins(objects, tmp_path):
    lib = tmp_path / "liboracle.so"
    _link(objects, lib)
    for pin_file in ("test_oracle_search.py", "test_oracle_mlp.py", "test_oracle_quant.py", "test_oracle_build.py",
                     "test_capi_host.py"):
        r = _run_pins(lib, pin_file)
        assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_a_planted_mistake_fails_a_pin(name, objects, tmp_path):
    src, text, planted, pin_file, *sites = MUTATIONS[name]
    code = (objects / src).read_text()
    assert code.count(text) == (sites[0] if sites else 1), f"unexpected sites of the mistake in {src}"
    (tmp_path / src).write_text(code.replace(text, planted))
    for f in os.listdir(objects):
        if f.endswith(".h"):
            shutil.copy(objects / f, tmp_path / f)
    obj = tmp_path / (src + ".o")
    subprocess.run(["g++", "-O2", "-std=c++17", "-fPIC", "-c", str(tmp_path / src), "-o", str(obj)], check=True)
    lib = tmp_path / "liboracle.so"
    _link(objects, lib, replaced=obj)
    r = _run_pins(lib, pin_file)
    assert r.returncode == 1, f"{name}: no pin failed\n{r.stdout[-2000:]}"
