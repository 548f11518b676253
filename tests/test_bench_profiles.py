"""Host logic of bench.py's roofline: which committed ncu counters apply.

bench.py attaches a kernel's DRAM traffic from its summary under profiles/
only while the kernel's code is the code that was captured. The summary
records code_sha256, a hash of the source with comments and whitespace runs
removed; these tests check that the hash ignores comment edits, changes with
any code edit, keeps string literals, and that the summaries bench.py reads
parse.
"""
import os
import re

import numpy as np

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_1705_03524_gb300", "csrc")


def _hash_of(tmp_path, text, name="k.cu"):
    p = tmp_path / name
    p.write_text(text)
    return bench.code_sha256(str(p))


def test_code_hash_ignores_comments_and_whitespace(tmp_path):
    base = "int f(int a) { return a + 1; }  // one\n/* two */\n"
    assert _hash_of(tmp_path, base) == _hash_of(tmp_path, "int f(int a)\n{\n  return a + 1;  /* other */ }\n")
    assert _hash_of(tmp_path, base) == _hash_of(tmp_path, "// a new header line\n" + base)


def test_code_hash_changes_with_code_and_literals(tmp_path):
    base = 'const char *s = "a // b"; int x = 1;\n'
    assert _hash_of(tmp_path, base) != _hash_of(tmp_path, 'const char *s = "a // c"; int x = 1;\n')
    assert _hash_of(tmp_path, base) != _hash_of(tmp_path, 'const char *s = "a // b"; int x = 2;\n')
    assert _hash_of(tmp_path, "char c = '/'; int y = 3;") != _hash_of(tmp_path, "char c = '/'; int y = 4;")


def test_the_summaries_bench_reads_parse():
    for name, src in (("gather_gaussian_1024", "k3_tiled_kernels.cuh"), ("ih_scan_gaussian_1024", "k2_ih_scan.cu")):
        text = open(os.path.join(ROOT, "profiles", name + ".md")).read()
        assert re.search(r"code_sha256:\s*[0-9a-f]{64}", text), name
        t = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
        assert t and float(t.group(1)) > 0, name
        assert os.path.exists(os.path.join(SRC, src))


def test_oracle_error_report_finds_a_planted_difference():
    """bench.oracle_errors compares maps with the oracle at sampled centres;
    maps made by the oracle itself (with float32 targets, as the GPU's) give
    zero, and a changed value at a sampled centre shows up in its map only."""
    from oracle import swih_oracle as O
    from paper_1705_03524_gb300 import synth

    img = synth.uniform_image(40, 52, 8, seed=4)
    B = 6
    jobs = [("manhattan", 5), ("gaussian", 9), ("euclidean", 3)]
    bins = O.quantize(img, 8, B)
    maps, targets = [], []
    for k, w in jobs:
        K = O.kernel_weights(k, w, w)
        q = O.target_hist(bins, B, K, 20, 18).astype(np.float32)
        targets.append(q)
        maps.append(O.likelihood_map(bins, B, K, q.astype(np.float64)).astype(np.float32))
    res = bench.oracle_errors(img, B, jobs, maps, np.stack(targets), n=64, seed=3)
    assert res["max_abs"] <= 1e-6, res
    # every valid centre is sampled on maps this small with enough draws: plant one error
    bad = [m.copy() for m in maps]
    bad[1][0, 0] += 0.25
    res = bench.oracle_errors(img, B, jobs, bad, np.stack(targets), n=4000, seed=3)
    assert abs(res["per_map"]["gaussian_9"] - 0.25) < 1e-3, res
    assert res["per_map"]["manhattan_5"] <= 1e-6 and res["per_map"]["euclidean_3"] <= 1e-6, res
