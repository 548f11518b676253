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
