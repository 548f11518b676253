"""Host logic of bench.py: which committed ncu counters apply to the
roofline, and how the step's CUDA events become stage means and step periods.

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


def test_oracle_error_reports_the_true_gaussian_distance():
    """The Gaussian maps also get their distance from the likelihood under
    exact Gaussian weights, labelled as approximation error; it is well above
    the parity tolerance for the degree-2 stand-in and absent for other kernels."""
    from oracle import swih_oracle as O
    from paper_1705_03524_gb300 import synth

    img = synth.blob_scene(64, 64, 8, 5, n_blobs=2, axes=(6, 14), margin=12).image
    B = 8
    jobs = [("gaussian", 21), ("manhattan", 9)]
    bins = O.quantize(img, 8, B)
    maps, targets = [], []
    for k, w in jobs:
        K = O.kernel_weights(k, w, w)
        q = O.target_hist(bins, B, K, 30, 30).astype(np.float32)
        targets.append(q)
        maps.append(O.likelihood_map(bins, B, K, q.astype(np.float64)).astype(np.float32))
    res = bench.oracle_errors(img, B, jobs, maps, np.stack(targets), n=256, seed=1)
    g = res["gaussian_vs_true_gaussian"]["per_map"]
    assert set(g) == {"gaussian_21"}
    assert 1e-5 < g["gaussian_21"] < 0.2, g
    # without a Gaussian map the report carries no approximation entry, and it
    # names where its maps came from
    res = bench.oracle_errors(img, B, jobs[1:], maps[1:], np.stack(targets[1:]), n=64, seed=1,
                              source="the maps of the block's last step")
    assert "gaussian_vs_true_gaussian" not in res and res["max_abs"] <= 1e-6
    assert res["sample"].endswith("the maps of the block's last step")


def test_sampled_error_reports_of_the_extra_blocks_find_planted_differences():
    """regions_error, serving_error and large_frame_error index the values the
    bench copied back by centre; fed values computed by the oracle itself they
    report zero, and a changed value shows up."""
    from oracle import swih_oracle as O
    from paper_1705_03524_gb300 import synth

    rng = np.random.default_rng(2)
    # search regions of a u16 frame, Gaussian kernel
    img16 = synth.uniform_image(90, 120, 16, seed=3)
    B = 16
    rois = [(5, 7, 40, 30), (50, 20, 60, 55)]
    targets = rng.gamma(0.5, size=(2, B))
    targets /= targets.sum(1, keepdims=True)
    samples = []
    for i, (x0, y0, w, h) in enumerate(rois):
        bins = O.quantize(img16[y0:y0 + h, x0:x0 + w], 16, B)
        for k in (5, 9):
            r = k // 2
            cx, cy = rng.integers(r, w - r, 20), rng.integers(r, h - r, 20)
            m = O.likelihood_map(bins, B, O.kernel_weights("gaussian", k, k), targets[i]).astype(np.float32)
            samples.append((i, k, cx, cy, m[cy - r, cx - r]))
    assert bench.regions_error(img16, B, rois, samples, targets)["max_abs"] <= 1e-6
    samples[3][4][2] += 0.125
    assert abs(bench.regions_error(img16, B, rois, samples, targets)["max_abs"] - 0.125) < 1e-4

    # served queries: crops of u8 / u16 frames, several targets and windows
    frames = [(synth.uniform_image(70, 80, 8, seed=5), 8), (synth.uniform_image(70, 80, 16, seed=6), 16)]
    qs = [dict(frame=1, x0=3, y0=4, w=50, h=40, B=8, kernel="euclidean", windows=[(5, 5), (9, 7)],
               targets=(np.full((2, 8), 1 / 8.0) + np.arange(8) / 80.0).astype(np.float32)),
          dict(frame=0, x0=10, y0=2, w=33, h=61, B=4, kernel="manhattan", windows=[(3, 3)],
               targets=np.array([[0.1, 0.2, 0.3, 0.4]], dtype=np.float32))]
    for q in qs:
        q["targets"] /= q["targets"].sum(1, keepdims=True)
    samples = []
    for i, q in enumerate(qs):
        img, bd = frames[q["frame"]]
        bins = O.quantize(img[q["y0"]:q["y0"] + q["h"], q["x0"]:q["x0"] + q["w"]], bd, q["B"])
        for t in range(len(q["targets"])):
            for (w, h) in q["windows"]:
                m = O.likelihood_map(bins, q["B"], O.kernel_weights(q["kernel"], w, h),
                                     q["targets"][t].astype(np.float64)).astype(np.float32)
                cx = rng.integers(0, q["w"] - w + 1, 8) + (w - 1) // 2
                cy = rng.integers(0, q["h"] - h + 1, 8) + (h - 1) // 2
                samples.append((i, t, w, h, cx, cy, m[cy - (h - 1) // 2, cx - (w - 1) // 2]))
    assert bench.serving_error(frames, qs, samples)["max_abs"] <= 1e-6
    samples[-1][6][0] -= 0.5
    assert abs(bench.serving_error(frames, qs, samples)["max_abs"] - 0.5) < 1e-4

    # a block of centres of a streamed frame (sub-image with an R-pixel halo)
    R = 4
    sub = synth.uniform_image(16 + 2 * R, 16 + 2 * R, 16, seed=7)
    job_kw = [("gaussian", 9), ("euclidean", 5)]
    tg = np.stack([targets[0], targets[1]])
    bins = O.quantize(sub, 16, B)
    blocks = []
    for j, (k, w) in enumerate(job_kw):
        full = O.likelihood_rect(bins, B, O.kernel_weights(k, w, w), tg[j], R, R, 16, 16)
        blocks.append(full.astype(np.float32))
    res = bench.large_frame_error(sub, B, job_kw, tg, blocks, 100, 200, R, n=16)
    assert res["max_abs"] <= 1e-6, res
    blocks[1][15, 0] += 0.25
    res = bench.large_frame_error(sub, B, job_kw, tg, blocks, 100, 200, R, n=16)
    assert abs(res["per_map"]["euclidean_5"] - 0.25) < 1e-4 and res["per_map"]["gaussian_9"] <= 1e-6, res


# --------------------------------------------------------------------------- step timing
class _Ev:
    """A stand-in for a CUDA event: elapsed_time is the difference of the
    recorded times in ms."""

    def __init__(self, t):
        self.t = t

    def elapsed_time(self, other):
        return other.t - self.t


def test_stage_means_and_step_periods():
    # three steps: the Gaussian build starts each step on the main stream
    # (at 0, 2.5 and 4.9 ms), every stage has a begin and an end event
    starts = [0.0, 2.5, 4.9]
    events = []
    for i, t0 in enumerate(starts):
        events.append({"build_me": (_Ev(t0), _Ev(t0 + 0.5 + 0.1 * i)),
                       "build_g": (_Ev(t0), _Ev(t0 + 0.8)),
                       "gather_gaussian": (_Ev(t0 + 0.8), _Ev(t0 + 2.3))})
    ms = bench.FrameStep.stage_ms(events)
    assert np.isclose(ms["build_me"], 0.6) and np.isclose(ms["build_g"], 0.8)
    assert np.isclose(ms["gather_gaussian"], 1.5)
    per = bench.FrameStep.step_ms(events)
    assert per["periods"] == 2
    assert np.isclose(per["p50"], 2.45) and np.isclose(per["max"], 2.5)
    # one stream and no Gaussian plan: the periods start at the first stage
    me_only = [{"build_me": (_Ev(t), _Ev(t + 0.2))} for t in (0.0, 1.0, 2.2)]
    per = bench.FrameStep.step_ms(me_only)
    assert per["periods"] == 2 and np.isclose(per["max"], 1.2)
    assert bench.FrameStep.step_ms([]) is None
    assert bench.FrameStep.step_ms(me_only[:1]) is None


def test_cpu_model_names_the_host():
    name = bench.cpu_model()
    assert isinstance(name, str) and name


def test_clock_summary_of_a_region_shorter_than_the_sampling_period():
    """Samples inside the region are summarised; a region between two samples
    gets the samples that bracket it, marked as such."""
    class _Proc:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            pass

    row = "2070, 2070, 500.0, Not Active, Not Active, Not Active, {}"
    cs = bench.ClockSampler(0)
    cs.proc = _Proc()
    cs.lines = [(1.0, row.format("Not Active")), (1.2, row.format("Active").replace("2070, 2070", "1995, 2070", 1)),
                (2.0, row.format("Not Active"))]
    inside = cs.stop(0.9, 1.5)
    assert inside["samples"] == 2 and "bracketing" not in inside
    assert inside["reasons"] == ["sw_power_cap"] and inside["sm_mhz"] == (2070 + 1995) / 2
    short = cs.stop(1.05, 1.1)
    assert short["bracketing"] and short["samples"] == 2 and short["sm_max_mhz"] == 2070
    assert cs.stop(5.0, 6.0)["samples"] == 1
