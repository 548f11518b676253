"""The server (swih_server_*): each query's maps are the same whether it runs
alone or in a mix of concurrent queries (micro-batched, crops of one frame
merged into shared integral histograms, micro-batches overlapping on several
streams), they match the oracle, and admission respects the memory budget."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import swih_oracle as O  # noqa: E402
from paper_1705_03524_gb300 import swih as S  # noqa: E402
from paper_1705_03524_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-5
DEV = "cuda:0"
KERN = ["plain", "manhattan", "euclidean", "gaussian"]


def oracle_bins(img, bitdepth, B):
    vmax = (1 << bitdepth) - 1
    return O.quantize(np.minimum(img.astype(np.int64), vmax), bitdepth, B)


class Scene:
    def __init__(self, seed=4):
        f0 = synth.blob_scene(420, 560, 8, seed, n_blobs=8, margin=50).image
        f1 = synth.blob_scene(360, 500, 16, seed + 1, n_blobs=6, margin=50).image
        self.frames = [(f0, 8), (f1, 12)]  # the 16-bit frame is read at bit depth 12 (clamped)
        self.dev = [torch.from_numpy(f0).to(DEV), torch.from_numpy(f1.view(np.int16)).to(DEV)]

    def register(self, server):
        ids = []
        for (img, bd), d in zip(self.frames, self.dev):
            pt = S.SWIH_PIXEL_U8 if img.dtype == np.uint8 else S.SWIH_PIXEL_U16
            ids.append(server.add_frame(d, img.shape[0], img.shape[1], pixel_type=pt, bitdepth=bd))
        return ids


class QSpec:
    def __init__(self, frame, x0, y0, w, h, B, kernel, windows, targets):
        self.frame, self.x0, self.y0, self.w, self.h = frame, x0, y0, w, h
        self.B, self.kernel, self.windows = B, kernel, windows
        self.q = np.asarray(targets, dtype=np.float64)  # [n_targets][B]
        self.targets = torch.tensor(self.q, dtype=torch.float32, device=DEV)

    def query(self, frame_ids, out, tag=0):
        return S.make_query(frame_ids[self.frame], self.x0, self.y0, self.w, self.h, self.B, self.kernel,
                            self.windows, self.targets, out, n_targets=len(self.q), user_tag=tag)

    def new_out(self):
        q = self.query([0, 0], 0)
        return torch.full((S.swih_query_out_elems(q),), -1.0, device=DEV)


def make_specs(scene, n, seed, overlap=True):
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(n):
        fi = int(rng.integers(0, 2))
        img, bd = scene.frames[fi]
        H, W = img.shape
        w = int(rng.integers(20, 220))
        h = int(rng.integers(20, 200))
        if overlap and i % 3 and specs:
            # near an earlier crop of this frame, so merging has something to share
            prev = [s for s in specs if s.frame == fi] or [None]
            p = prev[-1]
            x0 = int(np.clip((p.x0 if p else 0) + rng.integers(-30, 30), 0, W - w))
            y0 = int(np.clip((p.y0 if p else 0) + rng.integers(-30, 30), 0, H - h))
        else:
            x0 = int(rng.integers(0, W - w + 1))
            y0 = int(rng.integers(0, H - h + 1))
        B = int(rng.choice([8, 16, 32]))
        kernel = KERN[int(rng.integers(0, 4))]
        sizes = [s for s in (3, 9, 15, 25, 43) if s <= min(w, h)]
        ns = int(rng.integers(1, min(3, len(sizes)) + 1))
        pick = sorted(rng.choice(len(sizes), ns, replace=False))
        windows = [(sizes[k], sizes[min(k + int(rng.integers(0, 2)), len(sizes) - 1)]) for k in pick]
        nt = int(rng.integers(1, 4))
        targets = rng.gamma(0.5, 1.0, size=(nt, B))
        targets /= targets.sum(1, keepdims=True)
        specs.append(QSpec(fi, x0, y0, w, h, B, kernel, windows, targets))
    return specs


def run_mixed(scene, specs, **kw):
    outs = [sp.new_out() for sp in specs]
    with S.Server(**kw) as srv:
        ids = scene.register(srv)
        qids = [srv.submit(sp.query(ids, o, tag=i)) for i, (sp, o) in enumerate(zip(specs, outs))]
        srv.drain()
        comps = srv.poll(max_n=len(specs) + 8)
    return outs, qids, comps


def run_alone(scene, specs, **kw):
    outs = []
    with S.Server(**kw) as srv:
        ids = scene.register(srv)
        for sp in specs:
            o = sp.new_out()
            srv.submit(sp.query(ids, o))
            srv.drain()
            (c,) = srv.poll(max_n=4)
            assert c.status == S.SWIH_OK and c.batch_queries == 1
            outs.append(o)
    return outs


def check_oracle(scene, sp, out):
    img, bd = scene.frames[sp.frame]
    crop = img[sp.y0: sp.y0 + sp.h, sp.x0: sp.x0 + sp.w]
    bins = oracle_bins(crop, bd, sp.B)
    got = out.cpu().numpy().astype(np.float64)
    q = sp.query([0, 0], 0)
    shapes = S.query_map_shapes(q)
    k = 0
    for t in range(len(sp.q)):
        for (ww, wh) in sp.windows:
            off, (r, c) = shapes[k]
            K = O.kernel_weights(sp.kernel, ww, wh)
            ref = O.likelihood_map(bins, sp.B, K, sp.q[t])
            err = np.abs(got[off: off + r * c].reshape(r, c) - ref).max()
            assert err <= TOL, (sp.kernel, sp.w, sp.h, ww, wh, err)
            k += 1


def test_results_alone_equal_results_in_the_mix():
    scene = Scene()
    specs = make_specs(scene, 24, seed=7)
    kw = dict(hbm_budget_bytes=8 << 30, max_inflight=4, max_batch_queries=16, merge_regions=True)
    mixed, qids, comps = run_mixed(scene, specs, **kw)
    assert sorted(c.id for c in comps) == sorted(qids)
    assert all(c.status == S.SWIH_OK for c in comps)
    assert max(c.batch_queries for c in comps) > 1, "nothing was batched"
    alone = run_alone(scene, specs, **kw)
    exact = 0
    for sp, a, m in zip(specs, alone, mixed):
        assert (a >= 0).all() and (m >= 0).all(), "a map was not written"
        d = (a - m).abs().max().item()
        assert d <= TOL, (sp.kernel, d)
        exact += int(torch.equal(a, m))
    # integer integral histograms are exact wherever their origin lies, so the
    # maps are expected to agree bit for bit
    assert exact == len(specs)
    for sp, m in list(zip(specs, mixed))[:8]:
        check_oracle(scene, sp, m)


def test_tight_budget_waits_and_keeps_results():
    scene = Scene(seed=11)
    specs = make_specs(scene, 16, seed=3, overlap=False)
    with S.Server(hbm_budget_bytes=8 << 30) as probe:
        ids = scene.register(probe)
        need = [probe.query_bytes(sp.query(ids, 0)) for sp in specs]
    budget = int(max(need) * 1.6)
    mixed, qids, comps = run_mixed(scene, specs, hbm_budget_bytes=budget, max_inflight=4,
                                   max_batch_queries=8, merge_regions=True)
    assert all(c.status == S.SWIH_OK for c in comps) and len(comps) == len(specs)
    alone = run_alone(scene, specs, hbm_budget_bytes=budget, max_inflight=1, max_batch_queries=1)
    for a, m in zip(alone, mixed):
        assert torch.equal(a, m)
    for sp, m in list(zip(specs, mixed))[:4]:
        check_oracle(scene, sp, m)


def test_budget_refusal_and_argument_errors():
    scene = Scene(seed=2)
    # every query handed to submit carries real device buffers large enough for
    # its maps, so that even a validation mistake could not write out of bounds
    with S.Server(hbm_budget_bytes=64 << 20, max_inflight=2) as srv:
        ids = scene.register(srv)
        t = torch.full((1, 64), 1 / 64, device=DEV)
        big_out = torch.empty(500 * 400, device=DEV)
        big = S.make_query(ids[0], 0, 0, 500, 400, 64, "gaussian", [(25, 25)], t, big_out)
        assert S.swih_query_out_elems(big) <= big_out.numel()
        with pytest.raises(S.SwihError) as ei:
            srv.submit(big)
        assert ei.value.status == S.SWIH_ERR_BUDGET
        W0 = scene.frames[0][0].shape[1]
        small_out = torch.empty(30 * 20, device=DEV)
        for bad in (dict(frame=5), dict(x0=W0 - 29), dict(windows=[(31, 9)]), dict(windows=[(8, 9)])):
            args = dict(frame=ids[0], x0=0, y0=0, windows=[(9, 9)])
            args.update(bad)
            q = S.make_query(args["frame"], args["x0"], args["y0"], 30, 20, 8, "manhattan", args["windows"],
                             t, small_out)
            with pytest.raises(S.SwihError) as ei:
                srv.submit(q)
            assert ei.value.status == S.SWIH_ERR_INVALID_ARG
        # the server still serves after refusals
        sp = QSpec(0, 10, 10, 60, 50, 8, "manhattan", [(9, 9)], [np.full(8, 1 / 8)])
        out = sp.new_out()
        srv.submit(sp.query(ids, out))
        srv.drain()
        (c,) = srv.poll()
        assert c.status == S.SWIH_OK
        check_oracle(scene, sp, out)


def test_completion_records():
    scene = Scene(seed=5)
    specs = make_specs(scene, 10, seed=9)
    mixed, qids, comps = run_mixed(scene, specs, hbm_budget_bytes=4 << 30, max_inflight=2,
                                   max_batch_queries=4)
    by_id = {c.id: c for c in comps}
    assert len(by_id) == len(specs)
    for i, qid in enumerate(qids):
        c = by_id[qid]
        assert c.user_tag == i
        assert c.submit_ns <= c.start_ns <= c.done_ns
        assert 1 <= c.batch_queries <= 4


def test_wide_window_multi_target_uses_direct_gather():
    """A 2001-wide Euclidean window needs the 64-bit ring and row segments
    larger than a CTA's shared memory, so its job runs through the direct
    gather; three targets share each window histogram there too."""
    img = synth.uniform_image(2012, 2010, 8, seed=17)
    d = torch.from_numpy(img).to(DEV)
    B = 4
    rng = np.random.default_rng(2)
    q = rng.gamma(0.5, 1.0, size=(3, B))
    q /= q.sum(1, keepdims=True)
    sp = QSpec(0, 3, 1, 2005, 2010, B, "euclidean", [(2001, 2001), (9, 9)], q)
    out = sp.new_out()
    with S.Server(hbm_budget_bytes=8 << 30, max_inflight=2) as srv:
        fid = srv.add_frame(d, img.shape[0], img.shape[1])
        srv.submit(sp.query([fid], out))
        srv.drain()
        (c,) = srv.poll()
        assert c.status == S.SWIH_OK
    crop = img[1: 1 + 2010, 3: 3 + 2005]
    bins = oracle_bins(crop, 8, B)
    got = out.cpu().numpy().astype(np.float64)
    shapes = S.query_map_shapes(sp.query([0], 0))
    k = 0
    for t in range(3):
        for (ww, wh) in sp.windows:
            off, (r, cc) = shapes[k]
            k += 1
            K = O.kernel_weights("euclidean", ww, wh)
            x0, y0, nx, ny = O.valid_centres(2010, 2005, ww, wh)
            cx = np.concatenate([rng.integers(x0, x0 + nx, 12), [x0, x0 + nx - 1]])
            cy = np.concatenate([rng.integers(y0, y0 + ny, 12), [y0 + ny - 1, y0]])
            ref = O.likelihood_at(bins, B, K, q[t], cx, cy)
            m = got[off: off + r * cc].reshape(r, cc)
            err = np.abs(m[cy - y0, cx - x0] - ref).max()
            assert err <= TOL, (t, ww, err)


def test_cancel_queued_queries():
    scene = Scene(seed=12)
    specs = make_specs(scene, 30, seed=13, overlap=False)
    outs = [sp.new_out() for sp in specs]
    cancelled, refused = set(), 0
    with S.Server(hbm_budget_bytes=8 << 30, max_inflight=1, max_batch_queries=1) as srv:
        ids = scene.register(srv)
        qids = [srv.submit(sp.query(ids, o, tag=i)) for i, (sp, o) in enumerate(zip(specs, outs))]
        for i in range(10, 30, 2):
            try:
                srv.cancel(qids[i])
                cancelled.add(qids[i])
            except S.SwihError as e:  # already admitted or being admitted
                assert e.status == S.SWIH_ERR_INVALID_ARG
                refused += 1
        with pytest.raises(S.SwihError):
            srv.cancel(10 ** 9)  # unknown id
        srv.drain()
        comps = srv.poll(64)
    assert len(comps) == 30 and len(cancelled) >= 5
    for c in comps:
        i = c.user_tag
        if c.id in cancelled:
            assert c.status == S.SWIH_ERR_CANCELLED
            assert (outs[i] == -1.0).all(), "a cancelled query wrote its maps"
        else:
            assert c.status == S.SWIH_OK
    for i in (0, 1, 11, 29):
        if qids[i] not in cancelled:
            check_oracle(scene, specs[i], outs[i])


# ---------------------------------------------------------------- resident integral histograms
def one_query(srv, ids, sp):
    out = sp.new_out()
    n0 = S.swih_launch_count()
    srv.submit(sp.query(ids, out))
    srv.drain()
    (c,) = srv.poll(max_n=4)
    assert c.status == S.SWIH_OK
    return out, c, S.swih_launch_count() - n0


def test_a_crop_inside_a_resident_region_skips_quantise_and_scan():
    scene = Scene(seed=21)
    q = np.full((2, 16), 1.0 / 16)
    big = QSpec(0, 40, 30, 300, 250, 16, "euclidean", [(15, 15), (25, 21)], q)
    inner = QSpec(0, 90, 70, 120, 100, 16, "euclidean", [(9, 9), (25, 25)], q[:1])
    other_bins = QSpec(0, 90, 70, 120, 100, 32, "euclidean", [(9, 9)], np.full((1, 32), 1.0 / 32))
    with S.Server(hbm_budget_bytes=4 << 30, max_inflight=1, keep_ih=True) as srv:
        ids = scene.register(srv)
        _, c1, n1 = one_query(srv, ids, big)
        assert c1.ih_reused == 0 and n1 >= 4  # quantise, scan, row map, gather
        out, c2, n2 = one_query(srv, ids, inner)
        assert c2.ih_reused == 1 and n2 == n1 - 3, (n1, n2)  # the gather alone
        _, c3, n3 = one_query(srv, ids, other_bins)
        assert c3.ih_reused == 0 and n3 == n1, "another bin count cannot read these integral histograms"
        st = srv.stats()
        assert st["queries"] == 3 and st["ih_reused"] == 1 and st["regions_built"] == 2
        assert st["resident_bytes"] > 0
    check_oracle(scene, inner, out)
    with S.Server(hbm_budget_bytes=4 << 30, max_inflight=1) as srv:  # no residency: same maps
        ids = scene.register(srv)
        ref, c, _ = one_query(srv, ids, inner)
        assert c.ih_reused == 0
    assert torch.equal(ref, out)


def test_resident_reuse_in_the_mix_equals_alone():
    scene = Scene()
    specs = make_specs(scene, 24, seed=7)
    kw = dict(hbm_budget_bytes=8 << 30, max_inflight=4, max_batch_queries=16, merge_regions=True)
    alone = run_alone(scene, specs, **kw)
    outs = [sp.new_out() for sp in specs]
    with S.Server(keep_ih=True, **kw) as srv:
        ids = scene.register(srv)
        for rep in range(2):  # the second pass finds every crop resident
            for o in outs:
                o.fill_(-1.0)
            for i, (sp, o) in enumerate(zip(specs, outs)):
                srv.submit(sp.query(ids, o, tag=i))
            srv.drain()
            comps = srv.poll(max_n=len(specs) + 8)
            assert all(c.status == S.SWIH_OK for c in comps) and len(comps) == len(specs)
            if rep == 1:
                assert all(c.ih_reused == 1 for c in comps)
            for sp, a, m in zip(specs, alone, outs):
                assert torch.equal(a, m), (rep, sp.kernel)
        st = srv.stats()
        assert st["queries"] == 48 and st["ih_reused"] >= 24


def test_resident_regions_are_evicted_under_a_tight_budget():
    scene = Scene(seed=11)
    specs = make_specs(scene, 16, seed=3, overlap=False)
    with S.Server(hbm_budget_bytes=8 << 30) as probe:
        ids = scene.register(probe)
        need = [probe.query_bytes(sp.query(ids, 0)) for sp in specs]
    alone = run_alone(scene, specs, hbm_budget_bytes=8 << 30)
    outs = [sp.new_out() for sp in specs]
    with S.Server(hbm_budget_bytes=int(max(need) * 1.6), max_inflight=2, max_batch_queries=4,
                  keep_ih=True) as srv:
        ids = scene.register(srv)
        for i, (sp, o) in enumerate(zip(specs, outs)):
            srv.submit(sp.query(ids, o, tag=i))
        srv.drain()
        comps = srv.poll(max_n=32)
        assert all(c.status == S.SWIH_OK for c in comps) and len(comps) == len(specs)
        assert srv.stats()["evictions"] > 0
    for a, m in zip(alone, outs):
        assert torch.equal(a, m)


def test_frame_changed_drops_its_resident_regions():
    scene = Scene(seed=5)
    sp = QSpec(0, 20, 20, 200, 150, 16, "manhattan", [(15, 15)], np.full((1, 16), 1.0 / 16))
    with S.Server(hbm_budget_bytes=2 << 30, max_inflight=1, keep_ih=True) as srv:
        ids = scene.register(srv)
        one_query(srv, ids, sp)
        _, c, _ = one_query(srv, ids, sp)
        assert c.ih_reused == 1
        # new pixels in frame 0, announced to the server
        new = synth.blob_scene(420, 560, 8, 99, n_blobs=8, margin=50).image
        scene.dev[0].copy_(torch.from_numpy(new))
        scene.frames[0] = (new, 8)
        srv.frame_changed(ids[0])
        out, c, _ = one_query(srv, ids, sp)
        assert c.ih_reused == 0
    check_oracle(scene, sp, out)
