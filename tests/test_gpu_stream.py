"""Streamed frames (swih_stream_*): a frame processed band by band gives the
maps one plan over the whole frame gives, and matches the oracle, including
centres next to band boundaries; the band height follows the memory budget."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import swih_oracle as O  # noqa: E402
from paper_1705_03524_gb300 import swih as S  # noqa: E402
from paper_1705_03524_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu
TOL = 1e-5
DEV = "cuda:0"


def oracle_bins(img, bitdepth, B):
    vmax = (1 << bitdepth) - 1
    return O.quantize(np.minimum(img.astype(np.int64), vmax), bitdepth, B)


JOBS = [("manhattan", 9, 9), ("euclidean", 15, 15), ("euclidean", 43, 21), ("gaussian", 25, 25),
        ("gaussian", 41, 41), ("gaussian", 7, 45)]


def setup_frame(seed=6):
    img = synth.blob_scene(500, 700, 16, seed, n_blobs=8, margin=60).image
    d = torch.from_numpy(img.view(np.int16)).to(DEV)
    return img, d


def make_jobs(img, bd, B, jobs):
    H, W = img.shape
    bins = oracle_bins(img, bd, B)
    out = []
    for i, (k, w, h) in enumerate(jobs):
        K = O.kernel_weights(k, w, h)
        x0, y0, nx, ny = O.valid_centres(H, W, w, h)
        q = O.target_hist(bins, B, K, x0 + (7 * i) % nx, y0 + (11 * i) % ny)
        t = torch.tensor(q, dtype=torch.float32, device=DEV)
        m = torch.full((ny, nx), -1.0, device=DEV)
        out.append(dict(kernel=k, w=w, h=h, q=q, target=t, map=m, K=K))
    return bins, out


def desc_for(img, bd, B, **kw):
    H, W = img.shape
    return S.make_desc(H, W, pixel_type=S.SWIH_PIXEL_U16, bitdepth=bd, bins=B,
                       kernels=("manhattan", "euclidean", "gaussian"), max_win=(43, 45), **kw)


def run_stream(img, d, bd, B, jobs, band_height=0, budget=0):
    desc = desc_for(img, bd, B, hbm_budget_bytes=budget)
    fj = [S.make_frame_job(j["kernel"], j["w"], j["h"], j["target"], j["map"]) for j in jobs]
    with S.Stream(desc, fj, d, band_height=band_height) as st:
        st.run()
        st.sync_status()
        info = st.info()
        st.run()  # a second replay of the captured pass gives the same maps
        st.sync_status()
    return info


def test_bands_equal_one_plan_and_the_oracle():
    img, d = setup_frame()
    bd, B = 12, 16
    bins, jobs = make_jobs(img, bd, B, JOBS)
    info = run_stream(img, d, bd, B, jobs, band_height=37)
    assert info["band_height"] == 37 and info["n_bands"] > 10
    with S.Plan(desc_for(img, bd, B)) as p:
        p.build_ih(d)
        for j in jobs:
            whole = torch.empty_like(j["map"])
            p.likelihood(j["kernel"], j["w"], j["h"], j["target"], whole)
            p.sync_status()
            assert (j["map"] >= 0).all(), "a centre was not written"
            assert (whole - j["map"]).abs().max().item() <= 1e-6, j["kernel"]
    for j in jobs[:4]:
        ref = O.likelihood_map(bins, B, j["K"], j["q"])
        err = np.abs(j["map"].cpu().numpy() - ref).max()
        assert err <= TOL, (j["kernel"], j["w"], j["h"], err)


def test_budget_sets_the_band_height():
    img, d = setup_frame(seed=8)
    bd, B = 12, 16
    _bins, jobs = make_jobs(img, bd, B, JOBS)
    full = S.swih_plan_workspace_bytes(desc_for(img, bd, B))
    info = run_stream(img, d, bd, B, jobs, budget=full // 4)
    assert info["workspace_bytes"] <= full // 4 and info["n_bands"] >= 3
    maps = [j["map"].clone() for j in jobs]
    for j in jobs:
        j["map"].fill_(-1.0)
    run_stream(img, d, bd, B, jobs, band_height=13)
    for a, j in zip(maps, jobs):
        assert (a - j["map"]).abs().max().item() <= 1e-6
    with pytest.raises(S.SwihError) as ei:
        run_stream(img, d, bd, B, jobs, budget=1 << 20)
    assert ei.value.status == S.SWIH_ERR_BUDGET


@pytest.mark.parametrize("band_height", [37, 0])
def test_host_maps_copied_band_by_band(band_height):
    """With host maps set, each pass leaves every map in its page-locked host
    buffer (copied band by band during the pass) equal to the device map; a
    second pass into freshly cleared buffers does the same, and turning the
    copies off leaves the buffers untouched."""
    img, d = setup_frame(seed=11)
    bd, B = 12, 16
    _bins, jobs = make_jobs(img, bd, B, JOBS)
    full = S.swih_plan_workspace_bytes(desc_for(img, bd, B))
    desc = desc_for(img, bd, B, hbm_budget_bytes=0 if band_height else full // 4)
    fj = [S.make_frame_job(j["kernel"], j["w"], j["h"], j["target"], j["map"]) for j in jobs]
    hosts = [torch.full(j["map"].shape, -2.0).pin_memory() for j in jobs]
    with S.Stream(desc, fj, d, band_height=band_height) as st:
        assert st.info()["n_bands"] >= 3
        st.set_host_maps(hosts)
        for _ in range(2):
            for h in hosts:
                h.fill_(-2.0)
            st.run()
            st.sync_status()
            for h, j in zip(hosts, jobs):
                assert torch.equal(h, j["map"].cpu()), (j["kernel"], j["w"], j["h"])
        st.set_host_maps(None)
        for h in hosts:
            h.fill_(-2.0)
        st.run()
        st.sync_status()
        assert all((h == -2.0).all() for h in hosts)


def test_large_frame_sampled():
    """8192 x 8192 u16 frame, B = 64, Gaussian and Euclidean kernels at windows
    15/25/43/75/127, streamed in bands within a 100 GB budget; sampled centres
    (many at band boundaries) and one 512 x 512 block of centres vs the oracle."""
    cfg = synth.config4()
    img = cfg["image"]
    H, W = img.shape
    B = cfg["B"]
    d = torch.from_numpy(img.view(np.int16)).to(DEV)
    bins = oracle_bins(img, 16, B)
    tx, ty = cfg["object_centres"][0]
    jobs = []
    for k in cfg["kernels"]:
        for w in cfg["windows"]:
            K = O.kernel_weights(k, w, w)
            r = w // 2
            q = O.target_hist(bins, B, K, min(max(tx, r), W - 1 - r), min(max(ty, r), H - 1 - r))
            jobs.append(dict(kernel=k, w=w, h=w, q=q, K=K, target=torch.tensor(q, dtype=torch.float32, device=DEV),
                             map=torch.full((H - w + 1, W - w + 1), -1.0, device=DEV)))
    desc = S.make_desc(H, W, pixel_type=S.SWIH_PIXEL_U16, bitdepth=16, bins=B, kernels=cfg["kernels"],
                       max_win=(127, 127), hbm_budget_bytes=100 << 30)
    fj = [S.make_frame_job(j["kernel"], j["w"], j["h"], j["target"], j["map"]) for j in jobs]
    with S.Stream(desc, fj, d) as st:
        st.run()
        st.sync_status()
        info = st.info()
    assert info["n_bands"] > 1
    Hb, R = info["band_height"], 63
    rng = np.random.default_rng(5)
    for j in jobs:
        m = j["map"]
        r = j["w"] // 2
        assert m.min().item() >= 0.0 and m.max().item() <= 1.0 + 1e-5
        x0, y0, nx, ny = O.valid_centres(H, W, j["w"], j["h"])
        # rows on both sides of every band boundary, and random rows
        edges = [R + k * Hb + dd for k in range(1, info["n_bands"]) for dd in (-1, 0)]
        cy = np.array([c for c in edges if y0 <= c < y0 + ny] + list(rng.integers(y0, y0 + ny, 200)))
        cx = rng.integers(x0, x0 + nx, cy.size)
        ref = O.likelihood_at(bins, B, j["K"], j["q"], cx, cy)
        got = m[torch.from_numpy(cy - y0).to(DEV), torch.from_numpy(cx - x0).to(DEV)].cpu().numpy()
        err = np.abs(got - ref).max()
        assert err <= TOL, (j["kernel"], j["w"], err)
    # one 512 x 512 block of centres for the smallest window of each kernel
    for j in (jobs[0], jobs[len(cfg["windows"])]):
        r = j["w"] // 2
        bx, by = 3000, R + Hb - 256  # straddles the first band boundary
        ref = O.likelihood_rect(bins, B, j["K"], j["q"], bx, by, 512, 512)
        got = j["map"][by - r: by - r + 512, bx - r: bx - r + 512].cpu().numpy()
        err = np.abs(got - ref).max()
        assert err <= TOL, (j["kernel"], j["w"], err)


def test_timed_pass_equals_the_graph_pass_and_counts_loaded_bytes():
    """swih_stream_run_timed (stage by stage, with events) writes the maps the
    captured pass writes; its stage times are positive for the scan and for
    each kernel used; the gathers' load counters grow with each pass and reset."""
    img, d = setup_frame(seed=9)
    bd, B = 12, 16
    _bins, jobs = make_jobs(img, bd, B, JOBS)
    desc = desc_for(img, bd, B)
    fj = [S.make_frame_job(j["kernel"], j["w"], j["h"], j["target"], j["map"]) for j in jobs]
    with S.Stream(desc, fj, d, band_height=101) as st:
        st.run()
        st.sync_status()
        ref = [j["map"].clone() for j in jobs]
        for j in jobs:
            j["map"].fill_(-1.0)
        st.load_bytes(reset=True)
        ms = st.run_timed()
        st.sync_status()
        one = st.load_bytes()
        assert set(ms) == {"scan", "manhattan", "euclidean", "gaussian"}, ms
        assert all(v > 0 for v in ms.values()), ms
        for a, j in zip(ref, jobs):
            assert torch.equal(a, j["map"])
        assert one["gaussian"] > 0 and one["euclidean"] > 0 and one["manhattan"] > 0, one
        assert one["plain"] == 0 and one["wedding"] == 0
        st.run()
        two = st.load_bytes(reset=True)
        assert two == {k: 2 * v for k, v in one.items()}, (one, two)
        assert all(v == 0 for v in st.load_bytes().values())


def test_frames_wider_than_8192_columns_in_column_tiles():
    """A 12000-column frame runs as column tiles of at most 8192 columns (plus
    row bands): the maps equal those of plans over the left and right 8192
    columns bit for bit, and the oracle at centres on both sides of the tile
    boundary."""
    H, W, bd, B = 420, 12000, 12, 8
    img = synth.blob_scene(H, W, 16, 31, n_blobs=40, margin=60).image
    d = torch.from_numpy(img.view(np.int16)).to(DEV)
    jobs_spec = [("manhattan", 9, 9), ("euclidean", 43, 21), ("gaussian", 41, 41), ("gaussian", 25, 25)]
    bins, jobs = make_jobs(img, bd, B, jobs_spec)
    desc = S.make_desc(H, W, pixel_type=S.SWIH_PIXEL_U16, bitdepth=bd, bins=B,
                       kernels=("manhattan", "euclidean", "gaussian"), max_win=(43, 41))
    fj = [S.make_frame_job(j["kernel"], j["w"], j["h"], j["target"], j["map"]) for j in jobs]
    hosts = [torch.full(j["map"].shape, -2.0).pin_memory() for j in jobs]
    with S.Stream(desc, fj, d, band_height=150) as st:
        st.run()
        st.sync_status()
        info = st.info()
        # host maps: each band's rows go down after its last column tile and that
        # tile's copies into the frame maps
        st.set_host_maps(hosts)
        st.run()
        st.sync_status()
    assert info["n_bands"] == 3
    for h, j in zip(hosts, jobs):
        assert (j["map"] >= 0).all(), "a centre was not written"
        assert torch.equal(h, j["map"].cpu()), (j["kernel"], j["w"])
    # plans over the left and right 8192 columns (frame pitch): every centre of
    # the frame lies in one of them
    for x0 in (0, W - 8192):
        pd = S.make_desc(H, 8192, pitch_bytes=W * 2, pixel_type=S.SWIH_PIXEL_U16, bitdepth=bd, bins=B,
                         kernels=("manhattan", "euclidean", "gaussian"), max_win=(43, 41))
        with S.Plan(pd) as p:
            p.build_ih(d.data_ptr() + 2 * x0)
            for j in jobs:
                m = torch.empty((H - j["h"] + 1, 8192 - j["w"] + 1), device=DEV)
                p.likelihood(j["kernel"], j["w"], j["h"], j["target"], m)
                p.sync_status()
                assert torch.equal(m, j["map"][:, x0: x0 + m.shape[1]]), (x0, j["kernel"], j["w"])
    # the oracle across the tile boundary (tile 0 owns centre columns below 21 + 8150)
    rng = np.random.default_rng(3)
    for j in jobs:
        rx, ry = (j["w"] - 1) // 2, (j["h"] - 1) // 2
        cx = rng.integers(8150, 8195, 400)
        cy = rng.integers(ry, H - ry, 400)
        ref = O.likelihood_at(bins, B, j["K"], j["q"], cx, cy)
        got = j["map"].cpu().numpy()[cy - ry, cx - rx]
        assert np.abs(got - ref).max() <= TOL, j["kernel"]
