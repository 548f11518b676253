"""Host logic of the server, without a GPU: the first-fit arena allocator and
the crop-merging rule (compiled from csrc/serve_policy.h with g++ and driven
by randomised checks), the server structs' layout against the header, and the
output-size helper of the C ABI."""
import ctypes
import json
import os
import subprocess
import tempfile

import pytest

from paper_1705_03524_gb300 import swih as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1705_03524_gb300", "csrc")

HARNESS = r'''
#include <cstdio>
#include <map>
#include <random>
#include <set>
#include <string>
#include "serve_policy.h"
using namespace swih;

int main() {
    std::mt19937_64 rng(12345);
    // ---- arena: random allocations and releases against an interval model
    const uint64_t size = 1 << 24;
    Arena a(size);
    std::vector<std::pair<uint64_t, uint64_t>> live;  // (offset, granule-rounded bytes)
    int fails = 0, overlap = 0, oob = 0, misaligned = 0, used_bad = 0, allocs = 0;
    for (int it = 0; it < 20000; ++it) {
        if (live.empty() || (rng() % 3)) {
            const uint64_t bytes = 1 + rng() % (size / 16);
            uint64_t off = 0;
            if (a.alloc(bytes, off)) {
                ++allocs;
                const uint64_t len = Arena::granules(bytes);
                if (off % Arena::kAlign) ++misaligned;
                if (off + len > size) ++oob;
                for (auto &l : live)
                    if (off < l.first + l.second && l.first < off + len) ++overlap;
                live.push_back({off, len});
            } else {
                // a failure must mean no free block was large enough
                if (a.largest_free() >= Arena::granules(bytes)) ++fails;
            }
        } else {
            const size_t k = rng() % live.size();
            a.release(live[k].first, live[k].second);
            live.erase(live.begin() + (long)k);
        }
        uint64_t u = 0;
        for (auto &l : live) u += l.second;
        if (u != a.used()) ++used_bad;
    }
    for (auto &l : live) a.release(l.first, l.second);
    const bool whole = a.free_blocks() == 1 && a.largest_free() == size && a.used() == 0;

    // ---- crop merging: invariants on random crops
    int not_covered = 0, extra_pixels = 0, too_wide = 0, bad_index = 0, cases = 0, merged_some = 0;
    for (int t = 0; t < 300; ++t) {
        const int n = 1 + (int)(rng() % 24);
        std::vector<Rect> crops;
        for (int i = 0; i < n; ++i) {
            const int w = 3 + (int)(rng() % 400), h = 3 + (int)(rng() % 400);
            crops.push_back(Rect{(int)(rng() % 600), (int)(rng() % 600), w, h});
        }
        if (t % 3 == 0) crops.push_back(crops[0]);  // a repeated crop
        std::vector<Rect> reg;
        const int max_w = (t % 5 == 0) ? 500 : 8192;
        std::vector<int> of = merge_crops(crops, reg, max_w);
        ++cases;
        if (reg.size() < crops.size()) ++merged_some;
        std::vector<int64_t> member_area(reg.size(), 0);
        for (size_t i = 0; i < crops.size(); ++i) {
            if (of[i] < 0 || of[i] >= (int)reg.size()) { ++bad_index; continue; }
            const Rect &r = reg[of[i]], &c = crops[i];
            if (c.x0 < r.x0 || c.y0 < r.y0 || c.x0 + c.w > r.x0 + r.w || c.y0 + c.h > r.y0 + r.h) ++not_covered;
            member_area[of[i]] += c.area();
        }
        for (size_t r = 0; r < reg.size(); ++r) {
            if (reg[r].area() > member_area[r]) ++extra_pixels;
            if (reg[r].w > max_w && member_area[r] != reg[r].area()) ++too_wide;
        }
    }
    // identical crops share one region; far-apart crops do not
    std::vector<Rect> reg;
    std::vector<int> same = merge_crops({Rect{10, 10, 50, 40}, Rect{10, 10, 50, 40}}, reg, 8192);
    const bool same_ok = reg.size() == 1 && same[0] == 0 && same[1] == 0;
    merge_crops({Rect{0, 0, 10, 10}, Rect{500, 500, 10, 10}}, reg, 8192);
    const bool apart_ok = reg.size() == 2;
    // a crop inside another joins it
    std::vector<int> in = merge_crops({Rect{0, 0, 100, 100}, Rect{20, 30, 10, 10}}, reg, 8192);
    const bool inside_ok = reg.size() == 1 && reg[0].w == 100 && reg[0].h == 100 && in[1] == 0;

    // ---- resident integral histograms: random operations against a model
    int cache_bad = 0, cache_ops = 0, evicted_in_use = 0, found_wrong = 0, freed_twice = 0, hits = 0;
    {
        ResidentCache c;
        struct M { int frame; Rect r; std::string key; int block; };
        std::vector<M> model;                 // live entries
        std::map<int, int> users, entries;    // per live block
        std::map<int, std::pair<uint64_t, uint64_t>> where;
        std::set<int> gone;                   // blocks freed or evicted
        uint64_t next_off = 0;
        auto forget = [&](int id) {
            if (gone.count(id)) ++freed_twice;
            gone.insert(id);
            users.erase(id);
            entries.erase(id);
            where.erase(id);
        };
        for (int it = 0; it < 20000; ++it) {
            const int op = (int)(rng() % 6);
            ++cache_ops;
            if (op == 0) {  // a build becomes resident: a block with 1-3 entries
                const uint64_t bytes = 256 * (1 + rng() % 64);
                const int id = c.add_block(next_off, bytes);
                where[id] = {next_off, bytes};
                next_off += bytes;
                users[id] = 0;
                const int n = 1 + (int)(rng() % 3);
                for (int k = 0; k < n; ++k) {
                    M m{(int)(rng() % 4), Rect{(int)(rng() % 200), (int)(rng() % 200), 20 + (int)(rng() % 200),
                                               20 + (int)(rng() % 200)}, (rng() % 2) ? "a" : "b", id};
                    c.add_entry(id, m.frame, m.r, m.key, k);
                    model.push_back(m);
                    ++entries[id];
                }
            } else if (op == 1) {  // lookup: the answer holds the crop, and one exists iff the model has one
                const int f = (int)(rng() % 4);
                const std::string key = (rng() % 2) ? "a" : "b";
                const Rect q{(int)(rng() % 300), (int)(rng() % 300), 3 + (int)(rng() % 60), 3 + (int)(rng() % 60)};
                const int e = c.find(f, key, q);
                bool any = false;
                for (auto &m : model)
                    any |= m.frame == f && m.key == key && q.x0 >= m.r.x0 && q.y0 >= m.r.y0 &&
                           q.x0 + q.w <= m.r.x0 + m.r.w && q.y0 + q.h <= m.r.y0 + m.r.h;
                if ((e >= 0) != any) ++found_wrong;
                if (e >= 0) {
                    ++hits;
                    const auto &E = c.entry(e);
                    if (E.frame != f || E.key != key || q.x0 < E.rect.x0 || q.y0 < E.rect.y0 ||
                        q.x0 + q.w > E.rect.x0 + E.rect.w || q.y0 + q.h > E.rect.y0 + E.rect.h || gone.count(E.block))
                        ++found_wrong;
                    if (rng() % 2) {  // a micro-batch reads it
                        c.acquire(E.block);
                        ++users[E.block];
                    }
                }
            } else if (op == 2 && !users.empty()) {  // a micro-batch that read a block retires
                auto it2 = users.begin();
                std::advance(it2, (long)(rng() % users.size()));
                if (it2->second > 0) {
                    const int id = it2->first;
                    --it2->second;
                    uint64_t off = 0, bytes = 0;
                    const bool fr = c.release(id, off, bytes);
                    const bool should = users[id] == 0 && entries[id] == 0;
                    if (fr != should || (fr && where[id] != std::make_pair(off, bytes))) ++cache_bad;
                    if (fr) forget(id);
                }
            } else if (op == 3) {  // evict one
                uint64_t off = 0, bytes = 0;
                int id = -1;
                const bool ok = c.evict_one(off, bytes, &id);
                bool idle = false;
                for (auto &kv : users) idle |= kv.second == 0;
                if (ok != idle) ++cache_bad;
                if (ok) {
                    if (users[id] != 0) ++evicted_in_use;
                    if (where[id] != std::make_pair(off, bytes)) ++cache_bad;
                    for (size_t i = 0; i < model.size();)
                        if (model[i].block == id) model.erase(model.begin() + (long)i); else ++i;
                    forget(id);
                }
            } else if (op == 4) {  // a frame's pixels change
                const int f = (int)(rng() % 4);
                std::vector<std::pair<uint64_t, uint64_t>> freed;
                std::vector<int> ids;
                c.invalidate_frame(f, freed, &ids);
                for (size_t i = 0; i < model.size();)
                    if (model[i].frame == f) { --entries[model[i].block]; model.erase(model.begin() + (long)i); } else ++i;
                for (size_t k = 0; k < ids.size(); ++k) {
                    if (users[ids[k]] != 0 || entries[ids[k]] != 0 || where[ids[k]] != freed[k]) ++cache_bad;
                    forget(ids[k]);
                }
                for (auto &kv : entries)
                    if (kv.second == 0 && users[kv.first] == 0 && !std::count(ids.begin(), ids.end(), kv.first)) ++cache_bad;
            }
            if (c.n_entries() != model.size()) ++cache_bad;
            uint64_t live = 0;
            for (auto &kv : where) live += kv.second.second;
            if (c.resident_bytes() != live || c.n_blocks() != where.size()) ++cache_bad;
        }
    }

    std::printf("{\"cache_ops\": %d, \"cache_bad\": %d, \"evicted_in_use\": %d, \"found_wrong\": %d, "
                "\"freed_twice\": %d, \"hits\": %d, ", cache_ops, cache_bad, evicted_in_use, found_wrong,
                freed_twice, hits);
    std::printf("\"allocs\": %d, \"fails\": %d, \"overlap\": %d, \"oob\": %d, \"misaligned\": %d, "
                "\"used_bad\": %d, \"whole\": %d, \"cases\": %d, \"merged_some\": %d, \"not_covered\": %d, "
                "\"extra_pixels\": %d, \"too_wide\": %d, \"bad_index\": %d, \"same\": %d, \"apart\": %d, "
                "\"inside\": %d}\n",
                allocs, fails, overlap, oob, misaligned, used_bad, (int)whole, cases, merged_some, not_covered,
                extra_pixels, too_wide, bad_index, (int)same_ok, (int)apart_ok, (int)inside_ok);
    return 0;
}
'''


@pytest.fixture(scope="module")
def policy_results():
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "h.cpp")
        exe = os.path.join(d, "h")
        open(src, "w").write(HARNESS)
        subprocess.run(["g++", "-std=c++17", "-O1", "-I", CSRC, src, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    return json.loads(out)


def test_arena_allocator(policy_results):
    r = policy_results
    assert r["allocs"] > 1000
    assert r["fails"] == 0, "an allocation failed although a free block was large enough"
    assert r["overlap"] == 0 and r["oob"] == 0 and r["misaligned"] == 0
    assert r["used_bad"] == 0
    assert r["whole"] == 1, "free blocks did not coalesce back into one"


def test_crop_merging_invariants(policy_results):
    r = policy_results
    assert r["cases"] == 300 and r["merged_some"] > 0
    assert r["bad_index"] == 0 and r["not_covered"] == 0
    assert r["extra_pixels"] == 0, "a merged region has more pixels than its crops apart"
    assert r["too_wide"] == 0
    assert r["same"] == 1 and r["apart"] == 1 and r["inside"] == 1


def test_resident_cache_against_a_model(policy_results):
    """Resident integral histograms: lookups answer exactly when a live entry
    of the frame and key holds the crop; a block in use is never evicted; a
    block is freed once, when it has neither users nor entries; invalidating a
    frame drops exactly its entries; the resident byte count stays exact."""
    r = policy_results
    assert r["cache_ops"] == 20000 and r["hits"] > 100
    assert r["cache_bad"] == 0 and r["found_wrong"] == 0
    assert r["evicted_in_use"] == 0 and r["freed_twice"] == 0


def test_server_struct_layout_matches_header():
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "swih.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(swih_server_desc),
         offsetof(swih_server_desc, gauss_sigma_frac), offsetof(swih_server_desc, staging_bytes),
         sizeof(swih_frame_desc), offsetof(swih_frame_desc, pitch_bytes), sizeof(swih_query),
         offsetof(swih_query, d_targets), offsetof(swih_query, user_tag), sizeof(swih_completion),
         offsetof(swih_completion, done_ns), offsetof(swih_server_desc, keep_ih),
         offsetof(swih_completion, ih_reused), sizeof(swih_server_stats));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "probe.c")
        exe = os.path.join(d, "probe")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True,
                                               check=True).stdout.split()]
    assert vals == [ctypes.sizeof(S.swih_server_desc), S.swih_server_desc.gauss_sigma_frac.offset,
                    S.swih_server_desc.staging_bytes.offset, ctypes.sizeof(S.swih_frame_desc),
                    S.swih_frame_desc.pitch_bytes.offset, ctypes.sizeof(S.swih_query),
                    S.swih_query.d_targets.offset, S.swih_query.user_tag.offset,
                    ctypes.sizeof(S.swih_completion), S.swih_completion.done_ns.offset,
                    S.swih_server_desc.keep_ih.offset, S.swih_completion.ih_reused.offset,
                    ctypes.sizeof(S.swih_server_stats)]


def test_query_out_elems_and_validation():
    q = S.make_query(0, 5, 7, 100, 60, 16, "manhattan", [(9, 9), (21, 15)], 0, 0, n_targets=3)
    per_target = (60 - 9 + 1) * (100 - 9 + 1) + (60 - 15 + 1) * (100 - 21 + 1)
    assert S.swih_query_out_elems(q) == 3 * per_target
    shapes = S.query_map_shapes(q)
    assert len(shapes) == 6 and shapes[1] == ((60 - 8) * (100 - 8), (46, 80))
    assert shapes[-1][0] + 46 * 80 == 3 * per_target
    for bad in (dict(n_targets=9), dict(n_targets=0)):
        q2 = S.make_query(0, 0, 0, 100, 60, 16, "manhattan", [(9, 9)], 0, 0, **bad)
        with pytest.raises(S.SwihError) as ei:
            S.swih_query_out_elems(q2)
        assert ei.value.status == S.SWIH_ERR_INVALID_ARG
    q3 = S.make_query(0, 0, 0, 100, 60, 16, "manhattan", [(9, 61)], 0, 0)
    with pytest.raises(S.SwihError):
        S.swih_query_out_elems(q3)  # window taller than the crop
    q4 = S.make_query(0, 0, 0, 100, 60, 300, "manhattan", [(9, 9)], 0, 0)
    with pytest.raises(S.SwihError):
        S.swih_query_out_elems(q4)  # bins above 256


def test_server_create_rejects_bad_descriptions():
    for kw in (dict(hbm_budget_bytes=1000), dict(max_inflight=0), dict(max_inflight=33),
               dict(max_batch_queries=0), dict(gauss_degree=3)):
        base = dict(hbm_budget_bytes=1 << 30)
        base.update(kw)
        with pytest.raises(S.SwihError) as ei:
            S.Server(**base)  # rejected before any CUDA call
        assert ei.value.status in (S.SWIH_ERR_INVALID_ARG, S.SWIH_ERR_UNSUPPORTED)
    for fn, args in [(S.LIB.swih_server_submit, (None, None, None)),
                     (S.LIB.swih_server_drain, (None,)),
                     (S.LIB.swih_server_add_frame, (None, None, None))]:
        assert fn(*args) == S.SWIH_ERR_INVALID_ARG
    assert S.LIB.swih_server_destroy(None) == S.SWIH_OK
