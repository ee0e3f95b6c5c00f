"""bench.py host logic: recorded ncu figures are reported only for the sources
they were captured on; timed frames cover the whole orbit."""
import json
import os

import bench


def _record(tmp_path, sha):
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "traffic.json").write_text(json.dumps({"march_tex_kernel": {"hi": {
        "kernel_source_sha": sha, "dram_bytes_per_launch": 9.0e9, "thread_inst_per_sample": 98.5}}}))


def test_records_follow_the_source_hash(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "abc")
    _record(tmp_path, "abc")
    assert bench.recorded_traffic("march_tex_kernel", "hi") == 9.0e9
    assert bench.recorded_inst_per_sample("march_tex_kernel", "hi") == 98.5
    assert bench.recorded_traffic("march_tex_kernel", "hi_f16") is None
    assert bench.recorded_inst_per_sample("march_kernel", "hi") is None


def test_stale_records_are_not_reported(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "changed")
    _record(tmp_path, "abc")
    assert bench.recorded_traffic("march_tex_kernel", "hi") is None
    assert bench.recorded_inst_per_sample("march_tex_kernel", "hi") is None


def test_no_record_file(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.recorded_traffic("march_tex_kernel", "hi") is None
    assert bench.recorded_inst_per_sample("march_tex_kernel", "hi") is None


def test_timed_frames_span_the_orbit():
    idx = [bench.orbit_index(k, 20, 120) for k in range(20)]
    assert idx == list(range(0, 120, 6))
    assert sorted(bench.orbit_index(k, 120, 120) for k in range(120)) == list(range(120))
    assert [bench.orbit_index(k, 240, 120) for k in (0, 119, 120, 239)] == [0, 119, 0, 119]
    assert [bench.orbit_index(2 * k + 1, 10, 120) for k in range(5)] == [12, 36, 60, 84, 108]


def test_xl_training_slabs_cover_every_brick_layer_once():
    """The ~200 GiB cube's training slabs: consecutive layer ranges covering all
    layers (the last one shorter), and the decoder slabs spread over them."""
    for nbz, layers in ((50, 4), (50, 7), (3, 4), (1, 1)):
        slabs = bench.xl_slabs(nbz, layers)
        assert slabs[0][0] == 0 and slabs[-1][1] == nbz
        assert all(b1 - b0 <= layers and b1 > b0 for b0, b1 in slabs)
        assert all(a[1] == b[0] for a, b in zip(slabs, slabs[1:]))
    slabs = bench.xl_slabs(50, 4)
    picked = bench.spread(slabs, 3)
    assert len(picked) == 3 and len(set(picked)) == 3 and all(p in slabs for p in picked)
    assert picked[0][0] < 20 and picked[-1][0] > 30          # from both ends of the cube
    assert bench.spread(slabs[:2], 3) == slabs[:2]


def test_out_of_core_march_names():
    """The bench's names for VR_OPT_OOC_MARCH values, against the header."""
    import re
    assert bench.OOC_MARCH == {"direct": 0, "tex": 1, "auto": 2, "texz": 3, "texxz": 4}
    header = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "vr.h")).read()
    doc = header[header.index("#define VR_OPT_OOC_MARCH"):header.index("#define VR_OPT_PROVIDER_THREADS")]
    for v in (0, 1, 2, 3, 4):
        assert re.search(rf"\b{v}( \(default\))?:", doc), v
