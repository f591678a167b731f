"""Tile tables (include/flowroi.h, "tile shapes"): the JSON form the
library reads at create and that flowroi_autotune writes.  Validation is
host-side (no device used); a committed table, if any, must validate."""
import glob
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def F():
    from paper_2511_14419_gb300 import build, flowroi
    build()
    return flowroi


def _table(*entries, **top):
    t = {"format": "flowroi-tiles-1", "entries": list(entries)}
    t.update(top)
    return json.dumps(t)


GOOD = [
    {"param": "dwt_seg", "w": 2048, "storage": 32, "level": 1, "value": 48},
    {"param": "dwt_seg", "w": 512, "storage": 16, "level": 5, "value": 8},
    {"param": "update_rows", "storage": 32, "value": 8},
    {"param": "saliency_rows", "w": 8192, "storage": 32, "value": 64},
    {"param": "blocks_per_sm", "kernel": "window", "storage": 32, "value": 2},
    {"param": "blocks_per_sm", "kernel": "mask", "storage": 16, "value": 3},
    {"param": "dwt_variant", "storage": 32, "value": 6, "ms": 1.25},
]


def test_valid_tables_are_accepted(F):
    assert F.flowroi_tiles_check(_table()) == ""
    assert F.flowroi_tiles_check(_table(*GOOD, device="NVIDIA GB300", note="test")) == ""
    for e in GOOD:
        assert F.flowroi_tiles_check(_table(e)) == "", e


@pytest.mark.parametrize("text,why", [
    ("", "malformed"),
    ("{", "malformed"),
    ("[]", "object"),
    (_table()[:-1] + ", \"x\": 1}", "unknown key"),
    (json.dumps({"format": "other", "entries": []}), "format"),
    (json.dumps({"format": "flowroi-tiles-1"}), "entries"),
    (_table({"param": "bogus", "storage": 32, "value": 1}), "unknown param"),
    (_table({"param": "dwt_seg", "w": 2048, "storage": 32, "level": 1, "value": 3}), "dwt_seg"),
    (_table({"param": "dwt_seg", "w": 2048, "storage": 32, "level": 9, "value": 32}), "level"),
    (_table({"param": "dwt_seg", "w": 2000, "storage": 32, "level": 1, "value": 32}), "w must"),
    (_table({"param": "dwt_seg", "w": 2048, "storage": 8, "level": 1, "value": 32}), "storage"),
    (_table({"param": "update_rows", "storage": 32, "value": 6}), "4, 8, 16 or 32"),
    (_table({"param": "saliency_rows", "w": 2048, "storage": 32, "value": 12}), "multiple of 8"),
    (_table({"param": "saliency_rows", "w": 2048, "storage": 32, "value": 8.5}), "integer"),
    (_table({"param": "blocks_per_sm", "kernel": "nope", "storage": 32, "value": 2}), "kernel"),
    (_table({"param": "blocks_per_sm", "kernel": "dwt", "storage": 32, "value": 0}), "blocks_per_sm"),
    (_table({"param": "dwt_variant", "storage": 32, "value": 4}), "dwt_variant"),
    (_table({"param": "dwt_variant", "storage": 32, "value": 5, "extra": 1}), "unknown key"),
])
def test_malformed_tables_are_rejected_with_a_reason(F, text, why):
    err = F.flowroi_tiles_check(text)
    assert err and why in err, (text, err)


def test_committed_tables_validate(F):
    for path in glob.glob(os.path.join(ROOT, "paper_2511_14419_gb300", "tiles", "*.json")):
        with open(path) as f:
            assert F.flowroi_tiles_check(f.read()) == "", path


def test_create_rejects_an_unreadable_or_malformed_table_file(F, tmp_path):
    cfg = F.flowroi_default_config(tile_table=str(tmp_path / "missing.json"))
    with pytest.raises(F.FlowRoIError) as ei:
        F.flowroi_create(cfg)
    assert ei.value.code == F.EINVAL
    bad = tmp_path / "bad.json"
    bad.write_text(_table({"param": "dwt_variant", "storage": 32, "value": 9}))
    cfg = F.flowroi_default_config(tile_table=str(bad))
    with pytest.raises(F.FlowRoIError) as ei:
        F.flowroi_create(cfg)
    assert ei.value.code == F.EINVAL
