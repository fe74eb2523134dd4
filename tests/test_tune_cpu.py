"""The tuning table (host side, no GPU): record, look up, persist as JSON and reload."""
import json
import os

import pytest

from paper_1708_03912_gb300 import fraclap as F


@pytest.fixture
def lib():
    if not os.path.exists(F.LIB_PATH):
        pytest.skip("libfraclap.so not built")
    F.fl_tune_clear()
    yield F.lib()
    F.fl_tune_clear()


def test_record_lookup_replace(lib):
    assert F.fl_tune_lookup("batch_gemm", 8195, 64, 2) is None
    F.fl_tune_record("batch_gemm", 8195, 64, 2, 4, 152, 0.048)
    F.fl_tune_record("batch_gemm", 1887, 16, 1, 6, 120, 0.01)
    assert F.fl_tune_lookup("batch_gemm", 8195, 64, 2) == (4, 152)
    assert F.fl_tune_lookup("batch_gemm", 8195, 64, 1) is None
    F.fl_tune_record("batch_gemm", 8195, 64, 2, 3, 144, 0.047)  # replaces
    assert F.fl_tune_lookup("batch_gemm", 8195, 64, 2) == (3, 144)
    assert F.fl_tune_count() == 2


def test_save_load_round_trip(lib, tmp_path):
    F.fl_tune_record("batch_gemm", 8195, 64, 2, 4, 152, 0.048)
    F.fl_tune_record("resid_df", 33, 16, 1, 2, 304, 1.5)
    path = tmp_path / "tune.json"
    F.fl_tune_save(path)
    doc = json.loads(path.read_text())
    assert len(doc["entries"]) == 2 and doc["entries"][0]["p1"] == 152
    F.fl_tune_clear()
    assert F.fl_tune_count() == 0
    F.fl_tune_load(path)
    assert F.fl_tune_lookup("batch_gemm", 8195, 64, 2) == (4, 152)
    assert F.fl_tune_lookup("resid_df", 33, 16, 1) == (2, 304)


def test_other_device_entries_do_not_apply(lib, tmp_path):
    path = tmp_path / "tune.json"
    path.write_text(json.dumps({"entries": [{"device": "some other GPU", "kernel": "batch_gemm", "n": 10,
                                             "nrhs": 16, "nslices": 2, "p0": 3, "p1": 7, "ms": 1.0}]}))
    F.fl_tune_load(path)
    assert F.fl_tune_count() == 1
    assert F.fl_tune_lookup("batch_gemm", 10, 16, 2) is None


def test_bad_file_rejected(lib, tmp_path):
    path = tmp_path / "bad.json"
    path.write_text('{"entries": [{"kernel": }]}')
    with pytest.raises(F.FlError):
        F.fl_tune_load(path)
    with pytest.raises(F.FlError):
        F.fl_tune_load(tmp_path / "missing.json")
