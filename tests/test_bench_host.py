"""Host-side logic of bench.py, without a GPU: which kernel a record names,
when a committed DRAM-traffic figure may be used, and the roofline
arithmetic of the analysis kernel's record."""
import json
import os

import pytest

import bench


@pytest.mark.parametrize("prec,J,tuned,rows,ragged,want", [
    # untuned: one group of 32 events over 32-byte FP32 rows, two otherwise
    (1, 16, None, (32, True), False, "k_rows_packed<8,1,1,fixed>"),
    (2, 16, None, (32, True), False, "k_rows_packed<8,1,2,fixed>"),
    (1, 16, None, (64, True), False, "k_rows_packed<16,2,1,fixed>"),
    (1, 16, None, (64, False), False, "k_rows<16,2,1,fixed>"),
    (1, 8, None, (32, False), False, "k_rows<8,1,1,fixed>"),
    (0, 16, None, (32, True), False, "k_rows64<4,2,fixed>"),
    (0, 16, None, (64, True), True, "k_rows64<8,2,ragged>"),
    # tuned choices
    (1, 16, {"kernel": 2, "rows_in_flight": 2}, (32, True), False, "k_rows_packed<8,2,1,fixed>"),
    (0, 16, {"kernel": 2, "rows_in_flight": 1}, (32, True), True, "k_rows64<4,1,ragged>"),
    (0, 16, {"kernel": 3, "rows_in_flight": 2}, (64, False), False, "k_screen64<16,fixed>"),
    (0, 12, {"kernel": 1, "rows_in_flight": 2}, (128, False), False, "k_staged<double,12,fixed,ylt>"),
    (1, 20, {"kernel": 0, "rows_in_flight": 1}, (128, False), True, "k_sim_items<32,1,1,ragged>"),
    (1, 20, {"kernel": 1, "rows_in_flight": 2}, (128, False), False, "k_simulate_staged<32,1,fixed,epl2>"),
])
def test_kernel_names(prec, J, tuned, rows, ragged, want):
    assert bench.kernel_key(prec, J, tuned, rows, ragged=ragged) == want


def test_folded_kernel_name():
    assert bench.kernel_key("folded", 0) == "k_folded<fixed,smem_bits>"


def test_traffic_only_on_the_sources_it_was_taken_on(tmp_path, monkeypatch):
    """A committed DRAM figure counts only while the kernel's sources hash to
    the value recorded with it."""
    key = "k_rows_packed<8,1,1,fixed>"
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    rec = {key: {"dram_bytes_per_launch": 123, "sources_sha": bench.sources_sha(key)}}
    (prof / "traffic.json").write_text(json.dumps(rec))
    assert bench.ncu_traffic(key) == 123
    rec[key]["sources_sha"] = "0" * 16
    (prof / "traffic.json").write_text(json.dumps(rec))
    assert bench.ncu_traffic(key) is None
    assert bench.ncu_traffic("k_rows_packed<8,2,1,fixed>") is None     # no entry
    (prof / "traffic.json").write_text("not json")
    assert bench.ncu_traffic(key) is None


def test_every_kernel_family_hashes_existing_sources():
    for name, files in bench.KERNEL_SOURCES.items():
        for f in files:
            assert os.path.exists(os.path.join(bench.CSRC, f)), (name, f)
        assert bench.sources_sha(name + "<x>") is not None
    assert bench.sources_sha("k_unknown<1>") is None


def test_committed_traffic_entries_name_known_kernels():
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)
    for key, v in rec.items():
        assert key.split("<")[0] in bench.KERNEL_SOURCES, key
        assert v["dram_bytes_per_launch"] > 0
        assert os.path.exists(os.path.join(bench.ROOT, v["captured"])), v["captured"]


def test_roofline_arithmetic(monkeypatch):
    """1e9 events over 1e6 trials with 32-byte rows in 3.5 ms, against a
    gather ceiling of 3e11 rows/s and a 6700 GB/s HBM copy peak."""
    monkeypatch.setattr(bench, "hbm_peak", lambda: (6700.0, "measured"))
    monkeypatch.setattr(bench, "ncu_traffic", lambda key: 4.0e9)
    n_ev, n_tr, ms = 1_000_000_000, 1_000_000, 3.5
    shapes = [(1, 4, 3, 3.0e11), (0, 8, 8, 2.9e11)]
    r = bench.roofline(n_ev, n_tr, 16, 1, ms, None, (3.0e11, shapes), (32, True))
    algo = n_ev * (4 + 32) + 8 * n_tr
    assert r["bound"] == "l2_gather"
    assert r["algorithmic_bytes_per_launch"] == algo
    assert r["dense_formula_bytes_per_launch"] == n_ev * (4 + 64) + 8 * n_tr
    assert r["achieved"] == pytest.approx(algo / (ms * 1e-3) / 1e9, abs=0.1)
    assert r["peak"] == pytest.approx(algo / (n_ev / 3.0e11) / 1e9, abs=0.1)
    assert r["frac"] == pytest.approx((n_ev / (ms * 1e-3)) / 3.0e11, abs=1e-4)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], abs=1e-3)
    assert r["dram_frac"] == pytest.approx(4.0e9 / (ms * 1e-3) / 1e9 / 6700.0, abs=1e-4)
    assert r["kernel"] == "k_rows_packed<8,1,1,fixed>"
    assert r["l2_gather"]["ceiling_shape"]["in_flight"] == 4
    assert r["l2_gather"]["shapes_timed"] == 2
