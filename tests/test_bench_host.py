"""Host-side helpers of bench.py: the committed-traffic lookup and its source
hashes, the serving trace, and the CPU description (no GPU needed)."""
import hashlib
import math

import bench


def _fake_tree(tmp_path, src_text, recorded_text):
    csrc = tmp_path / "paper_2402_18311_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "k.cu").write_text(src_text)
    prof = tmp_path / "profiles"
    prof.mkdir()
    sha = hashlib.sha1(recorded_text.encode()).hexdigest()
    (prof / "traffic_w.txt").write_text(
        "# comment\n"
        "stage_a k_one 100\n"
        "stage_a k_two<4,4,6> 23\n"
        "stage_b k_three 7\n"
        f"sha stage_a k.cu {sha}\n")
    return tmp_path


def test_stage_traffic_sums_a_stage_while_its_sources_are_unchanged(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(_fake_tree(tmp_path, "kernel v1", "kernel v1")))
    assert bench.stage_traffic("stage_a", "w") == 123
    assert bench.stage_traffic("stage_b", "w") == 7      # no hash lines: kept
    assert bench.stage_traffic("stage_c", "w") is None   # no kernels recorded
    assert bench.stage_traffic("stage_a", "other") is None


def test_stage_traffic_is_null_once_a_source_changed(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(_fake_tree(tmp_path, "kernel v2", "kernel v1")))
    assert bench.stage_traffic("stage_a", "w") is None
    assert bench.stage_traffic("stage_b", "w") == 7


def test_serving_trace_is_reproducible_and_follows_its_recipe():
    jobs, designs = bench.serving_trace(12, 10_000, 40_000, seed=3)
    jobs2, designs2 = bench.serving_trace(12, 10_000, 40_000, seed=3)
    assert jobs == jobs2
    assert [d.n_movable for d in designs] == [d.n_movable for d in designs2]
    assert jobs[0][0] == "place"
    for kind, di, parent, _seed in jobs:
        if kind == "restart":
            assert jobs[parent][0] == "place" and jobs[parent][1] == di
    for d in designs:
        c = d.n_movable
        assert 10_000 <= c <= 40_000
        g = int(min(1024, max(128, 2 ** round(math.log2(math.sqrt(c))))))
        assert d.nx == d.ny == g
        assert 0.7 <= d.target_density <= 1.0


def test_cpu_model_names_something():
    m = bench.cpu_model()
    assert isinstance(m, str) and m


def test_spectral_pipe_flops_count_products_and_the_even_odd_split():
    from types import SimpleNamespace as NS
    d = NS(n_movable=10, n_cells=12, n_pins=40, n_nets=9, nx=1024, ny=512)
    n3 = 2 * 512 * 512 * 1024 + 2 * 1024 * 1024 * 512   # one 2D transform's two GEMMs
    plain = bench.algorithmic(d, NS(dct_mode=0, dct_fold=0))["spectral"]
    assert plain["flops"] == 2.0 * n3 * 1.5 == plain["flops_pipe"]     # three transforms
    bf = bench.algorithmic(d, NS(dct_mode=1, dct_fold=0))["spectral"]
    assert bf["flops_pipe"] == 3 * bf["flops"]                           # BF16x3
    fold = bench.algorithmic(d, NS(dct_mode=1, dct_fold=1))["spectral"]
    assert fold["flops"] == bf["flops"] and fold["flops_pipe"] == 1.5 * fold["flops"]
