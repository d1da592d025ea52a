"""Host-side helpers of the benchmark (no GPU): the profile lookup is keyed
to the pipeline's kernel code, and the byte model adds up."""
import bench


def test_profile_entries_require_the_current_kernel_code(tmp_path, monkeypatch):
    h = bench.kernel_source_hash()
    good = tmp_path / "good.md"
    good.write_text(f"kernel_sources: {h}\ntraffic_bytes_per_cell: build_doublets=20.0 fit_tracks=2.0\n"
                    f"fit_fp64_flops_per_track: 200.0\n")
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", str(good))
    assert bench.measured_traffic("build_doublets", 1000) == 20000.0
    assert bench.measured_traffic("connect_cells", 1000) is None
    assert bench.measured_fit_flops(10) == 2000.0
    stale = tmp_path / "stale.md"
    stale.write_text("kernel_sources: 0000000000000000\ntraffic_bytes_per_cell: build_doublets=20.0\n")
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", str(stale))
    assert bench.measured_traffic("build_doublets", 1000) is None


def test_algorithmic_bytes_per_stage():
    ab = bench.algorithmic_bytes(H=100, D=1000, E=50, T=20, K=10, nbar=3.5)
    assert ab["binning"] == 44 * 100
    assert ab["fishbone"] == 9 * 1000
    assert ab["connect"] == 13 * 1000 + 8 * 50
    assert ab["fit"] == 36 * 10 + 12 * 3.5 * 10 + 88 * 10
