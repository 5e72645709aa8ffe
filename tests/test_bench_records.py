"""Host-side checks of the bench's measured-traffic bookkeeping (no GPU): a recorded DRAM traffic figure is reported
only while the kernel's sources are the ones it was captured on, and the digest that decides this ignores comment
edits but not code edits."""
import os
import shutil

import bench


def _copy_sources(tmp_path, kernel):
    root = tmp_path / "root"
    for rel in bench.TRAFFIC_SOURCES[kernel]:
        dst = root / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        shutil.copy(os.path.join(bench.ROOT, rel), dst)
    return root


def test_digest_ignores_comments_but_not_code(tmp_path, monkeypatch):
    kernel = "k_momentum_df"
    root = _copy_sources(tmp_path, kernel)
    monkeypatch.setattr(bench, "ROOT", str(root))
    d0 = bench.sources_digest(kernel)
    main = root / bench.TRAFFIC_SOURCES[kernel][0]
    text = main.read_text()
    main.write_text(text + "\n// a comment added after the capture\n\n")
    assert bench.sources_digest(kernel) == d0
    main.write_text(text.replace("__syncthreads();", "__syncthreads();  // trailing comment", 1))
    assert bench.sources_digest(kernel) == d0
    main.write_text(text + "\nstatic const int evap_probe_constant = 1;\n")
    assert bench.sources_digest(kernel) != d0


def test_traffic_is_reported_only_for_the_captured_sources(tmp_path, monkeypatch):
    for (kernel, workload), (traffic, digest) in bench.MEASURED_TRAFFIC.items():
        assert traffic > 0
        if bench.sources_digest(kernel) == digest:
            assert bench.measured_traffic(kernel, workload) == traffic
    kernel, workload = next(iter(bench.MEASURED_TRAFFIC))
    root = _copy_sources(tmp_path, kernel)
    monkeypatch.setattr(bench, "ROOT", str(root))
    main = root / bench.TRAFFIC_SOURCES[kernel][0]
    main.write_text(main.read_text() + "\nstatic const int evap_probe_constant = 2;\n")
    assert bench.measured_traffic(kernel, workload) is None
    assert bench.measured_traffic(kernel, "no such workload") is None
