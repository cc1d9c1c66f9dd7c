"""Host-side pieces of bench.py (no GPU): the ncu-traffic lookup in the
committed dedispersion profile, the kernel-source hash it is keyed by, and the
launch-list table built from an ncu CSV."""
import os
import shutil

import pytest

import bench


def test_profile_traffic_covers_both_tied_shapes():
    """The committed ncu summary was taken on the current dedispersion
    sources, for the two tile shapes the autotuner finds tied on the
    single-beam band; traffic is close to the algorithmic bytes (no
    re-reads) and any other shape has none."""
    algo = 1024 * ((1 << 19) + 20464) // 4 + 1500 * (1 << 19) * 4
    for shape in ((8, 5, 64), (16, 3, 64)):
        t = bench.profiled_traffic(shape)
        assert t is not None, f"profile does not match the kernel sources for {shape}"
        assert 0.9 * algo < t < 1.05 * algo
    assert bench.profiled_traffic((16, 3, 32)) is None


def test_kernel_hash_ignores_whole_line_comments(tmp_path, monkeypatch):
    """Editing a // comment line leaves the hash (and the profile's validity)
    unchanged; editing code changes it."""
    srcs = []
    for p in bench.KERNEL_SRCS:
        q = tmp_path / os.path.basename(p)
        shutil.copy(p, q)
        srcs.append(str(q))
    monkeypatch.setattr(bench, "KERNEL_SRCS", srcs)
    h0 = bench.kernel_source_hash()
    with open(srcs[1], "a") as f:
        f.write("    // a comment added at the end\n")
    assert bench.kernel_source_hash() == h0
    with open(srcs[1], "a") as f:
        f.write("static_assert(true, \"code\");\n")
    assert bench.kernel_source_hash() != h0


def test_launch_table_per_step(tmp_path, capsys):
    """Two gulps' launches: per-step times and shares, the most frequent
    dedispersion shape kept (an autotuner trial of another shape dropped),
    PyTorch's and CUB's kernels left out."""
    rows = [
        ("void dd::tiled::dd_tiled_kernel<1, 5, 11, 64>(dd::tiled::TiledArgs)", "ms", "10.0"),
        ("void dd::tiled::dd_tiled_kernel<2, 3, 11, 64>(dd::tiled::TiledArgs)", "ms", "11.0"),
        ("void dd::<unnamed>::dd_median_kernel<0>(const unsigned int *)", "ms", "4.0"),
        ("void at::native::elementwise_kernel<128, 2>(int)", "us", "50"),
        ("void cub::DeviceScanKernel<int>(int)", "us", "20"),
        ("void dd::tiled::dd_tiled_kernel<1, 5, 11, 64>(dd::tiled::TiledArgs)", "ms", "10.0"),
        ("void dd::<unnamed>::dd_median_kernel<0>(const unsigned int *)", "ms", "4.0"),
    ]
    path = tmp_path / "launches.csv"
    with open(path, "w") as f:
        f.write('"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"\n')
        for i, (k, u, v) in enumerate(rows):
            f.write(f'"{i}","{k}","gpu__time_duration.sum","{u}","{v}"\n')
    assert bench.launch_table(str(path)) == 0
    out = capsys.readouterr().out
    assert "| dd_tiled_kernel<1, 5, 11, 64> | 1 | 10.000 |" in out
    assert "dd_tiled_kernel<2, 3, 11, 64>" not in out
    assert "| dd_median_kernel<0> | 1 | 4.000 |" in out
    assert "elementwise" not in out and "cub" not in out
    assert "| total | | 14.000 | 100 % |" in out
