"""The benchmark's kernel accounting on CPU: which library kernels a build and
a find launch (the basis of the reported `gpu_launches` and of the names in
`kernel_functions` and `roofline.kernel`), and the algorithmic bytes per key
of the roofline (4 + 4 + 128 p for a find, 8 + 128 p + 8 / LF for a build)."""

import pytest

import bench


def _st(**kw):
    st = {"last_build_split": 0, "last_build_grouped": 0, "last_build_ranked": 0, "last_find_grouped": 0,
          "find_staged": 1, "num_hashes": 3}
    st.update(kw)
    return st


def test_build_kernels_follow_the_build_path():
    # two grouping levels, block placement, overflow insert; no fill
    two_level = bench.build_kernels(_st(last_build_split=1, last_build_grouped=1, last_build_ranked=1))
    assert two_level == ["region_cursors_kernel", "group_scatter_kernel", "region_cursors_kernel",
                         "group_scatter_kernel", "block_place_kernel", "bucketed_insert_kernel"]
    assert "fill_kernel" not in two_level
    # input order: a fill and the insert of every key
    assert bench.build_kernels(_st()) == ["fill_kernel", "bucketed_insert_kernel"]
    # grouped with exact offsets and the L2-counter placement (the fallback)
    assert bench.build_kernels(_st(last_build_grouped=1, last_build_ranked=1)) == [
        "fill_kernel", "region_cursors_kernel", "group_scatter_kernel", "rank_place_kernel", "bucketed_insert_kernel"]
    assert bench.build_kernels(_st(last_build_grouped=1)) == [
        "fill_kernel", "group_count_kernel", "group_scan_kernel", "group_scatter_kernel", "bucketed_insert_kernel"]


@pytest.mark.parametrize("h", [2, 3, 4])
def test_find_kernels_follow_the_find_path(h):
    assert bench.find_kernels(_st(num_hashes=h)) == ["bcht_find_async_kernel"]
    assert bench.find_kernels(_st(num_hashes=h, find_staged=0)) == ["bucketed_find_kernel"]
    grouped = bench.find_kernels(_st(num_hashes=h, last_find_grouped=1))
    # per round two groupings (each with its cursor reset) and the lookup;
    # then the spill pass and the return: two position groupings and the windows
    assert len(grouped) == 5 * h + 6
    assert grouped.count("grouped_lookup_kernel") == h
    assert grouped.count("group_scatter_kernel") == 2 * h + 2
    assert grouped[-1] == "window_write_kernel"


def test_algorithmic_bytes_per_key():
    assert bench.bytes_per_key("find", 1.0, 0.99) == 136.0
    assert bench.bytes_per_key("find", 2.8, 0.99) == pytest.approx(4 + 4 + 128 * 2.8)
    assert bench.bytes_per_key("insert", 1.4, 0.99) == pytest.approx(8 + 128 * 1.4 + 8 / 0.99)
    assert bench.bytes_per_key("fill", 0.0, 0.9) == pytest.approx(8 / 0.9)
    with pytest.raises(ValueError):
        bench.bytes_per_key("scan", 1.0, 0.9)
