"""Host logic of the benchmark that needs no GPU: the coordinate descent that refines the lanes
per cell of each tetrahedron-count bin by whole-step timings, the HBM peak lookup, and the table
of the root search's captured DRAM traffic."""
import bench


def test_coordinate_descent_finds_a_separable_minimum():
    # a cost with its minimum at 8 lanes in bin 1 and 1 lane in bin 2; bins 0, 3, 4 hold no cells
    calls = []

    def cost(G):
        calls.append(list(G))
        assert G[0] == 0 and G[3] == 0 and G[4] == 0
        return (G[1] - 8) ** 2 + 3 * (G[2] - 1) ** 2

    assert bench.coordinate_descent([0, 2, 4, 0, 0], cost) == [0, 8, 1, 0, 0]
    assert len(calls) == 1 + 5 + 5  # the start, then five other lane counts per populated bin


def test_coordinate_descent_keeps_the_start_on_ties():
    assert bench.coordinate_descent([1, 4, 0, 16, 0], lambda G: 1.0) == [1, 4, 0, 16, 0]


def test_coordinate_descent_follows_the_coupling_in_bin_order():
    # bin 2's best depends on bin 1's value: the first pass settles bin 1, then bin 2 under it
    def cost(G):
        return abs(G[1] - 4) * 10 + abs(G[2] - G[1])

    assert bench.coordinate_descent([0, 32, 32, 0, 0], cost) == [0, 4, 4, 0, 0]


def test_hbm_peak_reads_the_measured_rate_else_falls_back(tmp_path):
    p = tmp_path / "peaks.json"
    p.write_text('{"hbm_gbs": 6785.5, "bf16_tflops": 1906.3}')
    v, src = bench.hbm_peak_gbs(str(p))
    assert v == 6785.5 and "of measured" in src
    v, src = bench.hbm_peak_gbs(str(tmp_path / "absent.json"))
    assert v == 6800.0 and "of fallback" in src
    p.write_text('{"bf16_tflops": 1906.3}')
    assert bench.hbm_peak_gbs(str(p))[0] == 6800.0


def test_root_traffic_entries_scale_with_the_interface():
    # the full pipe's entry is three 200-layer cuts; the 200-layer cut about twice the 100-layer one
    key = lambda L: ("pipe8m", L, "learned", (0, 8, 1, 0, 0))
    t = bench.ROOT_TRAFFIC
    assert t[key(600)] == 3 * t[key(200)]
    assert 2.0 <= t[key(200)] / t[key(100)] <= 2.1
    # the 5-8 bin's lane count changes the captured bytes by well under 1 %
    for G in (4, 16, 32):
        k = ("pipe8m", 600, "learned", (0, G, 1, 0, 0))
        assert abs(t[k] / t[key(600)] - 1) < 0.01
