"""Host logic of the benchmark that needs no GPU: the coordinate descent that refines the lanes
per cell of each tetrahedron-count bin by whole-step timings."""
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
