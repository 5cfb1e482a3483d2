"""Host logic of bench.py's roofline line: the committed DRAM traffic of the
dominant kernel is reported only for the launch shape it was captured on."""
import bench

TABLE = {"ct512_2_0": 974000000, "ct512_2_0_shape": {"tile": 4096, "stages": 6, "lanes": 16, "map": 1},
         "ct512_2_1": 971000000, "ct512_2_1_shape": {"tile": 1024, "stages": 13, "lanes": 32, "map": 2}}
INFO = {"strategy": 2, "tile": 4096, "stages": 6, "lanes_per_row": 16, "map": 1,
        "col_tile": 1024, "col_stages": 13, "col_lanes": 32, "col_map": 2}


def test_matching_shape_reports_the_capture():
    assert bench.measured_traffic(TABLE, INFO, 0) == 974000000
    assert bench.measured_traffic(TABLE, INFO, 1) == 971000000


def test_another_shape_or_strategy_reports_none():
    for k, v in (("lanes_per_row", 32), ("map", 2), ("tile", 2048), ("stages", 3)):
        assert bench.measured_traffic(TABLE, dict(INFO, **{k: v}), 0) is None
    assert bench.measured_traffic(TABLE, dict(INFO, col_map=1), 1) is None
    assert bench.measured_traffic(TABLE, dict(INFO, strategy=1), 0) is None
    assert bench.measured_traffic({"ct512_2_0": 1}, INFO, 0) is None
