"""Host logic of bench.py's roofline line: the algorithmic bytes of a sweep
follow the measurement plan (A's values and indices once, 16 B per row and
per unknown), a second read of A is traffic and never algorithmic, and the
committed DRAM traffic of the sweep is reported only for the strategy and
launch shape it was captured on."""
import bench

TABLE = {"ct512_sweep_strategy2": {"bytes_per_sweep": 1945000000.0,
                                   "shape": {"tile": 4096, "stages": 6, "map": 1}},
         "ct512_sweep_strategy3": {"bytes_per_sweep": 780000000.0,
                                   "shape": {"tiles": 152, "chunks": 250, "tile_ring": 172032}}}
INFO2 = {"strategy": 2, "tile": 4096, "stages": 6, "map": 1}
INFO3 = {"strategy": 3, "tiles": 152, "chunks": 250, "tile_ring": 172032}


def test_sweep_alg_bytes_is_the_plans_formula():
    m, n, nnz = 261000, 262144, 120309216
    assert bench.sweep_alg_bytes(m, n, nnz, 4) == nnz * 8 + m * 16 + n * 16
    assert bench.sweep_alg_bytes(m, n, nnz, 2) == nnz * 6 + m * 16 + n * 16


def test_second_read_of_A_is_not_algorithmic():
    m, n, nnz = 1000, 2000, 50000
    row = bench.kernel_alg_bytes(2, 0, m, n, nnz, 4)
    col = bench.kernel_alg_bytes(2, 1, m, n, nnz, 4)
    assert col < nnz       # the column pass carries no bytes of A
    assert row >= nnz * 8  # the row pass carries A once
    assert bench.kernel_alg_bytes(3, 0, m, n, nnz, 4) == bench.sweep_alg_bytes(m, n, nnz, 4)
    assert bench.kernel_alg_bytes(3, 1, m, n, nnz, 4) == 0


def test_matching_shape_reports_the_capture():
    assert bench.sweep_traffic_from(TABLE, INFO2)[0] == 1945000000.0
    assert bench.sweep_traffic_from(TABLE, INFO3)[0] == 780000000.0


def test_another_shape_or_strategy_reports_none():
    for k, v in (("tile", 2048), ("stages", 3), ("map", 2)):
        assert bench.sweep_traffic_from(TABLE, dict(INFO2, **{k: v}))[0] is None
    assert bench.sweep_traffic_from(TABLE, dict(INFO3, chunks=300))[0] is None
    assert bench.sweep_traffic_from(TABLE, dict(INFO2, strategy=1))[0] is None


def test_a_list_of_captures_is_matched_by_shape():
    table = {"ct512_sweep_strategy2": [dict(TABLE["ct512_sweep_strategy2"]),
                                       {"bytes_per_sweep": 1947000000,
                                        "shape": dict(TABLE["ct512_sweep_strategy2"]["shape"],
                                                      transposed_rows=5)}]}
    table["ct512_sweep_strategy2"][0]["shape"] = dict(TABLE["ct512_sweep_strategy2"]["shape"],
                                                      transposed_rows=0)
    assert bench.sweep_traffic_from(table, dict(INFO2, transposed_rows=0))[0] == 1945000000.0
    assert bench.sweep_traffic_from(table, dict(INFO2, transposed_rows=5))[0] == 1947000000.0
    assert bench.sweep_traffic_from(table, dict(INFO2, transposed_rows=7))[0] is None


def test_pinned_configuration_parses_into_create_options():
    """--pin strategy,tile,stages,lanes,map,col_map[,numbering] becomes the
    from_problem options that rebuild a tuned configuration without timing."""
    o = bench.pinned_opts(None, "1,4096,6,32,2,2,2")
    assert o == dict(strategy=1, stream_shape=(4096, 6, 32), stream_map=2, stream_col_map=2,
                     scatter_transpose=2)
    # without the seventh field the pixel numbering is off
    assert bench.pinned_opts(None, "2,2048,13,16,1,2")["scatter_transpose"] == -1


def test_committed_traffic_table_keys_the_patch_numbering():
    """The committed captures are told apart by the numbering flag: the patch
    form's DRAM bytes are not reported for the row-/column-major form of the
    same ring shape, and the reverse."""
    import json
    import os
    table = json.load(open(os.path.join(os.path.dirname(bench.__file__), "profiles", "traffic.json")))
    base = dict(strategy=1, tile=4096, stages=6, lanes_per_row=32, map=2, transposed_rows=116363)
    patch, _ = bench.sweep_traffic_from(table, dict(base, scatter_patch=1))
    plain, _ = bench.sweep_traffic_from(table, dict(base, scatter_patch=0))
    assert patch is not None and plain is not None and patch != plain
    # both read A once: about its 0.96 GB plus the vectors
    assert 0.95e9 < patch < 1.0e9 and 0.95e9 < plain < 1.0e9
