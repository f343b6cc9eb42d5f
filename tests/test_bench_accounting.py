"""The benchmark's roofline accounting (CPU): the algorithmic bytes of one PCG iteration written out word by word for
the layout, and the choice of the ncu traffic record for a launch shape."""
import importlib.util
import json
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_pcg_bytes_per_iteration_counts_every_stream_once():
    b = _bench()
    n, nb, w = 219314, 1092558, 4
    blocks = nb * 33 * w                      # factored off-diagonal bond blocks, read once
    diag = n * 21 * w + n * 21 * w            # diagonal blocks (product) and their inverses (update)
    product = n * (2 * 6 + 6) * w             # read z, r; write w
    update = n * (6 * 6 + 5 * 6) * w          # read z, w, p, s, x, r; write p, s, x, r, z
    assert b.pcg_bytes_per_iter(n, nb, 0, w) == blocks + diag + product + update == 254751912
    # an active contact entry: its neighbour index and the rank-one block (direction and weight)
    assert b.pcg_bytes_per_iter(n, nb, 10, w) - b.pcg_bytes_per_iter(n, nb, 0, w) == 10 * (4 + 4 * w)
    # FP64 words double every stream but the contact index
    assert b.pcg_bytes_per_iter(n, nb, 0, 8) == 2 * 254751912


def test_traffic_record_is_taken_for_the_launch_shapes_product():
    b = _bench()
    rec = {"records": [
        {"product": 2, "lanes_per_row": 2, "dram_bytes_per_pcg_iter": 1.0, "dram_bytes_once": 0},
        {"product": 3, "lanes_per_row": 1, "dram_bytes_per_pcg_iter": 2.0, "dram_bytes_once": 0},
        {"product": 3, "lanes_per_row": 2, "dram_bytes_per_pcg_iter": 3.0, "dram_bytes_once": 0},
    ]}
    pick = b.traffic_for_shape
    assert pick(rec, {"product": 2, "lanes_per_row": 2})["dram_bytes_per_pcg_iter"] == 1.0
    assert pick(rec, {"product": 3, "lanes_per_row": 2})["dram_bytes_per_pcg_iter"] == 3.0
    assert pick(rec, {"product": 2, "lanes_per_row": 8})["dram_bytes_per_pcg_iter"] == 1.0  # other lanes: same data
    assert pick(rec, {"product": 0, "lanes_per_row": 2}) is None  # a product never captured
    assert pick(None, {"product": 2, "lanes_per_row": 2}) is None
    assert pick(rec, None) is None


def test_committed_traffic_record_describes_the_products_it_names():
    with open(os.path.join(ROOT, "profiles", "k_pcg_traffic.json")) as f:
        rec = json.load(f)
    assert len(rec["pcg_source_sha256"]) == 64
    algorithmic = _bench().pcg_bytes_per_iter(219314, 1092558, 0, 4)
    for r in rec["records"]:
        assert r["product"] in (0, 1, 2, 3) and r["lanes_per_row"] in (1, 2, 4, 8)
        # DRAM traffic of a capture can exceed the algorithmic bytes (padding words, second reads that miss L2) but
        # not fall below them: a record under them would describe a kernel that skipped work
        assert algorithmic <= r["dram_bytes_per_pcg_iter"] <= 2 * algorithmic
