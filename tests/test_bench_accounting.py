"""Host-side accounting of bench.py (no GPU): algorithmic bytes and gathers per
run, and the code hash that ties committed ncu counters to the kernel source."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_rounds_bytes_by_hand():
    # rounds 1..3: |U| = 10, 6, 2; entries read 40, 24, 5; 2-byte color state
    sizes, vols, elem = [10, 6, 2], [40, 24, 5], 2
    # k = 2: reads 4*24 + 2*24 + 16*6 + 2*6 (no static masks yet); writes 4*5 + 16*2 + 32*2 + 2*6 + 4*4
    k2 = (96 + 48 + 96 + 12) + (20 + 32 + 64 + 12 + 16)
    # k = 3 (last): reads 4*5 + 2*5 + 16*2 + 2*2 + 32*2; writes 2*2 + 4*2 (both settle)
    k3 = (20 + 10 + 32 + 4 + 64) + (4 + 8)
    assert bench.algorithmic_bytes_rounds(sizes, vols, elem) == k2 + k3


def test_block_per_graph_bytes_by_hand():
    # N = 10 vertices; rounds 1..3: |U| = 10, 6, 2; rows read 40, 24, 5
    sizes, vols = [10, 6, 2], [40, 24, 5]
    r1 = 4 * 40 + 8 * 10 + 16 * 6
    r2 = 4 * 24 + 8 * 6 + 4 * 6 + 16 * 2
    r3 = 4 * 5 + 8 * 2 + 4 * 2
    assert bench.algorithmic_bytes_batch_blocks(10, sizes, vols) == 4 * 10 + r1 + r2 + r3


def test_shared_grid_batch_bytes_by_hand():
    N, NNZ, sizes, vols, elem = 10, 40, [10, 6, 2], [40, 24, 5], 2
    u2 = 6
    want = (8 * NNZ + (4 * (N + 1) + 4 * NNZ + 2 * elem * N + 8 * (N - u2) + 16 * u2)
            + bench.algorithmic_bytes_rounds(sizes, vols, elem) + 4 * u2 + 8 * N)
    assert bench.algorithmic_bytes_batch(N, NNZ, sizes, vols, elem) == want


def test_gathers_skip_round_one():
    assert bench.gathers_rounds([40, 24, 5]) == 29
    assert bench.gathers_rounds([7]) == 0


def test_code_hash_ignores_comments_only(tmp_path):
    a = tmp_path / "a.cuh"
    a.write_text("// header\nint f(int x) {  // note\n  return x + 1;\n}\n\n/* block\n comment */\n")
    b = tmp_path / "b.cuh"
    b.write_text("int f(int x) {\n  return x + 1;\n}\n")
    c = tmp_path / "c.cuh"
    c.write_text("int f(int x) {\n  return x + 2;\n}\n")
    assert bench.kernel_code_hash(str(a)) == bench.kernel_code_hash(str(b))
    assert bench.kernel_code_hash(str(b)) != bench.kernel_code_hash(str(c))


def test_batch_cpu_baseline_on_a_small_sample():
    import graphgen as gg
    gs = gg.batch_mix(8, 4, n_min=100, n_max=400)
    r = bench.batch_cpu_baseline(gs, stride=4)
    assert r["kind"] == "oracle" and r["cores"] == 1 and r["value"] > 0
    assert r["sample"].startswith("every 4th graph of the batch: 2 graphs")


def test_fixed_full_row_bytes_by_hand():
    # rounds 1..3: |U| = 10, 6, 2; degree volumes (whole rows) 40, 30, 9
    sizes, dv = [10, 6, 2], [40, 30, 9]
    k2 = 16 * 6 + 8 * 30 + 8 * 2
    k3 = 16 * 2 + 8 * 9
    assert bench.fixed_bytes_rounds(sizes, dv) == k2 + k3


def test_stored_degree_volumes_match_only_the_stored_run():
    import json
    entry = json.load(open(os.path.join(ROOT, "tests", "golden", "fullsize.json")))["rmat_b_s24_seed3"]
    got = bench.stored_degree_volumes(entry["n"], entry["nnz"], entry["round_sizes"])
    assert got == entry["round_degree_volumes"] and got[0] == entry["nnz"]
    assert all(a >= b for a, b in zip(got, got[1:]))            # U_k shrinks round by round
    assert bench.stored_degree_volumes(entry["n"], entry["nnz"], entry["round_sizes"][:-1]) is None
    # whole rows read at least what the active lists read: 23.8 nnz after round 1 on this graph
    assert abs(sum(got[1:]) / entry["nnz"] - 23.8) < 0.05


def test_fixed_bytes_of_a_whole_call_by_hand():
    n, nnz, sizes, dv = 10, 40, [10, 6, 2], [40, 30, 9]
    want = 4 * 11 + 4 * 40 + 4 * 10 + 8 * 6 + bench.fixed_bytes_rounds(sizes, dv) + 8 * 10
    assert bench.fixed_bytes_call(n, nnz, sizes, dv) == want


def test_golden_degree_volumes_follow_their_definition():
    """make_fullsize.degree_volumes (suffix sums of degrees by settle round) equals
    the definition vol_k = sum of deg(v) over U_k = {v : settle(v) >= k}."""
    import graphgen as gg
    import oracle
    sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
    import make_fullsize
    for g in (gg.rmat(11, 8, gg.RMAT_B, 3), gg.complete(12), gg.edgeless(3), gg.path(9)):
        r = oracle.iterative(g.rowptr, g.colidx)
        want = [int(g.degrees[r.settle_round >= k].sum()) for k in range(1, r.rounds + 1)]
        assert make_fullsize.degree_volumes(g, r) == want


def test_profile_counters_only_for_the_captured_code(tmp_path):
    """load_profile returns the stored ncu counters only while the kernel source
    (comments aside) is the one they were captured from."""
    src = tmp_path / "k.cuh"
    src.write_text("__global__ void k() { int x = 1; }\n")
    prof = tmp_path / "p.json"
    prof.write_text(json.dumps({"kernel_code_sha256": bench.kernel_code_hash(str(src)), "command": "ncu ...",
                                "per_launch": {"dram__bytes_read.sum": 5, "dram__bytes_write.sum": 7}}))
    d = bench.load_profile(str(src), str(prof))
    assert d["per_launch"]["dram__bytes_read.sum"] == 5
    src.write_text("// a comment\n__global__ void k() { int x = 1; }\n")
    assert bench.load_profile(str(src), str(prof))["command"] == "ncu ..."
    src.write_text("__global__ void k() { int x = 2; }\n")
    assert bench.load_profile(str(src), str(prof)) == {}
    assert bench.load_profile(str(src), str(tmp_path / "missing.json")) == {}
