"""The bench's host-side bookkeeping: the op model's choice between the two
formulations of the greedy, and the code hash that keys the committed DRAM
traffic figures (comments and layout must not change it, code must)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_code_of_ignores_comments_and_layout():
    a = "int f(int x) { // one\n  return x + 1; /* two\n lines */ }\n"
    b = "int f(int x)\n{\n    return x + 1;\n}\n// trailing note\n"
    assert bench.code_of(a) == bench.code_of(b)
    assert bench.code_of(a) != bench.code_of(a.replace("x + 1", "x + 2"))


def test_kernel_hashes_are_stable_and_distinct():
    h1 = bench.kernel_source_hash("k_rw_uniform")
    assert h1 == bench.kernel_source_hash("k_rw_uniform")
    assert h1 != bench.kernel_source_hash("k_pack_fixed")
    assert len(h1) == 16


def test_op_model_takes_the_cheaper_formulation():
    # few rows, short runs: row words are cheaper
    ops, xu, form = bench.model_ops(2, words=20, iters=3, cols=60)
    assert form == "row words" and xu == 20
    assert ops == 20 * bench.K_WORD + 3 * 5 * bench.K_RED + 3 * bench.K_ITER
    # many rows: one word per column is cheaper, with no find-first
    ops, xu, form = bench.model_ops(10, words=150, iters=9, cols=66)
    assert form == "columns" and xu == 0
    assert ops == 66 * bench.K_COL + 9 * bench.K_ITER
    # more than 32 rows take several words per column
    assert bench.column_ops(40, iters=2, cols=10) == \
        10 * 3 * bench.K_COL + 2 * bench.K_ITER
    ops, _, form = bench.model_ops(40, words=10**9, iters=2, cols=10)
    assert form == "columns" and ops == bench.column_ops(40, 2, 10)


def test_op_model_on_oracle_counters():
    """On the headline workload the model switches formulation between
    E = 4 and E = 6, as the kernels do."""
    r, f = bench.oracle_sample(2000)
    _, stats = bench.time_oracle(r, f)
    model = bench.op_model(stats, 2000)
    assert model[4]["model"] == "row words"
    assert model[6]["model"] == "columns"
    for E in bench.SWEEP:
        assert model[E]["alu_ops_per_pair"] <= \
            model[E]["alu_ops_row_words_per_pair"] + 1e-9


def test_reference_arm_line():
    """`bench.py --impl reference` (the oracle on the host cores) prints one
    JSON line on the GPU arm's config, metric and unit, with the sample it
    timed described in cpu_baseline."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, bench.__file__, "--impl", "reference",
                        "--steps", "1", "--warmup", "1"],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == "pairs/s"
    assert line["higher_is_better"] is True
    assert line["config"] == bench.config_dict(1)
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
