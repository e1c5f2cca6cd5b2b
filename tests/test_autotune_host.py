"""Host logic of the autotuner: table lookup and its fallback (no GPU)."""
import json

from paper_1708_02207_gb300 import autotune


def test_choose_reads_the_table_and_falls_back(tmp_path):
    t = {"513/mixed": {"leaf": 8, "ir_max_iter": 3}, "513/fp64": {"leaf": 16, "ir_max_iter": 0}}
    assert autotune.choose(513, "mixed", t) == {"leaf": 8, "ir_max_iter": 3}
    assert autotune.choose(513, "fp64", t) == {"leaf": 16, "ir_max_iter": 0}
    assert autotune.choose(129, "mixed", t) == {"leaf": 4, "ir_max_iter": 2}
    assert autotune.choose(129, "fp64", t) == {"leaf": 4, "ir_max_iter": 0}
    p = tmp_path / "t.json"
    p.write_text(json.dumps(t))
    assert autotune.load_table(str(p)) == t
    assert autotune.load_table(str(tmp_path / "missing.json")) == {}


def test_committed_table_is_well_formed():
    table = autotune.load_table()
    for key, e in table.items():
        N, prec = key.split("/")
        assert int(N) >= 3 and prec in ("mixed", "fp64")
        assert e["leaf"] in autotune.LEAVES
        ok = [c for c in e["candidates"] if c.get("failed_samples") == 0]
        # the winner is the fastest candidate that met the tolerance
        best = min(ok, key=lambda c: c["ms_per_sample"])
        assert (best["leaf"], best["ir_max_iter"]) == (e["leaf"], e["ir_max_iter"])
