"""Host logic of the autotuner: selection and the JSON table (no GPU)."""
import json

from paper_2109_14403_gb300 import autotune


def test_choose_takes_the_fastest_and_breaks_ties_low():
    assert autotune.choose({2: 15.4, 3: 12.6, 4: 13.0}) == 3
    assert autotune.choose({2: 10.0, 3: 10.0, 4: 11.0}) == 2


def test_lookup_reads_the_table(tmp_path):
    p = tmp_path / "t.json"
    p.write_text(json.dumps({autotune.key(8, "mixed"): {"variant": 4}}))
    assert autotune.lookup(8, "mixed", str(p)) == 4
    assert autotune.lookup(7, "mixed", str(p)) == 0
    assert autotune.lookup(8, "mixed", str(tmp_path / "missing.json")) == 0
