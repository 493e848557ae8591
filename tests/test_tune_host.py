"""The batched form's tuner on the host: the header it writes round-trips its
table, and the committed table is one it can write (one entry per n bucket,
each a candidate value)."""
import re

from paper_2111_11148_gb300 import tune_batched


def _table(text):
    n = re.search(r"kBatchTuneN\[kBatchTuneBuckets\] = \{([^}]*)\}", text).group(1)
    c = re.search(r"kBatchCtasPerSm\[kBatchTuneBuckets\] = \{([^}]*)\}", text).group(1)
    k = int(re.search(r"kBatchTuneBuckets = (\d+);", text).group(1))
    return k, [int(v) for v in n.split(",")], [int(v) for v in c.split(",")]


def test_header_round_trip(tmp_path):
    path = tmp_path / "batched_tuning.h"
    table = [4, 8, 16, 64, 128]
    tune_batched.write_header(table, 1234.5, "a note", str(path))
    text = path.read_text()
    k, ns, cs = _table(text)
    assert k == len(tune_batched.BUCKETS) and ns == list(tune_batched.BUCKETS) and cs == table
    assert "1234.5 ms" in text and "#pragma once" in text


def test_committed_table_is_writable():
    with open(tune_batched.HEADER) as f:
        k, ns, cs = _table(f.read())
    assert k == len(tune_batched.BUCKETS) and ns == list(tune_batched.BUCKETS)
    assert len(cs) == k and all(c in tune_batched.CANDIDATES for c in cs)
