"""The autotuner's record and the table the library compiles agree
(CPU only): every define in csrc/tuning.h equals the table of
data/autotune_gb300.json, and every table entry is the fastest of the
candidates measured for it."""
import json
import os
import re

from paper_2111_11538_gb300 import autotune

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_table():
    txt = open(autotune.HEADER_PATH).read()
    return {k: int(v) for k, v in re.findall(r"#define\s+(\w+)\s+(-?\d+)", txt)}


def test_compiled_table_matches_the_measured_one():
    rec = json.load(open(autotune.JSON_PATH))
    assert _header_table() == rec["table"]
    # the library source includes the generated header and uses every entry
    src = open(os.path.join(ROOT, "paper_2111_11538_gb300", "csrc", "pf_lib.cu")).read()
    assert '#include "tuning.h"' in src
    for k in rec["table"]:
        assert re.search(r"\b%s\b" % k, src), k


def test_every_entry_is_the_fastest_candidate():
    rec = json.load(open(autotune.JSON_PATH))
    keys = set()
    for row in rec["rows"]:
        times, cands = row["times"], row["candidates"]
        best = min(range(len(times)), key=lambda k: (times[k], cands[k]))
        assert row["best"] == cands[best], row["key"]
        assert rec["table"][row["key"]] == row["best"]
        keys.add(row["key"])
    assert keys == set(rec["table"])


def test_chunk_model_is_monotone_in_the_startup_weight():
    # a larger start-up cost per chunk never picks a shorter chunk; with
    # fewer chunks than blocks the shortest chunk is taken
    assert autotune.model_chunk(1, 8, 456, 3) == 1
    for cols, nm in ((256, 256), (8, 2048), (16, 64)):
        chunks = [autotune.model_chunk(cols, nm, 456, w) for w in autotune.STARTUP_CANDIDATES]
        assert all(1 <= c <= nm for c in chunks)
        assert chunks == sorted(chunks), (cols, nm, chunks)
