"""The tuning table read by ba_init (ba_tune_table_lookup, host only): lines
written by the binding's formatter round-trip, entries of other GPUs or
precisions are ignored, missing keys keep their defaults, malformed or
out-of-range entries are rejected, and the committed table parses."""
import os

import pytest

import paper_2511_06152_gb300 as ba

DEFAULTS = dict(chunk_tiles=0, lin_ctas_per_sm=8, back_ctas_per_sm=16, factor_nb=8, factor_threads=512,
                big_panel_w=4, batch_chains=4)


def _write(tmp_path, lines):
    p = tmp_path / "tuning.txt"
    p.write_text("\n".join(lines) + "\n")
    return str(p)


def test_formatted_line_round_trips(tmp_path):
    t = dict(chunk_tiles=12, lin_ctas_per_sm=4, back_ctas_per_sm=8, factor_nb=16, factor_threads=384, big_panel_w=2,
             batch_chains=3, ms_default=71.5, ms_tuned=68.25)
    path = _write(tmp_path, ["# header", ba.tune_table_line("NVIDIA GB300", 152, ba.BA_MIXED, t)])
    got = ba.tune_table_lookup(path, "NVIDIA GB300", 152, ba.BA_MIXED)
    assert got == t


def test_other_gpus_and_precisions_are_ignored_and_the_last_line_wins(tmp_path):
    lines = ["NVIDIA_GB300 152 fp64 chunk_tiles=4", "NVIDIA_B200 148 mixed chunk_tiles=8",
             "NVIDIA_GB300 152 mixed chunk_tiles=8  # first", "NVIDIA_GB300 144 mixed chunk_tiles=12",
             "NVIDIA_GB300 152 mixed chunk_tiles=12 factor_nb=4  # last"]
    path = _write(tmp_path, lines)
    got = ba.tune_table_lookup(path, "NVIDIA GB300", 152, ba.BA_MIXED)
    assert got == dict(DEFAULTS, chunk_tiles=12, factor_nb=4, ms_default=0.0, ms_tuned=0.0)
    assert ba.tune_table_lookup(path, "NVIDIA GB300", 152, ba.BA_FP64)["chunk_tiles"] == 4
    assert ba.tune_table_lookup(path, "NVIDIA H100", 132, ba.BA_MIXED) is None
    assert ba.tune_table_lookup(str(tmp_path / "missing.txt"), "NVIDIA GB300", 152, ba.BA_MIXED) is None


@pytest.mark.parametrize("entry", ["chunk_tiles=3", "chunk_tiles=17", "factor_threads=300", "big_panel_w=3",
                                   "lin_ctas_per_sm=0", "factor_nb=64", "batch_chains=0", "batch_chains=9",
                                   "unknown_key=1", "chunk_tiles", "factor_nb=x"])
def test_bad_entries_are_rejected(tmp_path, entry):
    path = _write(tmp_path, [f"NVIDIA_GB300 152 mixed {entry}"])
    with pytest.raises(ba.BAError) as ei:
        ba.tune_table_lookup(path, "NVIDIA GB300", 152, ba.BA_MIXED)
    assert ei.value.status == ba.BA_ERR_INVALID


def test_fp64_chunk_limit(tmp_path):
    path = _write(tmp_path, ["NVIDIA_GB300 152 fp64 chunk_tiles=12"])
    with pytest.raises(ba.BAError):
        ba.tune_table_lookup(path, "NVIDIA GB300", 152, ba.BA_FP64)


def test_committed_table_parses():
    with open(ba.TUNE_TABLE) as f:
        entries = [ln.split("#")[0].split() for ln in f]
    entries = [e for e in entries if e]
    for e in entries:
        prec = ba.BA_MIXED if e[2] == "mixed" else ba.BA_FP64
        got = ba.tune_table_lookup(ba.TUNE_TABLE, e[0].replace("_", " "), int(e[1]), prec)
        assert got is not None
        for kv in e[3:]:
            k, v = kv.split("=")
            assert got[k] == pytest.approx(float(v))
