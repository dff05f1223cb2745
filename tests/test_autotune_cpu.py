"""The 32-column apply's tile table (csrc/mapply_tune.h): the committed
header parses into four front-size buckets with ascending edges and tile
rows of 32 or 64, and the autotuner's writer changes only the tile rows
(CPU; the timing itself needs a GPU)."""
import re
import shutil

from paper_2105_07791_gb300 import autotune


def _without_table(txt: str) -> str:
    return re.sub(r"MAPPLY_TILE_ROWS\[[^\]]*\]\s*=\s*\{[^}]*\}", "", txt)


def test_committed_table_parses():
    t = autotune.current_table()
    edges = t["bucket_edges"]
    assert len(edges) == 3 and edges == sorted(edges) and len(set(edges)) == 3
    rows = list(t["tile_rows"].values())
    assert len(rows) == 4 and set(rows) <= {32, 64}
    assert list(t["tile_rows"])[0] == f"rows < {edges[0]}" and list(t["tile_rows"])[-1] == f"rows >= {edges[-1]}"


def test_writer_replaces_only_the_tile_rows(tmp_path, monkeypatch):
    dst = tmp_path / "mapply_tune.h"
    shutil.copy(autotune.HEADER, dst)
    before = dst.read_text()
    monkeypatch.setattr(autotune, "HEADER", str(dst))
    autotune.write_header((64, 32, 64, 32), [])
    assert list(autotune.current_table()["tile_rows"].values()) == [64, 32, 64, 32]
    after = dst.read_text()
    assert _without_table(before) == _without_table(after)
    autotune.write_header((32, 32, 32, 32), [])
    assert list(autotune.current_table()["tile_rows"].values()) == [32, 32, 32, 32]
