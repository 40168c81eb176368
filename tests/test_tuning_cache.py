"""The autotuner's per-size tiling cache: export / import through the C ABI (host only, no GPU)."""
import pytest

from paper_2602_07354_gb300 import binding as B


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2602_07354_gb300 import build

    build.build()


def test_round_trip_and_validation(tmp_path):
    B.elas_tuning_import("100 100 100 8 152 19 18 17\n64 64 64 4 152 15 15 8\n")
    text = B.elas_tuning_export()
    assert "100 100 100 8 152 19 18 17" in text and "64 64 64 4 152 15 15 8" in text
    path = tmp_path / "tiles.txt"
    B.save_tuning(str(path))
    B.load_tuning(str(path))
    assert B.elas_tuning_export() == text
    # a tile wider than a block's threads allow is not a tiling of that grid: nothing is recorded
    with pytest.raises(B.ElasError):
        B.elas_tuning_import("48 48 48 4 152 15 15 8\n48 48 48 8 152 200 200 4\n")
    assert "48 48 48" not in B.elas_tuning_export()
    with pytest.raises(B.ElasError):
        B.elas_tuning_import("1 2 3\n")
