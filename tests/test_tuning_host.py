"""The tuning table's host logic (no GPU): defaults, keys by (k, log2 mean row
length), validation, text save / load."""
import pytest

from paper_2302_05176_gb300 import gm


def setup_function():
    gm.tuning_clear()


def teardown_function():
    gm.tuning_clear()


def test_defaults_and_keys():
    d = gm.tuning_default()
    assert d == pytest.approx({"p_first": 0.05, "light_max": 4.0, "medium_max": 64.0, "heavy_max": 256.0})
    assert gm.tuning_get(1024, 3000) is None
    gm.tuning_set(1024, 3000, p_first=0.1, light_max=4, medium_max=32, heavy_max=512)
    # same bucket: floor(log2 3000) = floor(log2 2048) = 11; not 4095 -> 11 too, 4096 -> 12
    assert gm.tuning_get(1024, 2048)["light_max"] == 4.0
    assert gm.tuning_get(1024, 4095)["heavy_max"] == 512.0
    assert gm.tuning_get(1024, 4096) is None and gm.tuning_get(256, 3000) is None


@pytest.mark.parametrize("bad", [{"p_first": 0.0}, {"p_first": 1.0}, {"light_max": 0.0},
                                 {"light_max": 70.0}, {"medium_max": 300.0}, {"heavy_max": float("inf")}])
def test_invalid_tunings_are_refused(bad):
    with pytest.raises(gm.GmError):
        gm.tuning_set(64, 100, **bad)


def test_save_and_load(tmp_path):
    gm.tuning_set(256, 100, p_first=0.2, light_max=3, medium_max=24, heavy_max=128)
    gm.tuning_set(4096, 1 << 20, p_first=0.01, light_max=11, medium_max=96, heavy_max=1024)
    path = str(tmp_path / "tune.txt")
    gm.tuning_save(path)
    gm.tuning_clear()
    assert gm.tuning_get(256, 100) is None
    gm.tuning_load(path)
    assert gm.tuning_get(256, 100) == pytest.approx({"p_first": 0.2, "light_max": 3, "medium_max": 24, "heavy_max": 128})
    assert gm.tuning_get(4096, 1 << 20)["heavy_max"] == 1024.0
    bad = tmp_path / "bad.txt"
    bad.write_text("64 5 0.5 9 8 7\n")  # light > medium
    with pytest.raises(gm.GmError) as e:
        gm.tuning_load(str(bad))
    assert e.value.code == gm.GM_EDATA
