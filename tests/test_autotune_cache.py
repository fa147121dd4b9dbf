"""The autotuner's per-GPU cache on the host: tables round-trip through JSON,
GPU names map to safe file names, $SFX_AUTOTUNE_CACHE relocates the cache, and
an absent cache reads as None (the tuner then measures)."""
from paper_1711_02473_gb300 import autotune


def test_cache_round_trip_and_location(tmp_path, monkeypatch):
    monkeypatch.setenv("SFX_AUTOTUNE_CACHE", str(tmp_path / "tune"))
    name = "NVIDIA GB300 (x/y)"
    assert autotune.load(name) is None
    table = {"mixed": {8: {"best": 2, "ms": {"1": 1.9, "2": 1.8}}}, "fp64": {3: {"best": 4, "ms": {"4": 0.5}}}}
    autotune.save(table, name)
    path = autotune.cache_path(name)
    assert path.startswith(str(tmp_path / "tune"))
    assert all(c.isalnum() or c in "_." for c in path.rsplit("/", 1)[1])
    back = autotune.load(name)
    assert back["mixed"]["8"]["best"] == 2 and back["fp64"]["3"]["ms"]["4"] == 0.5


def test_default_location_is_the_build_directory(monkeypatch):
    monkeypatch.delenv("SFX_AUTOTUNE_CACHE", raising=False)
    assert autotune.cache_dir().endswith("_build")


def test_candidates_are_valid_team_counts():
    for p in range(1, 9):
        n2 = (p + 1) ** 2
        fp = autotune.candidates("fp64", p)
        assert fp and all(1 <= c <= max(1, 256 // n2) for c in fp)
        assert all(1 <= c <= 32 for c in autotune.candidates("mixed", p))


def test_warp_specialised_candidates_and_switch():
    """The warp-specialised kind has candidates only at p >= 3 (its kernel needs
    n >= 4), -1 among them (switch it off for that degree); applying a table
    entry sets the library's switch and cells per batch (host-only calls)."""
    import paper_1711_02473_gb300 as sfx
    for p in range(1, 9):
        c = autotune.candidates("mixed_ws", p)
        assert (c == []) == (p < 3)
        if c:
            assert -1 in c and all(v == -1 or 1 <= v <= 32 for v in c)
    try:
        autotune.set_value("mixed_ws", 5, -1)
        assert not sfx.sfx_tune_get_warp_specialised(5)
        autotune.set_value("mixed_ws", 5, 3)
        assert sfx.sfx_tune_get_warp_specialised(5) and sfx.sfx_tune_get_cells_per_cta("mixed_ws", 5) == 3
        autotune.set_value("mixed_ws", 2, 3)  # no kernel at p = 2: ignored
        assert not sfx.sfx_tune_get_warp_specialised(2)
        with __import__("pytest").raises(sfx.SfxError):
            sfx.sfx_tune_set_warp_specialised(2, True)
    finally:
        sfx.sfx_tune_set_warp_specialised(5, True)
        sfx.sfx_tune_set_cells_per_cta("mixed_ws", 5, 0)


def test_structured_candidates_fit_the_team_limit():
    for kind in ("hdivcurl", "elastic", "linearised"):
        for p in range(1, 9):
            c = autotune.candidates(kind, p)
            assert c and all(1 <= v <= max(1, 256 // (p + 1) ** 2) for v in c)
    for kind in ("linearised_mixed", "hdivcurl_mixed"):
        assert all(1 <= v <= 32 for v in autotune.candidates(kind, 4))
    assert set(autotune.STRUCTURED) == {"hdivcurl", "elastic", "linearised", "linearised_mixed", "hdivcurl_mixed"}
