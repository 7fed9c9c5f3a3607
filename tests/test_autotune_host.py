"""Host logic of the autotuner: candidate selection and filtering (no GPU)."""
import pytest

from paper_2507_20239_gb300 import autotune as at
from paper_2507_20239_gb300.step import StepConfig


def test_select_keeps_the_fastest_and_the_first_of_ties():
    c = [StepConfig((16, 16)), StepConfig((8, 8)), StepConfig((16, 32)), StepConfig((16, 16), 8, 1)]
    times = {c[0]: 3.0, c[1]: 2.0, c[2]: 2.0, c[3]: 2.5}
    best, ms, table = at.select(c, lambda cfg: times[cfg])
    assert best == c[1] and ms == 2.0
    assert [t[0] for t in table] == [x.label() for x in c]


def test_select_skips_inapplicable_and_failing_candidates():
    c = [StepConfig((16, 16)), StepConfig((8, 8)), StepConfig((16, 32))]

    def measure(cfg):
        if cfg.tile == (16, 16):
            return None
        if cfg.tile == (8, 8):
            raise RuntimeError("gs_bin_sort: capacity")
        return 4.0

    best, ms, table = at.select(c, measure)
    assert best == c[2] and ms == 4.0
    notes = {lbl: note for lbl, _, note in table}
    assert notes[c[0].label()] == "not applicable" and "capacity" in notes[c[1].label()]
    with pytest.raises(RuntimeError):
        at.select(c[:2], measure)


def test_fused_bits_must_fit_the_tile_ids():
    class Cam:
        width, height = 64, 48               # 16x16 tiles: 4 x 3 = 12 tiles, 4-bit ids
    assert at._fits(StepConfig((16, 16), 4), [Cam()])
    assert not at._fits(StepConfig((16, 16), 5), [Cam()])
    assert at._fits(StepConfig((16, 16), 0), [Cam()])
    assert at._fits(StepConfig((8, 8), 6), [Cam()])          # 48 tiles: 6-bit ids


def test_default_candidates_cover_the_tile_shapes():
    c = at.default_candidates()
    assert {x.tile for x in c} == {(16, 16), (8, 8), (16, 32)}
    assert {x.stage_depth for x in c if x.backward == "pixel"} == {0, 1}
    # per (tile, fused bits): two per-pixel staging depths and the per-splat backward,
    # the latter with the per-tile and with the queued forward
    assert sum(x.backward == "splat" for x in c) == 12
    assert sum(x.queue for x in c) == 6 and all(x.backward == "splat" for x in c if x.queue)
    assert len(set(c)) == len(c) == 24
    assert len({x.label() for x in c}) == 24
    assert len(at.default_candidates(splat=False)) == 12
    assert len(at.default_candidates(queue=False)) == 18


def test_step_config_backward_is_validated():
    assert StepConfig((8, 8), 2, 0, "splat").label() == "8x8/f2/splat"
    assert StepConfig((16, 16), 0, 1).label() == "16x16/f0/s1"
    assert StepConfig((16, 16), 0, 0, "splat", True).label() == "16x16/f0/splat/queue"
    with pytest.raises(ValueError):
        StepConfig(backward="tile")
