"""Host logic of the snake sweep (Sec. 4.4), CPU only: the window positions,
the two-tile exchanges and the coverage of the grid, and agreement of the
library's order with the oracle's independent statement of it."""
import pytest

torch = pytest.importorskip("torch")

from paper_2507_01631_b300.sweep import exchanges, snake_order, window_members
from oracle import sweep as OSW
from synth import workloads as W


@pytest.mark.parametrize("g", [(2, 2), (3, 3), (4, 3), (8, 8), (5, 2)])
def test_snake_order(g):
    order = snake_order(*g)
    assert order == OSW.snake_positions(*g)
    assert len(order) == (g[0] - 1) * (g[1] - 1) and len(set(order)) == len(order)
    for a, b in zip(order[:-1], order[1:]):
        assert abs(a[0] - b[0]) + abs(a[1] - b[1]) == 1  # neighbouring positions
    for (leave, enter), a, b in zip(exchanges(order), order[:-1], order[1:]):
        assert len(leave) == 2 and len(enter) == 2
        assert set(window_members(a)) - set(leave) == set(window_members(b)) - set(enter)
    seen = {t for p in order for t in window_members(p)}
    assert seen == {(x, y) for x in range(g[0]) for y in range(g[1])}
    assert window_members(order[0]) == OSW.window_tiles(order[0])


def test_a_tile_that_leaves_does_not_enter_at_the_next_move():
    ex = exchanges(snake_order(8, 8))
    for (leave, _), (_, enter) in zip(ex[:-1], ex[1:]):
        assert not set(leave) & set(enter)


def test_window_at_a_grid_position_is_offset_in_the_scene():
    w = W.get("tiny_sweep")
    win = w.window((1, 1), slot=(3, 2, 1, 0))
    assert list(win.origin) == [w.tile[0], w.tile[1], 0.0]
    lo, hi = w.scene_box()
    assert list(hi[:2]) == [3 * w.tile[0], 3 * w.tile[1]] and tuple(win.slot) == (3, 2, 1, 0)
