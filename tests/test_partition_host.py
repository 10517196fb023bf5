"""The chunk bounds of the dynamic work partition (best_chunk_bounds, host
arithmetic, no GPU): every chunk count is 16 x grid, the bounds run from 0
to the iteration's cost without decreasing, a large iteration is cut into
eight stages of 2 x grid equal chunks covering 1/2, 1/4, ... of the cost
(each within one cost unit of its share), and a small one into
max(grid, cost / 98304) equal chunks followed by empty ones."""
import numpy as np
import pytest

from paper_2603_28848_gb300 import BestError, chunk_bounds

UNIT = 8192 * 12          # the minimum chunk cost: 8192 samples of a 2 -> 2 task


@pytest.mark.parametrize("grid", [1, 7, 152, 608, 1216])
@pytest.mark.parametrize("cost", [0, 1, 12345, UNIT * 100, UNIT * 16 * 608 - 1, 6_144_000_000, 3 * 10**12])
def test_bounds_cover_the_cost_in_order(cost, grid):
    b = chunk_bounds(cost, grid)
    assert len(b) == 16 * grid + 1
    assert b[0] == 0 and b[-1] == cost
    assert np.all(np.diff(b) >= 0)


@pytest.mark.parametrize("grid", [152, 608])
def test_large_iteration_is_staged(grid):
    cost = 512 * 1_000_000 * 12            # a full-size 2 -> 2 iteration: 5.12e8 samples x 12
    assert cost >= 16 * grid * UNIT
    b = chunk_bounds(cost, grid)
    per = 2 * grid
    for s in range(8):
        lo, hi = b[s * per], b[(s + 1) * per]
        start = cost - (cost >> s)
        assert lo == start
        # stage s covers half of what the earlier stages left (the last stage the rest)
        want = (cost >> s) - (cost >> (s + 1)) if s < 7 else cost >> 7
        assert hi - lo == want
        sizes = np.diff(b[s * per:(s + 1) * per + 1])
        assert sizes.max() - sizes.min() <= 1           # equal chunks within a stage
    sizes = np.diff(b)
    assert sizes[:per].min() > sizes[-per:].max()       # the chunks taken last are the small ones


@pytest.mark.parametrize("grid,cost", [(608, UNIT * 100), (608, UNIT * 5000), (152, UNIT * 3)])
def test_small_iteration_has_equal_chunks_then_empty_ones(grid, cost):
    b = chunk_bounds(cost, grid)
    k = max(grid, cost // UNIT)
    sizes = np.diff(b)
    assert np.all(sizes[k:] == 0)
    assert sizes[:k].max() - sizes[:k].min() <= 1
    assert b[k] == cost


def test_invalid_arguments_are_rejected():
    with pytest.raises(BestError):
        chunk_bounds(-1, 608)
    with pytest.raises(BestError):
        chunk_bounds(100, 0)
