"""bench.py's command-line pieces that need no GPU: the launch-shape syntax
it reports the tuned shapes in and reads back with --lanes-per-row."""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_bench_shape_syntax_round_trips():
    # The bench reports the tuned launch shapes in the syntax its
    # --lanes-per-row option reads, so a profile can fix the same shapes.
    levels = [
        {"lanes_per_row": 0, "threads_per_block": 256, "sweep": 0, "carveout": -1},
        {"lanes_per_row": 0, "threads_per_block": 256, "sweep": 0, "carveout": 58},
        {"lanes_per_row": 4, "threads_per_block": 128, "sweep": 1, "carveout": -1},
        {"lanes_per_row": 8, "threads_per_block": 256, "sweep": 0, "carveout": -1},
        {"lanes_per_row": 0, "threads_per_block": 0, "sweep": 0, "carveout": -1},  # coarsest
    ]
    text = bench.shape_string(levels)
    assert text == "0,0c58,4hs,8"
    assert bench.parse_lanes(text) == [(0, 0, None), (0, 0, 58), (4 | 0x100, 128, None), (8, 0, None)]
    with pytest.raises(ValueError):
        bench.parse_lanes("0,x3")
