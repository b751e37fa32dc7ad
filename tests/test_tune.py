"""The autotuner's candidate list (host logic, no GPU): shapes that give the
same launch are timed once."""
from __future__ import annotations

import itertools

from paper_2405_07079_gb300.tune import GRID_WAVES, SMEM_BYTES, THREADS, effective_launch


def test_same_launch_shapes_collapse():
    # warp mode: 4,096 arenas need 512 CTAs; asking for 608 or 1,216 is the same launch
    assert effective_launch(32, 0, 0, 4096) == effective_launch(32, 608, 0, 4096) == (32, 512, 0)
    assert effective_launch(32, 304, 0, 4096) == (32, 304, 0)
    # CTA mode: the default budget is 24 KiB, and a grid at or above the arena count is one CTA per arena
    assert effective_launch(128, 0, 0, 100) == effective_launch(128, 608, 24 * 1024, 100)
    assert effective_launch(128, 50, 0, 100) == (128, 50, 24 * 1024)


def test_candidate_count_for_the_full_batched_configuration():
    seen = {effective_launch(t, 0 if w == 0 else w * 152, s, 4096)
            for t, w, s in itertools.product(THREADS, GRID_WAVES, SMEM_BYTES)}
    assert len(seen) == 21


def test_tlsf_warp_mode_runs_four_arenas_per_cta():
    # the two-level lists run four arenas (warps) per CTA in warp mode
    assert effective_launch(32, 0, 0, 4096, "tlsf") == effective_launch(32, 1216, 0, 4096, "tlsf") == (32, 1024, 0)
    assert effective_launch(32, 608, 0, 4096, "tlsf") == (32, 608, 0)
    assert effective_launch(128, 0, 0, 100, "tlsf") == effective_launch(128, 0, 0, 100)
