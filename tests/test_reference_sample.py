"""The reference arm's bounded sample of one frame (bench.oracle_frame_sample)
on a small scene: it runs the oracle's Stage I, emission, a sampled sort and
sampled tiles, and scales them to a frame.  With the sort cap above the
frame's pair count and a budget that blends every tile, the estimate is the
whole frame's oracle time (so the scaling adds nothing); with a small cap it
stays positive and finite."""
import time

import numpy as np

from oracle import oracle as O
from paper_2510_09997_gb300 import synth as S


def test_frame_sample_bounds():
    import bench
    O.build()
    sc = S.tiny_scene(n=3000, seed=5)
    v = S.tiny_view(2.0).replace(width=96, height=64)
    rng = np.random.default_rng(1)
    t0 = time.perf_counter()
    full = bench.oracle_frame_sample(O, sc, v, rng, budget_s=1e9, sort_cap=10 ** 9)
    wall = time.perf_counter() - t0
    assert 0.0 < full <= wall * 1.05 + 1e-3
    capped = bench.oracle_frame_sample(O, sc, v, rng, budget_s=0.0, sort_cap=100)
    assert np.isfinite(capped) and capped > 0.0
