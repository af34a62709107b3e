"""Host-side check of the per-warp contribution-mask layout the forward writes and the
backward reads: tile t's chunk c of forward warp w lives at word (off[t] >> 2) + 16 t +
8 c + w, for the ceil(n_t / 32) chunks of its n_t entries, inside a region of
(key_capacity >> 2) + 16 (n_tiles + 1) + 8 words. For random tile lengths (empty tiles,
lengths that are and are not multiples of 4 and 32, a list filling the key capacity)
every word is inside the region and no two (tile, chunk, warp) share one."""
import numpy as np
import pytest


@pytest.mark.parametrize("seed", range(6))
def test_mask_words_are_disjoint_and_in_bounds(seed):
    rng = np.random.default_rng(seed)
    n_tiles = int(rng.integers(1, 300))
    lens = rng.integers(0, 200, n_tiles)
    lens[rng.random(n_tiles) < 0.2] = 0
    if seed % 2:
        lens[rng.integers(0, n_tiles)] = 4097
    off = np.concatenate([[0], np.cumsum(lens)])
    key_cap = int(off[-1]) + int(rng.integers(0, 64))
    region = (key_cap >> 2) + 16 * (n_tiles + 1) + 8
    used = np.zeros(region, np.int32)
    for t in range(n_tiles):
        chunks = (int(lens[t]) + 31) // 32
        base = (int(off[t]) >> 2) + 16 * t
        for c in range(chunks):
            for w in range(8):
                i = base + 8 * c + w
                assert 0 <= i < region
                used[i] += 1
    assert used.max(initial=0) <= 1
