"""The bookkeeping of the medoid tiles, on the host.

The medoid kernel computes each pair of a mode's members once, in 32 x 32 tiles (ti <= tj),
and writes one partial per (member, tile): a row sum over tile tj for pairs in the upper
tiles, a column sum over tile ti for the lower ones, and on a diagonal tile the row sum
over the pairs above the diagonal plus the column sum over those below.  Summing a member's
partials over the tiles in order must give its full sum of distances, for sizes that are
and are not multiples of 32, and every entry must be written exactly once.
"""
import numpy as np
import pytest


def _tiled_sums(D):
    s = D.shape[0]
    nt = (s + 31) // 32
    P = np.full((s, nt), np.nan)
    writes = np.zeros((s, nt), int)
    for ti in range(nt):
        for tj in range(ti, nt):
            diag = ti == tj
            col = np.zeros((32, 32))
            row = np.zeros(32)
            for r in range(32):
                ra = ti * 32 + r
                if ra >= s:
                    continue
                d = np.zeros(32)
                for lane in range(32):
                    cb = tj * 32 + lane
                    if cb < s and not (diag and cb <= ra):
                        d[lane] = D[ra, cb]
                col[r] = d
                if diag:
                    row[r] = d.sum()
                else:
                    P[ra, tj] = d.sum()
                    writes[ra, tj] += 1
            for c in range(32):
                cb = tj * 32 + c
                if cb < s:
                    P[cb, ti] = (row[c] if diag else 0.0) + col[:, c].sum()
                    writes[cb, ti] += 1
    return P, writes


@pytest.mark.parametrize("s", [1, 2, 31, 32, 33, 70, 96])
def test_medoid_tiles_cover_every_pair_once(s):
    rng = np.random.Generator(np.random.PCG64(s))
    A = rng.uniform(0.0, 1.0, (s, s))
    D = np.triu(A, 1) + np.triu(A, 1).T            # symmetric, zero diagonal
    P, writes = _tiled_sums(D)
    assert np.all(writes == 1)
    assert np.allclose(P.sum(axis=1), D.sum(axis=1), rtol=1e-13, atol=1e-13)


def _tile_rc(t, nb):
    """The pairwise-link kernel's map from a linear tile index to the tile pair (bi <= bj):
    row bi holds tiles bi..nb-1 and starts at bi*nb - bi*(bi-1)/2; an FP64 square-root
    estimate of the row, then corrected by whole steps."""
    B = 2.0 * nb + 1.0
    r = int((B - np.sqrt(max(B * B - 8.0 * t, 0.0))) * 0.5)
    r = max(0, min(r, nb - 1))
    start = lambda b: b * nb - b * (b - 1) // 2
    while r > 0 and start(r) > t:
        r -= 1
    while r + 1 < nb and start(r + 1) <= t:
        r += 1
    return r, r + (t - start(r))


@pytest.mark.parametrize("nb", [1, 2, 3, 7, 32, 101, 416, 2000])
def test_link_tile_map_covers_each_pair_once(nb):
    seen = set()
    for t in range(nb * (nb + 1) // 2):
        bi, bj = _tile_rc(t, nb)
        assert 0 <= bi <= bj < nb
        seen.add((bi, bj))
    assert len(seen) == nb * (nb + 1) // 2
