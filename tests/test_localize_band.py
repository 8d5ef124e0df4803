"""The band of observations visited by each 32-row tile of the partial-localization kernel
(enkf_localized_update), transcribed from the kernel's index arithmetic and checked on the CPU:
every (state, observation) pair inside the radius of influence is visited exactly once, whatever
the wrap-around of the periodic ring, and no pair is visited twice.  The weights decide the rest,
so this is what makes the banded sum equal the full one."""
import math

import numpy as np
import pytest

TI = 32   # state rows per CTA


def band_of(nstate, radius):
    """ceil(radius) when a tile's band is narrower than the ring, else -1 (visit every observation)."""
    if radius is None or radius < 0 or radius >= nstate:
        return -1
    rc = math.ceil(radius)
    return rc if TI + 2 * rc < nstate else -1


def tile_ranges(nstate, nobs, stride, band, i0):
    """Observation index ranges [lo, hi] of the tile starting at state row i0 (at most two)."""
    if band < 0:
        return [(0, nobs - 1)]
    p, q = i0 - band, i0 + TI - 1 + band
    if p < 0:
        segs = [(p + nstate, nstate - 1), (0, q)]
    elif q >= nstate:
        segs = [(p, nstate - 1), (0, q - nstate)]
    else:
        segs = [(p, q)]
    out = []
    for a, b in segs:
        jl = (a + stride - 1) // stride
        jh = min(b // stride, nobs - 1)
        if jl <= jh:
            out.append((jl, jh))
    return out


@pytest.mark.parametrize("nstate,stride,radius", [
    (1000, 4, 30.5), (1000, 4, None), (513, 1, 5.0), (300, 5, 0.0), (130, 1, 64.0), (2000, 2, 250.0),
    (97, 3, 31.9), (1024, 7, 12.0), (4096, 2, 64.0), (33, 1, 0.4), (65, 2, 16.0), (64, 1, 15.9)])
def test_every_pair_inside_the_radius_is_visited_once(nstate, stride, radius):
    nobs = (nstate - 1) // stride + 1
    band = band_of(nstate, radius)
    visits = np.zeros((nstate, nobs), dtype=np.int64)
    for i0 in range(0, nstate, TI):
        rows = slice(i0, min(i0 + TI, nstate))
        for lo, hi in tile_ranges(nstate, nobs, stride, band, i0):
            assert 0 <= lo <= hi < nobs
            visits[rows, lo:hi + 1] += 1
    assert visits.max() <= 1
    i = np.arange(nstate)[:, None]
    j = np.arange(nobs)[None, :]
    d = np.abs(i - j * stride)
    d = np.minimum(d, nstate - d)
    inside = np.ones_like(d, dtype=bool) if radius is None else d <= radius
    assert np.all(visits[inside] == 1)
