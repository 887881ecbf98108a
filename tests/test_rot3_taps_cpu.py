"""The eight-tap form of the three-pass rotation (CPU).

The CUDA path runs the three 1D linear-interpolation passes of reading R13 as
one gather of eight taps per output -- the pixels the three passes reach, each
weighted by the product of its three pass weights -- and A' as eight-entry
lists that enumerate the same (output, pixel, weight) triples from the
pixel's side.  This test builds both index maps the way the plan does (FP64
shifts, products rounded to FP32) in numpy and checks them against the oracle's
pass-by-pass rotation and its scatter transpose, so the fused construction is
pinned on the CPU independently of the kernels.
"""
import math

import numpy as np
import pytest

import oracle


def _view(theta):
    r = float(np.rint(theta / (math.pi / 2)))
    phi = theta - r * (math.pi / 2)
    return int(r) % 4, math.tan(0.5 * phi), math.sin(phi)


def _shift(d):
    f = math.floor(d)
    return int(f), (1.0 - (d - f), d - f)


def _from(n, q, i, j):
    return [(i, j), (j, n - 1 - i), (n - 1 - i, n - 1 - j), (n - 1 - j, i)][q]


def _to(n, q, si, sj):
    return [(si, sj), (n - 1 - sj, si), (n - 1 - si, n - 1 - sj), (sj, n - 1 - si)][q]


def _taps(n, theta):
    """Forward taps per output (i, j) and adjoint entries per pixel (qi, qj)."""
    q, t, s = _view(theta)
    c = 0.5 * (n - 1)
    rows = [_shift(t * (m - c)) for m in range(n)]
    cols = [_shift(-s * (m - c)) for m in range(n)]
    fwd = {}
    for j in range(n):
        for i in range(n):
            taps = []
            for m3 in range(2):
                i2 = i + rows[j][0] + m3
                if not 0 <= i2 < n:
                    continue
                co, cw = cols[i2]
                for mp in range(2):
                    r = j + co + mp
                    if not 0 <= r < n:
                        continue
                    for m in range(2):
                        hi = i2 + rows[r][0] + m
                        if 0 <= hi < n:
                            taps.append((_from(n, q, hi, r), np.float32((cw[mp] * rows[r][1][m]) * rows[j][1][m3])))
            fwd[(i, j)] = taps
    adj = {}
    for qj in range(n):
        for qi in range(n):
            hi, hj = _to(n, q, qi, qj)
            ent = []
            for m in range(2):
                c1 = hi - rows[hj][0] - m
                if not 0 <= c1 < n:
                    continue
                co, cw = cols[c1]
                for mp in range(2):
                    r = hj - co - mp
                    if not 0 <= r < n:
                        continue
                    for m3 in range(2):
                        c3 = c1 - rows[r][0] - m3
                        w = np.float32((cw[mp] * rows[hj][1][m]) * rows[r][1][m3])
                        if 0 <= c3 < n and w != 0:
                            ent.append(((c3, r), w))
            adj[(qi, qj)] = ent
    return fwd, adj


@pytest.mark.parametrize("n", [7, 10, 16])
@pytest.mark.parametrize("theta", [0.0, 0.37, 1.5707963267948966, 2.2, 3.9, 5.5, -0.3])
def test_eight_taps_reproduce_the_three_passes(n, theta):
    fwd, adj = _taps(n, theta)
    assert max(len(v) for v in fwd.values()) <= 8 and max(len(v) for v in adj.values()) <= 8
    rng = np.random.default_rng(int(1000 * abs(theta)) + n)
    img = rng.uniform(-1, 1, (n, n))
    out = np.zeros((n, n))
    for (i, j), taps in fwd.items():
        out[j, i] = sum(float(w) * img[pj, pi] for (pi, pj), w in taps)
    # FP32-rounded weights: agreement to a few FP32 ulps of the interpolated values
    np.testing.assert_allclose(out, oracle.rotate3_slice(img, theta), rtol=0, atol=2e-7)
    t = rng.uniform(-1, 1, (n, n))
    back = np.zeros((n, n))
    for (qi, qj), ent in adj.items():
        back[qj, qi] = sum(float(w) * t[pj, pi] for (pi, pj), w in ent)
    np.testing.assert_allclose(back, oracle.rotate3_adjoint_slice(t, theta), rtol=0, atol=2e-7)


def test_adjoint_entries_are_the_forward_taps_transposed():
    """Every nonzero forward tap (output p reads pixel q with weight w) appears as
    exactly one adjoint entry (pixel q receives from output p with the same FP32 w)."""
    n = 12
    fwd, adj = _taps(n, 0.81)
    pairs_f = {}
    for (i, j), taps in fwd.items():
        for (pi, pj), w in taps:
            if w != 0:
                pairs_f[((pi, pj), (i, j))] = pairs_f.get(((pi, pj), (i, j)), []) + [w]
    pairs_a = {}
    for (qi, qj), ent in adj.items():
        for (ci, cj), w in ent:
            pairs_a[((qi, qj), (ci, cj))] = pairs_a.get(((qi, qj), (ci, cj)), []) + [w]
    assert pairs_f.keys() == pairs_a.keys()
    for k in pairs_f:
        assert sorted(pairs_f[k]) == sorted(pairs_a[k])
