"""Host logic of the sweep gridding (G_l^H, Sec. 2.1, step 12) on the CPU:
the work lists the plan builds (hs_sweep_lists) satisfy the conditions the
kernel relies on, and the kernel's algorithm run on them in NumPy (three 4-row
register bands per 32-column strip, groups of windows with disjoint columns)
equals direct gridding of the same windows."""

import numpy as np
import pytest

from paper_1806_04596_gb300 import hypersara as hs

T = 32


def _windows(seed, Kx, Ky, L, M):
    rng = np.random.default_rng(seed)
    off = np.concatenate([[0], np.cumsum(M)]).astype(np.int64)
    n = int(off[-1])
    k0x = rng.integers(0, Kx, n)
    k0y = rng.integers(0, Ky, n)
    # a dense band of start rows around row 0 (rows cut short, windows wrapping the edge)
    dense = rng.random(n) < 0.4
    k0y[dense] = rng.integers(-4, 4, dense.sum()) % Ky
    return off, k0x, k0y, rng


def _rel_row(k0y, row0, Ky):
    return ((k0y - row0 + 7) % Ky) - 7


def _rel_col(k0x, c0, Kx):
    return ((k0x - c0 + 7) % Kx) - 7


# the autotuner's candidates (rows per item, window cap); (0, 0) = the defaults (64, 1024)
CANDIDATES = [(0, 0), (32, 512), (128, 2048)]


@pytest.mark.parametrize("hmax_req,cap", CANDIDATES)
@pytest.mark.parametrize("Kx,Ky", [(64, 64), (128, 64), (64, 256), (160, 96)])
def test_lists_meet_the_kernel_conditions(Kx, Ky, hmax_req, cap):
    off, k0x, k0y, _ = _windows(3, Kx, Ky, 3, (1500, 0, 900))
    items, ent = hs.sweep_lists(Kx, Ky, off, k0x, k0y, hmax_req, cap)
    L = len(off) - 1
    hmax = min(hmax_req or 64, Ky - 8)
    rows = {}
    for (l, s, r0, r1, e0, e1) in items:
        assert 1 <= r1 - r0 <= hmax and (e1 - e0) % 4 == 0
        rows.setdefault((l, s), []).append((r0, r1))
        c0, H = s * T, r1 - r0
        seen = []
        band_prev = -2
        for g in range(e0, e1, 4):
            slots = ent[g:g + 4]
            real = slots[slots >= 0]
            assert len(real) >= 1 and np.all(slots[:len(real)] >= 0)   # pads only at the end
            assert np.all((real >= off[l]) & (real < off[l + 1]))
            ry = _rel_row(k0y[real], r0, Ky)
            rx = _rel_col(k0x[real], c0, Kx)
            band = ry[0] // 4
            assert np.all(ry // 4 == band) and band >= band_prev
            band_prev = band
            lo, hi = np.maximum(rx, 0), np.minimum(rx + 8, T)
            assert np.all(np.diff(rx) > 0) and np.all(lo[1:] >= hi[:-1])   # disjoint, by column
            seen.extend(real.tolist())
        # exactly the windows of channel l that reach the strip and start in rows r0 - 7 .. r1 - 1
        idx = np.arange(off[l], off[l + 1])
        want = idx[(_rel_col(k0x[idx], c0, Kx) <= T - 1) & (_rel_row(k0y[idx], r0, Ky) < H)]
        assert sorted(seen) == sorted(want.tolist())
    for l in range(L):
        for s in range(Kx // T):
            rr = sorted(rows[(l, s)])
            assert rr[0][0] == 0 and rr[-1][1] == Ky and all(a[1] == b[0] for a, b in zip(rr, rr[1:]))
    work = (items[:, 5] - items[:, 4]) + 4 * (items[:, 3] - items[:, 2])
    assert np.all(np.diff(work) <= 0)   # heaviest first


@pytest.mark.parametrize("hmax_req,cap", CANDIDATES)
def test_sweep_on_the_lists_equals_direct_gridding(hmax_req, cap):
    Kx, Ky = 128, 64
    off, k0x, k0y, rng = _windows(7, Kx, Ky, 2, (1200, 700))
    n = int(off[-1])
    phx, phy = rng.standard_normal((n, 8)), rng.standard_normal((n, 8))
    val = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    ref = np.zeros((2, Ky, Kx), complex)
    for l in range(2):
        for i in range(off[l], off[l + 1]):
            rows = (k0y[i] + np.arange(8)) % Ky
            cols = (k0x[i] + np.arange(8)) % Kx
            ref[l][np.ix_(rows, cols)] += val[i] * np.outer(phy[i], phx[i])
    items, ent = hs.sweep_lists(Kx, Ky, off, k0x, k0y, hmax_req, cap)
    out = np.full((2, Ky, Kx), np.nan, complex)
    lanes = np.arange(T)
    for (l, s, r0, r1, e0, e1) in items:
        c0, H = s * T, r1 - r0
        banks = [np.zeros((4, T), complex) for _ in range(3)]   # band j in bank j mod 3
        jb = -2

        def advance():
            nonlocal jb
            A = banks[jb % 3]
            for k in range(4):
                r = 4 * jb + k
                if 0 <= r < H:
                    assert np.all(np.isnan(out[l, r0 + r, c0:c0 + T]))   # every cell stored once
                    out[l, r0 + r, c0:c0 + T] = A[k]
            A[:] = 0
            jb += 1

        for g in range(e0, e1, 4):
            slots = ent[g:g + 4]
            rx = np.array([_rel_col(k0x[i], c0, Kx) if i >= 0 else 1 << 20 for i in slots])
            ry0 = _rel_row(k0y[slots[0]], r0, Ky)
            while jb < ry0 // 4:
                advance()
            sel = (lanes >= rx[1]).astype(int) + (lanes >= rx[2]) + (lanes >= rx[3])
            for lane in range(T):
                i = slots[sel[lane]]
                dx = lane - rx[sel[lane]]
                if not 0 <= dx < 8:
                    continue
                o = _rel_row(k0y[i], r0, Ky) & 3
                for m in range(8):
                    banks[(jb + (o + m) // 4) % 3][(o + m) & 3, lane] += val[i] * phy[i, m] * phx[i, dx]
        while 4 * jb < H:
            advance()
    assert not np.isnan(out).any()
    assert np.max(np.abs(out - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_bad_arguments_are_rejected():
    off = np.array([0, 2], dtype=np.int64)
    with pytest.raises(hs.HSError):
        hs.sweep_lists(80, 64, off, [0, 1], [0, 1])    # columns not a multiple of the 32-column strip
    with pytest.raises(hs.HSError):
        hs.sweep_lists(32, 64, off, [0, 1], [0, 1])    # narrower than two strips
    with pytest.raises(hs.HSError):
        hs.sweep_lists(64, 64, off, [0, 64], [0, 1])   # start cell outside the grid
