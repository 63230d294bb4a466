"""Host logic of the layer work items (no GPU): the items pml_plan_layer_items reports for a
box must cover the layer frame -- every vertex outside the layer-free run, the run taken
from the oracle's layout of the same damping profile -- exactly once, keep the TMA
alignment of their boxes, stay within their row caps, and claim an undamped axis (the
narrower halo of 2) only where no aux field of that axis lies within 4 vertices of any of
their outputs."""
import numpy as np
import pytest

import oracle
from paper_1804_01390_gb300 import _lib

G = 4          # ghost ring width
COLS = 32      # columns of a 2D strip (one warp, one column per lane)
KINDS = {"quadratic": oracle.KIND_POWER, "constant": oracle.KIND_CONSTANT, "random": oracle.KIND_RANDOM}


def _profile(N, w, kind, wall, seed):
    """Damping per axis as the library builds it, and the host pointers of the draws."""
    rng = np.random.default_rng(seed)
    sigs, draws = [], []
    for n in N:
        d = rng.random(n + 2 * w) if kind == "random" else None
        s = oracle.sigma_profile(n, w, KINDS[kind], 2.0, 2.0, draws=d)
        if wall:
            s[-1] = 0.0   # a wall leaves no wrap edge (pml.h, PML_FLAG_WALL)
        sigs.append(s)
        draws.append(d)
    return sigs, draws


def _items(N, w, kind, wall, prec, sm_count, which, draws):
    user = None
    if kind == "random":
        user = [d.ctypes.data for d in draws]
    flags = _lib.PML_FLAG_WALL if wall else 0
    return _lib.pml_plan_layer_items(len(N), N, w, KINDS[kind], 2.0, 2.0, user, prec, flags, sm_count, which)


def _axis_tables(sig, w, n):
    """(aux support of the axis, layer-free run lo, hi) from the oracle."""
    phi, psi, inner = oracle.layout_axis(sig, w + n // 2)
    aux = (np.asarray(phi) != 0) | (np.asarray(psi) != 0)
    idx = np.flatnonzero(np.asarray(inner))
    return aux, int(idx[0]), int(idx[-1])


def _near(aux, coords):
    """For each coordinate: an aux field of the axis within 4 vertices (periodic index)."""
    T = aux.size
    return np.array([aux[np.arange(c - 4, c + 5) % T].any() for c in coords], dtype=bool)


CASES_2D = [
    ((200, 150), 16, "quadratic", False),
    ((97, 131), 12, "random", False),
    ((120, 90), 20, "constant", False),
    ((64, 64), 6, "quadratic", False),
    ((200, 150), 16, "quadratic", True),
    ((150, 97), 10, "random", True),
]


@pytest.mark.parametrize("N,w,kind,wall", CASES_2D)
@pytest.mark.parametrize("which,prec,sm", [(0, 32, 152), (0, 64, 152), (0, 32, 2), (1, 32, 152), (2, 32, 152),
                                           (4, 32, 152)])
def test_2d_items_cover_the_frame_once(N, w, kind, wall, which, prec, sm):
    sigs, draws = _profile(N, w, kind, wall, seed=sum(N) + w)
    t = _items(N, w, kind, wall, prec, sm, which, draws)
    T0, T1 = N[0] + 2 * w, N[1] + 2 * w
    (ax, xlo, xhi), (ay, ylo, yhi) = _axis_tables(sigs[0], w, N[0]), _axis_tables(sigs[1], w, N[1])
    k = {0: 0, 1: 6, 2: 2, 4: 0}[which]   # the run of the frame, shrunk for the two-step passes
    xlo, xhi, ylo, yhi = xlo + k, xhi - k, ylo + k, yhi - k
    cover = np.zeros((T1, T0), dtype=np.int32)
    band, slab = {0: (32, 32 if wall else 24), 1: (32, 32 if wall else 24), 2: (32, 32 if wall else 24),
                  4: (40, 40)}[which]
    for x0, y0, z0, ilo, ihi, jlo, jhi, zlo, zhi, fl in t:
        HX = 4 if fl & 1 else 2
        assert (x0 - HX + G) % 4 == 0, "box start off the 16-byte TMA alignment"
        xs = np.arange(max(x0, ilo), min(x0 + COLS - 2 * HX - 1, ihi) + 1)
        assert xs.size > 0 and xs[0] >= 0 and xs[-1] < T0
        ys = np.arange(jlo, jhi + 1)
        rows = ys.size
        assert 1 <= rows <= max(band, slab)
        if fl == 3:   # corners: 2/5 of the run length
            assert rows <= max(8, band * 2 // 5)
        if wall:
            assert ys[-1] < T1, "no band crosses the box end of a wall-backed box"
        if not fl & 1:
            assert not _near(ax, xs).any(), "an undamped-x item has x aux fields within reach"
        if not fl & 2:
            assert not _near(ay, ys % T1).any(), "an undamped-y item has y aux fields within reach"
        cover[np.ix_(ys % T1, xs)] += 1
    run = np.zeros_like(cover, dtype=bool)
    run[ylo:yhi + 1, xlo:xhi + 1] = True
    assert (cover[run] == 0).all(), "an item writes into the layer-free run"
    assert (cover[~run] == 1).all(), "frame vertices covered %s times" % sorted(set(cover[~run].tolist()))


def test_2d_corner_items_are_shorter_than_the_others():
    """On the headline box the corner strips (damped along both axes) take 2/5 of the
    band's run length and every item holds at most 32 rows."""
    N, w = (8192, 8192), 32
    sigs, draws = _profile(N, w, "quadratic", False, 0)
    t = _items(N, w, "quadratic", False, 32, 152, 1, draws)
    rows = t[:, 6] - t[:, 5] + 1
    assert rows.max() <= 32
    assert (t[:, 9] == 3).any() and rows[t[:, 9] == 3].max() <= 12
    # about one item per warp of a full launch (152 SMs x 16 warps)
    assert len(t) <= 152 * 16


@pytest.mark.parametrize("N,w,kind", [((40, 36, 44), 8, "quadratic"), ((33, 41, 30), 6, "random")])
def test_3d_slab_tiles_cover_the_frame_once(N, w, kind):
    sigs, draws = _profile(N, w, kind, False, seed=7)
    t = _items(N, w, kind, False, 32, 152, 3, draws)
    T = tuple(n + 2 * w for n in N)
    tabs = [_axis_tables(sigs[a], w, N[a]) for a in range(3)]
    cover = np.zeros((T[2], T[1], T[0]), dtype=np.int32)
    for x0, y0, z0, ilo, ihi, jlo, jhi, zlo, zhi, fl in t:
        assert (x0 + G) % 4 == 0, "region start off the 16-byte TMA alignment"
        rng = [np.arange(ilo, ihi + 1), np.arange(jlo, jhi + 1), np.arange(zlo, zhi + 1)]
        for a in range(3):
            assert rng[a].size > 0
            if not (fl >> a) & 1:
                assert not _near(tabs[a][0], rng[a] % T[a]).any(), "axis %d claimed undamped" % a
        assert rng[0][-1] < T[0] and rng[1][-1] < T[1] and rng[2][0] >= 0
        cover[np.ix_(rng[2] % T[2], rng[1], rng[0])] += 1
    run = np.zeros_like(cover, dtype=bool)
    run[tabs[2][1]:tabs[2][2] + 1, tabs[1][1]:tabs[1][2] + 1, tabs[0][1]:tabs[0][2] + 1] = True
    assert (cover[run] == 0).all()
    assert (cover[~run] == 1).all(), "frame vertices covered %s times" % sorted(set(cover[~run].tolist()))


def test_rejects_item_sets_of_other_boxes():
    with pytest.raises(RuntimeError):
        _lib.pml_plan_layer_items(2, (64, 64), 8, oracle.KIND_POWER, 2.0, 2.0, None, 64, 0, 152, 1)
    with pytest.raises(RuntimeError):
        _lib.pml_plan_layer_items(2, (64, 64), 8, oracle.KIND_POWER, 2.0, 2.0, None, 32, 0, 152, 3)
    with pytest.raises(RuntimeError):
        _lib.pml_plan_layer_items(3, (16, 16, 16), 4, oracle.KIND_POWER, 2.0, 2.0, None, 32, 0, 152, 0)
    with pytest.raises(RuntimeError):
        _lib.pml_plan_layer_items(2, (64, 64), 8, oracle.KIND_POWER, 2.0, 2.0, None, 32, 0, 0, 0)
