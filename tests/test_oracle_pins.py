"""Pins of the CPU oracle against facts fixed outside it: closed forms,
brute force on tiny maps, textbook/library routines and published vectors.

Each test names the passage of the paper (or the definition) it checks.
"""
import math
import os

import numpy as np
import pytest

from paper_2606_15846_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RES = 0.05


def ulp32(x):
    x = np.float32(abs(x))
    return float(np.spacing(x)) if x > 0 else float(np.spacing(np.float32(0)))


# --------------------------------------------------------------------------
# sin / cos used for headings and beams (Eq. 4)
# --------------------------------------------------------------------------
def test_sincos_within_two_ulp_of_fp64(oracle):
    xs = np.concatenate([np.linspace(-math.pi - 0.2, math.pi + 0.2, 20001, dtype=np.float32),
                         np.float32([0.0, -0.0, np.float32(math.pi), -np.float32(math.pi),
                                     np.float32(math.pi / 2), np.float32(math.pi / 4)])])
    worst = 0.0
    for x in xs:
        s, c = oracle.sincosf(float(x))
        ts, tc = math.sin(float(x)), math.cos(float(x))
        es = abs(float(s) - ts) / ulp32(ts)
        ec = abs(float(c) - tc) / ulp32(tc)
        worst = max(worst, es, ec)
    assert worst <= 2.0, worst


def test_sincos_special_values(oracle):
    s, c = oracle.sincosf(0.0)
    assert s == 0.0 and c == 1.0


# --------------------------------------------------------------------------
# counter-based reset RNG: SplitMix64 finaliser, published outputs
# --------------------------------------------------------------------------
def test_hash_matches_published_splitmix64(oracle):
    gamma = 0x9E3779B97F4A7C15
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "splitmix64.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert rows
    for s, k, want in rows:
        s, k, want = int(s), int(k), int(want)
        state = (s + (k - 1) * gamma) % (1 << 64)
        assert oracle.hash64(state, 0, 0, 0) == want


def test_hash_bits_uniform(oracle):
    n = 20000
    top = np.array([oracle.hash64(7, e, 3, 5) >> 60 for e in range(n)])
    cnt = np.bincount(top, minlength=16)
    chi2 = float(((cnt - n / 16) ** 2 / (n / 16)).sum())
    assert chi2 < 45.0  # 15 dof, p ~ 1e-4


# --------------------------------------------------------------------------
# Ray casting (Eq. 4-5): exact grid traversal
# --------------------------------------------------------------------------
@pytest.mark.parametrize("direction", ["+x", "-x", "+y", "-y"])
def test_axis_wall_range_is_analytic(oracle, direction):
    n = 64
    occ = np.zeros((n, n), np.uint8)
    c = 50
    x0, y0 = np.float32(10.37 * RES), np.float32(20.61 * RES)
    xc = float(np.float32(x0 * np.float32(1 / RES)))
    yc = float(np.float32(y0 * np.float32(1 / RES)))
    if direction == "+x":
        occ[:, c] = 1
        d, want = (1.0, 0.0), (c - xc)
    elif direction == "-x":
        occ[:, 3] = 1
        d, want = (-1.0, 0.0), (xc - 4)
    elif direction == "+y":
        occ[c, :] = 1
        d, want = (0.0, 1.0), (c - yc)
    else:
        occ[5, :] = 1
        d, want = (0.0, -1.0), (yc - 6)
    r, hit, vis = oracle.cast_ray(occ, RES, float(x0), float(y0), d[0], d[1], 10.0)
    assert abs(float(r) - want * RES) <= 2 * ulp32(want * RES)
    assert hit >= 0 and occ.flat[hit] == 1
    assert vis == int(abs(want)) + 2


def test_oblique_far_wall_range_is_analytic(oracle):
    """Eq. 4-5: a ray at an oblique angle crosses ~2000 column boundaries
    and ~1000 row boundaries before a wall at column 2000; its range is the
    analytic (c - xc) / dx within 3 ulp.  Each boundary parameter is one
    rounding of t0 + k tDelta; adding tDelta once per step instead drifts by
    hundreds of ulp over this ray."""
    n, c = 2048, 2000
    occ = np.zeros((n, n), np.uint8)
    occ[:, c] = 1
    inv = np.float32(1 / RES)
    for trial in range(20):
        rng = np.random.default_rng(trial)
        x0 = np.float32(rng.uniform(5, 15) * RES)
        y0 = np.float32(rng.uniform(300, 400) * RES)
        a = rng.uniform(0.2, 0.6)
        dx, dy = np.float32(math.cos(a)), np.float32(math.sin(a))
        r, hit, _ = oracle.cast_ray(occ, RES, float(x0), float(y0), float(dx), float(dy), 120.0)
        xc = float(np.float32(x0 * inv))
        want = (c - xc) / float(dx) * RES
        assert abs(float(r) - want) <= 3 * ulp32(want), (trial, float(r), want)
        assert hit % n == c


def test_empty_map_returns_max_range(oracle):
    n = 256
    occ = np.zeros((n, n), np.uint8)
    x = y = n * RES / 2
    for k in range(360):
        a = -math.pi + (k + 0.5) * 2 * math.pi / 360
        r, hit, _ = oracle.cast_ray(occ, RES, x, y, math.cos(a), math.sin(a), 4.0)
        assert r == np.float32(4.0) and hit == -2


def test_leaving_the_map_is_an_obstacle(oracle):
    occ = np.zeros((16, 16), np.uint8)
    r, hit, _ = oracle.cast_ray(occ, RES, 8.5 * RES, 8.5 * RES, 1.0, 0.0, 10.0)
    assert hit == -1
    assert abs(float(r) - 7.5 * RES) < 1e-6


def _march(occ, xc, yc, dx, dy, rmax_c, step=1e-4):
    """Brute force: sample the ray every `step` cells (float64); return the
    first blocked cell (or -1 off-map, -2 none), its first sample's t and the
    ordered list of distinct cells met before it."""
    h, w = occ.shape
    t = np.arange(0.0, rmax_c + step, step)
    px = xc + t * dx
    py = yc + t * dy
    ci = np.floor(px).astype(np.int64)
    cj = np.floor(py).astype(np.int64)
    out = (ci < 0) | (cj < 0) | (ci >= w) | (cj >= h)
    blocked = out.copy()
    inside = ~out
    blocked[inside] = occ[cj[inside], ci[inside]] != 0
    idx = np.flatnonzero(blocked)
    if idx.size == 0:
        return -2, None, None
    f = idx[0]
    cid = -1 if out[f] else int(cj[f] * w + ci[f])
    return cid, t[f], (ci[:f], cj[:f])


def _near_corner(xc, yc, dx, dy, rmax_c, eps=2e-4):
    """True when the ray passes within eps of a grid corner (tie cases)."""
    t = np.linspace(0, rmax_c, int(rmax_c * 400) + 1)
    px, py = xc + t * dx, yc + t * dy
    fx = np.abs(px - np.round(px))
    fy = np.abs(py - np.round(py))
    return bool(np.any((fx < eps) & (fy < eps)))


@pytest.mark.parametrize("size", [4, 8, 12, 16])
def test_dda_agrees_with_supersampled_march(oracle, size):
    rng = np.random.default_rng(size)
    n_checked = 0
    for trial in range(60):
        occ = (rng.random((size, size)) < 0.25).astype(np.uint8)
        free = np.argwhere(occ == 0)
        if len(free) == 0:
            continue
        j, i = free[rng.integers(len(free))]
        x = float(np.float32((i + rng.uniform(0.05, 0.95)) * RES))
        y = float(np.float32((j + rng.uniform(0.05, 0.95)) * RES))
        a = rng.uniform(-math.pi, math.pi)
        dx, dy = float(np.float32(math.cos(a))), float(np.float32(math.sin(a)))
        rmax = 0.4
        r, hit, _ = oracle.cast_ray(occ, RES, x, y, dx, dy, rmax)
        xc = float(np.float32(np.float32(x) * np.float32(1 / RES)))
        yc = float(np.float32(np.float32(y) * np.float32(1 / RES)))
        rmax_c = rmax / RES
        if _near_corner(xc, yc, dx, dy, rmax_c):
            continue
        cid, tb, _ = _march(occ, xc, yc, dx, dy, rmax_c)
        n_checked += 1
        assert hit == cid, (trial, hit, cid)
        if cid != -2:
            assert abs(float(r) - tb * RES) <= 1e-4 * RES + 1e-6
        else:
            assert r == np.float32(rmax)
    assert n_checked > 30


def test_dda_invariants(oracle):
    wl = W.config_small()
    occ = wl.maps[0]
    rng = np.random.default_rng(3)
    free = np.argwhere(occ == 0)
    for _ in range(300):
        j, i = free[rng.integers(len(free))]
        x, y = (i + 0.5) * RES, (j + 0.5) * RES
        a = rng.uniform(-math.pi, math.pi)
        r, hit, vis = oracle.cast_ray(occ, RES, x, y, math.cos(a), math.sin(a), 4.0)
        assert 0.0 <= r <= np.float32(4.0)
        if hit >= 0:
            assert occ.flat[hit] == 1
        assert vis >= 1


def test_quarter_turn_permutes_beams(oracle):
    """Rotating the map (and the position) by +90 deg while the heading stays
    put maps beam k to beam k + K/4 (360 deg field of view, K divisible by 4):
    beam k + K/4 of the unrotated robot points 90 deg left of beam k."""
    rng = np.random.default_rng(11)
    occ = W.make_map(5, 80, 64, 0.15)
    H = occ.shape[0]
    rot = np.zeros((occ.shape[1], H), np.uint8)  # W' = H, H' = W
    jj, ii = np.nonzero(occ)
    rot[ii, H - 1 - jj] = 1
    K = 360
    par = W.Params(goal_dmin=0.0, goal_dmax=1e9)
    mk = lambda m: oracle.OracleSim([m], np.zeros(1, np.int32), np.full(1, K, np.int32),
                                    np.zeros(1, np.int32), [W.DISC], 3.0, par, RES)
    s0, s1 = mk(occ), mk(rot)
    s0.reset(0)
    s1.reset(0)
    free = np.argwhere(occ == 0)
    agree = total = 0
    stay = np.array([[-1.0, 0.0]], np.float32)  # v = 0, w = 0
    tried = 0
    while total < 6 * K and tried < 200:
        tried += 1
        j, i = free[rng.integers(len(free))]
        x, y = (i + 0.37) * RES, (j + 0.71) * RES
        th = float(np.float32(rng.uniform(-math.pi, math.pi)))
        xr, yr = H * RES - y, x
        if oracle.footprint(occ, RES, W.DISC, x, y, th) or \
                oracle.footprint(rot, RES, W.DISC, xr, yr, th):
            continue
        s0.set_state(0, np.array([[x, y, th, 0, 0, -50, -50, 100]], np.float32),
                     np.zeros((1, 2), np.int32))
        s1.set_state(0, np.array([[xr, yr, th, 0, 0, -50, -50, 100]], np.float32),
                     np.zeros((1, 2), np.int32))
        _, _, d0 = s0.step(stay)
        _, _, d1 = s1.step(stay)
        assert d0[0] == 0 and d1[0] == 0
        r0, _, _ = s0.debug()
        r1, _, _ = s1.debug()
        for k in range(K):
            total += 1
            agree += abs(float(r0[k]) - float(r1[(k + K // 4) % K])) < 1e-4
    assert total >= 6 * K
    assert agree / total > 0.99, (agree, total)


# --------------------------------------------------------------------------
# Fixed-step march (Sec. 2.2.2, Table 7's 0.03 m step) and the beam fan
# --------------------------------------------------------------------------
@pytest.mark.parametrize("direction", ["+x", "-y"])
@pytest.mark.parametrize("step", [0.03, 0.011])
def test_march_axis_wall_is_first_sample_past_the_face(oracle, direction, step):
    """Towards a wall at distance D along an axis, the march stops at the
    first sample s * step >= D, after s + 1 samples."""
    n = 64
    occ = np.zeros((n, n), np.uint8)
    x0, y0 = 10.37 * RES, 40.61 * RES
    if direction == "+x":
        occ[:, 50] = 1
        d, D = (1.0, 0.0), 50 * RES - x0
    else:
        occ[5, :] = 1
        d, D = (0.0, -1.0), y0 - 6 * RES
    s_star = math.ceil(D / step)
    assert s_star * step - D > 1e-4 and D - (s_star - 1) * step > 1e-4  # no rounding tie
    r, hit, vis = oracle.march_ray(occ, RES, x0, y0, d[0], d[1], step, 10.0)
    assert abs(float(r) - s_star * step) < 2e-5
    assert hit >= 0 and occ.flat[hit] == 1
    assert vis == s_star + 1


def test_march_empty_map_and_off_map(oracle):
    occ = np.zeros((256, 256), np.uint8)
    r, hit, vis = oracle.march_ray(occ, RES, 6.4, 6.4, 0.6, 0.8, 0.03, 4.0)
    assert r == np.float32(4.0) and hit == -2 and vis == math.floor(4.0 / 0.03 + 1e-6) + 1
    small = np.zeros((16, 16), np.uint8)
    r, hit, _ = oracle.march_ray(small, RES, 8.5 * RES, 8.5 * RES, 1.0, 0.0, 0.03, 10.0)
    assert hit == -1 and abs(float(r) - 0.39) < 2e-5  # first sample at x >= 0.8 m


def _chord(i, j, xc, yc, dx, dy):
    """Length (cells) of the ray's segment inside cell (i, j), exact slabs."""
    lo, hi = 0.0, math.inf
    for p, d, a in ((xc, dx, i), (yc, dy, j)):
        if abs(d) < 1e-12:
            if not (a <= p < a + 1):
                return 0.0
            continue
        t0, t1 = (a - p) / d, (a + 1 - p) / d
        lo, hi = max(lo, min(t0, t1)), min(hi, max(t0, t1))
    return max(0.0, hi - lo)


@pytest.mark.parametrize("step", [0.03, 0.07])
def test_march_against_exact_traversal(oracle, step):
    """The march never stops before the exact first hit; it stops within one
    step after it unless the ray only clips that cell for less than a step;
    and the cell of its stopping sample is blocked or off the map."""
    wl = W.config_small()
    occ = wl.maps[0]
    h, w = occ.shape
    rng = np.random.default_rng(5)
    free = np.argwhere(occ == 0)
    clipped = 0
    for _ in range(600):
        j, i = free[rng.integers(len(free))]
        x, y = (i + rng.uniform(0.1, 0.9)) * RES, (j + rng.uniform(0.1, 0.9)) * RES
        a = rng.uniform(-math.pi, math.pi)
        dx, dy = math.cos(a), math.sin(a)
        rd, hd, _ = oracle.cast_ray(occ, RES, x, y, dx, dy, 4.0)
        rm, hm, vm = oracle.march_ray(occ, RES, x, y, dx, dy, step, 4.0)
        assert float(rm) >= float(rd) - 1e-5
        if hd >= 0 and float(rm) - float(rd) >= step + 1e-5:
            xc, yc = np.float32(x) * np.float32(1 / RES), np.float32(y) * np.float32(1 / RES)
            assert _chord(hd % w, hd // w, float(xc), float(yc), dx, dy) * RES < step + 1e-5
            clipped += 1
        if hm == -2:
            assert rm == np.float32(4.0)
            continue
        assert vm == round(float(rm) / step) + 1
        px, py = (x + float(rm) * dx) / RES, (y + float(rm) * dy) / RES
        if min(abs(px - round(px)), abs(py - round(py))) < 1e-3:
            continue  # the stopping sample sits on a grid line
        ci, cj = math.floor(px), math.floor(py)
        off = ci < 0 or cj < 0 or ci >= w or cj >= h
        assert off == (hm == -1)
        if not off:
            assert occ[cj, ci] == 1 and hm == cj * w + ci
    assert clipped < 60


def test_march_converges_to_exact_range(oracle):
    wl = W.config_small()
    occ = wl.maps[0]
    rng = np.random.default_rng(9)
    free = np.argwhere(occ == 0)
    diffs = []
    for _ in range(300):
        j, i = free[rng.integers(len(free))]
        x, y = (i + 0.5) * RES, (j + 0.5) * RES
        a = rng.uniform(-math.pi, math.pi)
        rd, _, _ = oracle.cast_ray(occ, RES, x, y, math.cos(a), math.sin(a), 4.0)
        rm, _, _ = oracle.march_ray(occ, RES, x, y, math.cos(a), math.sin(a), 1e-3, 4.0)
        diffs.append(float(rm) - float(rd))
    diffs = np.array(diffs)
    assert diffs.min() > -1e-5
    assert np.mean(diffs < 1e-3 + 1e-5) > 0.97


def _one_scan(oracle, occ, K, par, x, y, th, max_range):
    sim = oracle.OracleSim([occ], np.zeros(1, np.int32), np.full(1, K, np.int32),
                           np.zeros(1, np.int32), [W.DISC], max_range, par, RES)
    sim.reset(0)
    sim.set_state(0, np.array([[x, y, th, 0, 0, -50, -50, 100]], np.float32),
                  np.zeros((1, 2), np.int32))
    obs, _, done = sim.step(np.array([[-1.0, 0.0]], np.float32))  # v = 0, w = 0
    assert done[0] == 0
    r, _, _ = sim.debug()
    return obs, r


def test_fan_of_270_degrees_matches_the_square_border(oracle):
    """Eq. 4's fan alpha_k = -fov/2 + (k + 1/2) fov / K: from the centre of an
    empty L x L map, beam k ends on the border at (L/2) / max|cos|, |sin|."""
    n, K = 128, 1080
    occ = np.zeros((n, n), np.uint8)
    c = n * RES / 2
    th = 0.3
    par = W.Params(goal_dmin=0.0, goal_dmax=1e9, fov_deg=270.0)
    _, r = _one_scan(oracle, occ, K, par, c, c, th, 10.0)
    fov = math.radians(270.0)
    for k in range(K):
        a = th - fov / 2 + (k + 0.5) * fov / K
        want = c / max(abs(math.cos(a)), abs(math.sin(a)))
        assert abs(float(r[k]) - want) < 2e-5, (k, float(r[k]), want)


@pytest.mark.parametrize("sensor", [0, 1])
def test_sector_pooling_reduces_to_the_raw_scan(oracle, sensor):
    """Eq. 6 special cases and the 1080 -> 30 x 36 split of Table 7: with one
    beam per sector the pooled observation is the raw one; every pooled row
    is the minimum of its beams of the raw run; dynamics, rewards and flags
    do not depend on the pooling."""
    wl = W.config_small()
    K = 1080
    rng = np.random.default_rng(2)
    acts = rng.uniform(-1, 1, (25, 4, 2)).astype(np.float32)

    def run(m):
        par = W.Params(sensor=sensor, n_sectors=m, fov_deg=270.0)
        sim = oracle.OracleSim(wl.maps, np.zeros(4, np.int32), np.full(4, K, np.int32),
                               np.zeros(4, np.int32), [W.DISC], 4.0, par, RES)
        out = [sim.reset(3)]
        for t in range(25):
            out.append(sim.step(acts[t], want_final=True))
        return sim, out

    _, raw = run(0)
    for m in (K, 30, 1):
        sim, pooled = run(m)
        D = m
        for t, (a, b) in enumerate(zip(raw, pooled)):
            o_raw = (a if t == 0 else a[0]).reshape(4, K + 4)
            o_pool = (b if t == 0 else b[0]).reshape(4, D + 4)
            want = o_raw[:, :K].reshape(4, m, K // m).min(axis=2)
            np.testing.assert_array_equal(o_pool[:, :D], want)
            np.testing.assert_array_equal(o_pool[:, D:], o_raw[:, K:])
            if t:
                np.testing.assert_array_equal(a[1], b[1])
                np.testing.assert_array_equal(a[2], b[2])
                f_raw = a[3].reshape(4, K + 4)
                f_pool = b[3].reshape(4, D + 4)
                fin = (a[2] & 3) != 0
                np.testing.assert_array_equal(
                    f_pool[fin, :D], f_raw[fin, :K].reshape(-1, m, K // m).min(axis=2))
                np.testing.assert_array_equal(f_pool[fin, D:], f_raw[fin, K:])


# --------------------------------------------------------------------------
# Unicycle integration (Sec. 2.2.3): exact arc
# --------------------------------------------------------------------------
@pytest.mark.parametrize("w", [1.0, -1.5, 0.3, 1e-7])
def test_constant_omega_follows_the_circle(oracle, w):
    x0, y0, th0, v, dt = 2.0, 3.0, 0.4, 0.5, 0.1
    x, y, th = np.float32(x0), np.float32(y0), np.float32(th0)
    n = 20
    for _ in range(n):
        x, y, th = oracle.integrate(float(x), float(y), float(th), v, w, dt)
    w32 = float(np.float32(w))
    T = n * dt
    if abs(w32) > 1e-6:
        thn = th0 + w32 * T
        xe = x0 + (v / w32) * (math.sin(thn) - math.sin(th0))
        ye = y0 - (v / w32) * (math.cos(thn) - math.cos(th0))
    else:
        thn = th0 + w32 * T
        xe, ye = x0 + v * T * math.cos(th0), y0 + v * T * math.sin(th0)
    wrap = (thn + math.pi) % (2 * math.pi) - math.pi
    assert abs(float(x) - xe) < 1e-5 and abs(float(y) - ye) < 1e-5
    assert abs(float(th) - wrap) < 1e-5


def test_zero_omega_is_a_straight_line(oracle):
    x, y, th = oracle.integrate(1.0, 1.0, 0.0, 0.5, 0.0, 0.1)
    assert abs(float(x) - 1.05) < 1e-7 and float(y) == 1.0 and float(th) == 0.0


def test_heading_wraps_into_half_open_interval(oracle):
    _, _, th = oracle.integrate(1.0, 1.0, 3.1, 0.0, 1.5, 0.1)
    assert -math.pi <= float(th) < math.pi
    assert abs(float(th) - (3.25 - 2 * math.pi)) < 1e-6


# --------------------------------------------------------------------------
# Footprint collision (Sec. 2.2.3, Tables 8-9): exact, vs float64 geometry
# --------------------------------------------------------------------------
def _disc_exact(occ, xc, yc, rc):
    """float64: does the open disc meet a blocked closed cell?  Returns
    (hit, margin) where margin is the smallest |dist - r| over cells near."""
    h, w = occ.shape
    hit, margin = False, np.inf
    for j in range(int(math.floor(yc - rc)) - 1, int(math.ceil(yc + rc)) + 1):
        for i in range(int(math.floor(xc - rc)) - 1, int(math.ceil(xc + rc)) + 1):
            blocked = i < 0 or j < 0 or i >= w or j >= h or occ[j, i]
            if not blocked:
                continue
            dx = max(i - xc, xc - (i + 1), 0.0)
            dy = max(j - yc, yc - (j + 1), 0.0)
            d = math.hypot(dx, dy)
            margin = min(margin, abs(d - rc))
            hit |= d < rc
    return hit, margin


def _rect_exact(occ, xc, yc, th, hl, hw):
    """float64 separating-axis test of the open rectangle vs blocked cells."""
    h, w = occ.shape
    u = np.array([math.cos(th), math.sin(th)])
    nrm = np.array([-math.sin(th), math.cos(th)])
    c = np.array([xc, yc])
    P = np.array([c + hl * u + hw * nrm, c - hl * u + hw * nrm,
                  c - hl * u - hw * nrm, c + hl * u - hw * nrm])
    axes = [np.array([1.0, 0.0]), np.array([0.0, 1.0]), u, nrm]
    R = hl + hw + 2
    hit, margin = False, np.inf
    for j in range(int(math.floor(yc - R)), int(math.ceil(yc + R)) + 1):
        for i in range(int(math.floor(xc - R)), int(math.ceil(xc + R)) + 1):
            blocked = i < 0 or j < 0 or i >= w or j >= h or occ[j, i]
            if not blocked:
                continue
            S = np.array([[i, j], [i + 1, j], [i + 1, j + 1], [i, j + 1]], float)
            ov = min(min(max(P @ a), max(S @ a)) - max(min(P @ a), min(S @ a)) for a in axes)
            margin = min(margin, abs(ov))
            hit |= ov > 0
    return hit, margin


def test_disc_footprint_matches_exact_geometry(oracle):
    rng = np.random.default_rng(5)
    n = 0
    for trial in range(400):
        occ = (rng.random((12, 12)) < 0.2).astype(np.uint8)
        x = float(np.float32(rng.uniform(0.0, 12 * RES)))
        y = float(np.float32(rng.uniform(0.0, 12 * RES)))
        got = oracle.footprint(occ, RES, W.DISC, x, y, 0.0)
        xc = float(np.float32(np.float32(x) * np.float32(1 / RES)))
        yc = float(np.float32(np.float32(y) * np.float32(1 / RES)))
        rc = float(np.float32(np.float32(0.18) * np.float32(1 / RES)))
        want, margin = _disc_exact(occ, xc, yc, rc)
        if margin < 1e-5:
            continue
        n += 1
        assert got == want, trial
    assert n > 300


def test_rect_footprint_matches_exact_geometry(oracle):
    rng = np.random.default_rng(6)
    n = 0
    for trial in range(300):
        occ = (rng.random((24, 24)) < 0.08).astype(np.uint8)
        x = float(np.float32(rng.uniform(0.2, 24 * RES - 0.2)))
        y = float(np.float32(rng.uniform(0.2, 24 * RES - 0.2)))
        th = float(np.float32(rng.uniform(-math.pi, math.pi)))
        got = oracle.footprint(occ, RES, W.RECT, x, y, th)
        xc, yc = x / RES, y / RES
        want, margin = _rect_exact(occ, xc, yc, th, 0.35 / RES, 0.155 / RES)
        if margin < 1e-4:
            continue
        n += 1
        assert got == want, trial
    assert n > 200


def test_disc_touching_a_wall_is_not_a_collision(oracle):
    occ = np.zeros((16, 16), np.uint8)
    occ[:, 10] = 1
    # centre 3.6 cells left of the wall face at x = 10: the open disc touches
    # the face only when rc == 3.6 exactly; 1e-3 cells inside must collide
    rc = float(np.float32(np.float32(0.18) * np.float32(20.0)))
    xc_touch = 10.0 - rc
    assert not oracle.footprint(occ, RES, W.DISC, (xc_touch - 1e-3) * RES, 8.0 * RES, 0.0)
    assert oracle.footprint(occ, RES, W.DISC, (xc_touch + 1e-3) * RES, 8.0 * RES, 0.0)


# --------------------------------------------------------------------------
# Reward, goal, collision, timeout (Eq. 3, Sec. 2.2.3, Table 7)
# --------------------------------------------------------------------------
def _one_env(oracle, occ, robot=W.DISC, params=None):
    params = params or W.Params(goal_dmin=0.0, goal_dmax=1e9)
    sim = oracle.OracleSim([occ], np.zeros(1, np.int32), np.full(1, 8, np.int32),
                           np.zeros(1, np.int32), [robot], 2.0, params, RES)
    sim.reset(1)
    return sim


def _set(sim, x, y, th, gx, gy, dprev, step=0):
    f = np.array([[x, y, th, 0, 0, gx, gy, dprev]], np.float32)
    i = np.array([[step, 0]], np.int32)
    sim.set_state(1, f, i)


def test_progress_reward_and_no_flags(oracle):
    sim = _one_env(oracle, np.zeros((64, 64), np.uint8))
    _set(sim, 1.0, 1.6, 0.0, 1.5, 1.6, 0.5)
    # action (1, 0): v = 0.5 m/s, w = 0 -> moves 0.05 m towards the goal
    _, rew, done = sim.step(np.array([[1.0, 0.0]], np.float32))
    assert done[0] == 0
    assert abs(float(rew[0]) - (2.0 * 0.05 - 0.01)) < 1e-5


def test_goal_reached_inclusive_threshold(oracle):
    sim = _one_env(oracle, np.zeros((64, 64), np.uint8))
    _set(sim, 1.0, 1.6, 0.0, 1.21, 1.6, 0.21)
    _, rew, done = sim.step(np.array([[1.0, 0.0]], np.float32))
    assert done[0] & 1 and done[0] & 4 and not done[0] & 8 and not done[0] & 2
    assert abs(float(rew[0]) - (2.0 * 0.05 - 0.01 + 10.0)) < 1e-5


def test_goal_not_reached_just_outside(oracle):
    sim = _one_env(oracle, np.zeros((64, 64), np.uint8))
    _set(sim, 1.0, 1.6, 0.0, 1.30, 1.6, 0.30)
    _, rew, done = sim.step(np.array([[1.0, 0.0]], np.float32))
    assert done[0] == 0  # d = 0.25 > 0.2


def test_collision_flags_and_penalty(oracle):
    occ = np.zeros((64, 64), np.uint8)
    occ[:, 25] = 1  # wall face at x = 1.25 m
    sim = _one_env(oracle, occ)
    _set(sim, 1.06, 1.6, 0.0, 0.5, 1.6, 0.56)  # disc edge at 1.24, moves 0.05
    _, rew, done = sim.step(np.array([[1.0, 0.0]], np.float32))
    assert done[0] & 1 and done[0] & 8 and not done[0] & 4
    assert abs(float(rew[0]) - (2.0 * (0.56 - 0.61) - 0.01 - 10.0)) < 1e-5


def test_timeout_is_truncation_only(oracle):
    sim = _one_env(oracle, np.zeros((64, 64), np.uint8))
    _set(sim, 1.0, 1.6, 0.0, 2.5, 1.6, 1.5, step=199)
    _, _, done = sim.step(np.array([[-1.0, 0.0]], np.float32))  # v = 0
    assert done[0] == 2


def test_timeout_with_terminal_event_is_termination(oracle):
    sim = _one_env(oracle, np.zeros((64, 64), np.uint8))
    _set(sim, 1.0, 1.6, 0.0, 1.21, 1.6, 0.21, step=199)
    _, _, done = sim.step(np.array([[1.0, 0.0]], np.float32))
    assert done[0] == 1 | 4


def test_exclusive_reward_mode(oracle):
    sim = _one_env(oracle, np.zeros((64, 64), np.uint8),
                   params=W.Params(goal_dmin=0.0, goal_dmax=1e9, reward_mode=1))
    _set(sim, 1.0, 1.6, 0.0, 1.21, 1.6, 0.21)
    _, rew, _ = sim.step(np.array([[1.0, 0.0]], np.float32))
    assert float(rew[0]) == 10.0


def test_final_observation_is_pre_reset(oracle):
    sim = _one_env(oracle, np.zeros((64, 64), np.uint8))
    _set(sim, 1.0, 1.6, 0.0, 1.21, 1.6, 0.21)
    obs, _, done, fin = sim.step(np.array([[1.0, 0.0]], np.float32), want_final=True)
    assert done[0] & 1
    assert abs(float(fin[8]) - 0.16) < 1e-5  # goal distance at the terminal pose
    f, i, _ = sim.get_state()
    assert i[0, 0] == 0 and i[0, 1] == 1  # counters cleared, episode advanced
    assert abs(float(obs[8]) - float(f[0, 7])) < 1e-6


# --------------------------------------------------------------------------
# Reset (Sec. 2.2.3 sparse reset)
# --------------------------------------------------------------------------
def test_spawnable_cells_and_components_match_library_labelling(oracle):
    scipy_ndimage = pytest.importorskip("scipy.ndimage")
    wl = W.config_small()
    sim = oracle.OracleSim.from_workload(wl)
    occ = wl.maps[0]
    rc = float(np.float32(np.float32(0.18) * np.float32(1 / RES)))
    ok = np.zeros(occ.shape, bool)
    for j in range(occ.shape[0]):
        for i in range(occ.shape[1]):
            hit, margin = _disc_exact(occ, i + 0.5, j + 0.5, rc)
            ok[j, i] = not hit
    labels = sim.comp_labels(0)
    assert ((labels >= 0) == ok).all()
    ref, n = scipy_ndimage.label(ok)  # 4-connectivity by default
    assert n == len(np.unique(labels[labels >= 0]))
    for lab in range(1, n + 1):
        assert len(np.unique(labels[ref == lab])) == 1


def test_reset_is_deterministic_and_valid(oracle):
    wl = W.config_small()
    s1 = oracle.OracleSim.from_workload(wl)
    s2 = oracle.OracleSim.from_workload(wl)
    o1, o2 = s1.reset(42), s2.reset(42)
    assert np.array_equal(o1, o2)
    f, i, _ = s1.get_state()
    occ = wl.maps[0]
    labels = s1.comp_labels(0)
    for e in range(wl.n_envs):
        x, y, th, v, w, gx, gy, dprev = f[e]
        assert not oracle.footprint(occ, RES, W.DISC, float(x), float(y), float(th))
        ci, cj = int(x / RES), int(y / RES)
        gi, gj = int(gx / RES), int(gy / RES)
        assert labels[cj, ci] >= 0 and labels[cj, ci] == labels[gj, gi]
        assert v == 0 and w == 0 and i[e, 0] == 0 and i[e, 1] == 0
        assert -math.pi <= th < math.pi
    o3 = oracle.OracleSim.from_workload(wl).reset(43)
    assert not np.array_equal(o1, o3)


def test_goal_distance_in_band_when_possible(oracle):
    wl = W.config_throughput(n_envs=64, n_maps=2)
    sim = oracle.OracleSim.from_workload(wl)
    sim.reset(9)
    f, _, _ = sim.get_state()
    d = np.hypot(f[:, 5] - f[:, 0], f[:, 6] - f[:, 1])
    assert ((d >= 2.0 - 1e-5) & (d <= 8.0 + 1e-5)).mean() > 0.95


def test_spawn_cells_uniform_over_spawnable_list(oracle):
    occ = W.make_map(3, 24, 24, 0.10)
    n_env = 256
    sim = oracle.OracleSim([occ], np.zeros(n_env, np.int32), np.full(n_env, 4, np.int32),
                           np.zeros(n_env, np.int32), [W.DISC], 1.0,
                           W.Params(goal_dmin=0.0, goal_dmax=1e9), RES)
    counts = {}
    for seed in range(40):
        sim.reset(seed)
        f, _, _ = sim.get_state()
        for x, y in f[:, :2]:
            c = (int(x / RES), int(y / RES))
            counts[c] = counts.get(c, 0) + 1
    n_sp = sim.spawn_count(0, 0)
    assert len(counts) <= n_sp
    total = n_env * 40
    obs_c = np.array(list(counts.values()) + [0] * (n_sp - len(counts)), float)
    exp = total / n_sp
    chi2 = float(((obs_c - exp) ** 2 / exp).sum())
    dof = n_sp - 1
    assert chi2 < dof + 5 * math.sqrt(2 * dof)


# --------------------------------------------------------------------------
# Free-running invariants on the small workload
# --------------------------------------------------------------------------
def test_free_running_invariants(oracle):
    wl = W.config_small()
    sim = oracle.OracleSim.from_workload(wl)
    obs = sim.reset(1)
    acts = W.uniform_actions(1, 200, wl.n_envs)
    K = 180
    prev_ep = np.zeros(wl.n_envs, np.int64)
    for t in range(200):
        obs, rew, done = sim.step(acts[t])
        o = obs.reshape(wl.n_envs, K + 4)
        assert (o[:, :K] >= 0).all() and (o[:, :K] <= np.float32(4.0)).all()
        f, i, _ = sim.get_state()
        ended = (done & 3) != 0
        assert (i[ended, 0] == 0).all()
        assert (i[ended, 1] == prev_ep[ended] + 1).all()
        assert (i[~ended, 1] == prev_ep[~ended]).all()
        assert ((done & 1) != 0).sum() == (((done & 4) != 0) | ((done & 8) != 0)).sum()
        assert not ((done & 1) & ((done & 2) >> 1)).any()
        prev_ep = i[:, 1].astype(np.int64)


# --------------------------------------------------------------------------
# Moving discs (the workload's dynamic layer): stamping, bounce, collision
# --------------------------------------------------------------------------
def _one_env_discs(oracle, occ):
    return _one_env(oracle, occ, params=W.Params(goal_dmin=0.0, goal_dmax=1e9, n_dyn=1))


def _set_disc(sim, x, y, th, disc):
    f = np.array([[x, y, th, 0, 0, 0.5, 0.5, 1.0]], np.float32)
    i = np.array([[0, 0]], np.int32)
    sim.set_state(1, f, i, np.array([[disc]], np.float32))


STAY = np.array([[-1.0, 0.0]], np.float32)  # v = 0, w = 0


def test_disc_stamp_is_first_cell_meeting_the_open_disc(oracle):
    """A ray along +x meets the first cell whose closed square meets the open
    disc: with the disc centre at (40.0, 32.2) cells and radius 3.6, row 32
    holds x in (36.4, 43.6), so cell 36 ([36, 37]) is stamped and 35 is not;
    from x = 20 the range is 16 cells."""
    sim = _one_env_discs(oracle, np.zeros((64, 64), np.uint8))
    # beam 4 of 8 points along the heading + pi/8
    _set_disc(sim, 20.0 * RES, 32.2 * RES, -math.pi / 8, [40.0 * RES, 32.2 * RES, 0.0, 0.0])
    obs, _, done = sim.step(STAY)
    r, h, _ = sim.debug()
    assert done[0] == 0
    assert h[4] == 32 * 64 + 36
    assert abs(float(r[4]) - 16.0 * RES) < 1e-5
    assert abs(float(obs[4]) - 16.0 * RES) < 1e-5


def test_disc_with_integer_edge_stamps_the_cell_it_opens_into(oracle):
    """Exact binary32 geometry (1/16 m cells, disc radius 3 cells, centre at
    x = 40 cells): the open disc spans x in (37, 43) in its centre row, so
    cell 36, whose closed square [36, 37] touches it only at its boundary
    point, is not stamped, and the first stamped cell is 37."""
    res = 0.0625
    params = W.Params(goal_dmin=0.0, goal_dmax=1e9, n_dyn=1, dyn_radius=0.1875)
    sim = oracle.OracleSim([np.zeros((64, 64), np.uint8)], np.zeros(1, np.int32),
                           np.full(1, 8, np.int32), np.zeros(1, np.int32), [W.DISC], 2.0,
                           params, res)
    sim.reset(1)
    f = np.array([[20.0 * res, 32.5 * res, -math.pi / 8, 0, 0, 0.5, 0.5, 1.0]], np.float32)
    sim.set_state(1, f, np.array([[0, 0]], np.int32),
                  np.array([[[40.0 * res, 32.5 * res, 0.0, 0.0]]], np.float32))
    sim.step(STAY)
    r, h, _ = sim.debug()
    assert h[4] == 32 * 64 + 37
    assert abs(float(r[4]) - 17.0 * res) < 1e-5


def test_disc_bounces_off_a_wall_and_moves_in_free_space(oracle):
    """Constant velocity over dt = 0.1 s; a velocity component flips, and that
    coordinate stays, when the moved centre's cell is blocked."""
    occ = np.zeros((64, 64), np.uint8)
    occ[:, 30] = 1  # wall column: x in [1.50, 1.55] m
    sim = _one_env_discs(oracle, occ)
    _set_disc(sim, 0.5, 1.61, 0.0, [1.475, 1.61, 0.5, 0.0])  # +x into the wall
    sim.step(STAY)
    _, _, d = sim.get_state()
    assert np.allclose(d[0, 0], [1.475, 1.61, -0.5, 0.0], atol=1e-6)
    sim.step(STAY)  # now moving -x through free cells
    _, _, d = sim.get_state()
    assert np.allclose(d[0, 0], [1.425, 1.61, -0.5, 0.0], atol=1e-6)
    _set_disc(sim, 0.5, 1.61, 0.0, [1.2, 1.2, 0.0, 0.5])  # +y in free space
    sim.step(STAY)
    _, _, d = sim.get_state()
    assert np.allclose(d[0, 0], [1.2, 1.25, 0.0, 0.5], atol=1e-6)


def test_robot_collides_with_a_stamped_cell_only(oracle):
    """Robot disc (r 0.18 m) centred at x = 20 cells reaches x = 23.6 in row
    32.  A disc whose left edge is at 23.4 stamps cell 23 of row 32: the
    footprint meets it (collision).  With the edge at 24.4 the first stamped
    cell of that row is 24, which the robot does not reach: no collision."""
    sim = _one_env_discs(oracle, np.zeros((64, 64), np.uint8))
    _set_disc(sim, 1.0, 32.5 * RES, 0.0, [1.35, 32.5 * RES, 0.0, 0.0])
    _, _, done = sim.step(STAY)
    assert done[0] & 1 and done[0] & 8
    _set_disc(sim, 1.0, 32.5 * RES, 0.0, [1.40, 32.5 * RES, 0.0, 0.0])
    _, _, done = sim.step(STAY)
    assert done[0] == 0


def _pick(h, n):
    return ((h >> 32) * n) >> 32


def test_goal_falls_back_to_the_draw_nearest_the_band(oracle):
    """Sec. 2.2.3 reset with an unreachable band: in a 1.2 m room no two
    spawnable cells are 2 m apart, so all 64 goal draws miss [2, 8] m and the
    goal is the draw closest to the band (the farthest one; the first on
    ties).  Brute force over the 64 draws from the published hash and the
    component lists (both pinned above)."""
    occ = np.zeros((24, 24), np.uint8)
    params = W.Params(goal_dmin=2.0, goal_dmax=8.0)
    sim = oracle.OracleSim([occ], np.zeros(4, np.int32), np.full(4, 8, np.int32),
                           np.zeros(4, np.int32), [W.DISC], 2.0, params, RES)
    seed = 5
    sim.reset(seed)
    f, _, _ = sim.get_state()
    labels = sim.comp_labels(0).ravel()
    spawn = np.flatnonzero(labels >= 0)  # spawnable cells, ascending
    f32 = np.float32
    for e in range(4):
        cell = int(spawn[_pick(oracle.hash64(seed, e, 0, 0), len(spawn))])
        x = (f32(cell % 24) + f32(0.5)) * f32(RES)
        y = (f32(cell // 24) + f32(0.5)) * f32(RES)
        comp = spawn[labels[spawn] == labels[cell]]
        best, bx, by = np.inf, x, y
        for a in range(64):
            gc = int(comp[_pick(oracle.hash64(seed, e, 0, 2 + a), len(comp))])
            gx = (f32(gc % 24) + f32(0.5)) * f32(RES)
            gy = (f32(gc // 24) + f32(0.5)) * f32(RES)
            dx, dy = gx - x, gy - y
            d = np.sqrt(dx * dx + dy * dy)
            assert d < 2.0
            err = f32(2.0) - d
            if err < best:
                best, bx, by = err, gx, gy
        assert f[e, 0] == x and f[e, 1] == y
        assert f[e, 5] == bx and f[e, 6] == by


def test_moving_discs_drawn_at_reset_by_their_rule(oracle):
    """Moving discs at reset: disc q takes the first of 16 spawn-cell draws
    at least dyn_min_sep from the robot (else the 16th), speed U[0, max) and
    a uniform heading from one more draw; brute force from the published hash
    and the spawn list."""
    occ = np.zeros((40, 40), np.uint8)
    params = W.Params(goal_dmin=0.0, goal_dmax=1e9, n_dyn=3, dyn_min_sep=0.8,
                      dyn_speed_max=0.5)
    sim = oracle.OracleSim([occ], np.zeros(3, np.int32), np.full(3, 8, np.int32),
                           np.zeros(3, np.int32), [W.DISC], 2.0, params, RES)
    seed = 11
    sim.reset(seed)
    f, _, d = sim.get_state()
    spawn = np.flatnonzero(sim.comp_labels(0).ravel() >= 0)
    f32 = np.float32
    two_pi, pi = f32(6.2831853071795864769), f32(3.14159265358979323846)
    for e in range(3):
        x, y = f[e, 0], f[e, 1]
        for q in range(3):
            for a in range(16):
                oc = int(spawn[_pick(oracle.hash64(seed, e, 0, 1024 + 64 * q + a), len(spawn))])
                ox = (f32(oc % 40) + f32(0.5)) * f32(RES)
                oy = (f32(oc // 40) + f32(0.5)) * f32(RES)
                dx, dy = ox - x, oy - y
                if np.sqrt(dx * dx + dy * dy) >= f32(0.8):
                    break
            hv = oracle.hash64(seed, e, 0, 1024 + 64 * q + 48)
            sp = f32(hv >> 40) * f32(1.0 / 16777216.0) * f32(0.5)
            hd = f32((hv >> 8) & 0xFFFFFF) * f32(1.0 / 16777216.0) * two_pi - pi
            sh, ch = oracle.sincosf(float(hd))
            assert d[e, q, 0] == ox and d[e, q, 1] == oy
            assert d[e, q, 2] == sp * ch and d[e, q, 3] == sp * sh
