"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-derive the oracle's own formulas: each checks it against a
closed form, a brute-force restatement, an invariant of the paper's
delivery-state semantics, or central finite differences.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2606_17212_b300 import synth


def tiny_scene(mu, log_scale, quat, logit, colour, n_layers=1, res=None, u=None,
               clusters=None, sh_degree=0):
    n = len(mu)
    nc = 3 * (sh_degree + 1) ** 2
    if clusters is None:
        clusters = np.zeros(n, np.int64)
    C = int(np.max(clusters)) + 1
    order = np.argsort(clusters, kind="stable")
    assert np.all(order == np.arange(n)), "tiny scenes are built cluster-contiguous"
    offs = np.zeros(C + 1, np.int32)
    offs[1:] = np.cumsum(np.bincount(clusters, minlength=C))
    f = lambda a: np.ascontiguousarray(a, np.float32)
    R = 0 if u is None else len(u)
    K = 11 + nc
    return synth.Scene(n, C, n_layers, sh_degree, R, offs, f(mu),
                       f(np.zeros((0, n, 3)) if u is None else u), f(log_scale), f(quat),
                       f(logit), f(colour),
                       f(np.zeros((n_layers - 1, n, K)) if res is None else res))


def axis_camera(W=128, H=128, f=128.0):
    """Camera at (4,0,0) looking at the origin: image x = world y, image y = -world z."""
    return synth.ring_camera(0, 1, W, H, f)


def logit_of(o):
    return math.log(o / (1.0 - o))


def rodrigues(axis, angle):
    a = np.asarray(axis, np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * K @ K


# ---------------------------------------------------------------- closure
def test_closure_prefix_semantics():
    """Section 4 / 7.4: a layer is usable only when every layer below it is."""
    rng = np.random.default_rng(0)
    C, L = 9, 4
    for _ in range(200):
        bits = rng.uniform(size=C * L) < 0.6
        words = np.zeros(2, np.uint32)
        for b in np.nonzero(bits)[0]:
            words[b // 32] |= np.uint32(1 << (b % 32))
        d = oracle.closure(words, C, L)
        for c in range(C):
            row = bits[c * L:(c + 1) * L]
            assert 0 <= d[c] <= L
            assert row[:d[c]].all()                       # everything below is delivered
            assert d[c] == L or not row[d[c]]            # the first gap stops it
            # monotone: delivering any extra packet never lowers the depth
            for l in range(L):
                w2 = words.copy()
                b = c * L + l
                w2[b // 32] |= np.uint32(1 << (b % 32))
                assert oracle.closure(w2, C, L)[c] >= d[c]


def test_closure_of_prefix_masks_is_identity():
    rng = np.random.default_rng(1)
    d = synth.prefix_states(50, 7, 4, rng)
    masks = synth._pack(synth.depths_to_bits(d, 4))
    for s in range(50):
        assert np.array_equal(oracle.closure(masks[s], 7, 4), d[s])


# ---------------------------------------------------------------- closed forms
def _one_gaussian_at_pixel_centre(o=0.7, colour=(0.9, 0.2, 0.4), z_c=4.0):
    # ray through pixel (64,64)'s centre (64.5, 64.5): x_c/z_c = y_c/z_c = 1/256
    mu = [[4.0 - z_c, z_c / 256.0, -z_c / 256.0]]
    return mu, o, colour


def test_single_gaussian_centre_pixel_closed_form():
    """One Gaussian whose mean sits on a pixel centre: C = o c + (1 - o) bg."""
    mu, o, col = _one_gaussian_at_pixel_centre()
    sc = tiny_scene(mu, [[-2.5] * 3], [[1, 0, 0, 0]], [logit_of(o)], [col])
    bg = np.array([0.1, 0.3, 0.05])
    img, marg, _ = oracle.render(sc, np.array([1], np.uint8), 0.0, axis_camera(), bg)
    o32 = 1.0 / (1.0 + math.exp(-float(np.float32(logit_of(o)))))
    expect = o32 * np.array(col, np.float32).astype(np.float64) + (1 - o32) * bg
    assert np.allclose(img[64, 64], expect, rtol=0, atol=1e-12)
    assert not marg[64, 64]


def test_alpha_clamp_and_threshold_closed_forms():
    """S12: alpha = min(0.99, o e^power) and alpha < 1/255 is skipped.  On a pixel
    centre (power 0): o = 0.995 composites with alpha 0.99; o = 0.005 (between
    1/255 and 1/128) composites with alpha o; o = 0.003 (below 1/255) leaves bg."""
    mu, _, col = _one_gaussian_at_pixel_centre()
    bg = np.array([0.2, 0.4, 0.1])
    sig = lambda x: 1.0 / (1.0 + math.exp(-float(np.float32(x))))
    c = np.array(col, np.float32).astype(np.float64)
    for o, expect_alpha in [(0.995, 0.99), (0.005, None), (0.003, 0.0)]:
        sc = tiny_scene(mu, [[-2.5] * 3], [[1, 0, 0, 0]], [logit_of(o)], [col])
        img, _, _ = oracle.render(sc, np.array([1], np.uint8), 0.0, axis_camera(), bg)
        a = sig(logit_of(o)) if expect_alpha is None else expect_alpha
        assert np.allclose(img[64, 64], a * c + (1 - a) * bg, rtol=0, atol=1e-12), o


def test_two_gaussians_on_one_ray_closed_form():
    """Front-to-back order by depth, not by index: the nearer one is index 1."""
    o1, o2 = 0.6, 0.8
    c_far, c_near = (0.2, 0.9, 0.1), (0.7, 0.1, 0.3)
    mu = [[4.0 - 3.0, 3.0 / 256, -3.0 / 256], [4.0 - 2.0, 2.0 / 256, -2.0 / 256]]
    sc = tiny_scene(mu, [[-3.0] * 3] * 2, [[1, 0, 0, 0]] * 2, [logit_of(o2), logit_of(o1)],
                    [c_far, c_near])
    bg = np.array([0.05, 0.05, 0.5])
    img, marg, _ = oracle.render(sc, np.array([1], np.uint8), 0.0, axis_camera(), bg)
    sig = lambda x: 1.0 / (1.0 + math.exp(-float(np.float32(x))))
    a1, a2 = sig(logit_of(o1)), sig(logit_of(o2))
    c1 = np.array(c_near, np.float32).astype(float)
    c2 = np.array(c_far, np.float32).astype(float)
    expect = a1 * c1 + (1 - a1) * a2 * c2 + (1 - a1) * (1 - a2) * bg
    assert np.allclose(img[64, 64], expect, atol=1e-12)


def test_early_stop_after_thirteen_halvings():
    """Reading S13: a pixel stops before the Gaussian that would take T (1 - alpha)
    below 1e-4.  Twenty Gaussians with alpha = 1/2 on one ray: 2^-13 >= 1e-4 > 2^-14,
    so exactly 13 composite and the background enters with T = 2^-13."""
    zs = np.linspace(2.0, 3.9, 20)
    mu = [[4.0 - z, z / 256.0, -z / 256.0] for z in zs]
    col = 0.25
    sc = tiny_scene(mu, [[-3.0] * 3] * 20, [[1, 0, 0, 0]] * 20, [0.0] * 20, [[col] * 3] * 20)
    bg = np.array([1.0, 0.5, 0.0])
    img, marg, _ = oracle.render(sc, np.array([1], np.uint8), 0.0, axis_camera(), bg)
    T = 2.0 ** -13
    assert np.allclose(img[64, 64], col * (1 - T) + T * bg, rtol=0, atol=1e-9)


def _bracket_float32_logit(alpha_star):
    """Two float32 logits whose sigmoids (in FP64, as the oracle decodes them)
    lie just below and just above alpha_star."""
    sig = lambda x: 1.0 / (1.0 + math.exp(-float(x)))
    l = np.float32(logit_of(alpha_star))
    while sig(l) >= alpha_star:
        l = np.nextafter(l, np.float32(-np.inf))
    lo = l
    hi = np.nextafter(lo, np.float32(np.inf))
    while sig(hi) < alpha_star:
        hi = np.nextafter(hi, np.float32(np.inf))
    assert sig(lo) < alpha_star <= sig(hi)
    return float(lo), float(hi)


def test_derived_bound_covers_the_alpha_threshold_jump():
    """A Gaussian whose alpha straddles 1/255 on a pixel centre: the two sides
    differ by about (1/255) |c - bg| there, and the oracle's derived bound at
    that (flagged) pixel covers the jump on both sides; unflagged pixels carry
    a zero bound."""
    mu, _, col = _one_gaussian_at_pixel_centre()
    bg = np.array([0.1, 0.3, 0.05])
    out = []
    for lg in _bracket_float32_logit(1.0 / 255.0):
        sc = tiny_scene(mu, [[-2.5] * 3], [[1, 0, 0, 0]], [lg], [col])
        out.append(oracle.render(sc, np.array([1], np.uint8), 0.0, axis_camera(), bg, want_bound=True))
    (a, ma, _, ba), (b, mb, _, bb) = out
    jump = np.abs(a - b).max(axis=2)
    assert jump[64, 64] > 0.5 * (1.0 / 255.0) * 0.5          # the Gaussian is in one side only
    assert ma[64, 64] and mb[64, 64]
    # the decision jumps; the perturbation of the input moves other pixels continuously (<< 1e-7)
    assert np.all(jump <= np.minimum(ba, bb) + 1e-7)
    assert np.all(ba[~ma] == 0) and np.all(bb[~mb] == 0)


def test_derived_bound_covers_the_early_stop_jump():
    """Thirteen alpha = 1/2 Gaussians leave T = 2^-13 on one ray; a fourteenth
    whose alpha puts T (1 - alpha) on either side of 1e-4 stops the pixel or
    composites (then a fifteenth stops it).  The two sides differ by
    T alpha |c - bg| and the derived bound at the flagged pixel covers it."""
    T13 = 2.0 ** -13
    a_star = 1.0 - 1e-4 / T13
    zs = np.linspace(2.0, 3.9, 15)
    mu = [[4.0 - z, z / 256.0, -z / 256.0] for z in zs]
    bg = np.array([1.0, 0.5, 0.0])
    cols = [[0.25] * 3] * 13 + [[0.0, 0.9, 0.6], [0.3, 0.3, 0.3]]
    out = []
    for lg in _bracket_float32_logit(a_star):
        sc = tiny_scene(mu, [[-3.0] * 3] * 15, [[1, 0, 0, 0]] * 15, [0.0] * 13 + [lg, 0.0], cols)
        out.append(oracle.render(sc, np.array([1], np.uint8), 0.0, axis_camera(), bg, want_bound=True))
    (a, ma, _, ba), (b, mb, _, bb) = out
    jump = np.abs(a - b).max(axis=2)
    assert jump[64, 64] > 0.5 * T13 * a_star * 0.5
    assert ma[64, 64] and mb[64, 64]
    # the decision jumps; the perturbation of the input moves other pixels continuously (<< 1e-7)
    assert np.all(jump <= np.minimum(ba, bb) + 1e-7)


def test_derived_bound_covers_a_depth_order_swap():
    """Two Gaussians on one ray at depths one float32 ulp apart (flagged as a
    near tie): swapping their order moves the pixel by T a1 a2 |c1 - c2|, within
    the derived bound of both orders."""
    z1 = np.float32(2.5)
    z2 = np.nextafter(z1, np.float32(np.inf))
    bg = np.array([0.05, 0.05, 0.5])
    cols = [(0.7, 0.1, 0.3), (0.2, 0.9, 0.1)]
    out = []
    for za, zb in ((z1, z2), (z2, z1)):
        mu = [[4.0 - float(za), float(za) / 256.0, -float(za) / 256.0],
              [4.0 - float(zb), float(zb) / 256.0, -float(zb) / 256.0]]
        sc = tiny_scene(mu, [[-3.0] * 3] * 2, [[1, 0, 0, 0]] * 2, [logit_of(0.6), logit_of(0.8)], cols)
        out.append(oracle.render(sc, np.array([1], np.uint8), 0.0, axis_camera(), bg, want_bound=True))
    (a, ma, _, ba), (b, mb, _, bb) = out
    jump = np.abs(a - b).max(axis=2)
    assert jump[64, 64] > 0.01
    assert ma[64, 64] and mb[64, 64]
    # the decision jumps; the perturbation of the input moves other pixels continuously (<< 1e-7)
    assert np.all(jump <= np.minimum(ba, bb) + 1e-7)


def test_on_axis_covariance_and_radius_closed_form():
    """On the optical axis J = diag(f/z, f/z) | 0, so Sigma2D = (f/z)^2 [W Sigma3 W^T]_2x2 + 0.3 I."""
    rng = np.random.default_rng(5)
    cam = axis_camera()
    f, z = 128.0, 4.0
    for trial in range(20):
        ls = rng.normal(-3.0, 0.4, size=3)
        axis = rng.normal(size=3)
        ang = rng.uniform(0, np.pi)
        axis = axis / np.linalg.norm(axis)
        q = np.concatenate([[math.cos(ang / 2)], math.sin(ang / 2) * axis])
        sc = tiny_scene([[0.0, 0.0, 0.0]], [ls], [q], [0.0], [[0.5, 0.5, 0.5]])
        rec = oracle.project(sc, np.array([1], np.uint8), 0.0, cam)[0]
        Rr = rodrigues(axis, ang)
        s = np.exp(np.float32(ls).astype(np.float64))
        S3 = Rr @ np.diag(s * s) @ Rr.T
        W = cam.R_wc.astype(np.float64)
        S2 = (f / z) ** 2 * (W @ S3 @ W.T)[:2, :2] + 0.3 * np.eye(2)
        conic = np.linalg.inv(S2)
        qf = np.float32(q).astype(np.float64)
        # the float32 quaternion is the input; rebuild the exact rotation it encodes
        qf = qf / np.linalg.norm(qf)
        ang_f = 2 * math.acos(max(-1.0, min(1.0, qf[0])))
        ax_f = qf[1:] / max(np.linalg.norm(qf[1:]), 1e-300)
        Rr = rodrigues(ax_f, ang_f)
        S3 = Rr @ np.diag(s * s) @ Rr.T
        S2 = (f / z) ** 2 * (W @ S3 @ W.T)[:2, :2] + 0.3 * np.eye(2)
        conic = np.linalg.inv(S2)
        got = np.array([[rec[3], rec[4]], [rec[4], rec[5]]])
        assert np.allclose(got, conic, rtol=1e-9, atol=1e-12), (trial, got, conic)
        lam = np.linalg.eigvalsh(S2).max()
        assert rec[11] == math.ceil(3 * math.sqrt(lam))
        assert rec[1] == pytest.approx(64.0, abs=1e-12) and rec[2] == pytest.approx(64.0, abs=1e-12)


def test_neighbour_pixel_falloff_closed_form():
    """Axis-aligned Gaussian on the axis: alpha at pixel offsets follows the dilated conic."""
    cam = axis_camera()
    ls = np.array([-3.2, -2.9, -3.4], np.float32)
    o = 0.9
    sc = tiny_scene([[0.0, 0.0, 0.0]], [ls], [[1, 0, 0, 0]], [logit_of(o)], [[1.0, 1.0, 1.0]])
    img, _, _ = oracle.render(sc, np.array([1], np.uint8), 0.0, cam, np.zeros(3))
    s = np.exp(ls.astype(np.float64))
    # image x = world y, image y = -world z
    vx = (128.0 / 4.0 * s[1]) ** 2 + 0.3
    vy = (128.0 / 4.0 * s[2]) ** 2 + 0.3
    o32 = 1.0 / (1.0 + math.exp(-float(np.float32(logit_of(o)))))
    for kx, ky in [(0, 0), (1, 0), (2, 1), (-3, 0), (0, -2), (2, 2)]:
        dx, dy = 64 + kx + 0.5 - 64.0, 64 + ky + 0.5 - 64.0
        a = min(0.99, o32 * math.exp(-0.5 * (dx * dx / vx + dy * dy / vy)))
        expect = a if a >= 1 / 255 else 0.0
        assert img[64 + ky, 64 + kx, 0] == pytest.approx(expect, abs=1e-12), (kx, ky)


def _num_jacobian(cam, p):
    """Finite-difference Jacobian of the pinhole image position w.r.t. world position."""
    def proj(x):
        sc = tiny_scene([x], [[-4.0] * 3], [[1, 0, 0, 0]], [0.0], [[0.5] * 3])
        r = oracle.project(sc, np.array([1], np.uint8), 0.0, cam)[0]
        return np.array([r[1], r[2]])
    J = np.zeros((2, 3))
    h = 1e-3
    for k in range(3):
        e = np.zeros(3); e[k] = h
        hi = np.float32(p + e).astype(np.float64)   # the oracle reads float32 inputs:
        lo = np.float32(p - e).astype(np.float64)   # divide by the step actually taken
        J[:, k] = (proj(hi) - proj(lo)) / (hi[k] - lo[k])
    return J


def test_off_axis_covariance_matches_linearised_projection():
    """EWA: Sigma2D = Jp Sigma3 Jp^T + 0.3 I with Jp the derivative of the projection
    (taken here numerically), evaluated at the clamped direction outside 1.3 x FOV."""
    rng = np.random.default_rng(7)
    cam = synth.ring_camera(1, 8, 160, 120, 150.0)
    for trial in range(12):
        if trial < 8:
            p = rng.normal(0, 0.6, size=3)
        else:  # far outside the clamp on image x
            p = np.array(cam.R_wc, np.float64).T @ (np.array([5.0, 0.3, 3.0]) - cam.t_wc.astype(np.float64))
        p = np.float32(p).astype(np.float64)
        ls = np.float32(rng.normal(-3.0, 0.3, size=3))
        q = rng.normal(size=4); q /= np.linalg.norm(q)
        q = np.float32(q)
        sc = tiny_scene([p], [ls], [q], [0.0], [[0.5] * 3])
        rec = oracle.project(sc, np.array([1], np.uint8), 0.0, cam)[0]
        W = cam.R_wc.astype(np.float64)
        pc = W @ p + cam.t_wc.astype(np.float64)
        limx = 1.3 * (cam.width / 2) / cam.fx
        limy = 1.3 * (cam.height / 2) / cam.fy
        pcl = pc.copy()
        pcl[0] = np.clip(pc[0] / pc[2], -limx, limx) * pc[2]
        pcl[1] = np.clip(pc[1] / pc[2], -limy, limy) * pc[2]
        pw = W.T @ (pcl - cam.t_wc.astype(np.float64))
        Jp = _num_jacobian(cam, pw)
        qd = q.astype(np.float64); qd /= np.linalg.norm(qd)
        ang = 2 * math.acos(np.clip(qd[0], -1, 1))
        Rr = rodrigues(qd[1:] if np.linalg.norm(qd[1:]) > 0 else [1, 0, 0], ang)
        s = np.exp(ls.astype(np.float64))
        S3 = Rr @ np.diag(s * s) @ Rr.T
        S2 = Jp @ S3 @ Jp.T + 0.3 * np.eye(2)
        got = np.linalg.inv(np.array([[rec[3], rec[4]], [rec[4], rec[5]]]))
        assert np.allclose(got, S2, rtol=2e-5, atol=1e-9), (trial, got, S2)


# ---------------------------------------------------------------- brute force
def test_row_filter_equals_full_scan():
    w = synth.config("c1_plain_4k")
    sc = w.scene
    D = oracle.state_depths(w.states, sc.n_clusters, sc.n_layers)
    a = oracle.render(sc, D[0], 0.0, w.cams[0], w.bg)
    b = oracle.render(sc, D[0], 0.0, w.cams[0], w.bg, full_scan=True)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]


def test_composite_equals_product_form_brute_force():
    """Tiny scenes: C = sum_k c_k a_k prod_{j<k}(1-a_j) + prod(1-a_j) bg over the
    included list, recomputed in Python from the projected records."""
    rng = np.random.default_rng(11)
    cam = synth.ring_camera(0, 1, 32, 32, 40.0)
    for trial in range(4):
        n = 16
        mu = rng.normal(0, 0.5, size=(n, 3))
        ls = rng.normal(-2.0, 0.3, size=(n, 3))
        q = rng.normal(size=(n, 4)); q /= np.linalg.norm(q, axis=1, keepdims=True)
        lg = rng.normal(0, 1.5, size=n)
        col = rng.uniform(size=(n, 3))
        sc = tiny_scene(mu, ls, q, lg, col)
        bg = rng.uniform(size=3)
        d = np.array([1], np.uint8)
        img, marg, _ = oracle.render(sc, d, 0.0, cam, bg)
        rec = oracle.project(sc, d, 0.0, cam)
        live = np.nonzero(rec[:, 0] > 0)[0]
        order = sorted(live, key=lambda i: (np.float32(rec[i, 6]), i))
        for py in range(32):
            for px in range(32):
                alphas, cols = [], []
                for i in order:
                    r = rec[i]
                    if not (r[12] <= px <= r[13] and r[14] <= py <= r[15]):
                        continue
                    dx, dy = r[1] - (px + 0.5), r[2] - (py + 0.5)
                    pw = -0.5 * (r[3] * dx * dx + r[5] * dy * dy) - r[4] * dx * dy
                    if pw > 0:
                        continue
                    a = min(0.99, r[7] * math.exp(pw))
                    if a < 1 / 255:
                        continue
                    if np.prod([1 - x for x in alphas + [a]]) < 1e-4:
                        break
                    alphas.append(a); cols.append(r[8:11])
                acc = np.zeros(3)
                for k, (a, c) in enumerate(zip(alphas, cols)):
                    acc += np.asarray(c) * a * np.prod([1 - x for x in alphas[:k]])
                acc += np.prod([1 - x for x in alphas]) * bg
                assert np.allclose(img[py, px], acc, atol=1e-12), (trial, px, py)


def test_tile_lists_brute_force():
    """bin_tiles == per tile, every record whose pixel box meets the tile, by (depth bits, rank)."""
    rng = np.random.default_rng(3)
    n, tile, tx, ty = 300, 16, 5, 4
    W, H = 70, 60
    xlo = rng.integers(0, W, n); xhi = np.minimum(W - 1, xlo + rng.integers(0, 30, n))
    ylo = rng.integers(0, H, n); yhi = np.minimum(H - 1, ylo + rng.integers(0, 30, n))
    z = rng.uniform(0.5, 8.0, n).astype(np.float32)
    z[::7] = z[3]                       # exact depth ties
    live = rng.uniform(size=n) < 0.9
    vg = rng.integers(0, 3, n)
    keys, vals, ranges = oracle.bin_tiles(xlo, xhi, ylo, yhi, oracle.float_key(z), live, tile,
                                          tx, ty, view_group=vg)
    for v in range(3):
        for t in range(tx * ty):
            x0, y0 = (t % tx) * tile, (t // tx) * tile
            brute = [r for r in range(n) if live[r] and vg[r] == v
                     and xlo[r] <= x0 + tile - 1 and xhi[r] >= x0
                     and ylo[r] <= y0 + tile - 1 and yhi[r] >= y0]
            brute.sort(key=lambda r: (z[r], r))
            lo, hi = ranges[v * tx * ty + t]
            assert list(vals[lo:hi]) == brute


# ---------------------------------------------------------------- invariants
def _c1_like():
    w = synth.config("c1_plain_4k")
    return w.scene, w.cams[0], w.bg


def test_empty_delivery_is_background():
    sc, cam, _ = _c1_like()
    bg = np.array([0.2, 0.4, 0.6])
    img, marg, ne = oracle.render(sc, np.zeros(sc.n_clusters, np.uint8), 0.0, cam, bg)
    assert np.all(img == bg) and not marg.any() and ne == 0


def test_full_delivery_equals_complete_render_and_mse_zero():
    sc, cam, bg = _c1_like()
    words = synth.mask_words(sc.n_clusters, sc.n_layers)
    full_mask = np.full(words, 0xFFFFFFFF, np.uint32)
    a = oracle.render(sc, oracle.closure(full_mask, sc.n_clusters, sc.n_layers), 0.0, cam, bg)
    b = oracle.render(sc, oracle.full_depth(sc), 0.0, cam, bg)
    assert np.array_equal(a[0], b[0])
    mse, psnr = oracle.mse_psnr(a[0], b[0])
    assert mse == 0.0 and psnr == float("inf")


def test_mse_psnr_definition():
    a = np.zeros((4, 5, 3)); b = np.full((4, 5, 3), 0.1)
    mse, psnr = oracle.mse_psnr(a, b)
    assert mse == pytest.approx(0.01, rel=1e-12) and psnr == pytest.approx(20.0, rel=1e-12)


def test_undelivered_packets_never_change_a_pixel():
    """Packets above a gap, and the residual data of undelivered layers, are invisible."""
    rng = np.random.default_rng(21)
    w = synth.config("c2_dynamic_250k", scale=0.02, n_states=4)
    sc, cam = w.scene, w.cams[0]
    C, L = sc.n_clusters, sc.n_layers
    d = rng.integers(0, L, size=C)        # at most L-1: layer d is a gap
    bits = synth.depths_to_bits(d[None], L)[0]
    base_mask = synth._pack(bits[None])[0]
    ref = oracle.render(sc, oracle.closure(base_mask, C, L), 0.3, cam, w.bg)
    # deliver random packets strictly above each cluster's gap
    extra = bits.copy()
    for c in range(C):
        for l in range(d[c] + 1, L):
            extra[c * L + l] = rng.uniform() < 0.7
    m2 = synth._pack(extra[None])[0]
    got = oracle.render(sc, oracle.closure(m2, C, L), 0.3, cam, w.bg)
    assert np.array_equal(ref[0], got[0])
    # poison the residual layers no cluster uses
    res = sc.res.copy()
    cl = sc.cluster_of()
    for i in range(sc.n):
        res[d[cl[i]]:, i, :] = np.nan    # layers l >= d (index l-1 >= d-1 ... keep l < d)
        if d[cl[i]] >= 1:
            res[:d[cl[i]] - 1, i, :] = sc.res[:d[cl[i]] - 1, i, :]
    poisoned = synth.Scene(**{**sc.__dict__, "res": res})
    got2 = oracle.render(poisoned, oracle.closure(base_mask, C, L), 0.3, cam, w.bg)
    assert np.array_equal(ref[0], got2[0])


def test_decode_is_base_plus_delivered_refinements():
    """Rendering at depth d equals rendering a base-only scene whose base already
    holds base + res_1 + ... + res_{d-1} (Section 3)."""
    w = synth.config("c2_dynamic_250k", scale=0.02, n_states=1)
    sc, cam = w.scene, w.cams[0]
    for d in range(1, sc.n_layers + 1):
        depth = np.full(sc.n_clusters, d, np.uint8)
        ref, marg, _ = oracle.render(sc, depth, 0.0, cam, w.bg)
        acc = sc.res[:d - 1].astype(np.float64).sum(0)
        nb = synth.Scene(sc.n, sc.n_clusters, 1, sc.sh_degree, sc.temporal_rank,
                         sc.cluster_offsets,
                         (sc.mu0 + acc[:, 0:3]).astype(np.float32), sc.u,
                         (sc.log_scale + acc[:, 3:6]).astype(np.float32),
                         (sc.quat + acc[:, 6:10]).astype(np.float32),
                         (sc.opacity_logit + acc[:, 10]).astype(np.float32),
                         (sc.colour + acc[:, 11:]).astype(np.float32),
                         np.zeros((0, sc.n, sc.res_width), np.float32))
        got, marg2, _ = oracle.render(nb, np.ones(sc.n_clusters, np.uint8), 0.0, cam, w.bg)
        ok = ~(marg | marg2)
        assert ok.mean() > 0.98
        assert np.abs(got - ref)[ok].max() < 1e-4


def test_temporal_basis_order_and_period():
    """Eq. 1 basis b1 = cos 2 pi t, b2 = sin 2 pi t: t = 0 moves by u1, t = 1/4 by u2,
    and t + 1 renders like t."""
    w = synth.config("c2_dynamic_250k", scale=0.02, n_states=1)
    sc, cam = w.scene, w.cams[0]
    depth = np.ones(sc.n_clusters, np.uint8)
    for t, k in [(0.0, 0), (0.25, 1)]:
        ref, m1, _ = oracle.render(sc, depth, t, cam, w.bg)
        moved = synth.Scene(**{**sc.__dict__, "temporal_rank": 0,
                               "u": np.zeros((0, sc.n, 3), np.float32),
                               "mu0": (sc.mu0.astype(np.float64) + sc.u[k]).astype(np.float32)})
        got, m2, _ = oracle.render(moved, depth, 0.0, cam, w.bg)
        ok = ~(m1 | m2)
        assert np.abs(got - ref)[ok].max() < 1e-4
    a, ma, _ = oracle.render(sc, depth, 0.375, cam, w.bg)
    b, mb, _ = oracle.render(sc, depth, 1.375, cam, w.bg)
    ok = ~(ma | mb)
    assert np.abs(a - b)[ok].max() < 1e-9


# ---------------------------------------------------------------- SH
def test_sh_basis_orthonormal_by_quadrature():
    """Gauss-Legendre in cos(theta) x uniform phi integrates products exactly to degree 6."""
    xs, ws = np.polynomial.legendre.leggauss(12)
    nphi = 24
    G = np.zeros((16, 16))
    for z, wz in zip(xs, ws):
        for k in range(nphi):
            ph = 2 * np.pi * k / nphi
            r = math.sqrt(1 - z * z)
            Y = oracle.sh_basis([r * math.cos(ph), r * math.sin(ph), z], 3)
            G += wz * (2 * np.pi / nphi) * np.outer(Y, Y)
    assert np.allclose(G, np.eye(16), atol=1e-12)


def test_sh_degree0_equivalence():
    """SH3 colour with only the DC coefficient = SH0 colour Y00 k0 + 0.5."""
    w = synth.config("c1_plain_4k")
    sc = w.scene
    rng = np.random.default_rng(4)
    k0 = rng.normal(0, 0.5, size=(sc.n, 3)).astype(np.float32)
    sh = np.zeros((sc.n, 48), np.float32); sh[:, :3] = k0
    sc3 = synth.Scene(**{**sc.__dict__, "sh_degree": 3, "colour": sh,
                         "res": np.zeros((1, sc.n, 59), np.float32)})
    Y00 = 0.5 / math.sqrt(math.pi)
    sc0 = synth.Scene(**{**sc.__dict__, "colour": (Y00 * k0.astype(np.float64) + 0.5).astype(np.float32),
                         "res": np.zeros((1, sc.n, 14), np.float32)})
    d = oracle.full_depth(sc)
    a, ma, _ = oracle.render(sc3, d, 0.0, w.cams[0], w.bg)
    b, mb, _ = oracle.render(sc0, d, 0.0, w.cams[0], w.bg)
    ok = ~(ma | mb)
    assert np.abs(a - b)[ok].max() < 1e-6


# ---------------------------------------------------------------- adjoint
def _fd_case(sh_degree=0, n=256, seed=9):
    if sh_degree == 0:
        w = synth.config("c3_fwdbwd_250k", scale=0.004, n_states=2)
        sc = w.scene
    else:
        sc = synth.make_scene(n, 8, 4, seed=seed, sh_degree=3)
        w = synth.config("c3_fwdbwd_250k", scale=0.004, n_states=2)
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(sc.n, size=min(n, sc.n), replace=False))
    sub = sc.subset(idx)
    cam = synth.ring_camera(1, 8, 48, 40, 60.0)
    return sub, cam


def _loss(sc, depth, t, cam, bg, target):
    img, _, _ = oracle.render(sc, depth, t, cam, bg)
    return float(np.mean((img - target) ** 2)), img


@pytest.mark.parametrize("sh_degree", [0, 3])
def test_adjoint_matches_central_differences(sh_degree):
    """Gradient of L = mean((I - target)^2) vs central differences, h = 1e-3
    (parameters whose FD at h and h/2 disagree by >1e-2 straddle a threshold
    and are excluded and counted)."""
    sc, cam = _fd_case(sh_degree)
    rng = np.random.default_rng(17)
    depth = rng.integers(1, sc.n_layers + 1, size=sc.n_clusters).astype(np.uint8)
    depth[0] = sc.n_layers
    t = 0.3125
    bg = np.array([0.1, 0.2, 0.3])
    target = rng.uniform(size=(cam.height, cam.width, 3))
    L0, img = _loss(sc, depth, t, cam, bg, target)
    dL = 2.0 * (img - target) / img.size
    g = oracle.render_backward(sc, depth, t, cam, bg, dL)
    checked = excluded = 0
    names = ["mu0", "u", "log_scale", "quat", "opacity_logit", "colour", "res"]
    cl = sc.cluster_of()
    for name in names:
        arr = getattr(sc, name)
        G = g[name]
        flat = arr.reshape(-1)
        scale = max(np.abs(G).max(), 1e-12)
        cand = np.argsort(-np.abs(G).reshape(-1))[:12]
        cand = np.concatenate([cand, rng.choice(flat.size, size=8, replace=False)])
        for j in cand:
            def fd(h):
                orig = flat[j]
                flat[j] = np.float32(orig + h); lp, _ = _loss(sc, depth, t, cam, bg, target); up = float(flat[j])
                flat[j] = np.float32(orig - h); lm, _ = _loss(sc, depth, t, cam, bg, target); dn = float(flat[j])
                flat[j] = orig
                return (lp - lm) / (up - dn)
            f1, f2 = fd(1e-3), fd(5e-4)
            if abs(f1 - f2) > 1e-2 * max(abs(f1), abs(f2), 1e-3 * scale):
                excluded += 1
                continue
            checked += 1
            assert abs(G.reshape(-1)[j] - f2) <= 2e-3 * scale + 1e-9, (name, j, G.reshape(-1)[j], f1, f2)
    assert checked >= 60 and excluded <= checked // 4, (checked, excluded)


def test_undelivered_residuals_get_exactly_zero_gradient():
    sc, cam = _fd_case(0)
    depth = np.array([1, 2] + [4] * (sc.n_clusters - 2), np.uint8)
    rng = np.random.default_rng(2)
    dL = rng.normal(size=(cam.height, cam.width, 3))
    g = oracle.render_backward(sc, depth, 0.1, cam, np.zeros(3), dL)
    cl = sc.cluster_of()
    for i in range(sc.n):
        d = depth[cl[i]]
        assert np.all(g["res"][d - 1:, i] == 0.0)


@pytest.mark.parametrize("tile", [16, 32])
def test_footprint_tiles_are_where_a_lone_gaussian_changes_the_image(tile):
    """Tile membership from the footprint, pinned to the compositing: rendered
    alone over a background it never matches, a Gaussian changes exactly the
    pixels it composites at, so the tiles holding a changed pixel must include
    every tile footprint_tiles marks sure and lie within its sure and marginal
    tiles."""
    rng = np.random.default_rng(8)
    cam = synth.ring_camera(0, 1, 96, 80, 110.0)
    bg = np.array([-1.0, -1.0, -1.0])
    tiles_x = -(-96 // tile)
    n_sure = 0
    for k in range(60):
        mu = rng.normal(0, 0.6, size=(1, 3))
        ls = rng.normal(-2.8, 0.5, size=(1, 3))
        q = rng.normal(size=(1, 4)); q /= np.linalg.norm(q, axis=1, keepdims=True)
        lg = rng.normal(-1.0, 2.5, size=1)
        sc = tiny_scene(mu, ls, q, lg, rng.uniform(0.2, 1.0, size=(1, 3)))
        img, _, _ = oracle.render(sc, np.array([1], np.uint8), 0.0, cam, bg)
        ys, xs = np.nonzero(np.any(img != bg, axis=2))
        changed = set((ys // tile * tiles_x + xs // tile).tolist())
        g, tl, m = oracle.footprint_tiles(sc, np.array([1], np.uint8), 0.0, cam, tile)
        assert np.all(g == 0)
        sure, maybe = set(tl[~m].tolist()), set(tl[m].tolist())
        assert sure <= changed <= sure | maybe, k
        n_sure += len(sure)
    assert n_sure > 20


def test_row_band_render_equals_full_render_rows():
    """The row-band render used to time the oracle on a bounded sample gives
    exactly the rows of the whole-image render."""
    w = synth.config("c1_plain_4k")
    D = oracle.closure(w.states.masks[0], w.scene.n_clusters, w.scene.n_layers)
    full, marg, ne = oracle.render(w.scene, D, 0.0, w.cams[0], w.bg)
    band, bmarg, bne = oracle.render_rows(w.scene, D, 0.0, w.cams[0], w.bg, 40, 57)
    assert np.array_equal(band, full[40:57]) and np.array_equal(bmarg, marg[40:57])
    parts = [oracle.render_rows(w.scene, D, 0.0, w.cams[0], w.bg, y, min(y + 32, 128))[2] for y in range(0, 128, 32)]
    assert sum(parts) == ne


def test_utility_stats_hand_computed():
    """Eq. 4 on values computed by hand: Delta = 1..10 gives mean 5.5, population
    std sqrt(8.25), Q_0.1 at position 0.9 between 1 and 2 = 1.9."""
    import math
    mean, qv, std, u = oracle.utility_stats(np.arange(10, 0, -1, dtype=float))   # order must not matter
    assert mean == 5.5 and abs(qv - 1.9) < 1e-15 and abs(std - math.sqrt(8.25)) < 1e-15
    assert abs(u - (0.75 * 5.5 + 0.25 * 1.9) / (1 + 0.05 * math.sqrt(8.25))) < 1e-15
    # constant contributions: every statistic equals the value, utility too
    assert oracle.utility_stats(np.full(7, -0.3)) == pytest.approx((-0.3, -0.3, 0.0, -0.3), abs=1e-15)
    # one context: the quantile is that value
    assert oracle.utility_stats(np.array([2.0]), alpha=0.5, beta=1.0) == (2.0, 2.0, 0.0, 2.0)
    # q = 0 is the minimum, q = 1 the maximum
    assert oracle.utility_stats(np.array([3.0, -1.0, 2.0]), q=0.0)[1] == -1.0
    assert oracle.utility_stats(np.array([3.0, -1.0, 2.0]), q=1.0)[1] == 3.0


def test_group_utility_special_cases():
    """Eq. 3: a packet of a cluster with no Gaussian in view contributes exactly
    0 in every context; adding a base packet to the empty state changes D from
    the closed form mean((bg - I)^2) (an empty delivery renders the background)."""
    w = synth.config("c1_plain_4k")
    sc, cam, bg = w.scene, w.cams[0], np.array([0.2, 0.1, 0.0], np.float32)
    # a cluster entirely off-screen: push its Gaussians far behind the camera
    sc2 = synth.Scene(**{f.name: getattr(sc, f.name) for f in __import__("dataclasses").fields(sc)})
    sc2.mu0 = sc.mu0.copy()
    c_off = 3
    lo, hi = sc.cluster_offsets[c_off], sc.cluster_offsets[c_off + 1]
    sc2.mu0[lo:hi] = cam.R_wc.T @ (np.array([0.0, 0.0, -50.0]) - cam.t_wc)   # z = -50 in camera space
    groups = np.array([[c_off, 0], [c_off, 1], [1, 0]], np.int32)
    rng = np.random.default_rng(7)
    M = 3
    ctx = synth.group_contexts(groups, M, sc.n_clusters, sc.n_layers, rng)
    delta, stats = oracle.group_utility(sc2, ctx, groups, M, cam, 0.0, bg)
    assert np.all(delta[0] == 0.0) and np.all(delta[1] == 0.0)
    assert np.all(stats[0] == 0.0)
    # empty state vs base of cluster 1 alone
    empty = np.zeros((1, ctx.shape[1]), np.uint32)
    d, _ = oracle.group_utility(sc2, empty, groups[2:3], 1, cam, 0.0, bg)
    full, _, _ = oracle.render(sc2, oracle.full_depth(sc2), 0.0, cam, bg)
    depth = np.zeros(sc.n_clusters, np.uint8); depth[1] = 1
    one, _, _ = oracle.render(sc2, depth, 0.0, cam, bg)
    d_empty = np.mean((bg.astype(np.float64)[None, None, :] - full) ** 2)
    assert d[0, 0] == pytest.approx(d_empty - np.mean((one - full) ** 2), rel=1e-12)
    # contexts hold cluster c at exactly depth l, others anything
    D = np.stack([oracle.closure(m, sc.n_clusters, sc.n_layers) for m in ctx])
    for g, (c, l) in enumerate(groups):
        assert np.all(D[g * M:(g + 1) * M, c] == l)


# ------------------------------------------------------------ Eq. 2 objective
def test_ssim_window_and_identities():
    """The window is the normalised sampled Gaussian (ratio of neighbours
    exp(-(2k+1)/(2 sigma^2)) about the centre), SSIM(x, x) = 1 exactly, SSIM is
    symmetric, and on constant images the interior value (window inside the
    image) is the closed form (2ab + C1)/(a^2 + b^2 + C1)."""
    g = oracle.ssim_window()
    assert len(g) == 11 and abs(g.sum() - 1.0) < 1e-15 and np.allclose(g, g[::-1], rtol=0, atol=0)
    for k in range(5):
        assert g[6 + k] / g[5 + k] == pytest.approx(np.exp(-(2 * k + 1) / (2 * 1.5 ** 2)), rel=1e-13)
    rng = np.random.default_rng(3)
    x = rng.uniform(size=(19, 23, 3)); y = rng.uniform(size=(19, 23, 3))
    assert oracle.ssim(x, x) == 1.0
    assert oracle.ssim(x, y) == pytest.approx(oracle.ssim(y, x), rel=1e-14)
    assert oracle.ssim(x, y) < 1.0
    a, b = 0.3, 0.7
    f = oracle.ssim(np.full((20, 24, 3), a), np.full((20, 24, 3), b), want_grad="map")
    c1 = 0.01 ** 2
    assert np.allclose(f[5:-5, 5:-5], (2 * a * b + c1) / (a * a + b * b + c1), rtol=1e-12, atol=0)


def _fd(fun, x, idx, h=1e-6):
    xp = x.copy(); xp[idx] += h
    xm = x.copy(); xm[idx] -= h
    return (fun(xp) - fun(xm)) / (2 * h)


def test_objective_gradient_finite_differences_and_special_cases():
    """Every term of Eq. 2 (mean D, CVaR tail, temporal change F, prefix
    hinge M, complete-prefix anchor) against central differences of the
    oracle's own value; images equal to their references give L = 0 and no
    gradient; a prefix pair whose distortion falls adds nothing."""
    rng = np.random.default_rng(5)
    S, H, W = 6, 12, 14
    refs = rng.uniform(size=(2, H, W, 3))
    ridx = np.array([0, 1, 0, 1, 0, 1])
    imgs = refs[ridx] + rng.normal(0, [0.05, 0.1, 0.2, 0.02, 0.3, 0.15], size=(H, W, 3, S)).transpose(3, 0, 1, 2)
    kw = dict(pairs_t=[(0, 2), (1, 3)], pairs_m=[(0, 4), (4, 0), (1, 5)], anchors=[3, 5], cvar_q=0.34)
    L, D, grad = oracle.objective(imgs, refs, ridx, **kw)
    assert np.sum(D > D[3]) >= 1
    for idx in [(0, 3, 4, 1), (2, 0, 0, 0), (4, 11, 13, 2), (5, 6, 7, 1), (3, 5, 5, 0)]:
        fd = _fd(lambda z: oracle.objective(z, refs, ridx, **kw)[0], imgs, idx)
        assert fd == pytest.approx(grad[idx], rel=1e-5, abs=1e-11), idx
    # the definition term by term on these values
    k = int(np.ceil(0.34 * S))
    cvar = np.sort(D)[::-1][:k].mean()
    M = (max(0, D[4] - D[0]) + max(0, D[0] - D[4]) + max(0, D[5] - D[1])) / 3
    F = np.mean((((imgs[2] - imgs[0]) - (refs[0] - refs[0])) ** 2)) / 2 + \
        np.mean((((imgs[3] - imgs[1]) - (refs[1] - refs[1])) ** 2)) / 2
    assert L == pytest.approx(D.mean() + 0.30 * cvar + 0.10 * F + 2.0 * M + 0.5 * (D[3] + D[5]) / 2, rel=1e-12)
    # perfect renders: zero objective, zero gradient
    L0, D0, g0 = oracle.objective(refs[ridx], refs, ridx, **kw)
    assert L0 == 0.0 and np.all(D0 == 0.0) and np.abs(g0).max() < 1e-12   # SSIM is stationary at x = y


# ------------------------------------------------------------ cluster affine (Eq. 1)
def _affine_case():
    import dataclasses
    w = synth.config("c3_fwdbwd_250k", scale=0.004, n_states=1)
    sc = w.scene
    cam = synth.ring_camera(1, 8, 48, 40, 60.0)
    D = oracle.full_depth(sc)
    return sc, cam, D, dataclasses


def test_cluster_affine_special_cases():
    """Identity keyframes change nothing; a uniform scale by 2 equals rendering
    means doubled (exact in FP32); at a keyframe time only that keyframe counts,
    half way between two keyframes their average."""
    sc, cam, D, dc = _affine_case()
    bg = np.zeros(3)
    base, _, _ = oracle.render(sc, D, 0.3, cam, bg)
    C = sc.n_clusters
    eye = np.tile(np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], np.float32), (C, 4, 1))
    ident, _, _ = oracle.render(dc.replace(sc, affine=eye), D, 0.3, cam, bg)
    assert np.abs(ident - base).max() < 1e-12
    two = eye.copy(); two[..., [0, 5, 10]] = 2.0
    scaled, _, _ = oracle.render(dc.replace(sc, affine=two), D, 0.3, cam, bg)
    ref2, _, _ = oracle.render(dc.replace(sc, mu0=(sc.mu0 * 2).astype(np.float32)), D, 0.3, cam, bg)
    assert np.abs(scaled - ref2).max() < 1e-12
    # keyframes on a 2^-10 grid, so that the average of two is exact in FP32
    A = (np.round(synth.cluster_affine(C, 4, np.random.default_rng(9)) * 1024) / 1024).astype(np.float32)
    at_key, _, _ = oracle.render(dc.replace(sc, affine=A), D, 0.5, cam, bg)          # t = 2/4: keyframe 2
    one, _, _ = oracle.render(dc.replace(sc, affine=A[:, 2:3].copy()), D, 0.5, cam, bg)
    assert np.abs(at_key - one).max() < 1e-12
    mid, _, _ = oracle.render(dc.replace(sc, affine=A), D, 0.125, cam, bg)            # half way 0 -> 1
    avg = (0.5 * A[:, 0:1].astype(np.float64) + 0.5 * A[:, 1:2].astype(np.float64))
    avg32 = avg.astype(np.float32)
    assert np.array_equal(avg32.astype(np.float64), avg)                               # exactly representable?
    mid_ref, _, _ = oracle.render(dc.replace(sc, affine=avg32), D, 0.125, cam, bg)
    assert np.abs(mid - mid_ref).max() < 1e-12


def test_cluster_affine_gradient_finite_differences():
    """dL/dA (keyframes, between two of them) and dL/dmubar through A against
    central differences on a sparse scene; parameters whose differences at h
    and h/2 disagree straddle a threshold and are excluded and counted."""
    import dataclasses
    sc, cam = _fd_case(0)
    A = synth.cluster_affine(sc.n_clusters, 3, np.random.default_rng(4))
    sca = dataclasses.replace(sc, affine=A)
    D = oracle.full_depth(sca)
    t = 0.2                                                  # between keyframes 0 and 1 (w = 0.6)
    rng = np.random.default_rng(1)
    bg = np.array([0.1, 0.0, 0.2])
    target = rng.uniform(size=(cam.height, cam.width, 3))
    _, img = _loss(sca, D, t, cam, bg, target)
    g = oracle.render_backward(sca, D, t, cam, bg, 2.0 * (img - target) / img.size)
    checked = excluded = 0
    for name, arr in (("affine", A), ("mu0", sca.mu0)):
        G = g[name].reshape(-1)
        flat = arr.reshape(-1)
        scale = max(np.abs(G).max(), 1e-12)
        cand = np.argsort(-np.abs(G))[:16]
        for j in cand:
            def fd(h):
                orig = flat[j]
                flat[j] = np.float32(orig + h); lp, _ = _loss(sca, D, t, cam, bg, target); up = float(flat[j])
                flat[j] = np.float32(orig - h); lm, _ = _loss(sca, D, t, cam, bg, target); dn = float(flat[j])
                flat[j] = orig
                return (lp - lm) / (up - dn)
            f1, f2 = fd(1e-4), fd(5e-5)     # cluster parameters move many Gaussians: small steps
            if abs(f1 - f2) > 1e-2 * max(abs(f1), abs(f2), 1e-3 * scale):
                excluded += 1
                continue
            checked += 1
            assert abs(G[j] - f2) <= 2e-3 * scale + 1e-9, (name, j, G[j], f1, f2)
    assert checked >= 16 and excluded <= checked // 2, (checked, excluded)
    # keyframes the state's time does not touch get nothing
    assert np.all(g["affine"][:, 2] == 0.0)


# ------------------------------------------------------------ quantized refinements
def _quant_case():
    import dataclasses
    sc, cam = _fd_case(0)
    q, step = synth.quantize_residuals(sc)
    deq = (q.astype(np.float32) * step[:, None, :]).astype(np.float32)    # exact: steps are powers of two
    return sc, cam, q, step, deq, dataclasses


def test_quantized_refinement_decode_special_cases():
    """Decoding symbols (mode 1) equals the float refinements q * step; fake
    quantization (mode 2) equals rendering its dequantized values, and is the
    identity on values already on the step grid."""
    sc, cam, q, step, deq, dc = _quant_case()
    D = np.array([sc.n_layers] * sc.n_clusters, np.uint8)
    D[1] = 2
    bg = np.zeros(3)
    ref, _, _ = oracle.render(dc.replace(sc, res=deq), D, 0.4, cam, bg)
    m1, _, _ = oracle.render(dc.replace(sc, res_q=q, res_step=step, res_mode=1), D, 0.4, cam, bg)
    assert np.abs(m1 - ref).max() < 1e-12
    m2grid, _, _ = oracle.render(dc.replace(sc, res=deq, res_step=step, res_mode=2), D, 0.4, cam, bg)
    assert np.abs(m2grid - ref).max() < 1e-12
    m2, _, _ = oracle.render(dc.replace(sc, res_step=step, res_mode=2), D, 0.4, cam, bg)
    v = np.clip(np.rint(sc.res / step[:, None, :]), -32768, 32767)   # float32 division, as the definition
    ref2, _, _ = oracle.render(dc.replace(sc, res=(v * step[:, None, :]).astype(np.float32)), D, 0.4, cam, bg)
    assert np.abs(m2 - ref2).max() < 1e-12
    assert np.abs(m2 - oracle.render(sc, D, 0.4, cam, bg)[0]).max() > 0     # the quantization shows


def test_quantized_refinement_straight_through_gradients():
    """Mode 2: the refinement gradient is the gradient at the dequantized values
    (straight through the rounding), zero where the symbol clips; the step
    gradient is the sum of g (v - x / step), or g v where clipped."""
    sc, cam, q, step, deq, dc = _quant_case()
    res = sc.res.copy()
    res[0, 5, 11] = 40000.0 * step[0, 11]                   # clips at 32767
    scq = dc.replace(sc, res=res, res_step=step, res_mode=2)
    D = oracle.full_depth(sc)
    rng = np.random.default_rng(6)
    dL = rng.normal(size=(cam.height, cam.width, 3))
    g2 = oracle.render_backward(scq, D, 0.4, cam, np.zeros(3), dL)
    v = np.clip(np.rint(res / step[:, None, :]), -32768, 32767)
    g0 = oracle.render_backward(dc.replace(sc, res=(v * step[:, None, :]).astype(np.float32)), D, 0.4, cam,
                                np.zeros(3), dL)
    clipped = np.abs(res / step[:, None, :]) > 32767.5
    assert clipped.sum() == 1 and g2["res"][0, 5, 11] == 0.0
    assert np.allclose(g2["res"][~clipped], g0["res"][~clipped], rtol=1e-12, atol=1e-15)
    lsq = np.where(clipped, v, v - res / step[:, None, :])
    assert np.allclose(g2["res_step"], (g0["res"] * lsq).sum(axis=1), rtol=1e-9, atol=1e-14)
    assert np.abs(g2["res_step"]).max() > 0


def test_ssim_value_by_direct_window_sums():
    """SSIM at interior pixels from direct 2-D window sums (C1 = 1e-4, C2 = 9e-4)
    on an anti-correlated pair, where both constants matter."""
    rng = np.random.default_rng(12)
    y = rng.uniform(size=(24, 26, 3))
    x = 0.9 - 0.8 * y + 0.05 * rng.normal(size=y.shape)
    f = oracle.ssim(x, y, want_grad="map")
    a = np.arange(11) - 5.0
    w2 = np.exp(-(a[:, None] ** 2 + a[None, :] ** 2) / (2 * 1.5 ** 2))
    w2 /= w2.sum()
    for r, c in [(5, 5), (12, 13), (18, 20)]:
        for ch in range(3):
            px, py = x[r - 5:r + 6, c - 5:c + 6, ch], y[r - 5:r + 6, c - 5:c + 6, ch]
            mx, my = (w2 * px).sum(), (w2 * py).sum()
            sxx = (w2 * px * px).sum() - mx * mx
            syy = (w2 * py * py).sum() - my * my
            sxy = (w2 * px * py).sum() - mx * my
            exp = ((2 * mx * my + 1e-4) * (2 * sxy + 9e-4)) / ((mx * mx + my * my + 1e-4) * (sxx + syy + 9e-4))
            assert f[r, c, ch] == pytest.approx(exp, rel=1e-12), (r, c, ch)


def _golden_weights():
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "locked_weights.txt")
    out = {}
    with open(path) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()[:2]
                out[k] = float(v)
    return out


def test_locked_weights_are_the_papers():
    """The defaults of the oracle and of the binding are the weights the paper fixes
    (Eq. 2 and Eq. 4); the rate weight is 0, so the objective has no rate term."""
    import inspect
    from paper_2606_17212_b300 import dgs
    w = _golden_weights()
    assert w["lambda_r"] == 0.0
    obj = inspect.signature(oracle.objective).parameters
    for k in ("ssim_weight", "lambda_c", "cvar_q", "lambda_t", "lambda_m", "anchor_weight"):
        assert obj[k].default == w[k], k
        assert dgs.OBJECTIVE_DEFAULTS[k] == w[k], k
    for sig in (inspect.signature(oracle.utility_stats).parameters,
                inspect.signature(oracle.group_utility).parameters,
                inspect.signature(dgs.Renderer.group_utility).parameters):
        assert (sig["alpha"].default, sig["beta"].default, sig["q"].default) == \
            (w["utility_alpha"], w["utility_beta"], w["utility_q"])
    assert (oracle.SSIM_C1, oracle.SSIM_C2) == pytest.approx((w["ssim_c1"], w["ssim_c2"]), rel=1e-15)
