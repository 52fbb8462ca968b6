"""FP64 CPU oracle of delivery-state rendering (test infrastructure only).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never does.  It shares
no code with the CUDA library; inputs come from the seeded generators.

Functions and the passages of the paper they follow:

* :func:`closure` -- Section 4 ("dependencies are enforced after delivery, then
  converted to cluster-layer masks") and Section 7.4 (a chunk is usable only
  when its whole dependency closure is usable): delivered depth per cluster.
* :func:`project` -- Section 3 (base plus refinements) and Eq. 1 (low-rank
  temporal position model, cluster affine = identity) followed by the EWA
  projection of the external rasterizer the paper uses (Section 6).
* :func:`render` -- front-to-back alpha compositing of one delivery state;
  :func:`render_states` repeats it per state (the batched renderer of Section 6
  must equal this serial evaluation).
* :func:`mse_psnr` -- the distortion D of Eq. 3 taken as MSE (FP64) and PSNR.
* :func:`render_backward` -- adjoint of :func:`render`.
* :func:`bin_tiles` -- tile lists ordered by the 64-bit (tile | depth) key with
  ties by Gaussian index then variant (an integer function).
* :func:`group_utility` -- Eq. 3 marginal contribution of each completion group
  over its sampled contexts and the risk-adjusted utility of Eq. 4.

Every function is pinned by the CPU tests against closed forms, brute force,
invariants and finite differences (see ``tests/test_oracle_pins.py``).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dgs_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

REC_FIELDS = ("valid", "mx", "my", "A", "B", "C", "z", "o", "r", "g", "b", "radius",
              "xlo", "xhi", "ylo", "yhi", "marg_rad", "marg_near", "z32", "d")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, OpenMP over pixels)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-Wall",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _OScene(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_clusters", ctypes.c_int32),
                ("n_layers", ctypes.c_int32), ("sh_degree", ctypes.c_int32),
                ("temporal_rank", ctypes.c_int32),
                ("cluster_offsets", ctypes.c_void_p), ("mu0", ctypes.c_void_p),
                ("u", ctypes.c_void_p), ("log_scale", ctypes.c_void_p),
                ("quat", ctypes.c_void_p), ("opacity_logit", ctypes.c_void_p),
                ("colour", ctypes.c_void_p), ("res", ctypes.c_void_p),
                ("affine", ctypes.c_void_p), ("affine_T", ctypes.c_int32),
                ("res_q", ctypes.c_void_p), ("res_step", ctypes.c_void_p), ("res_mode", ctypes.c_int32)]


class _OCam(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3),
                ("fx", ctypes.c_double), ("fy", ctypes.c_double),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class _OEps(ctypes.Structure):
    _fields_ = [("box_px", ctypes.c_double), ("rel_alpha", ctypes.c_double),
                ("rel_T", ctypes.c_double), ("rel_depth", ctypes.c_double),
                ("rel_radius", ctypes.c_double), ("near_abs", ctypes.c_double)]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        lib.o_closure.argtypes = [ctypes.c_int, ctypes.c_int, P, P]
        lib.o_project.argtypes = [ctypes.POINTER(_OScene), P, ctypes.c_double, ctypes.POINTER(_OCam), P]
        lib.o_render.argtypes = [ctypes.POINTER(_OScene), P, ctypes.c_double, ctypes.POINTER(_OCam),
                                 P, ctypes.c_int, P, P, P, P, ctypes.c_int, ctypes.POINTER(_OEps), P]
        lib.o_render.restype = ctypes.c_int64
        lib.o_render_rows.argtypes = [ctypes.POINTER(_OScene), P, ctypes.c_double, ctypes.POINTER(_OCam), P,
                                      ctypes.c_int, ctypes.c_int, P, P, P]
        lib.o_render_rows.restype = ctypes.c_int64
        lib.o_render_backward.argtypes = [ctypes.POINTER(_OScene), P, ctypes.c_double,
                                          ctypes.POINTER(_OCam), P, P] + [P] * 10
        lib.o_sh_basis.argtypes = [P, ctypes.c_int, P]
        lib.o_rec_width.restype = ctypes.c_int
        lib.o_footprint_tiles.argtypes = [ctypes.POINTER(_OScene), P, ctypes.c_double, ctypes.POINTER(_OCam),
                                          ctypes.c_int, ctypes.c_int64, P, P, P]
        lib.o_footprint_tiles.restype = ctypes.c_int64
        _lib = lib
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class _Pinned:
    """Holds the contiguous arrays behind an _OScene for the call's duration."""

    def __init__(self, scene):
        c = lambda a, dt: np.ascontiguousarray(a, dtype=dt)
        self.keep = dict(offs=c(scene.cluster_offsets, np.int32), mu0=c(scene.mu0, np.float32),
                         u=c(scene.u, np.float32), ls=c(scene.log_scale, np.float32),
                         q=c(scene.quat, np.float32), lg=c(scene.opacity_logit, np.float32),
                         col=c(scene.colour, np.float32), res=c(scene.res, np.float32))
        k = self.keep
        if k["u"].size == 0:
            k["u"] = np.zeros(3, np.float32)
        if k["res"].size == 0:
            k["res"] = np.zeros(1, np.float32)
        aff = getattr(scene, "affine", None)
        if aff is not None:
            k["aff"] = c(aff, np.float32)
        mode = int(getattr(scene, "res_mode", 0))
        if mode:
            k["step"] = c(scene.res_step, np.float32)
            if mode == 1:
                k["rq"] = c(scene.res_q, np.int16)
        self.s = _OScene(scene.n, scene.n_clusters, scene.n_layers, scene.sh_degree,
                         scene.temporal_rank, k["offs"].ctypes.data, k["mu0"].ctypes.data,
                         k["u"].ctypes.data, k["ls"].ctypes.data, k["q"].ctypes.data,
                         k["lg"].ctypes.data, k["col"].ctypes.data, k["res"].ctypes.data,
                         k["aff"].ctypes.data if aff is not None else None,
                         int(aff.shape[1]) if aff is not None else 0,
                         k["rq"].ctypes.data if mode == 1 else None,
                         k["step"].ctypes.data if mode else None, mode)


def _cam(cam) -> _OCam:
    R = np.asarray(cam.R_wc, dtype=np.float64).reshape(9)
    t = np.asarray(cam.t_wc, dtype=np.float64).reshape(3)
    return _OCam((ctypes.c_double * 9)(*R), (ctypes.c_double * 3)(*t), float(cam.fx),
                 float(cam.fy), float(cam.cx), float(cam.cy), int(cam.width), int(cam.height))


def closure(mask_row: np.ndarray, n_clusters: int, n_layers: int) -> np.ndarray:
    lib = _load()
    m = np.ascontiguousarray(mask_row, dtype=np.uint32)
    out = np.zeros(n_clusters, dtype=np.uint8)
    lib.o_closure(n_clusters, n_layers, _ptr(m), _ptr(out))
    return out


def project(scene, depth: np.ndarray, t: float, cam) -> np.ndarray:
    """Per-Gaussian FP64 projection, columns named by :data:`REC_FIELDS`."""
    lib = _load()
    pin = _Pinned(scene)
    d = np.ascontiguousarray(depth, dtype=np.uint8)
    out = np.zeros((scene.n, lib.o_rec_width()), dtype=np.float64)
    oc = _cam(cam)
    lib.o_project(ctypes.byref(pin.s), _ptr(d), float(t), ctypes.byref(oc), _ptr(out))
    return out[:, :len(REC_FIELDS)]


def render(scene, depth, t, cam, bg, pix=None, full_scan=False, eps=None, want_bound=False):
    """Render one state.  Returns (image FP64, marginal flags, evaluations),
    and with ``want_bound`` also the per-pixel bound on how far an evaluation
    deciding the flagged thresholds the other way can move each channel.

    ``pix`` = int array [P,2] of (x, y) samples, else the whole [H,W,3] image."""
    lib = _load()
    pin = _Pinned(scene)
    d = np.ascontiguousarray(depth, dtype=np.uint8)
    oc = _cam(cam)
    bgd = np.ascontiguousarray(bg, dtype=np.float64)
    n_eval = np.zeros(1, np.int64)
    e = None if eps is None else _OEps(*eps)
    if pix is None:
        img = np.zeros((cam.height, cam.width, 3), np.float64)
        marg = np.zeros((cam.height, cam.width), np.uint8)
        bnd = np.zeros((cam.height, cam.width), np.float64)
        lib.o_render(ctypes.byref(pin.s), _ptr(d), float(t), ctypes.byref(oc), _ptr(bgd), 0,
                     None, _ptr(img), _ptr(marg), _ptr(n_eval), int(full_scan),
                     ctypes.byref(e) if e else None, _ptr(bnd))
    else:
        p = np.ascontiguousarray(pix, dtype=np.int32).reshape(-1, 2)
        img = np.zeros((p.shape[0], 3), np.float64)
        marg = np.zeros(p.shape[0], np.uint8)
        bnd = np.zeros(p.shape[0], np.float64)
        lib.o_render(ctypes.byref(pin.s), _ptr(d), float(t), ctypes.byref(oc), _ptr(bgd),
                     p.shape[0], _ptr(p), _ptr(img), _ptr(marg), _ptr(n_eval), 1,
                     ctypes.byref(e) if e else None, _ptr(bnd))
    if want_bound:
        return img, marg.astype(bool), int(n_eval[0]), bnd
    return img, marg.astype(bool), int(n_eval[0])


def render_rows(scene, depth, t, cam, bg, y0, y1):
    """Rows [y0, y1) of one state's image, rendered exactly as the whole image
    (same row filter); a bounded sample for timing the oracle.  Returns
    (image rows FP64 [y1-y0, W, 3], marginal flags, evaluations)."""
    lib = _load()
    pin = _Pinned(scene)
    d = np.ascontiguousarray(depth, dtype=np.uint8)
    oc = _cam(cam)
    bgd = np.ascontiguousarray(bg, dtype=np.float64)
    n_eval = np.zeros(1, np.int64)
    img = np.zeros((y1 - y0, cam.width, 3), np.float64)
    marg = np.zeros((y1 - y0, cam.width), np.uint8)
    lib.o_render_rows(ctypes.byref(pin.s), _ptr(d), float(t), ctypes.byref(oc), _ptr(bgd), int(y0), int(y1),
                      _ptr(img), _ptr(marg), _ptr(n_eval))
    return img, marg.astype(bool), int(n_eval[0])


def state_depths(states, n_clusters, n_layers) -> np.ndarray:
    return np.stack([closure(states.masks[s], n_clusters, n_layers) for s in range(states.n)])


def render_states(scene, states, cams, bg, which=None, want_bound=False):
    """Serial evaluation of every state (the definition batched rendering must equal)."""
    D = state_depths(states, scene.n_clusters, scene.n_layers)
    idx = range(states.n) if which is None else which
    out = []
    for s in idx:
        cam = cams[int(states.cam[s])]
        out.append(render(scene, D[s], float(states.t[s]), cam, bg, want_bound=want_bound))
    return out


def full_depth(scene) -> np.ndarray:
    return np.full(scene.n_clusters, scene.n_layers, dtype=np.uint8)


def mse_psnr(image: np.ndarray, ref: np.ndarray):
    """Eq. 3's D as mean squared error over all channels (FP64) and PSNR (peak 1)."""
    diff = np.asarray(image, np.float64) - np.asarray(ref, np.float64)
    mse = float(np.mean(diff * diff))
    psnr = float("inf") if mse == 0.0 else 10.0 * np.log10(1.0 / mse)
    return mse, psnr


def render_backward(scene, depth, t, cam, bg, dL_dimage, want_2d=False):
    """Adjoint of :func:`render`; returns FP64 gradients in the scene layout."""
    lib = _load()
    pin = _Pinned(scene)
    d = np.ascontiguousarray(depth, dtype=np.uint8)
    oc = _cam(cam)
    bgd = np.ascontiguousarray(bg, dtype=np.float64)
    g = np.ascontiguousarray(dL_dimage, dtype=np.float64)
    n, R, L = scene.n, scene.temporal_rank, scene.n_layers
    out = dict(mu0=np.zeros((n, 3)), u=np.zeros((max(R, 1), n, 3)), log_scale=np.zeros((n, 3)),
               quat=np.zeros((n, 4)), opacity_logit=np.zeros(n),
               colour=np.zeros((n, scene.n_colour)),
               res=np.zeros((max(L - 1, 1), n, scene.res_width)))
    g2 = np.zeros((n, 9))
    aff = getattr(scene, "affine", None)
    if aff is not None:
        out["affine"] = np.zeros(aff.shape)
    if int(getattr(scene, "res_mode", 0)) == 2:
        out["res_step"] = np.zeros(np.asarray(scene.res_step).shape)
    lib.o_render_backward(ctypes.byref(pin.s), _ptr(d), float(t), ctypes.byref(oc), _ptr(bgd),
                          _ptr(g), _ptr(out["mu0"]), _ptr(out["u"]), _ptr(out["log_scale"]),
                          _ptr(out["quat"]), _ptr(out["opacity_logit"]), _ptr(out["colour"]),
                          _ptr(out["res"]), _ptr(g2), _ptr(out["affine"]) if aff is not None else None,
                          _ptr(out["res_step"]) if "res_step" in out else None)
    out["u"] = out["u"][:R]
    out["res"] = out["res"][:max(L - 1, 0)]
    if want_2d:
        out["g2d"] = g2
    return out


def sh_basis(direction, degree: int = 3) -> np.ndarray:
    lib = _load()
    d = np.ascontiguousarray(direction, dtype=np.float64)
    Y = np.zeros(16, np.float64)
    lib.o_sh_basis(_ptr(d), int(degree), _ptr(Y))
    return Y[:(degree + 1) ** 2]


def footprint_tiles(scene, depth, t, cam, tile):
    """Tile membership from the footprint alone (S11/S12): every (Gaussian,
    tile) pair where the Gaussian can composite at some pixel centre of the
    tile (pixel box and alpha >= 1/255), with a flag for pairs only
    near-threshold pixels qualify for.  Returns (gaussian index, tile index,
    marginal) arrays in (Gaussian, tile) order."""
    lib = _load()
    pin = _Pinned(scene)
    d = np.ascontiguousarray(depth, dtype=np.uint8)
    oc = _cam(cam)
    n = lib.o_footprint_tiles(ctypes.byref(pin.s), _ptr(d), float(t), ctypes.byref(oc), int(tile), 0,
                              None, None, None)
    g = np.zeros(max(n, 1), np.int32)
    tl = np.zeros(max(n, 1), np.int32)
    m = np.zeros(max(n, 1), np.uint8)
    lib.o_footprint_tiles(ctypes.byref(pin.s), _ptr(d), float(t), ctypes.byref(oc), int(tile), int(n),
                          _ptr(g), _ptr(tl), _ptr(m))
    return g[:n], tl[:n], m[:n].astype(bool)


def float_key(z32: np.ndarray) -> np.ndarray:
    """Order-preserving uint32 image of positive float32 depths (their bit pattern)."""
    return np.asarray(z32, dtype=np.float32).view(np.uint32)


def bin_tiles(xlo, xhi, ylo, yhi, depth_bits, live, tile, tiles_x, tiles_y,
              view_group=None, rank=None):
    """Tile lists of live records (integer function).

    Every live record r emits one entry per tile of its pixel box
    [xlo, xhi] x [ylo, yhi]; the entries are ordered by the 64-bit key
    (view_group * tiles + tile) << 32 | depth_bits, ties by ``rank`` (the record
    order (Gaussian index, variant)).  Returns (keys uint64, values = record
    index, ranges [V*tiles, 2])."""
    n = len(xlo)
    vg = np.zeros(n, np.int64) if view_group is None else np.asarray(view_group, np.int64)
    rk = np.arange(n) if rank is None else np.asarray(rank, np.int64)
    keys, vals = [], []
    T = tiles_x * tiles_y
    for r in np.nonzero(np.asarray(live))[0]:
        for ty in range(int(ylo[r]) // tile, int(yhi[r]) // tile + 1):
            for tx in range(int(xlo[r]) // tile, int(xhi[r]) // tile + 1):
                key = ((int(vg[r]) * T + ty * tiles_x + tx) << 32) | int(depth_bits[r])
                keys.append(key)
                vals.append(r)
    keys = np.array(keys, dtype=np.uint64)
    vals = np.array(vals, dtype=np.int64)
    order = np.lexsort((rk[vals] if len(vals) else vals, keys))
    keys, vals = keys[order], vals[order]
    nv = int(vg.max()) + 1 if n else 1
    ranges = np.zeros((nv * T, 2), np.int64)
    tid = (keys >> np.uint64(32)).astype(np.int64)
    for k in range(nv * T):
        lo = np.searchsorted(tid, k, side="left")
        hi = np.searchsorted(tid, k, side="right")
        ranges[k] = (lo, hi)
    return keys, vals, ranges


def utility_stats(delta: np.ndarray, alpha: float = 0.25, beta: float = 0.05, q: float = 0.10):
    """Eq. 4 over one group's contexts: returns (mean, Q_q, std, risk-adjusted
    utility) with E_m the mean over the sampled contexts, Std_m the population
    standard deviation, Q_q the quantile by linear interpolation between order
    statistics (position q (M - 1) of the sorted values), and
    utility = ((1 - alpha) mean + alpha Q_q) / (1 + beta std)."""
    x = np.sort(np.asarray(delta, dtype=np.float64))
    mean = float(np.mean(x))
    std = float(np.sqrt(np.mean((x - mean) ** 2)))
    h = q * (x.size - 1)
    lo = int(np.floor(h))
    hi = min(lo + 1, x.size - 1)
    quant = float(x[lo] + (h - lo) * (x[hi] - x[lo]))
    return mean, quant, std, ((1.0 - alpha) * mean + alpha * quant) / (1.0 + beta * std)


def group_utility(scene, ctx_masks, groups, n_contexts, cam, t, bg, alpha=0.25, beta=0.05, q=0.10):
    """Eq. 3 and Eq. 4.  ``ctx_masks`` [G * M, words]: context j of group g is
    row g * M + j; ``groups`` [G, 2] = (cluster, layer) packets.  For every
    context m: Delta_g(m) = D(I, R(m)) - D(I, R(m u g)) with D the MSE against
    the complete render I at the same view (FP64 renders).  Returns
    (delta [G, M], stats [G, 4] = mean, Q_q, std, utility)."""
    G, M = len(groups), int(n_contexts)
    L = scene.n_layers
    full, _, _ = render(scene, full_depth(scene), t, cam, bg)
    delta = np.zeros((G, M))
    stats = np.zeros((G, 4))
    for g, (c, l) in enumerate(groups):
        bit = int(c) * L + int(l)
        for j in range(M):
            m = np.array(ctx_masks[g * M + j], dtype=np.uint32)
            mg = m.copy()
            mg[bit // 32] |= np.uint32(1 << (bit % 32))
            d0 = mse_psnr(render(scene, closure(m, scene.n_clusters, L), t, cam, bg)[0], full)[0]
            d1 = mse_psnr(render(scene, closure(mg, scene.n_clusters, L), t, cam, bg)[0], full)[0]
            delta[g, j] = d0 - d1
        stats[g] = utility_stats(delta[g], alpha, beta, q)
    return delta, stats


# ----------------------------------------------------------------- Eq. 2 objective
SSIM_C1, SSIM_C2 = 0.01 ** 2, 0.03 ** 2


def ssim_window(size: int = 11, sigma: float = 1.5) -> np.ndarray:
    """Normalised 1-D Gaussian window (the 2-D window is its outer product)."""
    x = np.arange(size, dtype=np.float64) - (size - 1) / 2.0
    g = np.exp(-x * x / (2.0 * sigma * sigma))
    return g / g.sum()


def _blur(img: np.ndarray, g: np.ndarray) -> np.ndarray:
    """'Same'-size 2-D filtering of [H, W, C] with the separable window g, zero padded."""
    r = len(g) // 2
    H, W = img.shape[:2]
    p = np.zeros((H + 2 * r, W + 2 * r) + img.shape[2:])
    p[r:r + H, r:r + W] = img
    h = sum(g[k] * p[:, k:k + W] for k in range(len(g)))
    return sum(g[k] * h[k:k + H] for k in range(len(g)))


def ssim(x: np.ndarray, y: np.ndarray, want_grad: bool = False):
    """Structural similarity of image x against reference y ([H, W, 3]) in FP64:
    local means, variances and covariance under an 11x11 Gaussian window
    (sigma 1.5, zero-padded same-size filtering), per-pixel
    ((2 mx my + C1)(2 sxy + C2)) / ((mx^2 + my^2 + C1)(sx^2 + sy^2 + C2)),
    averaged over pixels and channels.  With want_grad also returns dSSIM/dx
    (want_grad="map": the per-pixel, per-channel values instead of their mean)."""
    g = ssim_window()
    x = np.asarray(x, np.float64); y = np.asarray(y, np.float64)
    mx, my = _blur(x, g), _blur(y, g)
    exx, eyy, exy = _blur(x * x, g), _blur(y * y, g), _blur(x * y, g)
    sxx, syy, sxy = exx - mx * mx, eyy - my * my, exy - mx * my
    a1, a2 = 2 * mx * my + SSIM_C1, 2 * sxy + SSIM_C2
    b1, b2 = mx * mx + my * my + SSIM_C1, sxx + syy + SSIM_C2
    f = a1 * a2 / (b1 * b2)
    if want_grad == "map":
        return f
    s = float(np.mean(f))
    if not want_grad:
        return s
    # f as a function of (mx, exx, exy): chain through sxx = exx - mx^2, sxy = exy - mx my
    d_mx = f * (2 * my / a1 - 2 * my / a2 - 2 * mx / b1 + 2 * mx / b2)
    d_exx = -f / b2
    d_exy = 2 * f / a2
    n = f.size
    grad = (_blur(d_mx, g) + 2 * x * _blur(d_exx, g) + y * _blur(d_exy, g)) / n
    return s, grad


def objective(images, refs, ref_index, pairs_t=(), pairs_m=(), anchors=(), ssim_weight=0.20,
              lambda_c=0.30, cvar_q=0.05, lambda_t=0.10, lambda_m=2.0, anchor_weight=0.50):
    """Eq. 2 with the locked weights, in FP64, over a batch of rendered states.

    D_s = MSE(I_s, ref) + ssim_weight (1 - SSIM(I_s, ref)) against the state's
    reference image; then
      L = mean_s D_s + lambda_c CVaR_q(D) + lambda_t F + lambda_m M
          + anchor_weight mean_{s in anchors} D_s
    with CVaR_q(D) the mean of the ceil(q S) largest D (the upper tail of the
    loss), F the mean over temporal pairs (i, j) of the mean squared error
    between the rendered change I_j - I_i and the reference change, and M the
    mean over prefix pairs (i, j) (state j extends state i) of max(0, D_j - D_i).
    The rate term is absent (its locked weight is 0).  Returns (L, D [S],
    dL/dimages [S, H, W, 3])."""
    imgs = np.asarray(images, np.float64)
    rf = np.asarray(refs, np.float64)
    S = imgs.shape[0]
    n_val = imgs[0].size
    D = np.zeros(S)
    gD = np.zeros_like(imgs)                     # dD_s / dI_s
    for s in range(S):
        y = rf[int(ref_index[s])]
        d = imgs[s] - y
        sv, sg = ssim(imgs[s], y, want_grad=True)
        D[s] = np.mean(d * d) + ssim_weight * (1.0 - sv)
        gD[s] = 2.0 * d / n_val - ssim_weight * sg
    w = np.full(S, 1.0 / S)                      # dL / dD_s
    k = int(np.ceil(cvar_q * S)) if S else 0
    top = np.argsort(-D, kind="stable")[:k]
    cvar = float(np.mean(D[top])) if k else 0.0
    w[top] += lambda_c / k
    M = 0.0
    if len(pairs_m):
        for i, j in pairs_m:
            if D[j] > D[i]:
                M += (D[j] - D[i]) / len(pairs_m)
                w[j] += lambda_m / len(pairs_m)
                w[i] -= lambda_m / len(pairs_m)
    A = 0.0
    if len(anchors):
        for s in anchors:
            A += D[s] / len(anchors)
            w[s] += anchor_weight / len(anchors)
    grad = w[:, None, None, None] * gD
    F = 0.0
    if len(pairs_t):
        for i, j in pairs_t:
            e = (imgs[j] - imgs[i]) - (rf[int(ref_index[j])] - rf[int(ref_index[i])])
            F += np.mean(e * e) / len(pairs_t)
            gf = lambda_t * 2.0 * e / (n_val * len(pairs_t))
            grad[j] += gf
            grad[i] -= gf
    L = float(np.mean(D)) + lambda_c * cvar + lambda_t * F + lambda_m * M + anchor_weight * A
    return L, D, grad
