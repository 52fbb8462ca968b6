"""CUDA path vs the FP64 oracle, through the C ABI (needs a B300)."""
import math

import numpy as np
import pytest

import oracle
from paper_2606_17212_b300 import dgs, synth

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4          # max-abs per channel, plus the oracle's derived bound at flagged pixels
GRAD_TOL = 1e-3         # ||g - g_ref||_inf <= GRAD_TOL * max(||g_ref||_inf, 1e-6), per tensor


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    assert _t.cuda.is_available()
    return _t


@pytest.fixture(scope="module")
def R(torch):
    r = dgs.Renderer(0)
    yield r
    r.close()


def _compare_image(gpu, ref, bound):
    """Largest error in excess of the oracle's derived bound (zero except at
    pixels with a threshold decision FP32 may take the other way), over every
    pixel, and the count of bounded pixels."""
    err = np.abs(gpu.astype(np.float64) - ref) - bound[..., None]
    return (float(err.max()) if err.size else 0.0), int((bound > 0).sum())


def _mse_tol(d, e):
    """Bound on |MSE_gpu - MSE_ref| when the reference difference image is d and
    each value of the GPU difference image is within e (per pixel) of it:
    |(d + x)^2 - d^2| <= 2 |d| e + e^2, averaged, plus FP32 rounding of the
    squared errors (5 ulp of each)."""
    e = np.broadcast_to(e[..., None], d.shape)
    return float(np.mean(2 * np.abs(d) * e + e * e)) + 5 * 2.0 ** -24 * float(np.mean(d * d))


def _gpu_states(w):
    return dgs.DeviceStates.from_host(w.states)


# --------------------------------------------------------------------- forward
def test_c1_render_state_matches_oracle(R, torch):
    w = synth.config("c1_plain_4k")
    sc = dgs.DeviceScene.from_host(w.scene)
    st = _gpu_states(w)
    img = R.render_state(sc, st.masks[0], 0.0, w.cams[0], w.bg)
    torch.cuda.synchronize()
    D = oracle.closure(w.states.masks[0], w.scene.n_clusters, w.scene.n_layers)
    ref, marg, ne, bnd = oracle.render(w.scene, D, 0.0, w.cams[0], w.bg, want_bound=True)
    err, nm = _compare_image(img.cpu().numpy(), ref, bnd)
    assert err <= IMG_TOL, (err, nm)
    assert nm <= 0.002 * marg.size


@pytest.mark.parametrize("name,scale,n", [("c2_dynamic_250k", 0.02, 6), ("c3_fwdbwd_250k", 0.02, 6)])
def test_batched_matches_oracle_per_state(R, torch, name, scale, n):
    w = synth.config(name, scale=scale, n_states=n)
    sc = dgs.DeviceScene.from_host(w.scene)
    st = _gpu_states(w)
    imgs = R.render_states_batched(sc, st, w.cams, w.bg).cpu().numpy()
    refs = oracle.render_states(w.scene, w.states, w.cams, w.bg, want_bound=True)
    for s, (ref, marg, _, bnd) in enumerate(refs):
        err, nm = _compare_image(imgs[s], ref, bnd)
        assert err <= IMG_TOL, (s, err, nm)
        assert nm <= 0.01 * marg.size, (s, nm)


def test_batched_equals_per_state_bitwise(R, torch):
    """The abstract: batched rendering is bit-equivalent to serial evaluation."""
    w = synth.config("c3_fwdbwd_250k", scale=0.05, n_states=24)
    sc = dgs.DeviceScene.from_host(w.scene)
    st = _gpu_states(w)
    batched = R.render_states_batched(sc, st, w.cams, w.bg)
    for s in range(st.n):
        one = R.render_state(sc, st.masks[s], float(w.states.t[s]), w.cams[int(w.states.cam[s])], w.bg)
        assert torch.equal(one, batched[s]), s


def test_tile_size_changes_no_bit(R, torch):
    """The sort tile size is an acceleration structure: 16 and 32 px tiles give
    the same images and per-state MSE bit for bit (every pixel composites the
    same Gaussians in the same order; squared errors are summed over fixed
    16 x 16 blocks), and the same gradients up to the order of the float
    atomic adds (ragged image, several view groups)."""
    w = synth.config("c3_fwdbwd_250k", scale=0.03, n_states=12)
    w.cams = [synth.ring_camera(k, 8, 83, 57, 96.0) for k in range(8)]
    sc = dgs.DeviceScene.from_host(w.scene)
    st = _gpu_states(w)
    out = {}
    try:
        for tile in (16, 32):
            R.set_tile_size(tile)
            imgs = R.render_states_batched(sc, st, w.cams, w.bg)
            mse, psnr = R.state_utility(sc, st, w.cams, w.bg)
            dL = torch.sin(torch.arange(imgs.numel(), device="cuda", dtype=torch.float32) * 0.37).reshape(imgs.shape)
            g = R.render_backward(sc, st, w.cams, w.bg, dL * 1e-3, images=imgs)
            out[tile] = (imgs.clone(), mse.clone(), {k: v.clone() for k, v in g.items()})
    finally:
        R.set_tile_size(0)
    assert torch.equal(out[16][0], out[32][0])
    assert torch.equal(out[16][1], out[32][1])
    for k, v in out[16][2].items():
        ref = float(v.abs().max())
        err = float((out[32][2][k] - v).abs().max())
        assert err <= 1e-5 * max(ref, 1e-12), (k, err, ref)


def test_memory_budget_splits_the_batch_bit_identically(torch):
    """A context whose workspace budget cannot hold the whole batch renders it
    in parts: images and per-state MSE are bit-identical to one unbudgeted
    batch, gradients equal up to float addition order, and the workspace stays
    within the budget."""
    w = synth.config("c3_fwdbwd_250k", scale=0.02, n_states=20)
    sc = dgs.DeviceScene.from_host(w.scene)
    st = _gpu_states(w)
    dL = None
    out = []
    for budget in (0, None):
        r = dgs.Renderer(0)
        r.set_tile_size(16)
        if budget is None:
            budget = ws_full // 3
            r.set_memory_budget(budget)
        imgs = r.render_states_batched(sc, st, w.cams, w.bg)
        if dL is None:
            dL = torch.cos(torch.arange(imgs.numel(), device="cuda", dtype=torch.float32) * 0.05).reshape(imgs.shape)
        g = r.render_backward(sc, st, w.cams, w.bg, dL * 1e-3, images=imgs)
        mse, _ = r.state_utility(sc, st, w.cams, w.bg)
        ws, splits = r.memory_stats()
        if budget == 0:
            ws_full = ws
            assert splits == 0
        else:
            assert splits > 0 and ws <= budget, (splits, ws, budget)
        out.append((imgs.clone(), mse.clone(), {k: v.clone() for k, v in g.items()}))
        r.close()
    assert torch.equal(out[0][0], out[1][0])
    assert torch.equal(out[0][1], out[1][1])
    for k, v in out[0][2].items():
        ref = float(v.abs().max())
        assert float((out[1][2][k] - v).abs().max()) <= 1e-5 * max(ref, 1e-12), k


def test_ragged_image_and_edge_cases(R, torch):
    w = synth.config("c2_dynamic_250k", scale=0.01, n_states=3)
    cam = synth.ring_camera(2, 8, 97, 61, 110.0)          # ragged tiles on both axes
    sc = dgs.DeviceScene.from_host(w.scene)
    st = _gpu_states(w)
    imgs = R.render_states_batched(sc, st, [cam], w.bg).cpu().numpy()
    for s in range(st.n):
        D = oracle.closure(w.states.masks[s], w.scene.n_clusters, w.scene.n_layers)
        ref, marg, _, bnd = oracle.render(w.scene, D, float(w.states.t[s]), cam, w.bg, want_bound=True)
        err, nm = _compare_image(imgs[s], ref, bnd)
        assert err <= IMG_TOL, (s, err, nm)
    # empty delivery -> background everywhere
    bg = np.array([0.25, 0.5, 0.75], np.float32)
    empty = torch.zeros_like(st.masks[0])
    img = R.render_state(sc, empty, 0.0, cam, bg).cpu().numpy()
    assert np.all(img == bg[None, None, :])
    # no states: nothing to do
    st0 = dgs.DeviceStates(st.masks[:0], np.zeros(0, np.float32), np.zeros(0, np.int32))
    out = R.render_states_batched(sc, st0, [cam], bg)
    assert out.shape[0] == 0


def test_single_gaussian_closed_form_on_gpu(R, torch):
    """C = o c + (1 - o) bg at the pixel centre under the mean (Section 6 path, 1 Gaussian)."""
    o = 0.7
    sc_h = synth.Scene(1, 1, 1, 0, 0, np.array([0, 1], np.int32),
                       np.array([[0.0, 1 / 64, -1 / 64]], np.float32), np.zeros((0, 1, 3), np.float32),
                       np.full((1, 3), -2.5, np.float32), np.array([[1, 0, 0, 0]], np.float32),
                       np.array([math.log(o / (1 - o))], np.float32), np.array([[0.9, 0.2, 0.4]], np.float32),
                       np.zeros((0, 1, 14), np.float32))
    cam = synth.ring_camera(0, 1, 128, 128, 128.0)
    sc = dgs.DeviceScene.from_host(sc_h)
    mask = torch.ones(1, dtype=torch.int32, device="cuda")
    bg = np.array([0.1, 0.3, 0.05], np.float32)
    img = R.render_state(sc, mask, 0.0, cam, bg).cpu().numpy()
    o32 = 1.0 / (1.0 + math.exp(-float(np.float32(math.log(o / (1 - o))))))
    expect = o32 * np.array([0.9, 0.2, 0.4], np.float32) + (1 - o32) * bg
    assert np.allclose(img[64, 64], expect, atol=2e-6)


# --------------------------------------------------------------------- utility
def test_state_utility_matches_oracle(R, torch):
    """Eq. 3 D per state vs the oracle, every state: each value of the state
    and complete renders is within 1e-4 plus the oracle's derived bound of the
    FP64 one, so |dMSE| <= mean(2 |d| e + e^2) with e the sum of both."""
    w = synth.config("c2_dynamic_250k", scale=0.004, n_states=8)
    masks = w.states.masks.copy()
    masks[0] = 0xFFFFFFFF             # complete delivery: MSE exactly 0, PSNR +inf
    w.states.masks = masks
    sc = dgs.DeviceScene.from_host(w.scene)
    st = _gpu_states(w)
    mse, psnr = R.state_utility(sc, st, w.cams, w.bg)
    mse, psnr = mse.cpu().numpy(), psnr.cpu().numpy()
    assert mse[0] == 0.0 and math.isinf(psnr[0])
    refs = oracle.render_states(w.scene, w.states, w.cams, w.bg, want_bound=True)
    for s in range(1, st.n):
        full, mfull, _, bfull = oracle.render(w.scene, oracle.full_depth(w.scene), float(w.states.t[s]),
                                              w.cams[0], w.bg, want_bound=True)
        ref, marg, _, bnd = refs[s]
        d = ref - full
        m_ref = float(np.mean(d * d))
        bound = _mse_tol(d, 2 * IMG_TOL + bnd + bfull)
        assert abs(mse[s] - m_ref) <= bound, (s, mse[s], m_ref, bound)
        assert psnr[s] == pytest.approx(10 * math.log10(1 / mse[s]), rel=1e-12)


def test_utility_equals_images_then_mse(R, torch):
    """Fused FP64 epilogue == images written, then the separate MSE kernel (bitwise)."""
    w = synth.config("c2_dynamic_250k", scale=0.02, n_states=7)
    sc = dgs.DeviceScene.from_host(w.scene)
    st = _gpu_states(w)
    mse, _ = R.state_utility(sc, st, w.cams, w.bg)
    imgs = R.render_states_batched(sc, st, w.cams, w.bg)
    full_masks = torch.full_like(st.masks, -1)
    tvals = np.unique(w.states.t)
    fst = dgs.DeviceStates(full_masks[:len(tvals)], tvals, np.zeros(len(tvals), np.int32))
    fulls = R.render_states_batched(sc, fst, w.cams, w.bg)
    ridx = np.searchsorted(tvals, w.states.t)
    m2, p2, _ = R.image_mse(imgs, fulls, ridx)
    assert torch.allclose(mse, m2, rtol=1e-12, atol=0)


@pytest.mark.parametrize("name,scale,n,tile", [("c4_utility_2p7m", 0.02, 600, 16), ("c2_dynamic_250k", 0.03, 256, 16),
                                               ("c3_fwdbwd_250k", 0.05, 96, 16), ("c4_utility_2p7m", 0.02, 600, 32),
                                               ("c3_fwdbwd_250k", 0.05, 96, 32)])
def test_tile_reuse_is_bitwise(R, torch, name, scale, n, tile):
    """Reusing rendered tiles across the states of a view changes no bit of any
    state's MSE: reuse on == every (state, tile) rendered, for either sort tile size."""
    w = synth.config(name, scale=scale, n_states=n)
    masks = w.states.masks.copy()
    masks[1] = 0                       # empty delivery
    masks[2] = 0xFFFFFFFF              # complete delivery
    masks[3:6] = masks[6]              # duplicates
    if name == "c3_fwdbwd_250k":       # many states on few views: eight per (camera, time)
        w.states.t[:] = w.states.t[0]
        w.states.cam[:] = w.states.cam % 2
    w.states.masks = masks
    sc = dgs.DeviceScene.from_host(w.scene)
    st = _gpu_states(w)
    R.set_tile_size(tile)
    try:
        R.set_tile_reuse(False)
        try:
            m0, p0 = R.state_utility(sc, st, w.cams, w.bg)
        finally:
            R.set_tile_reuse(True)
        m1, p1 = R.state_utility(sc, st, w.cams, w.bg)
        pairs, rendered, rounds = R.tile_reuse_stats()
    finally:
        R.set_tile_size(0)
    tiles = -(-w.cams[0].width // tile) * -(-w.cams[0].height // tile)
    assert pairs == n * tiles and 0 < rendered <= pairs and 1 <= rounds <= 17
    assert torch.equal(m0, m1)
    assert torch.equal(p0.isinf(), p1.isinf()) and torch.equal(p0[~p0.isinf()], p1[~p1.isinf()])
    assert float(m1[2]) == 0.0


def test_tile_reuse_group_utility_bitwise(R, torch):
    """Eq. 3 / Eq. 4 group utility with and without tile reuse: identical bits."""
    w = synth.config("c4_utility_2p7m", scale=0.02, n_states=16)
    sc = dgs.DeviceScene.from_host(w.scene)
    rng = np.random.default_rng(5)
    C, L, M = w.scene.n_clusters, w.scene.n_layers, 12
    groups = np.array([[c, int(rng.integers(0, L))] for c in rng.choice(C, 6, replace=False)], np.int32)
    ctx = synth.group_contexts(groups, M, C, L, rng)
    n = len(groups) * M
    states = dgs.DeviceStates.from_host(synth.States(ctx, np.full(n, w.states.t[0], np.float32),
                                                     np.zeros(n, np.int32)))
    R.set_tile_reuse(False)
    try:
        d0, s0 = R.group_utility(sc, states, groups, M, w.cams, w.bg)
    finally:
        R.set_tile_reuse(True)
    d1, s1 = R.group_utility(sc, states, groups, M, w.cams, w.bg)
    assert torch.equal(d0, d1) and torch.equal(s0, s1)


def test_image_mse_and_gradient(R, torch):
    rng = np.random.default_rng(0)
    a = rng.uniform(size=(3, 37, 29, 3)).astype(np.float32)
    b = rng.uniform(size=(2, 37, 29, 3)).astype(np.float32)
    idx = np.array([1, 0, 1])
    ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    mse, psnr, dL = R.image_mse(ta, tb, idx, weight=0.25, want_grad=True)
    for s in range(3):
        d = a[s].astype(np.float64) - b[idx[s]].astype(np.float64)
        # each pixel's squared RGB error is an FP32 value within 5 * 2^-24 (first
        # order) of the exact one; the sum over pixels is FP64
        assert mse[s].item() == pytest.approx(np.mean(d * d), rel=5 * 2.0 ** -24)
        # the same per-pixel value emulated: FP32 differences, d0^2 rounded, then two
        # fused multiply-adds (the product is exact in FP64; one rounding to FP32)
        d32 = (a[s] - b[idx[s]]).astype(np.float32)
        e = d32.astype(np.float64)
        p0 = (d32[..., 0] * d32[..., 0]).astype(np.float64)
        p1 = (e[..., 1] * e[..., 1] + p0).astype(np.float32).astype(np.float64)
        p2 = (e[..., 2] * e[..., 2] + p1).astype(np.float32).astype(np.float64)
        assert mse[s].item() == pytest.approx(p2.sum() / d.size, rel=1e-12)
        g = 0.25 * 2 * (a[s] - b[idx[s]]) / d.size
        assert np.allclose(dL[s].cpu().numpy(), g, rtol=1e-6, atol=1e-12)


# --------------------------------------------------------------------- backward
def _grad_case(seed=0, sh=0):
    if sh == 0:
        w = synth.config("c3_fwdbwd_250k", scale=0.004, n_states=4)
        sc = w.scene
    else:
        w = synth.config("c3_fwdbwd_250k", scale=0.004, n_states=4)
        sc = synth.make_scene(1000, 8, 4, seed=77, sh_degree=3)
        w.states.masks = synth._pack(synth.depths_to_bits(
            synth.prefix_states(4, 8, 4, np.random.default_rng(5)), 4))
    cams = [synth.ring_camera(k, 8, 64, 48, 75.0) for k in range(8)]
    return sc, w.states, cams


@pytest.mark.parametrize("sh,with_images", [(0, False), (0, True), (3, False), (3, True)])
def test_backward_matches_oracle_adjoint(R, torch, sh, with_images):
    """Adjoint vs the oracle's, with the forward images given (one walk per
    tile) and without (final pixel values recomputed by a first walk)."""
    sc_h, states, cams = _grad_case(sh=sh)
    bg = np.array([0.1, 0.2, 0.3], np.float32)
    rng = np.random.default_rng(3)
    S = states.n
    H, W = cams[0].height, cams[0].width
    dL = rng.normal(size=(S, H, W, 3))
    D = oracle.state_depths(states, sc_h.n_clusters, sc_h.n_layers)
    ref = None
    for s in range(S):
        cam = cams[int(states.cam[s])]
        g = oracle.render_backward(sc_h, D[s], float(states.t[s]), cam, bg, dL[s])
        ref = g if ref is None else {k: ref[k] + g[k] for k in ref}
    sc = dgs.DeviceScene.from_host(sc_h)
    st = dgs.DeviceStates.from_host(states)
    imgs = R.render_states_batched(sc, st, cams, bg)
    grads = R.render_backward(sc, st, cams, bg, torch.from_numpy(dL.astype(np.float32)).cuda(),
                              images=imgs if with_images else None)
    for k in dgs.SCENE_FIELDS:
        gg = grads[k].cpu().numpy().astype(np.float64)
        gr = ref[k]
        if gr.size == 0:
            continue
        scale = max(np.abs(gr).max(), 1e-6)
        err = np.abs(gg - gr).max()
        assert err <= GRAD_TOL * scale, (k, err, scale)


def test_backward_undelivered_layers_exactly_zero_and_autograd(R, torch):
    sc_h, states, cams = _grad_case()
    # the two clusters with the most Gaussians in view of state 0 go to depth 1 and 2
    full = oracle.full_depth(sc_h)
    rec = oracle.project(sc_h, full, float(states.t[0]), cams[int(states.cam[0])])
    cl = sc_h.cluster_of()
    seen = np.bincount(cl, weights=rec[:, 0], minlength=sc_h.n_clusters)
    c1, c2 = np.argsort(-seen)[:2]
    D = synth.prefix_states(states.n, sc_h.n_clusters, sc_h.n_layers, np.random.default_rng(1))
    D[:, c1] = 1
    D[:, c2] = 2
    states.masks = synth._pack(synth.depths_to_bits(D, sc_h.n_layers))
    sc = dgs.DeviceScene.from_host(sc_h)
    st = dgs.DeviceStates.from_host(states)
    bg = np.zeros(3, np.float32)
    for v in sc.t.values():
        v.requires_grad_(True)
    img = dgs.render(R, sc, st, cams, bg)
    loss = (img ** 2).mean()
    loss.backward()
    res_g = sc.t["res"].grad.cpu().numpy()
    assert np.all(res_g[:, cl == c1] == 0.0)         # depth 1: no refinement rendered
    assert np.all(res_g[1:, cl == c2] == 0.0)        # depth 2: only layer 1
    assert np.abs(res_g[0, cl == c2]).max() > 0
    assert np.abs(sc.t["mu0"].grad.cpu().numpy()).max() > 0


def test_backward_after_masks_changed_in_place(R, torch):
    """The backward reuses the forward's lists only while the masks still hold
    the bits the forward rendered: masks edited in place between forward and
    backward give DGS_E_STALE when the forward's images are passed, and without
    images the gradients of the current masks (as a fresh forward + backward)."""
    sc_h, states, cams = _grad_case(seed=4)
    sc = dgs.DeviceScene.from_host(sc_h)
    st = dgs.DeviceStates.from_host(states)
    bg = np.zeros(3, np.float32)
    imgs = R.render_states_batched(sc, st, cams, bg)
    dL = torch.sin(torch.arange(imgs.numel(), device="cuda", dtype=torch.float32) * 0.11).reshape(imgs.shape)
    st.masks[0].zero_()                          # in place: same pointer, other bits
    with pytest.raises(RuntimeError, match="DGS_E_STALE"):
        R.render_backward(sc, st, cams, bg, dL, images=imgs)
    g_now = R.render_backward(sc, st, cams, bg, dL)          # no images: lists for the current masks
    st2 = dgs.DeviceStates.from_host(states)
    st2.masks.copy_(st.masks)
    R.render_states_batched(sc, st2, cams, bg)               # fresh forward of the edited masks
    g_ref = R.render_backward(sc, st2, cams, bg, dL)
    for k, v in g_ref.items():
        ref = float(v.abs().max())
        assert float((g_now[k] - v).abs().max()) <= 1e-5 * max(ref, 1e-12), k
    assert float(g_now["res"].abs().max()) > 0


# --------------------------------------------------------------------- tile lists
def _unpack_boxes(recs):
    bx, by, cd = recs[:, 9], recs[:, 10], recs[:, 11]
    return (bx & 0xFFFF).astype(np.int64), (bx >> 16).astype(np.int64), (by & 0xFFFF).astype(np.int64), \
        (by >> 16).astype(np.int64), ((cd >> 12) & 0xF).astype(np.int64), ((cd >> 16) & 0x7FFF).astype(np.int64), \
        (cd & 0x3FF).astype(np.int64)


@pytest.mark.parametrize("tile", [16, 32])
def test_tile_lists_bitwise_and_end_to_end(R, torch, tile):
    w = synth.config("c3_fwdbwd_250k", scale=0.01, n_states=10)
    sc_h = w.scene
    sc = dgs.DeviceScene.from_host(sc_h)
    st = _gpu_states(w)
    R.set_tile_size(tile)
    try:
        R.render_states_batched(sc, st, w.cams, w.bg)
        d = R.debug_tile_lists()
    finally:
        R.set_tile_size(0)
    n_rec, T = d["n_rec"], d["tiles"]
    W, H = w.cams[0].width, w.cams[0].height
    tx, ty = -(-W // tile), -(-H // tile)
    assert T == tx * ty
    recs = d["recs"]
    xlo, xhi, ylo, yhi, depth, vg, clus = _unpack_boxes(recs)
    live = depth != 0
    ds, dk = d["depth_slots"].astype(np.int64), d["depth_keys"].astype(np.uint64)
    n_live = int(live.sum())
    # the depth sort drops the culled records (key 0xFFFFFFFF): the live ones first, then the tail marker
    assert np.all(ds[n_live:] == 0xFFFFFFFF) and np.all(dk[n_live:] == 0xFFFFFFFF)
    dkey = np.full(n_rec, 0xFFFFFFFF, np.uint64)
    dkey[ds[:n_live]] = dk[:n_live]
    assert np.array_equal(dkey != 0xFFFFFFFF, live)
    # depth sort = stable sort of the live records by (view group, depth key)
    order = np.lexsort((dkey, vg))
    order = order[dkey[order] != 0xFFFFFFFF]
    assert np.array_equal(order, ds[:n_live])
    # (1) regression check, bitwise: the oracle's integer binning (tile
    # rectangles, 64-bit key order) applied to the GPU's own FP32 boxes and depths
    keys, vals, ranges = oracle.bin_tiles(xlo, xhi, ylo, yhi, dkey, live, tile, tx, ty, view_group=vg,
                                          rank=np.arange(n_rec))
    assert np.array_equal((keys >> np.uint64(32)).astype(np.uint32), d["entry_keys"])
    assert np.array_equal(vals.astype(np.uint32), d["entry_vals"])
    g_rng = d["ranges"].reshape(-1, 2).astype(np.int64)
    for k in range(len(g_rng)):
        lo, hi = ranges[k] if k < len(ranges) else (0, 0)
        if hi > lo:
            assert tuple(g_rng[k]) == (lo, hi), k
        else:
            assert g_rng[k][0] == g_rng[k][1], k
    # (2) end to end, against the footprint definition: every (Gaussian variant,
    # tile) pair where the FP64 footprint (pixel box and alpha >= 1/255) reaches a
    # pixel centre of the tile must be in the GPU run of that tile (the runs may
    # hold more: binning uses a conservative box); near-threshold pairs are
    # optional.  Slots follow the GPU's layout: view group, cluster, Gaussian, depth.
    views = []
    for s in range(w.states.n):
        key = (int(w.states.cam[s]), float(w.states.t[s]))
        if key not in views:
            views.append(key)
    D = oracle.state_depths(w.states, sc_h.n_clusters, sc_h.n_layers)
    vg_of = [views.index((int(w.states.cam[s]), float(w.states.t[s]))) for s in range(w.states.n)]
    need = [[set() for _ in range(sc_h.n_clusters)] for _ in views]
    for s in range(w.states.n):
        for c in range(sc_h.n_clusters):
            if D[s, c] > 0:
                need[vg_of[s]][c].add(int(D[s, c]))
    offs = sc_h.cluster_offsets
    cl = sc_h.cluster_of()
    slot_of = {}
    o_z = np.zeros(n_rec, np.float32); o_marg = np.zeros(n_rec, bool); o_valid = np.zeros(n_rec, bool)
    proj = {}
    slot = 0
    for v, (cam_i, t) in enumerate(views):
        for c in range(sc_h.n_clusters):
            ds = sorted(need[v][c])
            for i in range(offs[c], offs[c + 1]):
                for dd in ds:
                    if (v, dd) not in proj:
                        proj[(v, dd)] = oracle.project(sc_h, np.full(sc_h.n_clusters, dd, np.uint8), t,
                                                       w.cams[cam_i])
                    r = proj[(v, dd)][i]
                    o_valid[slot] = r[0] > 0
                    o_z[slot] = np.float32(r[18])
                    o_marg[slot] = bool(r[16] or r[17])
                    assert vg[slot] == v and clus[slot] == c and depth[slot] in (0, dd)
                    slot_of[(v, i, dd)] = slot
                    slot += 1
    assert slot == n_rec
    ev = d["entry_vals"].astype(np.int64)
    ek = d["entry_keys"].astype(np.int64)
    member = set((ek * n_rec + ev).tolist())            # (view group tile, slot) pairs of the GPU runs
    required = optional = 0
    for (v, dd) in proj:
        cam_i, t = views[v]
        g, tl, m = oracle.footprint_tiles(sc_h, np.full(sc_h.n_clusters, dd, np.uint8), t, w.cams[cam_i], tile)
        for gi, ti, mi in zip(g.tolist(), tl.tolist(), m.tolist()):
            if dd not in need[v][cl[gi]]:
                continue
            if mi:
                optional += 1
                continue
            sl = slot_of[(v, gi, dd)]
            assert live[sl], (v, gi, dd)
            assert (v * T + ti) * n_rec + sl in member, (v, gi, dd, ti)
            required += 1
    assert required > 1000 and optional < 0.03 * required, (required, optional)
    ok = ~o_marg
    both = ok & live & o_valid
    gz = dkey[both].astype(np.uint32).view(np.float32)
    assert np.all(np.abs(gz.astype(np.float64) - o_z[both]) <= 4e-7 * np.abs(o_z[both]))
    # per tile, the GPU run restricted to non-marginal records is the FP64 depth order
    for k in range(len(g_rng)):
        lo, hi = g_rng[k]
        seq = [x for x in ev[lo:hi] if ok[x] and o_valid[x]]
        zs = o_z[seq].astype(np.float64)
        bad = np.nonzero(np.diff(zs) < 0)[0]
        for b in bad:   # only near-ties (FP32 vs FP64 depth within a few ulps) may swap
            assert zs[b] - zs[b + 1] <= 8e-7 * zs[b], (k, b)


# --------------------------------------------------------------------- Eq. 3 / Eq. 4
def test_group_utility_matches_oracle(R, torch):
    """Counterfactual utility of completion groups.  (1) The per-group
    statistics equal the oracle's Eq. 4 on the GPU's own Delta values; (2) every
    Delta equals the MSE difference of the GPU's own rendered images of m and
    m u g; (3) every Delta matches the FP64 oracle within the bound a 1e-4
    per-value image error allows on non-marginal pixels plus, at pixels the
    oracle flags as marginal (a threshold FP32 may decide the other way), a
    change of up to one colour unit per value; (4) the statistics match the
    oracle's within the largest per-context bound of their group (mean,
    quantile and std move by at most the largest change of their inputs)."""
    w = synth.config("c3_fwdbwd_250k", scale=0.004)
    sc_h = w.scene
    cam, t, bg = synth.ring_camera(2, 8, 64, 48, 75.0), 0.25, np.array([0.05, 0.1, 0.0], np.float32)
    full_d = oracle.full_depth(sc_h)
    rec = oracle.project(sc_h, full_d, t, cam)
    seen = np.bincount(sc_h.cluster_of(), weights=rec[:, 0], minlength=sc_h.n_clusters)
    vis = np.argsort(-seen)
    groups = np.array([[vis[0], 0], [vis[0], 1], [vis[1], 2], [vis[2], 3], [vis[3], 0], [vis[5], 1]], np.int32)
    G, M = len(groups), 10
    ctx = synth.group_contexts(groups, M, sc_h.n_clusters, sc_h.n_layers, np.random.default_rng(11))
    states = synth.States(ctx, np.full(G * M, t, np.float32), np.zeros(G * M, np.int32))
    sc = dgs.DeviceScene.from_host(sc_h)
    delta_t, stats_t = R.group_utility(sc, dgs.DeviceStates.from_host(states), groups, M, [cam], bg)
    delta, stats = delta_t.cpu().numpy(), stats_t.cpu().numpy()
    for g in range(G):
        ref = oracle.utility_stats(delta[g])
        assert np.allclose(stats[g], ref, rtol=1e-12, atol=1e-15), (g, stats[g], ref)
    # paired masks (m rows, then m u g rows), rendered as images on the GPU
    L = sc_h.n_layers
    pairs = np.concatenate([ctx, ctx.copy()])
    for k in range(G * M):
        c, l = groups[k // M]
        pairs[G * M + k, (c * L + l) // 32] |= np.uint32(1 << ((c * L + l) % 32))
    pst = synth.States(pairs, np.full(2 * G * M, t, np.float32), np.zeros(2 * G * M, np.int32))
    imgs = R.render_states_batched(sc, dgs.DeviceStates.from_host(pst), [cam], bg)
    fullm = torch.full((1, pairs.shape[1]), -1, dtype=torch.int32, device="cuda")
    fimg = R.render_states_batched(sc, dgs.DeviceStates(fullm, np.full(1, t, np.float32), np.zeros(1, np.int32)),
                                   [cam], bg)
    mse_g, _, _ = R.image_mse(imgs, fimg, np.zeros(2 * G * M, np.int32))
    mse_g = mse_g.cpu().numpy()
    assert np.allclose(delta.ravel(), mse_g[:G * M] - mse_g[G * M:], rtol=1e-12, atol=1e-16)
    # the FP64 oracle, per state: every pixel within 1e-4 plus the oracle's
    # derived bound (both renders).  Tight check: Delta over the pixels neither
    # render flags, from the GPU's images (tied to the API's Delta above).
    full, mfull, _, bfull = oracle.render(sc_h, full_d, t, cam, bg, want_bound=True)
    imgs_h = imgs.cpu().numpy().astype(np.float64)
    fimg_h = fimg[0].cpu().numpy().astype(np.float64)
    n_val = full.size
    mse_o = np.zeros(2 * G * M); tol = np.zeros(2 * G * M)
    m_o = np.zeros(2 * G * M); m_g = np.zeros(2 * G * M); tol_m = np.zeros(2 * G * M)
    for k in range(2 * G * M):
        img, marg, _, bnd = oracle.render(sc_h, oracle.closure(pairs[k], sc_h.n_clusters, L), t, cam, bg,
                                          want_bound=True)
        d = img - full
        mse_o[k] = np.mean(d * d)
        flagged = np.broadcast_to((marg | mfull)[..., None], d.shape)
        tol[k] = _mse_tol(d, 2 * IMG_TOL + bnd + bfull)
        dg = imgs_h[k] - fimg_h
        m_o[k] = np.sum(np.where(flagged, 0.0, d * d)) / n_val
        m_g[k] = np.sum(np.where(flagged, 0.0, dg * dg)) / n_val
        tol_m[k] = np.sum(np.where(flagged, 0.0, 4 * IMG_TOL * np.abs(d) + 4 * IMG_TOL ** 2)) / n_val \
            + 5 * 2.0 ** -24 * m_o[k]
    delta_o = (mse_o[:G * M] - mse_o[G * M:]).reshape(G, M)
    tol_d = (tol[:G * M] + tol[G * M:]).reshape(G, M)
    assert np.all(np.abs(delta - delta_o) <= tol_d), np.max(np.abs(delta - delta_o) - tol_d)
    dm_o = (m_o[:G * M] - m_o[G * M:]).reshape(G, M)
    dm_g = (m_g[:G * M] - m_g[G * M:]).reshape(G, M)
    tol_dm = (tol_m[:G * M] + tol_m[G * M:]).reshape(G, M)
    assert np.all(np.abs(dm_g - dm_o) <= tol_dm), np.max(np.abs(dm_g - dm_o) - tol_dm)
    assert np.abs(dm_o).max() > 1e-3                 # the groups do change the image
    assert np.median(tol_dm) < 0.05 * np.abs(dm_o).max()
    for g in range(G):
        ref = np.array(oracle.utility_stats(delta_o[g]))
        bound = tol_d[g].max()
        assert np.all(np.abs(stats[g, :3] - ref[:3]) <= bound + 1e-15), (g, stats[g], ref, bound)
        assert abs(stats[g, 3] - ref[3]) <= 2 * bound + 1e-15
        # the same statistics of the masked Delta: tight
        sg, so = np.array(oracle.utility_stats(dm_g[g])), np.array(oracle.utility_stats(dm_o[g]))
        assert np.all(np.abs(sg[:3] - so[:3]) <= tol_dm[g].max() + 1e-15)


# --------------------------------------------------------------------- Eq. 2 objective
@pytest.mark.parametrize("S,H,W,cvar_q", [(9, 37, 53, 0.25), (1, 16, 16, 0.05), (300, 20, 33, 0.05)])
def test_objective_matches_oracle(R, torch, S, H, W, cvar_q):
    """Eq. 2 on the GPU against the FP64 oracle: per-state D, the loss and the
    gradient.  Images are references plus noise of distinct levels, so the CVaR
    tail and the prefix-hinge signs are far from ties.  Sizes span ragged 32x16
    SSIM tiles, a single state, and a non-power-of-two batch for the CVaR sort."""
    rng = np.random.default_rng(S)
    n_refs = min(3, S)
    refs = rng.uniform(size=(n_refs, H, W, 3))
    ridx = rng.integers(0, n_refs, size=S)
    levels = np.linspace(0.01, 0.3, S)[rng.permutation(S)]
    imgs = refs[ridx] + levels[:, None, None, None] * rng.normal(size=(S, H, W, 3))
    imgs = imgs.astype(np.float32).astype(np.float64)
    refs = refs.astype(np.float32).astype(np.float64)
    pt = [(i, i + 1) for i in range(0, S - 1, 3)]
    pm = [(i, (i + 2) % S) for i in range(0, S, 2)] if S > 1 else []
    an = [S - 1, 0] if S > 1 else [0]
    kw = dict(pairs_t=pt, pairs_m=pm, anchors=an)
    L_o, D_o, g_o = oracle.objective(imgs, refs, ridx, cvar_q=cvar_q, **kw)
    loss, D, dL = R.objective(torch.from_numpy(imgs.astype(np.float32)).cuda(),
                              torch.from_numpy(refs.astype(np.float32)).cuda(), ridx, params=dict(cvar_q=cvar_q), **kw)
    D, loss, dL = D.cpu().numpy(), float(loss.item()), dL.cpu().numpy().astype(np.float64)
    assert np.allclose(D, D_o, rtol=1e-5, atol=2e-7), np.abs(D - D_o).max()
    assert loss == pytest.approx(L_o, rel=1e-5, abs=2e-7)
    assert np.abs(dL - g_o).max() <= 2e-4 * np.abs(g_o).max(), (np.abs(dL - g_o).max(), np.abs(g_o).max())


def test_objective_through_autograd_to_the_scene(R, torch):
    """loss = Eq. 2 of the batched render; loss.backward() reaches every scene
    tensor through both library adjoints, and equals the chained library calls."""
    sc_h, states, cams = _grad_case()
    sc = dgs.DeviceScene.from_host(sc_h)
    st = dgs.DeviceStates.from_host(states)
    bg = np.zeros(3, np.float32)
    full = torch.full_like(st.masks, -1)
    refs = R.render_states_batched(sc, dgs.DeviceStates(full, states.t, states.cam), cams, bg)
    ridx = np.arange(states.n)
    for v in sc.t.values():
        v.requires_grad_(True)
    img = dgs.render(R, sc, st, cams, bg)
    loss, D = dgs.objective(R, img, refs, ridx, pairs_m=[(0, 1)], anchors=[2])
    loss.backward()
    g_auto = {k: sc.t[k].grad.clone() for k in dgs.SCENE_FIELDS}
    assert all(torch.isfinite(g).all() for g in g_auto.values())
    assert float(g_auto["mu0"].abs().max()) > 0 and float(g_auto["colour"].abs().max()) > 0
    # the same chain by hand
    imgs = R.render_states_batched(sc, st, cams, bg)
    l2, _, dL = R.objective(imgs, refs, ridx, pairs_m=[(0, 1)], anchors=[2])
    g_hand = R.render_backward(sc, st, cams, bg, dL, images=imgs)
    assert abs(float(l2.item()) - float(loss.item())) <= 1e-12 * abs(float(loss.item()))
    for k in dgs.SCENE_FIELDS:
        if g_hand[k].numel():
            assert torch.allclose(g_auto[k], g_hand[k], rtol=1e-4, atol=1e-6 * float(g_hand[k].abs().max()) + 1e-12)


# --------------------------------------------------------------------- cluster affine (Eq. 1)
def test_cluster_affine_matches_oracle_forward_backward_and_plan(R, torch):
    """Scenes with cluster affine keyframes: batched images against the oracle
    (non-marginal pixels), the adjoint (including the keyframe gradients)
    against the oracle's, and a capture-safe plan equal to the context calls."""
    import dataclasses
    sc_h, states, cams = _grad_case()
    A = synth.cluster_affine(sc_h.n_clusters, 3, np.random.default_rng(12))
    sca = dataclasses.replace(sc_h, affine=A)
    bg = np.array([0.1, 0.2, 0.3], np.float32)
    sc = dgs.DeviceScene.from_host(sca)
    st = dgs.DeviceStates.from_host(states)
    imgs = R.render_states_batched(sc, st, cams, bg)
    D = oracle.state_depths(states, sca.n_clusters, sca.n_layers)
    rng = np.random.default_rng(3)
    S, H, W = states.n, cams[0].height, cams[0].width
    dL = rng.normal(size=(S, H, W, 3))
    ref = None
    for s in range(S):
        cam = cams[int(states.cam[s])]
        img_o, marg, _, bnd = oracle.render(sca, D[s], float(states.t[s]), cam, bg, want_bound=True)
        err, _ = _compare_image(imgs[s].cpu().numpy(), img_o, bnd)
        assert err <= IMG_TOL, (s, err)
        g = oracle.render_backward(sca, D[s], float(states.t[s]), cam, bg, dL[s])
        ref = g if ref is None else {k: ref[k] + g[k] for k in ref}
    dLt = torch.from_numpy(dL.astype(np.float32)).cuda()
    grads = R.render_backward(sc, st, cams, bg, dLt, images=imgs)
    assert float(np.abs(ref["affine"]).max()) > 0
    for k in sc.fields:
        gg = grads[k].cpu().numpy().astype(np.float64)
        gr = ref[k]
        if gr.size == 0:
            continue
        scale = max(np.abs(gr).max(), 1e-6)
        assert np.abs(gg - gr).max() <= GRAD_TOL * scale, (k, np.abs(gg - gr).max(), scale)
    plan = dgs.Plan(R, sc, st, cams, bg, dgs.PLAN_RENDER, entry_headroom=2.0)
    out = torch.empty_like(imgs)
    plan.render(st.masks, out)
    assert torch.equal(out, imgs)
    gp = plan.backward(dLt, sc.zeros_like_grads(), images=out)
    for k in sc.fields:
        if grads[k].numel():
            assert torch.allclose(gp[k], grads[k], rtol=1e-4, atol=1e-5 * float(grads[k].abs().max()) + 1e-12), k
    plan.close()


# --------------------------------------------------------------------- quantized refinements
@pytest.mark.parametrize("mode", [1, 2])
def test_quantized_refinements_match_oracle(R, torch, mode):
    """Refinements read as int16 symbols times learned steps (mode 1) or
    quantized on the fly with straight-through gradients (mode 2): images
    against the oracle (derived bounds at flagged pixels) and the adjoint
    (refinements and steps) against the oracle's."""
    import dataclasses
    sc_h, states, cams = _grad_case()
    q, step = synth.quantize_residuals(sc_h, step_scale=1.0 / 16.0)      # coarse: the quantization shows
    scq = dataclasses.replace(sc_h, res_q=q, res_step=step, res_mode=mode)
    bg = np.array([0.1, 0.2, 0.3], np.float32)
    sc = dgs.DeviceScene.from_host(scq)
    st = dgs.DeviceStates.from_host(states)
    imgs = R.render_states_batched(sc, st, cams, bg)
    D = oracle.state_depths(states, scq.n_clusters, scq.n_layers)
    rng = np.random.default_rng(4)
    S, H, W = states.n, cams[0].height, cams[0].width
    dL = rng.normal(size=(S, H, W, 3))
    ref = None
    for s in range(S):
        cam = cams[int(states.cam[s])]
        img_o, marg, _, bnd = oracle.render(scq, D[s], float(states.t[s]), cam, bg, want_bound=True)
        err, _ = _compare_image(imgs[s].cpu().numpy(), img_o, bnd)
        assert err <= IMG_TOL, (s, err)
        g = oracle.render_backward(scq, D[s], float(states.t[s]), cam, bg, dL[s])
        ref = g if ref is None else {k: ref[k] + g[k] for k in ref}
    grads = R.render_backward(sc, st, cams, bg, torch.from_numpy(dL.astype(np.float32)).cuda(), images=imgs)
    if mode == 2:
        assert "res_step" in sc.fields and float(np.abs(ref["res_step"]).max()) > 0
    for k in sc.fields:
        gg = grads[k].cpu().numpy().astype(np.float64)
        gr = ref[k]
        if gr.size == 0:
            continue
        scale = max(np.abs(gr).max(), 1e-6)
        assert np.abs(gg - gr).max() <= GRAD_TOL * scale, (mode, k, np.abs(gg - gr).max(), scale)
