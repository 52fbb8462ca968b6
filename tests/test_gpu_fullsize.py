"""Parity at the workloads' full sizes, in the launch configuration bench.py times.

The oracle cannot render 250k-2.7M Gaussian scenes in full, so these tests check
sampled outputs it computes one pixel at a time (forward) and the adjoint of
sampled pixels (backward: dL/dI is non-zero only at sampled pixels, so the
oracle's adjoint costs one pixel scan per sample), plus properties that hold at
any size.  Every sampled pixel is compared: where the oracle flags a threshold
decision FP32 may take the other way, the tolerance adds the oracle's derived
bound on how far that decision moves the pixel.
"""
import numpy as np
import pytest

import oracle
from paper_2606_17212_b300 import dgs, synth

pytestmark = pytest.mark.gpu

IMG_TOL = 1e-4
GRAD_TOL = 1e-3


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


def _samples(rng, W, H, n):
    flat = rng.choice(W * H, size=n, replace=False)
    return np.stack([flat % W, flat // W], 1).astype(np.int32)


def _check_sampled(w, imgs, which, rng, n_pix=96):
    D = oracle.state_depths(w.states, w.scene.n_clusters, w.scene.n_layers)
    out = {}
    for s in which:
        cam = w.cams[int(w.states.cam[s])]
        pix = _samples(rng, cam.width, cam.height, n_pix)
        ref, marg, _, bnd = oracle.render(w.scene, D[s], float(w.states.t[s]), cam, w.bg, pix=pix,
                                          want_bound=True)
        got = imgs[s][pix[:, 1], pix[:, 0]].astype(np.float64)
        err = np.abs(got - ref) - bnd[:, None]
        assert err.max() <= IMG_TOL, (s, err.max(), int(marg.sum()))
        # ~150 Gaussians per pixel: near-threshold decisions are common, but their
        # derived bounds stay small; few pixels are checked only loosely
        assert (bnd > 1e-2).mean() <= 0.03, (s, np.sort(bnd)[-5:])
        out[s] = (pix, marg)
    return out


def test_fwdbwd_250k_full_size(R, torch):
    """Training workload: 250k Gaussians, 64 states, 512x512, 8 cameras."""
    w = synth.config("c3_fwdbwd_250k")
    sc = dgs.DeviceScene.from_host(w.scene)
    st = dgs.DeviceStates.from_host(w.states)
    imgs_t = R.render_states_batched(sc, st, w.cams, w.bg)
    imgs = imgs_t.cpu().numpy()
    rng = np.random.default_rng(0)
    which = [0, 7, 33, 62]
    samp = _check_sampled(w, imgs, which, rng)
    # batched == per-state, bit for bit, at full size
    for s in which:
        one = R.render_state(sc, st.masks[s], float(w.states.t[s]), w.cams[int(w.states.cam[s])], w.bg)
        assert torch.equal(one, imgs_t[s]), s
    # adjoint of the sampled pixels through the full 64-state batched backward
    S, H, W = st.n, w.cams[0].height, w.cams[0].width
    dL = np.zeros((S, H, W, 3), np.float32)
    D = oracle.state_depths(w.states, w.scene.n_clusters, w.scene.n_layers)
    ref = None
    for s in which:
        pix, marg = samp[s]
        keep = pix
        dL[s, keep[:, 1], keep[:, 0]] = rng.normal(size=(len(keep), 3)).astype(np.float32)
        g = oracle.render_backward(w.scene, D[s], float(w.states.t[s]), w.cams[int(w.states.cam[s])], w.bg,
                                   dL[s].astype(np.float64))
        ref = g if ref is None else {k: ref[k] + g[k] for k in ref}
    imgs_t = R.render_states_batched(sc, st, w.cams, w.bg)
    grads = R.render_backward(sc, st, w.cams, w.bg, torch.from_numpy(dL).cuda(), images=imgs_t)
    for k in dgs.SCENE_FIELDS:
        gr = ref[k]
        if gr.size == 0:
            continue
        gg = grads[k].cpu().numpy().astype(np.float64)
        scale = max(np.abs(gr).max(), 1e-6)
        assert np.abs(gg - gr).max() <= GRAD_TOL * scale, (k, np.abs(gg - gr).max(), scale)


def test_dynamic_forward_250k_full_size(R, torch):
    """Batched forward: 250k Gaussians, 256 states, 800x800, 16 times."""
    w = synth.config("c2_dynamic_250k")
    sc = dgs.DeviceScene.from_host(w.scene)
    st = dgs.DeviceStates.from_host(w.states)
    imgs_t = R.render_states_batched(sc, st, w.cams, w.bg)
    rng = np.random.default_rng(1)
    which = [0, 100, 255]
    _check_sampled(w, {s: imgs_t[s].cpu().numpy() for s in which}, which, rng)
    # PSNR per state from the fused utility path == from the written images
    mse, psnr = R.state_utility(sc, st, w.cams, w.bg)
    tv = np.unique(w.states.t)
    full = torch.full((len(tv), st.masks.shape[1]), -1, dtype=torch.int32, device="cuda")
    fulls = R.render_states_batched(sc, dgs.DeviceStates(full, tv, np.zeros(len(tv), np.int32)), w.cams, w.bg)
    m2, p2, _ = R.image_mse(imgs_t, fulls, np.searchsorted(tv, w.states.t))
    assert torch.allclose(mse, m2, rtol=1e-12, atol=0)
    assert torch.allclose(psnr, p2, rtol=1e-12, atol=0)


def test_utility_sweep_2p7m_full_size(R, torch):
    """Utility sweep: 2.7M Gaussians, 32,768 distinct states, 480x270, one launch."""
    w = synth.config("c4_utility_2p7m")
    sc = dgs.DeviceScene.from_host(w.scene)
    st = dgs.DeviceStates.from_host(w.states)
    mse, psnr = R.state_utility(sc, st, w.cams, w.bg)
    # tile reuse across the 32,768 states (on by default) changes no bit
    R.set_tile_reuse(False)
    try:
        mse_plain, _ = R.state_utility(sc, st, w.cams, w.bg)
    finally:
        R.set_tile_reuse(True)
    assert torch.equal(mse, mse_plain)
    mse = mse.cpu().numpy()
    # >= 0: pixels stop inside the front clusters of this dense scene, so a state that
    # delivers those completely renders bit-identically to the complete state (MSE 0)
    assert np.all(np.isfinite(mse)) and np.all(mse >= 0) and np.median(mse) > 0
    which = [0, 12345, 32767]
    sub = dgs.DeviceStates(st.masks[which], w.states.t[which], w.states.cam[which])
    imgs_t = R.render_states_batched(sc, sub, w.cams, w.bg)
    full = torch.full((1, st.masks.shape[1]), -1, dtype=torch.int32, device="cuda")
    fulls = R.render_states_batched(sc, dgs.DeviceStates(full, w.states.t[:1], np.zeros(1, np.int32)), w.cams,
                                    w.bg)
    m2, _, _ = R.image_mse(imgs_t, fulls, np.zeros(len(which), np.int32))
    assert np.allclose(mse[which], m2.cpu().numpy(), rtol=1e-12, atol=0)
    sub_states = synth.States(w.states.masks[which], w.states.t[which], w.states.cam[which])
    w_sub = synth.Workload(w.name, w.scene, w.cams, sub_states, w.bg)
    imgs = imgs_t.cpu().numpy()
    _check_sampled(w_sub, {k: imgs[k] for k in range(len(which))}, range(len(which)), np.random.default_rng(2),
                   n_pix=48)


def test_serving_mix_scenes_full_size(R, torch):
    """Serving-shaped mix (SH degree 3, 64 states per scene): the smallest
    scene, the largest (2.47M Gaussians) and a 960x540 one at full size;
    sampled pixels of the batched forward and the adjoint of sampled pixels
    through the batched backward against the oracle."""
    specs = synth.mix_specs()
    by_n = sorted(specs, key=lambda s: s.n)
    wide = [s for s in specs if (s.width, s.height) == (960, 540)]
    pick = [by_n[0], by_n[-1], wide[len(wide) // 2]]
    rng = np.random.default_rng(5)
    for spec in pick:
        w = synth.mix_workload(spec)
        sc = dgs.DeviceScene.from_host(w.scene)
        st = dgs.DeviceStates.from_host(w.states)
        imgs_t = R.render_states_batched(sc, st, w.cams, w.bg)
        which = [0, 37]
        samp = _check_sampled(w, {s: imgs_t[s].cpu().numpy() for s in which}, which, rng, n_pix=64)
        S, H, W = st.n, w.cams[0].height, w.cams[0].width
        dL = np.zeros((S, H, W, 3), np.float32)
        D = oracle.state_depths(w.states, w.scene.n_clusters, w.scene.n_layers)
        ref = None
        for s in which:
            pix, marg = samp[s]
            keep = pix
            dL[s, keep[:, 1], keep[:, 0]] = rng.normal(size=(len(keep), 3)).astype(np.float32)
            g = oracle.render_backward(w.scene, D[s], float(w.states.t[s]), w.cams[int(w.states.cam[s])], w.bg,
                                       dL[s].astype(np.float64))
            ref = g if ref is None else {k: ref[k] + g[k] for k in ref}
        grads = R.render_backward(sc, st, w.cams, w.bg, torch.from_numpy(dL).cuda(), images=imgs_t)
        for k in dgs.SCENE_FIELDS:
            gr = ref[k]
            if gr.size == 0:
                continue
            gg = grads[k].cpu().numpy().astype(np.float64)
            scale = max(np.abs(gr).max(), 1e-6)
            assert np.abs(gg - gr).max() <= GRAD_TOL * scale, (spec.index, k, np.abs(gg - gr).max(), scale)
        del sc, st, imgs_t, grads
