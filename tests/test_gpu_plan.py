"""Capture-safe plans: equal to the context calls, and replayable in a CUDA graph."""
import numpy as np
import pytest

from paper_2606_17212_b300 import dgs, synth

pytestmark = pytest.mark.gpu


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


def _masks(torch, w, seed):
    rng = np.random.default_rng(seed)
    sc = w.scene
    d = synth.prefix_states(w.states.n, sc.n_clusters, sc.n_layers, rng)
    bits = synth.erase_one_packet(synth.depths_to_bits(d, sc.n_layers), 0.2, rng)
    return torch.from_numpy(synth._pack(bits).view(np.int32)).cuda()


def test_plan_render_backward_match_and_replay_in_graph(R, torch):
    w = synth.config("c3_fwdbwd_250k", scale=0.05, n_states=12)
    sc = dgs.DeviceScene.from_host(w.scene)
    st = dgs.DeviceStates.from_host(w.states)
    S, H, W = st.n, w.cams[0].height, w.cams[0].width
    plan = dgs.Plan(R, sc, st, w.cams, w.bg, dgs.PLAN_RENDER, entry_headroom=2.0)
    masks = st.masks.clone()
    images = torch.empty((S, H, W, 3), device="cuda")
    plan.render(masks, images)
    ref = R.render_states_batched(sc, st, w.cams, w.bg)
    assert torch.equal(images, ref)
    rng = np.random.default_rng(0)
    dL = torch.from_numpy(rng.normal(size=(S, H, W, 3)).astype(np.float32)).cuda()
    g_plan = plan.backward(dL, sc.zeros_like_grads(), images=images)
    g_ref = R.render_backward(sc, st, w.cams, w.bg, dL)          # final pixels recomputed
    for k in dgs.SCENE_FIELDS:
        a, b = g_plan[k], g_ref[k]
        if b.numel():
            assert torch.allclose(a, b, rtol=1e-4, atol=1e-5 * float(b.abs().max()) + 1e-12), k
    # capture forward + backward once, replay with other masks
    grads = sc.zeros_like_grads()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        plan.render(masks, images)
        plan.backward(dL, grads, images=images)
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        for g in grads.values():
            g.zero_()
        plan.render(masks, images)
        plan.backward(dL, grads, images=images)
    for seed in (1, 2):
        new = _masks(torch, w, seed)
        masks.copy_(new)
        graph.replay()
        torch.cuda.synchronize()
        plan.status()
        st_new = dgs.DeviceStates(new, w.states.t, w.states.cam)
        assert torch.equal(images, R.render_states_batched(sc, st_new, w.cams, w.bg))
        g_ref = R.render_backward(sc, st_new, w.cams, w.bg, dL)
        for k in dgs.SCENE_FIELDS:
            if g_ref[k].numel():
                assert torch.allclose(grads[k], g_ref[k], rtol=1e-4,
                                      atol=1e-5 * float(g_ref[k].abs().max()) + 1e-12), (seed, k)
    plan.close()


def test_plan_utility_and_image_mse(R, torch):
    w = synth.config("c2_dynamic_250k", scale=0.02, n_states=20)
    sc = dgs.DeviceScene.from_host(w.scene)
    st = dgs.DeviceStates.from_host(w.states)
    plan = dgs.Plan(R, sc, st, w.cams, w.bg, dgs.PLAN_UTILITY)
    mse = torch.empty(st.n, dtype=torch.float64, device="cuda")
    psnr = torch.empty_like(mse)
    masks = st.masks.clone()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        plan.utility(masks, mse, psnr)
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        plan.utility(masks, mse, psnr)
    graph.replay()
    torch.cuda.synchronize()
    m_ref, p_ref = R.state_utility(sc, st, w.cams, w.bg)
    assert torch.equal(mse, m_ref) and torch.equal(psnr, p_ref)
    plan.close()
    # one view, many states: the context call reuses tiles, the plan renders every pair
    w4 = synth.config("c4_utility_2p7m", scale=0.02, n_states=96)
    sc4 = dgs.DeviceScene.from_host(w4.scene)
    st4 = dgs.DeviceStates.from_host(w4.states)
    plan4 = dgs.Plan(R, sc4, st4, w4.cams, w4.bg, dgs.PLAN_UTILITY)
    m4 = torch.empty(st4.n, dtype=torch.float64, device="cuda")
    p4 = torch.empty_like(m4)
    plan4.utility(st4.masks.clone(), m4, p4)
    torch.cuda.synchronize()
    m4_ref, _ = R.state_utility(sc4, st4, w4.cams, w4.bg)
    assert R.tile_reuse_stats()[2] > 0
    assert torch.equal(m4, m4_ref)
    plan4.close()
    # image MSE through a render plan with reference indices
    tv = np.unique(w.states.t)
    ridx = np.searchsorted(tv, w.states.t).astype(np.int32)
    plan2 = dgs.Plan(R, sc, st, w.cams, w.bg, dgs.PLAN_RENDER, ref_index=ridx, n_refs=len(tv))
    imgs = R.render_states_batched(sc, st, w.cams, w.bg)
    full = torch.full((len(tv), st.masks.shape[1]), -1, dtype=torch.int32, device="cuda")
    refs = R.render_states_batched(sc, dgs.DeviceStates(full, tv, np.zeros(len(tv), np.int32)), w.cams, w.bg)
    m1, p1, d1 = R.image_mse(imgs, refs, ridx, weight=0.5, want_grad=True)
    m2, p2, d2 = torch.empty_like(m1), torch.empty_like(p1), torch.empty_like(d1)
    plan2.image_mse(imgs, refs, m2, p2, d2, weight=0.5)
    torch.cuda.synchronize()
    assert torch.equal(m1, m2) and torch.equal(d1, d2)
    # the fused pass: the same images and dL/dI bits; the MSE sums the same FP32
    # squared errors in another FP64 order; a backward may follow it
    img3, m3, p3, d3 = torch.empty_like(imgs), torch.empty_like(m1), torch.empty_like(p1), torch.full_like(d1, 7.0)
    plan2.render_mse(st.masks.clone(), img3, refs, m3, p3, d3, weight=0.5)
    torch.cuda.synchronize()
    assert torch.equal(img3, imgs) and torch.equal(d3, d1)
    assert torch.allclose(m3, m1, rtol=1e-12, atol=0.0) and torch.allclose(p3, p1, rtol=1e-12, atol=0.0)
    g = plan2.backward(d3, sc.zeros_like_grads(), images=img3)
    g_ref = R.render_backward(sc, st, w.cams, w.bg, d1, images=imgs)
    for k in dgs.SCENE_FIELDS:
        if g_ref[k].numel():
            assert torch.allclose(g[k], g_ref[k], rtol=1e-4, atol=1e-5 * float(g_ref[k].abs().max()) + 1e-12), k
    plan2.close()


def test_plan_reports_entry_overflow_without_faulting(R, torch):
    """A plan sized on sparse masks, run on complete masks, drops entries past its
    capacity (every write stays inside the reserved buffers) and says so."""
    w = synth.config("c3_fwdbwd_250k", scale=0.3, n_states=4)    # ~2M entries when complete
    sc = dgs.DeviceScene.from_host(w.scene)
    sparse = torch.zeros((w.states.n, w.states.masks.shape[1]), dtype=torch.int32, device="cuda")
    sparse[:, 0] = 1                          # only cluster 0's base layer
    st = dgs.DeviceStates(sparse, w.states.t, w.states.cam)
    plan = dgs.Plan(R, sc, st, w.cams, w.bg, dgs.PLAN_RENDER, entry_headroom=1.0)
    images = torch.empty((st.n, w.cams[0].height, w.cams[0].width, 3), device="cuda")
    plan.render(sparse, images)
    plan.status()                             # fits
    full = torch.full_like(sparse, -1)
    plan.render(full, images)
    with pytest.raises(RuntimeError, match="DGS_E_CAPACITY"):
        plan.status()
    plan.status()                             # the flag was cleared
    plan.close()


def _mix_case(torch, R, spec, n_states):
    w = synth.mix_workload(spec, n_states=n_states)
    sc = dgs.DeviceScene.from_host(w.scene)
    st = dgs.DeviceStates.from_host(w.states)
    views = sorted(set(zip(w.states.cam.tolist(), w.states.t.tolist())))
    ridx = np.array([views.index(v) for v in zip(w.states.cam.tolist(), w.states.t.tolist())], np.int32)
    full = torch.full((len(views), st.masks.shape[1]), -1, dtype=torch.int32, device="cuda")
    fv = dgs.DeviceStates(full, np.array([v[1] for v in views], np.float32), np.array([v[0] for v in views], np.int32))
    targets = R.render_states_batched(sc, fv, w.cams, w.bg)
    return w, sc, st, ridx, targets


def test_arena_plans_of_several_scenes_in_one_graph(R, torch):
    """Three scenes of the serving mix (SH degree 3, different sizes and
    resolutions), one plan each in a shared arena, the training step of all
    three captured in one CUDA graph: images equal the context calls bit for
    bit, gradients up to float atomic order, after replays with new masks."""
    specs = synth.mix_specs(scale=0.02)
    pick = [specs[0], specs[1], specs[2]]
    assert len({(s.width, s.height) for s in pick}) >= 2
    arena = dgs.Arena(R)
    cases = []
    for spec in pick:
        w, sc, st, ridx, targets = _mix_case(torch, R, spec, 12)
        plan = dgs.Plan(R, sc, st, w.cams, w.bg, dgs.PLAN_RENDER, ref_index=ridx, n_refs=int(targets.shape[0]),
                        entry_headroom=2.0, arena=arena)
        S, H, W = st.n, w.cams[0].height, w.cams[0].width
        cases.append(dict(w=w, sc=sc, st=st, ridx=ridx, targets=targets, plan=plan, masks=st.masks.clone(),
                          images=torch.empty((S, H, W, 3), device="cuda"),
                          mse=torch.empty(S, dtype=torch.float64, device="cuda"),
                          psnr=torch.empty(S, dtype=torch.float64, device="cuda"),
                          dL=torch.empty((S, H, W, 3), device="cuda"), grads=sc.zeros_like_grads()))

    def step():
        for c in cases:
            for g in c["grads"].values():
                g.zero_()
            c["plan"].render(c["masks"], c["images"])
            c["plan"].image_mse(c["images"], c["targets"], c["mse"], c["psnr"], c["dL"], weight=1.0 / c["st"].n)
            c["plan"].backward(c["dL"], c["grads"], images=c["images"])

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for seed in (3, 4):
        for c in cases:
            c["masks"].copy_(_masks(torch, c["w"], seed))
        graph.replay()
        torch.cuda.synchronize()
        for c in cases:
            c["plan"].status()
            w, sc = c["w"], c["sc"]
            st_new = dgs.DeviceStates(c["masks"], w.states.t, w.states.cam)
            imgs = R.render_states_batched(sc, st_new, w.cams, w.bg)
            assert torch.equal(c["images"], imgs)
            mse, _, dL = R.image_mse(imgs, c["targets"], c["ridx"], weight=1.0 / st_new.n, want_grad=True)
            assert torch.equal(c["mse"], mse)
            g_ref = R.render_backward(sc, st_new, w.cams, w.bg, dL, images=imgs)
            for k in dgs.SCENE_FIELDS:
                if g_ref[k].numel():
                    assert torch.allclose(c["grads"][k], g_ref[k], rtol=1e-4,
                                          atol=1e-5 * float(g_ref[k].abs().max()) + 1e-12), (seed, k)
    # a plan's backward must follow its own render within the arena
    a, b = cases[0], cases[1]
    a["plan"].render(a["masks"], a["images"])
    b["plan"].render(b["masks"], b["images"])
    with pytest.raises(RuntimeError, match="another plan of the arena"):
        a["plan"].backward(a["dL"], a["grads"], images=a["images"])
    with pytest.raises(RuntimeError, match="still alive"):
        arena.close()
    for c in cases:
        c["plan"].close()
    arena.close()


def test_scenes_batched_one_launch_equals_per_scene_calls(R, torch):
    """dgs_render_scenes_batched over three serving-mix scenes of different sizes
    and resolutions: every image equals dgs_render_states_batched of its scene,
    bit for bit; dgs_render_scenes_backward gives the per-scene gradients up to
    float atomic order; masks changed in place after the forward are refused."""
    specs = synth.mix_specs(scale=0.02)
    cases = []
    for spec in (specs[0], specs[1], specs[2]):
        w, sc, st, ridx, targets = _mix_case(torch, R, spec, 10)
        S, H, W = st.n, w.cams[0].height, w.cams[0].width
        cases.append(dict(w=w, sc=sc, st=st, images=torch.full((S, H, W, 3), 9.0, device="cuda")))
    assert len({(c["w"].cams[0].width, c["w"].cams[0].height) for c in cases}) >= 2
    jobs = [(c["sc"], c["st"], c["w"].cams, c["w"].bg, c["images"]) for c in cases]
    R.set_tile_size(32)
    try:
        R.render_scenes_batched(jobs)
        torch.cuda.synchronize()
        rng = np.random.default_rng(5)
        dls = [torch.from_numpy(rng.normal(size=tuple(c["images"].shape)).astype(np.float32)).cuda() for c in cases]
        grads = [c["sc"].zeros_like_grads() for c in cases]
        R.render_scenes_backward(jobs, dls, grads)
        torch.cuda.synchronize()
        for c, dl, g in zip(cases, dls, grads):
            ref = R.render_states_batched(c["sc"], c["st"], c["w"].cams, c["w"].bg)
            assert torch.equal(c["images"], ref)
            g_ref = R.render_backward(c["sc"], c["st"], c["w"].cams, c["w"].bg, dl, images=ref)
            for k in dgs.SCENE_FIELDS:
                if g_ref[k].numel():
                    assert torch.allclose(g[k], g_ref[k], rtol=1e-4, atol=1e-5 * float(g_ref[k].abs().max()) + 1e-12), k
        # a second call reuses the scene workspaces; masks edited in place after it are refused
        R.render_scenes_batched(jobs)
        cases[1]["st"].masks.copy_(_masks(torch, cases[1]["w"], 11))
        with pytest.raises(RuntimeError, match="STALE"):
            R.render_scenes_backward(jobs, dls, [c["sc"].zeros_like_grads() for c in cases])
    finally:
        R.set_tile_size(0)


def test_plan_objective_training_step_in_one_graph(R, torch):
    """Render, the Eq. 2 objective (with its image gradient) and the adjoint,
    all through one plan, captured in one CUDA graph: the loss, D and dL/dI
    carry the bits of the context calls, and the replayed step with new masks
    equals the context calls on those masks."""
    w = synth.config("c3_fwdbwd_250k", scale=0.05, n_states=12)
    sc = dgs.DeviceScene.from_host(w.scene)
    st = dgs.DeviceStates.from_host(w.states)
    S, H, W = st.n, w.cams[0].height, w.cams[0].width
    tv = np.unique(w.states.t)
    ridx = np.searchsorted(tv, w.states.t).astype(np.int32)
    full = torch.full((len(tv), st.masks.shape[1]), -1, dtype=torch.int32, device="cuda")
    refs = R.render_states_batched(sc, dgs.DeviceStates(full, tv, np.zeros(len(tv), np.int32)), w.cams, w.bg)
    plan = dgs.Plan(R, sc, st, w.cams, w.bg, dgs.PLAN_RENDER, ref_index=ridx, n_refs=len(tv), entry_headroom=2.0)
    kw = dict(pairs_t=[(0, 1), (2, 3), (5, 4)], pairs_m=[(0, 2), (6, 7)], anchors=[1, 11])
    prm = dict(cvar_q=0.25, lambda_c=0.4)
    with pytest.raises(RuntimeError):
        plan.objective(refs, refs, torch.empty(1, dtype=torch.float64, device="cuda"))   # not set yet
    with pytest.raises(RuntimeError):
        plan.set_objective(pairs_t=[(0, S)])                                          # out of range
    plan.set_objective(params=prm, **kw)
    masks = st.masks.clone()
    images = torch.empty((S, H, W, 3), device="cuda")
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    D = torch.empty(S, dtype=torch.float64, device="cuda")
    dL = torch.empty_like(images)
    grads = sc.zeros_like_grads()

    def step():
        for g in grads.values():
            g.zero_()
        plan.render(masks, images)
        plan.objective(images, refs, loss, D, dL)
        plan.backward(dL, grads, images=images)

    def check(states):
        img_ref = R.render_states_batched(sc, states, w.cams, w.bg)
        assert torch.equal(images, img_ref)
        l_ref, D_ref, dL_ref = R.objective(img_ref, refs, ridx, params=prm, **kw)
        assert torch.equal(loss, l_ref) and torch.equal(D, D_ref) and torch.equal(dL, dL_ref)
        g_ref = R.render_backward(sc, states, w.cams, w.bg, dL_ref, images=img_ref)
        for k in dgs.SCENE_FIELDS:
            if g_ref[k].numel():
                assert torch.allclose(grads[k], g_ref[k], rtol=1e-4,
                                      atol=1e-5 * float(g_ref[k].abs().max()) + 1e-12), k

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    check(st)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    for seed in (3, 4):
        new = _masks(torch, w, seed)
        masks.copy_(new)
        graph.replay()
        torch.cuda.synchronize()
        plan.status()
        check(dgs.DeviceStates(new, w.states.t, w.states.cam))
    plan.close()
