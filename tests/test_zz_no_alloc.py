"""dgs_image_mse_noalloc against dgs_image_mse (needs a GPU).

The no-allocation entry point serves callers that cannot allocate device
memory (code inside a memory pool or arena it does not own, real-time loops,
hosts that forbid a library from touching the allocator).  Its output must
match the allocating entry point's on consecutive calls, which share one fixed
scratch array; sizes beyond that scratch must be refused before any launch.
"""
import numpy as np
import pytest

from paper_2606_17212_b300 import dgs

pytestmark = pytest.mark.gpu


def test_noalloc_matches_image_mse_on_two_calls_in_a_row():
    import torch
    R = dgs.Renderer(0)
    rng = np.random.default_rng(42)
    shapes = [(5, 37, 29, 2, 0.2), (3, 64, 48, 3, 1.0)]   # S, H, W, refs, weight
    for S, H, W, n_refs, weight in shapes:
        images = torch.from_numpy(rng.uniform(size=(S, H, W, 3)).astype(np.float32)).cuda()
        refs = torch.from_numpy(rng.uniform(size=(n_refs, H, W, 3)).astype(np.float32)).cuda()
        idx = rng.integers(0, n_refs, size=S).astype(np.int32)
        mse_ref, psnr_ref, dL_ref = R.image_mse(images, refs, idx, weight=weight, want_grad=True)
        idx_dev = torch.from_numpy(idx).cuda()
        mse = torch.empty(S, dtype=torch.float64, device="cuda")
        psnr = torch.empty(S, dtype=torch.float64, device="cuda")
        dL = torch.empty_like(images)
        rc = dgs.image_mse_noalloc(images, refs, idx_dev, mse, psnr, dL, weight=weight)
        assert rc == dgs.DGS_OK
        torch.cuda.synchronize()
        assert torch.allclose(mse, mse_ref, rtol=1e-12, atol=0)
        assert torch.allclose(psnr, psnr_ref, rtol=1e-12, atol=0)
        assert torch.allclose(dL, dL_ref, rtol=1e-6, atol=1e-12)
    R.close()


def test_noalloc_out_of_range_reference_gives_nan_for_that_image_only():
    """An index equal to n_refs or negative makes that image's MSE and its
    dL/dimages NaN (the read is redirected to refs[0], never past refs); the
    other images still match dgs_image_mse."""
    import torch
    R = dgs.Renderer(0)
    rng = np.random.default_rng(7)
    S, H, W, n_refs = 4, 33, 21, 2
    images = torch.from_numpy(rng.uniform(size=(S, H, W, 3)).astype(np.float32)).cuda()
    refs = torch.from_numpy(rng.uniform(size=(n_refs, H, W, 3)).astype(np.float32)).cuda()
    idx = np.array([1, n_refs, 0, -1], np.int32)
    good = [0, 2]
    mse_ref, _, dL_ref = R.image_mse(images[good], refs, idx[good], weight=0.5, want_grad=True)
    mse = torch.empty(S, dtype=torch.float64, device="cuda")
    dL = torch.empty_like(images)
    for _ in range(2):
        rc = dgs.image_mse_noalloc(images, refs, torch.from_numpy(idx).cuda(), mse, None, dL, weight=0.5)
        assert rc == dgs.DGS_OK
        torch.cuda.synchronize()
        assert torch.isnan(mse[1]) and torch.isnan(mse[3])
        assert torch.isnan(dL[1]).all() and torch.isnan(dL[3]).all()
        assert torch.allclose(mse[good], mse_ref, rtol=1e-12, atol=0)
        assert torch.allclose(dL[good], dL_ref, rtol=1e-6, atol=1e-12)
    R.close()


def test_noalloc_refuses_sizes_beyond_its_scratch():
    """400 images of 512 x 512 need 400 * ceil(512 * 512 / 1024) = 102,400 partial
    sums > 65,536: refused before any launch.  Every buffer is sized for the shape
    it is passed with, so even a refusal that failed could not read out of bounds."""
    import torch
    S, H, W = 400, 512, 512
    parts = -(-H * W // 1024)
    assert S * parts > dgs.NOALLOC_MAX_PARTS
    images = torch.zeros((S, H, W, 3), dtype=torch.float32, device="cuda")
    refs = torch.zeros((1, H, W, 3), dtype=torch.float32, device="cuda")
    idx = torch.zeros(S, dtype=torch.int32, device="cuda")
    mse = torch.full((S,), -1.0, dtype=torch.float64, device="cuda")
    rc = dgs.image_mse_noalloc(images, refs, idx, mse)
    assert rc == dgs.DGS_E_SCRATCH
    torch.cuda.synchronize()
    assert torch.all(mse == -1.0)          # nothing was launched
    del images
