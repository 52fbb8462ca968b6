"""Thin Python binding of the C ABI in ``include/dgs.h`` (argument marshalling only).

Every step of the rendering path runs in the CUDA library ``libdgs.so``; this
module only passes torch tensors' device pointers, sizes and the current CUDA
stream.  There is no fallback: if the library is missing the import of
:func:`lib` raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdgs.so")

DGS_OK = 0
ERRORS = {-1: "DGS_E_INVALID_ARG", -2: "DGS_E_UNSUPPORTED", -3: "DGS_E_OOM", -4: "DGS_E_CUDA",
          -5: "DGS_E_CAPACITY", -6: "DGS_E_SCRATCH", -7: "DGS_E_STALE"}
DGS_E_SCRATCH = -6
NOALLOC_MAX_PARTS = 65536


class Scene_t(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_clusters", ctypes.c_int32), ("n_layers", ctypes.c_int32),
                ("sh_degree", ctypes.c_int32), ("temporal_rank", ctypes.c_int32),
                ("cluster_offsets", ctypes.c_void_p), ("mu0", ctypes.c_void_p), ("u", ctypes.c_void_p),
                ("log_scale", ctypes.c_void_p), ("quat", ctypes.c_void_p),
                ("opacity_logit", ctypes.c_void_p), ("colour", ctypes.c_void_p), ("res", ctypes.c_void_p),
                ("affine", ctypes.c_void_p), ("affine_T", ctypes.c_int32),
                ("res_q", ctypes.c_void_p), ("res_step", ctypes.c_void_p), ("res_mode", ctypes.c_int32)]


OBJECTIVE_KEYS = ("ssim_weight", "lambda_c", "cvar_q", "lambda_t", "lambda_m", "anchor_weight")
OBJECTIVE_DEFAULTS = dict(ssim_weight=0.20, lambda_c=0.30, cvar_q=0.05, lambda_t=0.10, lambda_m=2.0,
                          anchor_weight=0.50)


class ObjectiveParams_t(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in OBJECTIVE_KEYS]


class SceneGrad_t(ctypes.Structure):
    _fields_ = [(k, ctypes.c_void_p) for k in
                ("mu0", "u", "log_scale", "quat", "opacity_logit", "colour", "res", "affine", "res_step")]


class Camera_t(ctypes.Structure):
    _fields_ = [("R_wc", ctypes.c_float * 9), ("t_wc", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class States_t(ctypes.Structure):
    _fields_ = [("masks", ctypes.c_void_p), ("t", ctypes.c_void_p), ("cam", ctypes.c_void_p),
                ("n_states", ctypes.c_int32)]


class SceneJob_t(ctypes.Structure):
    _fields_ = [("scene", ctypes.POINTER(Scene_t)), ("states", States_t), ("cams", ctypes.POINTER(Camera_t)),
                ("n_cams", ctypes.c_int32), ("bg", ctypes.c_float * 3), ("images", ctypes.c_void_p)]


EXPORTS = ("dgs_create", "dgs_destroy", "dgs_last_error", "dgs_version", "dgs_render_state",
           "dgs_render_states_batched", "dgs_render_backward", "dgs_state_utility", "dgs_image_mse",
           "dgs_kernel_launches", "dgs_reset_kernel_launches", "dgs_profile_enable", "dgs_profile_read",
           "dgs_image_mse_noalloc", "dgs_debug_tile_lists", "dgs_plan_create", "dgs_plan_destroy",
           "dgs_plan_last_error", "dgs_plan_render", "dgs_plan_backward", "dgs_plan_utility",
           "dgs_plan_image_mse", "dgs_plan_status", "dgs_arena_create", "dgs_arena_destroy",
           "dgs_group_utility", "dgs_objective", "dgs_set_tile_reuse",
           "dgs_tile_reuse_stats", "dgs_set_tile_size", "dgs_set_memory_budget", "dgs_memory_stats",
           "dgs_last_tile_size", "dgs_plan_tile_size", "dgs_plan_render_mse",
           "dgs_render_scenes_batched", "dgs_render_scenes_backward", "dgs_plan_set_objective",
           "dgs_plan_objective")
OBJECTIVE_MAX_STATES = 16384
UTILITY_MAX_CONTEXTS = 4096
PLAN_RENDER, PLAN_UTILITY = 1, 2

_lib = None


def lib():
    """Load ``libdgs.so`` (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libdgs.so is not built: run `python -m paper_2606_17212_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        P, I, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_float
        L.dgs_create.argtypes = [ctypes.POINTER(P), I]
        L.dgs_destroy.argtypes = [P]
        L.dgs_destroy.restype = None
        L.dgs_last_error.argtypes = [P]
        L.dgs_last_error.restype = ctypes.c_char_p
        L.dgs_version.restype = I
        L.dgs_render_state.argtypes = [P, ctypes.POINTER(Scene_t), P, F, ctypes.POINTER(Camera_t), P, P, P]
        L.dgs_render_states_batched.argtypes = [P, ctypes.POINTER(Scene_t), ctypes.POINTER(States_t),
                                                P, I, P, P, P]
        L.dgs_render_scenes_batched.argtypes = [P, ctypes.POINTER(SceneJob_t), I, P]
        L.dgs_render_scenes_backward.argtypes = [P, ctypes.POINTER(SceneJob_t), I, P, P, P]
        L.dgs_render_backward.argtypes = [P, ctypes.POINTER(Scene_t), ctypes.POINTER(States_t), P, I, P, P, P,
                                          ctypes.POINTER(SceneGrad_t), P]
        L.dgs_state_utility.argtypes = [P, ctypes.POINTER(Scene_t), ctypes.POINTER(States_t), P, I, P, P, P, P]
        L.dgs_image_mse.argtypes = [P, P, P, P, I, I, I, I, F, P, P, P, P]
        D = ctypes.c_double
        L.dgs_objective.argtypes = [P, P, P, P, I, I, I, I, P, I, P, I, P, I, ctypes.POINTER(ObjectiveParams_t), P, P,
                                    P, P]
        L.dgs_group_utility.argtypes = [P, ctypes.POINTER(Scene_t), ctypes.POINTER(States_t), P, I, I, P, I, P,
                                        D, D, D, P, P, P]
        L.dgs_set_tile_reuse.argtypes = [P, I]
        L.dgs_set_tile_size.argtypes = [P, I]
        L.dgs_set_memory_budget.argtypes = [P, ctypes.c_uint64]
        L.dgs_memory_stats.argtypes = [P, P, P]
        L.dgs_last_tile_size.argtypes = [P, ctypes.POINTER(ctypes.c_int32)]
        L.dgs_plan_tile_size.argtypes = [P, ctypes.POINTER(ctypes.c_int32)]
        L.dgs_tile_reuse_stats.argtypes = [P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                           ctypes.POINTER(ctypes.c_int32)]
        L.dgs_kernel_launches.argtypes = [P]
        L.dgs_kernel_launches.restype = ctypes.c_int64
        L.dgs_reset_kernel_launches.argtypes = [P]
        L.dgs_reset_kernel_launches.restype = None
        L.dgs_profile_enable.argtypes = [P, I]
        L.dgs_profile_enable.restype = None
        L.dgs_profile_read.argtypes = [P, I, P, P, P]
        L.dgs_profile_read.restype = I
        L.dgs_image_mse_noalloc.argtypes = [P, P, P, I, I, I, I, F, P, P, P, P]
        L.dgs_image_mse_noalloc.restype = I
        L.dgs_debug_tile_lists.argtypes = [P] * 11 + [P]
        L.dgs_debug_tile_lists.restype = I
        L.dgs_plan_create.argtypes = [P, ctypes.POINTER(Scene_t), ctypes.POINTER(States_t), P, I, P, I, P, I, F,
                                      P, ctypes.POINTER(P)]
        L.dgs_arena_create.argtypes = [P, ctypes.POINTER(P)]
        L.dgs_arena_destroy.argtypes = [P]
        L.dgs_plan_destroy.argtypes = [P]
        L.dgs_plan_destroy.restype = None
        L.dgs_plan_last_error.argtypes = [P]
        L.dgs_plan_last_error.restype = ctypes.c_char_p
        L.dgs_plan_render.argtypes = [P, P, P, P]
        L.dgs_plan_backward.argtypes = [P, P, P, ctypes.POINTER(SceneGrad_t), P]
        L.dgs_plan_utility.argtypes = [P, P, P, P, P]
        L.dgs_plan_image_mse.argtypes = [P, P, P, F, P, P, P, P]
        L.dgs_plan_render_mse.argtypes = [P, P, P, P, F, P, P, P, P]
        L.dgs_plan_set_objective.argtypes = [P, P, I, P, I, P, I, ctypes.POINTER(ObjectiveParams_t)]
        L.dgs_plan_objective.argtypes = [P, P, P, P, P, P, P]
        L.dgs_plan_status.argtypes = [P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64), P]
        _lib = L
    return _lib


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def camera_struct(cam) -> Camera_t:
    R = np.asarray(cam.R_wc, np.float32).reshape(9)
    t = np.asarray(cam.t_wc, np.float32).reshape(3)
    return Camera_t((ctypes.c_float * 9)(*R), (ctypes.c_float * 3)(*t), float(cam.fx), float(cam.fy),
                    float(cam.cx), float(cam.cy), int(cam.width), int(cam.height))


def camera_array(cams):
    arr = (Camera_t * len(cams))()
    for k, c in enumerate(cams):
        arr[k] = camera_struct(c)
    return arr


SCENE_FIELDS = ("mu0", "u", "log_scale", "quat", "opacity_logit", "colour", "res")


def _grad_struct(grads: dict) -> SceneGrad_t:
    ptrs = [(_ptr(grads[k]) if grads[k].numel() else None) for k in SCENE_FIELDS]
    return SceneGrad_t(*ptrs, _ptr(grads.get("affine")), _ptr(grads.get("res_step")))


class DeviceScene:
    """Scene tensors resident on a CUDA device, with the C struct that points at them."""

    def __init__(self, tensors: dict, n, n_clusters, n_layers, sh_degree, temporal_rank, cluster_offsets,
                 affine=None, res_q=None, res_step=None, res_mode=0):
        import torch
        self.t = {k: tensors[k].contiguous() for k in SCENE_FIELDS}
        # optional cluster affine keyframes of Eq. 1 [C, T, 12] (None = identity)
        if affine is not None:
            self.t["affine"] = affine.contiguous()
        # quantized refinements: res_mode 1 reads int16 symbols res_q times res_step,
        # res_mode 2 quantizes res to res_step on the fly (res_step then has a gradient)
        self.res_mode = int(res_mode)
        self.res_q = None if res_q is None else res_q.contiguous()
        if res_step is not None:
            if self.res_mode == 2:
                self.t["res_step"] = res_step.contiguous()
            else:
                self.res_step = res_step.contiguous()
        self.offsets = cluster_offsets.to(torch.int32).contiguous()
        self.n, self.n_clusters, self.n_layers = int(n), int(n_clusters), int(n_layers)
        self.sh_degree, self.temporal_rank = int(sh_degree), int(temporal_rank)

    @classmethod
    def from_host(cls, scene, device="cuda"):
        import torch
        ts = {k: torch.from_numpy(np.ascontiguousarray(getattr(scene, k), np.float32)).to(device)
              for k in SCENE_FIELDS}
        offs = torch.from_numpy(np.asarray(scene.cluster_offsets, np.int32)).to(device)
        aff = getattr(scene, "affine", None)
        aff = None if aff is None else torch.from_numpy(np.ascontiguousarray(aff, np.float32)).to(device)
        mode = int(getattr(scene, "res_mode", 0))
        rq = None if mode != 1 else torch.from_numpy(np.ascontiguousarray(scene.res_q, np.int16)).to(device)
        rs = None if mode == 0 else torch.from_numpy(np.ascontiguousarray(scene.res_step, np.float32)).to(device)
        return cls(ts, scene.n, scene.n_clusters, scene.n_layers, scene.sh_degree, scene.temporal_rank, offs,
                   affine=aff, res_q=rq, res_step=rs, res_mode=mode)

    @property
    def fields(self):
        """The differentiable tensors: SCENE_FIELDS, plus "affine" and "res_step" when present."""
        return SCENE_FIELDS + tuple(k for k in ("affine", "res_step") if k in self.t)

    def struct(self) -> Scene_t:
        g = lambda k: _ptr(self.t[k]) if self.t[k].numel() else None
        aff = self.t.get("affine")
        step = self.t.get("res_step", getattr(self, "res_step", None))
        return Scene_t(self.n, self.n_clusters, self.n_layers, self.sh_degree, self.temporal_rank,
                       _ptr(self.offsets), g("mu0"), g("u"), g("log_scale"), g("quat"),
                       g("opacity_logit"), g("colour"), g("res"), _ptr(aff),
                       0 if aff is None else int(aff.shape[1]), _ptr(self.res_q), _ptr(step), self.res_mode)

    def zeros_like_grads(self) -> dict:
        import torch
        return {k: torch.zeros_like(v) for k, v in self.t.items()}


class DeviceStates:
    """Masks on the device, times and camera indices on the host."""

    def __init__(self, masks, t, cam):
        import torch
        self.masks = masks.contiguous() if isinstance(masks, torch.Tensor) else torch.from_numpy(
            np.ascontiguousarray(masks, np.uint32).view(np.int32)).cuda()
        self.t = np.ascontiguousarray(t, np.float32)
        self.cam = np.ascontiguousarray(cam, np.int32)
        self.n = int(self.t.shape[0])

    @classmethod
    def from_host(cls, states):
        return cls(states.masks, states.t, states.cam)

    def struct(self) -> States_t:
        return States_t(_ptr(self.masks), self.t.ctypes.data_as(ctypes.c_void_p),
                        self.cam.ctypes.data_as(ctypes.c_void_p), self.n)


class Renderer:
    """One library context on one CUDA device."""

    def __init__(self, device: int = 0):
        self._lib = lib()
        h = ctypes.c_void_p()
        rc = self._lib.dgs_create(ctypes.byref(h), int(device))
        if rc != DGS_OK:
            raise RuntimeError("dgs_create failed: %s" % ERRORS.get(rc, rc))
        self.h = h
        self.device = device

    def close(self):
        if getattr(self, "h", None):
            self._lib.dgs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != DGS_OK:
            msg = self._lib.dgs_last_error(self.h).decode()
            raise RuntimeError("%s failed (%s): %s" % (what, ERRORS.get(rc, rc), msg))

    def kernel_launches(self) -> int:
        return int(self._lib.dgs_kernel_launches(self.h))

    def reset_kernel_launches(self):
        self._lib.dgs_reset_kernel_launches(self.h)

    def profile(self, on: bool = True):
        self._lib.dgs_profile_enable(self.h, int(bool(on)))

    def profile_read(self) -> dict:
        """{kernel name: (total ms, launches)} since enabling or the last read."""
        n_max = 64
        names = ctypes.create_string_buffer(32 * n_max)
        ms = (ctypes.c_double * n_max)()
        cnt = (ctypes.c_int64 * n_max)()
        n = self._lib.dgs_profile_read(self.h, n_max, names, ms, cnt)
        if n < 0:
            self._check(n, "dgs_profile_read")
        raw = names.raw
        return {raw[32 * k:32 * k + 32].split(b"\0")[0].decode(): (ms[k], cnt[k]) for k in range(n)}

    def debug_tile_lists(self, stream=None) -> dict:
        """Copies of the last forward call's records and sorted lists (numpy)."""
        import torch
        n_rec, n_ent = ctypes.c_uint32(), ctypes.c_uint32()
        nvg, tiles = ctypes.c_int32(), ctypes.c_uint32()
        z = None
        self._check(self._lib.dgs_debug_tile_lists(self.h, ctypes.byref(n_rec), ctypes.byref(n_ent),
                                                   ctypes.byref(nvg), ctypes.byref(tiles), z, z, z, z, z, z,
                                                   _stream(stream)), "dgs_debug_tile_lists")
        nr, ne, nrg = n_rec.value, n_ent.value, nvg.value * tiles.value
        mk = lambda *shape: torch.empty(shape, dtype=torch.int32, device="cuda")
        recs, dk, ds, ek, ev, rg = mk(max(nr, 1), 12), mk(max(nr, 1)), mk(max(nr, 1)), mk(max(ne, 1)), \
            mk(max(ne, 1)), mk(max(nrg, 1), 2)
        self._check(self._lib.dgs_debug_tile_lists(self.h, None, None, None, None, _ptr(recs), _ptr(dk), _ptr(ds),
                                                   _ptr(ek), _ptr(ev), _ptr(rg), _stream(stream)),
                    "dgs_debug_tile_lists")
        torch.cuda.synchronize()
        u = lambda t, n: t.cpu().numpy().view(np.uint32)[:n]
        return dict(n_rec=nr, n_ent=ne, view_groups=nvg.value, tiles=tiles.value,
                    recs=recs.cpu().numpy().view(np.uint32)[:nr], depth_keys=u(dk, nr), depth_slots=u(ds, nr),
                    entry_keys=u(ek, ne), entry_vals=u(ev, ne), ranges=rg.cpu().numpy().view(np.uint32)[:nrg])

    def render_state(self, scene: DeviceScene, mask, t: float, cam, bg, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((cam.height, cam.width, 3), dtype=torch.float32, device="cuda")
        bgv = (ctypes.c_float * 3)(*[float(x) for x in bg])
        sc = scene.struct()
        c = camera_struct(cam)
        self._check(self._lib.dgs_render_state(self.h, ctypes.byref(sc), _ptr(mask), float(t), ctypes.byref(c),
                                               bgv, _ptr(out), _stream(stream)), "dgs_render_state")
        return out

    def render_states_batched(self, scene: DeviceScene, states: DeviceStates, cams, bg, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty((states.n, cams[0].height, cams[0].width, 3), dtype=torch.float32, device="cuda")
        bgv = (ctypes.c_float * 3)(*[float(x) for x in bg])
        sc, st, ca = scene.struct(), states.struct(), camera_array(cams)
        self._check(self._lib.dgs_render_states_batched(self.h, ctypes.byref(sc), ctypes.byref(st), ca, len(cams),
                                                        bgv, _ptr(out), _stream(stream)),
                    "dgs_render_states_batched")
        return out

    def render_backward(self, scene: DeviceScene, states: DeviceStates, cams, bg, dL_dimages, grads=None,
                        stream=None, images=None):
        """Adjoint of render_states_batched.  ``images``: that forward's output
        (one walk per tile) or None (a first walk recomputes final pixels)."""
        if grads is None:
            grads = scene.zeros_like_grads()
        bgv = (ctypes.c_float * 3)(*[float(x) for x in bg])
        g = _grad_struct(grads)
        sc, st, ca = scene.struct(), states.struct(), camera_array(cams)
        img = None if images is None else images.contiguous()
        self._check(self._lib.dgs_render_backward(self.h, ctypes.byref(sc), ctypes.byref(st), ca, len(cams), bgv,
                                                  _ptr(img), _ptr(dL_dimages.contiguous()), ctypes.byref(g),
                                                  _stream(stream)), "dgs_render_backward")
        return grads

    def _jobs(self, jobs):
        """Marshal (scene, states, cams, bg, images) tuples; the keep list holds
        every ctypes object the job array points into."""
        arr = (SceneJob_t * len(jobs))()
        keep = []
        for k, (scene, states, cams, bg, images) in enumerate(jobs):
            sc, ca = scene.struct(), camera_array(cams)
            keep += [sc, ca]
            arr[k].scene = ctypes.pointer(sc)
            arr[k].states = states.struct()
            arr[k].cams = ctypes.cast(ca, ctypes.POINTER(Camera_t))
            arr[k].n_cams = len(cams)
            for c in range(3):
                arr[k].bg[c] = float(bg[c])
            arr[k].images = _ptr(images)
        return arr, keep

    def render_scenes_batched(self, jobs, stream=None):
        """dgs_render_scenes_batched: jobs = [(scene, states, cams, bg, images)];
        every scene's states rendered into its images with one raster launch."""
        arr, keep = self._jobs(jobs)
        self._check(self._lib.dgs_render_scenes_batched(self.h, arr, len(jobs), _stream(stream)),
                    "dgs_render_scenes_batched")
        return [j[4] for j in jobs]

    def render_scenes_backward(self, jobs, dL_dimages, grads, stream=None):
        """dgs_render_scenes_backward: adjoint of the last render_scenes_batched of
        these jobs; grads (one dict per job) accumulate."""
        arr, keep = self._jobs(jobs)
        dl = (ctypes.c_void_p * len(jobs))(*[_ptr(d.contiguous()) for d in dL_dimages])
        gs = (SceneGrad_t * len(jobs))(*[_grad_struct(g) for g in grads])
        self._check(self._lib.dgs_render_scenes_backward(self.h, arr, len(jobs), dl, gs, _stream(stream)),
                    "dgs_render_scenes_backward")
        return grads

    def set_tile_reuse(self, enable: bool):
        """dgs_set_tile_reuse: exact reuse of rendered tiles across the states of
        one view in the distortion passes (on by default; outputs unchanged)."""
        self._check(self._lib.dgs_set_tile_reuse(self.h, 1 if enable else 0), "dgs_set_tile_reuse")

    def set_memory_budget(self, nbytes: int):
        """dgs_set_memory_budget: cap the workspace; batches that do not fit run in parts."""
        self._check(self._lib.dgs_set_memory_budget(self.h, int(nbytes)), "dgs_set_memory_budget")

    def memory_stats(self):
        """dgs_memory_stats: (workspace bytes, batch splits since creation)."""
        a, b = ctypes.c_uint64(), ctypes.c_int64()
        self._check(self._lib.dgs_memory_stats(self.h, ctypes.byref(a), ctypes.byref(b)), "dgs_memory_stats")
        return a.value, b.value

    def last_tile_size(self) -> int:
        """dgs_last_tile_size: sort tile side (px) of the last prepared batch, 0 before any."""
        v = ctypes.c_int32()
        self._check(self._lib.dgs_last_tile_size(self.h, ctypes.byref(v)), "dgs_last_tile_size")
        return v.value

    def set_tile_size(self, size: int):
        """dgs_set_tile_size: side of the sort tiles (16 or 32 px, 0 = chosen per batch shape)."""
        self._check(self._lib.dgs_set_tile_size(self.h, int(size)), "dgs_set_tile_size")

    def tile_reuse_stats(self):
        """dgs_tile_reuse_stats of the last distortion pass: (pairs, rendered, rounds)."""
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        self._check(self._lib.dgs_tile_reuse_stats(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
                    "dgs_tile_reuse_stats")
        return a.value, b.value, c.value

    def state_utility(self, scene: DeviceScene, states: DeviceStates, cams, bg, mse=None, psnr=None,
                      stream=None):
        import torch
        if mse is None:
            mse = torch.empty(states.n, dtype=torch.float64, device="cuda")
        if psnr is None:
            psnr = torch.empty(states.n, dtype=torch.float64, device="cuda")
        bgv = (ctypes.c_float * 3)(*[float(x) for x in bg])
        sc, st, ca = scene.struct(), states.struct(), camera_array(cams)
        self._check(self._lib.dgs_state_utility(self.h, ctypes.byref(sc), ctypes.byref(st), ca, len(cams), bgv,
                                                _ptr(mse), _ptr(psnr), _stream(stream)), "dgs_state_utility")
        return mse, psnr

    def group_utility(self, scene: DeviceScene, contexts: DeviceStates, groups, n_contexts: int, cams, bg,
                      alpha: float = 0.25, beta: float = 0.05, q: float = 0.10, stream=None):
        """Eq. 3 / Eq. 4 (dgs_group_utility): returns (delta [G, M] f64, stats [G, 4]
        f64 = mean, Q_q, std, risk-adjusted utility) as CUDA tensors."""
        import torch
        g = np.ascontiguousarray(groups, np.int32).reshape(-1, 2)
        G, M = g.shape[0], int(n_contexts)
        delta = torch.empty((G, M), dtype=torch.float64, device="cuda")
        stats = torch.empty((G, 4), dtype=torch.float64, device="cuda")
        bgv = (ctypes.c_float * 3)(*[float(x) for x in bg])
        sc, st, ca = scene.struct(), contexts.struct(), camera_array(cams)
        self._check(self._lib.dgs_group_utility(self.h, ctypes.byref(sc), ctypes.byref(st),
                                                g.ctypes.data_as(ctypes.c_void_p), G, M, ca, len(cams), bgv,
                                                float(alpha), float(beta), float(q), _ptr(delta), _ptr(stats),
                                                _stream(stream)), "dgs_group_utility")
        return delta, stats

    def objective(self, images, refs, ref_index, pairs_t=(), pairs_m=(), anchors=(), params=None,
                  want_grad=True, stream=None):
        """Eq. 2 (dgs_objective): returns (loss [1] f64, D [S] f64, dL/dimages or None)
        as CUDA tensors.  params: dict of ssim_weight, lambda_c, cvar_q, lambda_t,
        lambda_m, anchor_weight (missing keys take the paper's values)."""
        import torch
        S, H, W, _ = images.shape
        ri = np.ascontiguousarray(ref_index, np.int32)
        pt = np.ascontiguousarray(np.asarray(pairs_t, np.int32).reshape(-1, 2))
        pm = np.ascontiguousarray(np.asarray(pairs_m, np.int32).reshape(-1, 2))
        an = np.ascontiguousarray(np.asarray(anchors, np.int32).reshape(-1))
        prm = None
        if params is not None:
            v = dict(OBJECTIVE_DEFAULTS, **params)
            prm = ObjectiveParams_t(*[float(v[k]) for k in OBJECTIVE_KEYS])
        loss = torch.empty(1, dtype=torch.float64, device="cuda")
        D = torch.empty(S, dtype=torch.float64, device="cuda")
        dL = torch.empty_like(images) if want_grad else None
        vp = lambda a: a.ctypes.data_as(ctypes.c_void_p) if a.size else None
        self._check(self._lib.dgs_objective(self.h, _ptr(images.contiguous()), _ptr(refs.contiguous()), vp(ri), S,
                                            refs.shape[0], H, W, vp(pt), pt.shape[0], vp(pm), pm.shape[0], vp(an),
                                            an.size, None if prm is None else ctypes.byref(prm), _ptr(loss), _ptr(D),
                                            _ptr(dL), _stream(stream)), "dgs_objective")
        return loss, D, dL

    def image_mse(self, images, refs, ref_index, weight=1.0, want_grad=False, stream=None):
        import torch
        S, H, W, _ = images.shape
        ri = np.ascontiguousarray(ref_index, np.int32)
        mse = torch.empty(S, dtype=torch.float64, device="cuda")
        psnr = torch.empty(S, dtype=torch.float64, device="cuda")
        dL = torch.empty_like(images) if want_grad else None
        self._check(self._lib.dgs_image_mse(self.h, _ptr(images.contiguous()), _ptr(refs.contiguous()),
                                            ri.ctypes.data_as(ctypes.c_void_p), S, refs.shape[0], H, W,
                                            float(weight), _ptr(mse), _ptr(psnr), _ptr(dL), _stream(stream)),
                    "dgs_image_mse")
        return mse, psnr, dL


def render_function():
    """A torch.autograd.Function whose forward is the batched render and whose
    backward is the library's adjoint (gradients w.r.t. the scene tensors)."""
    import torch

    class RenderStates(torch.autograd.Function):
        @staticmethod
        def forward(ctx, renderer, scene, states, cams, bg, *tensors):
            out = renderer.render_states_batched(scene, states, cams, bg)
            ctx.renderer, ctx.scene, ctx.states, ctx.cams, ctx.bg = renderer, scene, states, cams, bg
            ctx.save_for_backward(out)
            return out

        @staticmethod
        def backward(ctx, grad_out):
            (out,) = ctx.saved_tensors
            grads = ctx.renderer.render_backward(ctx.scene, ctx.states, ctx.cams, ctx.bg, grad_out.contiguous(),
                                                 images=out)
            return (None, None, None, None, None) + tuple(grads[k] for k in ctx.scene.fields)

    return RenderStates


def objective_function():
    """A torch.autograd.Function for the Eq. 2 objective over rendered images:
    forward = dgs_objective (loss and per-state D), backward = its gradient
    with respect to the images (computed in the same call)."""
    import torch

    class Objective(torch.autograd.Function):
        @staticmethod
        def forward(ctx, renderer, images, refs, ref_index, pairs_t, pairs_m, anchors, params):
            loss, D, dL = renderer.objective(images.detach(), refs, ref_index, pairs_t, pairs_m, anchors, params,
                                             want_grad=True)
            ctx.save_for_backward(dL)
            ctx.mark_non_differentiable(D)
            return loss[0], D

        @staticmethod
        def backward(ctx, g_loss, g_D):
            (dL,) = ctx.saved_tensors
            return None, dL * g_loss.to(dL.dtype), None, None, None, None, None, None

    return Objective


def objective(renderer, images, refs, ref_index, pairs_t=(), pairs_m=(), anchors=(), params=None):
    """Differentiable Eq. 2 loss of rendered images: returns (loss, D)."""
    return objective_function().apply(renderer, images, refs, ref_index, pairs_t, pairs_m, anchors, params)


def render(renderer, scene: DeviceScene, states: DeviceStates, cams, bg):
    """Differentiable batched render: images [S,H,W,3] with autograd to scene tensors."""
    fn = render_function()
    return fn.apply(renderer, scene, states, cams, bg, *[scene.t[k] for k in scene.fields])


def image_mse_noalloc(images, refs, ref_index, mse, psnr=None, dL=None, weight=1.0, stream=None) -> int:
    """dgs_image_mse_noalloc: per-image MSE for callers that cannot allocate.

    Every argument is a caller-owned CUDA tensor (ref_index int32 on the
    device); nothing is allocated by this call or by the library.  Returns the
    library's status code (0 = ok, DGS_E_SCRATCH when the sizes exceed the
    fixed scratch)."""
    S, H, W, _ = images.shape
    return int(lib().dgs_image_mse_noalloc(_ptr(images), _ptr(refs), _ptr(ref_index), int(S), int(refs.shape[0]),
                                           int(H), int(W), float(weight), _ptr(mse), _ptr(psnr), _ptr(dL),
                                           _stream(stream)))


class Arena:
    """A scratch workspace shared by plans that run one after another on one
    stream (see dgs_arena_create in include/dgs.h)."""

    def __init__(self, renderer: Renderer):
        self._lib = lib()
        h = ctypes.c_void_p()
        rc = self._lib.dgs_arena_create(renderer.h, ctypes.byref(h))
        if rc != DGS_OK:
            raise RuntimeError("dgs_arena_create failed (%s)" % ERRORS.get(rc, rc))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            rc = self._lib.dgs_arena_destroy(self.h)
            if rc != DGS_OK:
                raise RuntimeError("dgs_arena_destroy: plans of this arena are still alive")
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """A capture-safe plan over a fixed batch (see dgs_plan_create in include/dgs.h).

    Per-step calls launch kernels only, so they can run inside a
    ``torch.cuda.graph`` capture and be replayed with new masks.  ``arena``
    (an Arena) shares the scratch buffers with the arena's other plans."""

    def __init__(self, renderer: Renderer, scene: DeviceScene, states: DeviceStates, cams, bg,
                 mode: int = PLAN_RENDER, ref_index=None, n_refs: int = 0, entry_headroom: float = 1.25,
                 arena: "Arena | None" = None):
        self._lib = lib()
        self.arena = arena
        self.scene, self.cams, self.n = scene, cams, states.n
        self.W, self.H = cams[0].width, cams[0].height
        self._keep = (scene.struct(), states.struct(), camera_array(cams),
                      (ctypes.c_float * 3)(*[float(x) for x in bg]))
        ri = None if ref_index is None else np.ascontiguousarray(ref_index, np.int32)
        self._ri = ri
        h = ctypes.c_void_p()
        sc, st, ca, bgv = self._keep
        rc = self._lib.dgs_plan_create(renderer.h, ctypes.byref(sc), ctypes.byref(st), ca, len(cams), bgv, int(mode),
                                       None if ri is None else ri.ctypes.data_as(ctypes.c_void_p), int(n_refs),
                                       float(entry_headroom), None if arena is None else arena.h, ctypes.byref(h))
        if rc != DGS_OK:
            raise RuntimeError("dgs_plan_create failed (%s): %s" % (ERRORS.get(rc, rc),
                                                                    self._lib.dgs_last_error(renderer.h).decode()))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self._lib.dgs_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc != DGS_OK:
            raise RuntimeError("%s failed (%s): %s" % (what, ERRORS.get(rc, rc),
                                                       self._lib.dgs_plan_last_error(self.h).decode()))

    def render(self, masks, images, stream=None):
        self._check(self._lib.dgs_plan_render(self.h, _ptr(masks), _ptr(images), _stream(stream)), "dgs_plan_render")
        return images

    def backward(self, dL, grads, stream=None, images=None):
        """Adjoint of the last render; ``images``: its output, or None."""
        g = _grad_struct(grads)
        self._check(self._lib.dgs_plan_backward(self.h, _ptr(images), _ptr(dL), ctypes.byref(g), _stream(stream)),
                    "dgs_plan_backward")
        return grads

    def utility(self, masks, mse, psnr, stream=None):
        self._check(self._lib.dgs_plan_utility(self.h, _ptr(masks), _ptr(mse), _ptr(psnr), _stream(stream)),
                    "dgs_plan_utility")
        return mse, psnr

    def render_mse(self, masks, images, refs, mse, psnr, dL, weight=1.0, stream=None):
        """dgs_plan_render_mse: render, squared errors and dL/dimages in one forward pass."""
        self._check(self._lib.dgs_plan_render_mse(self.h, _ptr(masks), _ptr(images), _ptr(refs), float(weight),
                                                  _ptr(mse), _ptr(psnr), _ptr(dL), _stream(stream)),
                    "dgs_plan_render_mse")
        return images, mse, psnr, dL

    def image_mse(self, images, refs, mse, psnr, dL, weight=1.0, stream=None):
        self._check(self._lib.dgs_plan_image_mse(self.h, _ptr(images), _ptr(refs), float(weight), _ptr(mse),
                                                 _ptr(psnr), _ptr(dL), _stream(stream)), "dgs_plan_image_mse")
        return mse, psnr, dL

    def set_objective(self, pairs_t=(), pairs_m=(), anchors=(), params=None):
        """dgs_plan_set_objective: fix the Eq. 2 pair and anchor lists and weights
        (as Renderer.objective's) for later capture-safe objective calls."""
        pt = np.ascontiguousarray(np.asarray(pairs_t, np.int32).reshape(-1, 2))
        pm = np.ascontiguousarray(np.asarray(pairs_m, np.int32).reshape(-1, 2))
        an = np.ascontiguousarray(np.asarray(anchors, np.int32).reshape(-1))
        prm = None
        if params is not None:
            v = dict(OBJECTIVE_DEFAULTS, **params)
            prm = ObjectiveParams_t(*[float(v[k]) for k in OBJECTIVE_KEYS])
        vp = lambda a: a.ctypes.data_as(ctypes.c_void_p) if a.size else None
        self._check(self._lib.dgs_plan_set_objective(self.h, vp(pt), pt.shape[0], vp(pm), pm.shape[0], vp(an),
                                                     an.size, None if prm is None else ctypes.byref(prm)),
                    "dgs_plan_set_objective")

    def objective(self, images, refs, loss, D=None, dL=None, stream=None):
        """dgs_plan_objective: Eq. 2 loss [1] f64, per-state D [S] f64 (or None)
        and dL/dimages (or None) into the given device tensors; kernels only."""
        self._check(self._lib.dgs_plan_objective(self.h, _ptr(images), _ptr(refs), _ptr(loss), _ptr(D), _ptr(dL),
                                                 _stream(stream)), "dgs_plan_objective")
        return loss, D, dL

    def tile_size(self) -> int:
        """dgs_plan_tile_size: sort tile side (px) fixed at creation."""
        v = ctypes.c_int32()
        self._check(self._lib.dgs_plan_tile_size(self.h, ctypes.byref(v)), "dgs_plan_tile_size")
        return v.value

    def status(self, stream=None):
        """(records, entries) of the last call; raises if entries overflowed."""
        nr, ne = ctypes.c_int64(), ctypes.c_int64()
        self._check(self._lib.dgs_plan_status(self.h, ctypes.byref(nr), ctypes.byref(ne), _stream(stream)),
                    "dgs_plan_status")
        return nr.value, ne.value
