"""Seeded synthetic inputs: dynamic Gaussian scenes, delivery masks, times and cameras.

This module only draws inputs.  It holds none of the renderer's arithmetic (no
decode, deformation, projection, compositing or scoring); both the CUDA library
and the FP64 oracle consume what it produces, and random numbers the method
would draw (masks, times, erasures) are drawn here and passed in as inputs.

Scene layout (the layout the C-ABI takes, Section 3 of the paper: N Gaussians
with base attributes plus three additive refinements, grouped in clusters):

* Gaussians are stored cluster-contiguous; ``cluster_offsets[c]:cluster_offsets[c+1]``
  are the Gaussians of cluster ``c``.
* ``mu0 [n,3]``, ``u [R,n,3]`` (the per-Gaussian temporal coefficients q_{i,r} of
  Eq. 1), ``log_scale [n,3]``, ``quat [n,4]`` (w,x,y,z), ``opacity_logit [n]``,
  ``colour [n, 3*(sh+1)^2]`` (SH coefficient-major, 3 channels innermost).
* ``res [L-1, n, K]`` with ``K = 11 + 3*(sh+1)^2``: per refinement layer l=1..L-1
  the residual vector (dmu[3], dlog_scale[3], dquat[4], dlogit[1], dcolour[...]).
* A delivery state is a bitmask with bit ``c*L + l`` set when packet (cluster c,
  layer l) arrived, packed little-endian into uint32 words, plus a time t and a
  camera index.

Distributions follow the workload descriptions of the benchmark configurations:
means ~N(0,1)^3, log-scales ~N(-3.5,0.4), random unit quaternions, opacity
logits ~N(0,1.5), RGB ~U[0,1] (SH degree 0) or 48 SH coefficients ~N(0,0.2^2)
(degree 3), temporal coefficients ~N(0,0.1^2), residual std 0.05 halving per
layer.  Cameras are OpenCV pinholes (x right, y down, z forward) on a ring of
radius 4 in the z=0 plane looking at the origin with world up +z.
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = [
    "Scene", "Camera", "States", "Workload",
    "make_scene", "ring_camera", "prefix_states", "bernoulli_states",
    "erase_one_packet", "mask_words", "config", "CONFIG_NAMES", "MixSpec", "mix_specs", "mix_workload",
    "completion_groups", "group_contexts", "cluster_affine", "quantize_residuals",
]


@dataclasses.dataclass
class Scene:
    n: int
    n_clusters: int
    n_layers: int
    sh_degree: int
    temporal_rank: int
    cluster_offsets: np.ndarray  # int32 [C+1]
    mu0: np.ndarray              # f32 [n,3]
    u: np.ndarray                # f32 [R,n,3]
    log_scale: np.ndarray        # f32 [n,3]
    quat: np.ndarray             # f32 [n,4]
    opacity_logit: np.ndarray    # f32 [n]
    colour: np.ndarray           # f32 [n, 3*(sh+1)^2]
    res: np.ndarray              # f32 [L-1, n, K]
    affine: np.ndarray | None = None   # f32 [C, T, 12] cluster affine keyframes of Eq. 1 (None = identity)
    res_q: np.ndarray | None = None    # i16 [L-1, n, K] quantized refinement symbols (res_mode 1)
    res_step: np.ndarray | None = None  # f32 [L-1, K] quantization steps (res_mode 1 and 2)
    res_mode: int = 0                  # 0: res as given; 1: res_q * res_step; 2: res quantized to res_step

    @property
    def n_colour(self) -> int:
        return 3 * (self.sh_degree + 1) ** 2

    @property
    def res_width(self) -> int:
        return 11 + self.n_colour

    def cluster_of(self) -> np.ndarray:
        sizes = np.diff(self.cluster_offsets)
        return np.repeat(np.arange(self.n_clusters, dtype=np.int32), sizes)

    def subset(self, idx: np.ndarray) -> "Scene":
        """Scene restricted to Gaussians ``idx`` (sorted), clusters kept."""
        idx = np.sort(np.asarray(idx, dtype=np.int64))
        cl = self.cluster_of()[idx]
        counts = np.bincount(cl, minlength=self.n_clusters)
        offs = np.zeros(self.n_clusters + 1, dtype=np.int32)
        offs[1:] = np.cumsum(counts)
        return Scene(len(idx), self.n_clusters, self.n_layers, self.sh_degree,
                     self.temporal_rank, offs, self.mu0[idx].copy(),
                     self.u[:, idx].copy(), self.log_scale[idx].copy(),
                     self.quat[idx].copy(), self.opacity_logit[idx].copy(),
                     self.colour[idx].copy(), self.res[:, idx].copy(),
                     None if self.affine is None else self.affine.copy(),
                     None if self.res_q is None else self.res_q[:, idx].copy(),
                     None if self.res_step is None else self.res_step.copy(), self.res_mode)

    def arrays(self):
        return dict(mu0=self.mu0, u=self.u, log_scale=self.log_scale, quat=self.quat,
                    opacity_logit=self.opacity_logit, colour=self.colour, res=self.res)


@dataclasses.dataclass
class Camera:
    R_wc: np.ndarray   # f32 [3,3] world -> camera rotation (row-major)
    t_wc: np.ndarray   # f32 [3]
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int


@dataclasses.dataclass
class States:
    masks: np.ndarray  # uint32 [S, words]
    t: np.ndarray      # f32 [S]
    cam: np.ndarray    # int32 [S]

    @property
    def n(self) -> int:
        return int(self.masks.shape[0])


@dataclasses.dataclass
class Workload:
    name: str
    scene: Scene
    cams: list
    states: States
    bg: np.ndarray               # f32 [3]
    target_scene: Scene | None = None   # teacher scene for training targets


def mask_words(n_clusters: int, n_layers: int) -> int:
    return (n_clusters * n_layers + 31) // 32


def _kmeans(x: np.ndarray, k: int, rng: np.random.Generator, iters: int = 8) -> np.ndarray:
    """Seeded Lloyd iterations; returns a cluster id per row (input grouping only)."""
    n = x.shape[0]
    k = min(k, n)
    cent = x[rng.choice(n, size=k, replace=False)].astype(np.float64)
    assign = np.zeros(n, dtype=np.int64)
    chunk = 1 << 16
    for _ in range(iters):
        c2 = (cent * cent).sum(1)
        for s in range(0, n, chunk):
            xs = x[s:s + chunk].astype(np.float64)
            d = c2[None, :] - 2.0 * xs @ cent.T
            assign[s:s + chunk] = np.argmin(d, axis=1)
        for j in range(k):
            sel = assign == j
            if sel.any():
                cent[j] = x[sel].mean(0)
    return assign


def _nearest(x: np.ndarray, cent: np.ndarray) -> np.ndarray:
    out = np.zeros(x.shape[0], dtype=np.int64)
    c2 = (cent * cent).sum(1)
    for s in range(0, x.shape[0], 1 << 16):
        xs = x[s:s + (1 << 16)].astype(np.float64)
        out[s:s + (1 << 16)] = np.argmin(c2[None, :] - 2.0 * xs @ cent.T, axis=1)
    return out


def _fast_normal(seed: int, tag: int, shape, mean: float, std: float) -> np.ndarray:
    """float32 N(mean, std^2) filled in 16 fixed chunks, each from its own
    PCG64 stream spawned from (seed, tag), on a thread pool: the values depend
    only on (seed, tag, shape), not on the number of threads."""
    from concurrent.futures import ThreadPoolExecutor
    out = np.empty(int(np.prod(shape)), dtype=np.float32)
    n = out.size
    chunks = 16
    gens = [np.random.Generator(np.random.PCG64(ss))
            for ss in np.random.SeedSequence([seed, tag]).spawn(chunks)]

    def fill(i):
        lo, hi = i * n // chunks, (i + 1) * n // chunks
        v = out[lo:hi]
        gens[i].standard_normal(out=v, dtype=np.float32)
        v *= np.float32(std)
        v += np.float32(mean)

    with ThreadPoolExecutor(8) as ex:
        list(ex.map(fill, range(chunks)))
    return out.reshape(shape)


def make_scene(n: int, n_clusters: int, n_layers: int, *, seed: int,
               temporal_rank: int = 2, sh_degree: int = 0,
               residual_std: float = 0.05, residual_attrs: str = "all",
               mean_std: float = 1.0, log_scale_mean: float = -3.5,
               log_scale_std: float = 0.4, logit_std: float = 1.5,
               u_std: float = 0.1, sh_std: float = 0.2, fast: bool = False) -> Scene:
    """Draw a scene; ``residual_attrs`` is "all" or "colour_opacity".

    ``fast`` (for the many large scenes of the serving mix) draws float32
    values from parallel streams, fits the k-means centroids on a 65,536-point
    subsample and assigns every Gaussian to its nearest centroid, and draws the
    attributes that do not enter the clustering directly in cluster order."""
    if fast:
        return _make_scene_fast(n, n_clusters, n_layers, seed, temporal_rank, sh_degree, residual_std,
                                mean_std, log_scale_mean, log_scale_std, logit_std, u_std, sh_std)
    rng = np.random.default_rng(seed)
    mu0 = rng.normal(0.0, mean_std, size=(n, 3))
    ls = rng.normal(log_scale_mean, log_scale_std, size=(n, 3))
    q = rng.normal(0.0, 1.0, size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    logit = rng.normal(0.0, logit_std, size=n)
    nc = 3 * (sh_degree + 1) ** 2
    if sh_degree == 0:
        col = rng.uniform(0.0, 1.0, size=(n, 3))
    else:
        col = rng.normal(0.0, sh_std, size=(n, nc))
    u = rng.normal(0.0, u_std, size=(temporal_rank, n, 3))
    feats = mu0 if temporal_rank == 0 else np.concatenate(
        [mu0] + [u[r] for r in range(temporal_rank)], axis=1)
    assign = _kmeans(feats, n_clusters, rng)
    K = 11 + nc
    res = np.zeros((max(n_layers - 1, 0), n, K))
    for l in range(1, n_layers):
        std = residual_std * 2.0 ** (-(l - 1))
        r = rng.normal(0.0, std, size=(n, K))
        if residual_attrs == "colour_opacity":
            r[:, 0:10] = 0.0
        elif l == 1:
            r[:, 0:3] = 0.0   # Eq. 1: position residuals only on the two finer levels
        res[l - 1] = r
    order = np.argsort(assign, kind="stable")
    counts = np.bincount(assign, minlength=n_clusters)
    offs = np.zeros(n_clusters + 1, dtype=np.int32)
    offs[1:] = np.cumsum(counts)
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return Scene(n, n_clusters, n_layers, sh_degree, temporal_rank, offs,
                 f32(mu0[order]), f32(u[:, order]), f32(ls[order]), f32(q[order]),
                 f32(logit[order]), f32(col[order]), f32(res[:, order]))


def _make_scene_fast(n, n_clusters, n_layers, seed, temporal_rank, sh_degree, residual_std, mean_std,
                     log_scale_mean, log_scale_std, logit_std, u_std, sh_std) -> Scene:
    rng = np.random.default_rng(seed)
    mu0 = _fast_normal(seed, 0, (n, 3), 0.0, mean_std)
    u = _fast_normal(seed, 1, (temporal_rank, n, 3), 0.0, u_std)
    feats = mu0 if temporal_rank == 0 else np.concatenate(
        [mu0] + [u[r] for r in range(temporal_rank)], axis=1)
    if n > 65536:
        sub = rng.choice(n, size=65536, replace=False)
        a_sub = _kmeans(feats[sub], n_clusters, rng)
        cent = np.stack([feats[sub][a_sub == j].mean(0) if (a_sub == j).any() else feats[sub][0]
                         for j in range(n_clusters)]).astype(np.float64)
        assign = _nearest(feats, cent)
    else:
        assign = _kmeans(feats, n_clusters, rng)
    order = np.argsort(assign, kind="stable")
    counts = np.bincount(assign, minlength=n_clusters)
    offs = np.zeros(n_clusters + 1, dtype=np.int32)
    offs[1:] = np.cumsum(counts)
    mu0 = np.ascontiguousarray(mu0[order])
    u = np.ascontiguousarray(u[:, order])
    # the remaining attributes are i.i.d. per Gaussian: drawn in cluster order
    ls = _fast_normal(seed, 2, (n, 3), log_scale_mean, log_scale_std)
    q = _fast_normal(seed, 3, (n, 4), 0.0, 1.0)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    logit = _fast_normal(seed, 4, (n,), 0.0, logit_std)
    nc = 3 * (sh_degree + 1) ** 2
    if sh_degree == 0:
        col = rng.uniform(0.0, 1.0, size=(n, 3)).astype(np.float32)
    else:
        col = _fast_normal(seed, 5, (n, nc), 0.0, sh_std)
    K = 11 + nc
    res = np.empty((max(n_layers - 1, 0), n, K), dtype=np.float32)
    for l in range(1, n_layers):
        res[l - 1] = _fast_normal(seed, 5 + l, (n, K), 0.0, residual_std * 2.0 ** (-(l - 1)))
        if l == 1:
            res[0, :, 0:3] = 0.0   # Eq. 1: position residuals only on the two finer levels
    return Scene(n, n_clusters, n_layers, sh_degree, temporal_rank, offs, mu0, u, ls, q, logit, col, res)


def ring_camera(k: int, n_ring: int, width: int, height: int, focal: float,
                radius: float = 4.0) -> Camera:
    """Pinhole at angle 2*pi*k/n_ring on a ring of ``radius``, looking at the origin."""
    th = 2.0 * np.pi * k / n_ring
    pos = np.array([radius * np.cos(th), radius * np.sin(th), 0.0])
    fwd = -pos / np.linalg.norm(pos)
    up = np.array([0.0, 0.0, 1.0])
    right = np.cross(fwd, up)
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd])
    t = -R @ pos
    return Camera(R.astype(np.float32), t.astype(np.float32), float(focal), float(focal),
                  width / 2.0, height / 2.0, int(width), int(height))


def _pack(bits: np.ndarray) -> np.ndarray:
    """bits [S, C*L] bool -> uint32 [S, words], bit b in word b//32 at position b%32."""
    S, nb = bits.shape
    words = (nb + 31) // 32
    out = np.zeros((S, words), dtype=np.uint64)
    for b in range(nb):
        out[:, b // 32] |= bits[:, b].astype(np.uint64) << np.uint64(b % 32)
    return out.astype(np.uint32)


def prefix_states(n_states: int, n_clusters: int, n_layers: int, rng: np.random.Generator,
                  distinct: bool = False) -> np.ndarray:
    """Prefix-valid masks: per cluster a delivered depth ~U{0..L}; returns depths [S,C]."""
    d = rng.integers(0, n_layers + 1, size=(n_states, n_clusters))
    if distinct:
        while True:
            _, first = np.unique(d, axis=0, return_index=True)
            dup = np.setdiff1d(np.arange(n_states), first)
            if dup.size == 0:
                break
            d[dup] = rng.integers(0, n_layers + 1, size=(dup.size, n_clusters))
    return d


def depths_to_bits(d: np.ndarray, n_layers: int) -> np.ndarray:
    S, C = d.shape
    lay = np.arange(n_layers)
    return (lay[None, None, :] < d[:, :, None]).reshape(S, C * n_layers)


def bernoulli_states(n_states: int, n_clusters: int, n_layers: int, rng: np.random.Generator,
                     p: float = 0.5) -> np.ndarray:
    return rng.uniform(size=(n_states, n_clusters * n_layers)) < p


def erase_one_packet(bits: np.ndarray, frac: float, rng: np.random.Generator) -> np.ndarray:
    """For a fraction of states clear one delivered packet chosen uniformly."""
    bits = bits.copy()
    S = bits.shape[0]
    chosen = rng.uniform(size=S) < frac
    for s in np.nonzero(chosen)[0]:
        on = np.nonzero(bits[s])[0]
        if on.size:
            bits[s, rng.choice(on)] = False
    return bits


def completion_groups(n_clusters: int, n_layers: int, n_groups: int, rng: np.random.Generator) -> np.ndarray:
    """n_groups distinct (cluster, layer) packets, uniformly drawn: [G, 2] int32."""
    allg = np.array([(c, l) for c in range(n_clusters) for l in range(n_layers)], dtype=np.int32)
    pick = rng.choice(len(allg), size=min(n_groups, len(allg)), replace=False)
    return allg[np.sort(pick)]


def group_contexts(groups: np.ndarray, n_contexts: int, n_clusters: int, n_layers: int,
                   rng: np.random.Generator) -> np.ndarray:
    """Valid partial receiver contexts for each completion group (cluster c,
    layer l): prefix-valid masks whose cluster c holds exactly layers 0..l-1
    (so adding the packet keeps the state valid and changes it) and every other
    cluster a delivered depth ~U{0..L}.  Row g * n_contexts + j is context j of
    group g; returns packed uint32 masks."""
    G = len(groups)
    d = rng.integers(0, n_layers + 1, size=(G * n_contexts, n_clusters))
    for g, (c, l) in enumerate(groups):
        d[g * n_contexts:(g + 1) * n_contexts, c] = l
    return _pack(depths_to_bits(d, n_layers))


def cluster_affine(n_clusters: int, n_keyframes: int, rng: np.random.Generator, linear_std: float = 0.05,
                   shift_std: float = 0.1) -> np.ndarray:
    """Cluster affine keyframes of Eq. 1 near the identity: [C, T, 12] float32,
    row-major 3x4 (linear part | translation), linear part I + N(0, linear_std^2),
    translation N(0, shift_std^2)."""
    A = np.zeros((n_clusters, n_keyframes, 3, 4))
    A[..., :3] = np.eye(3) + rng.normal(0.0, linear_std, size=(n_clusters, n_keyframes, 3, 3))
    A[..., 3] = rng.normal(0.0, shift_std, size=(n_clusters, n_keyframes, 3))
    return A.reshape(n_clusters, n_keyframes, 12).astype(np.float32)


def quantize_residuals(scene: Scene, step_scale: float = 1.0 / 256.0) -> tuple:
    """Quantization steps and symbols for a scene's refinements: one step per
    (layer, component), a power of two near step_scale times the component's
    standard deviation, and the signed 16-bit symbols round(res / step).
    Returns (res_q int16 [L-1, n, K], res_step float32 [L-1, K])."""
    r = np.asarray(scene.res, np.float32)
    sd = r.std(axis=1) + 1e-12
    step = (2.0 ** np.round(np.log2(sd * step_scale))).astype(np.float32)
    step[r.std(axis=1) == 0] = 1.0
    q = np.clip(np.rint(r / step[:, None, :]), -32768, 32767).astype(np.int16)
    return q, step


CONFIG_NAMES = ("c1_plain_4k", "c2_dynamic_250k", "c3_fwdbwd_250k", "c4_utility_2p7m", "c5_mix_48")

MIX_RESOLUTIONS = ((256, 256), (512, 512), (960, 540))


@dataclasses.dataclass
class MixSpec:
    """One scene of the serving-shaped mix: sizes drawn up front, scene drawn on demand."""
    index: int
    n: int
    n_clusters: int
    width: int
    height: int
    seed: int


def mix_specs(n_scenes: int = 48, *, scale: float = 1.0) -> list:
    """The uneven mix: Gaussian counts log-uniform in [50,000, 2,700,000],
    clusters ~U{16..64}, 4 layers, resolution drawn from MIX_RESOLUTIONS."""
    rng = np.random.default_rng(1005)
    specs = []
    for i in range(n_scenes):
        n = int(round(np.exp(rng.uniform(np.log(5e4), np.log(2.7e6)))))
        C = int(rng.integers(16, 65))
        W, H = MIX_RESOLUTIONS[int(rng.integers(0, len(MIX_RESOLUTIONS)))]
        if scale < 1.0:
            n = max(64, int(round(n * scale)))
            W, H = max(16, int(round(W * np.sqrt(scale)))), max(16, int(round(H * np.sqrt(scale))))
        specs.append(MixSpec(i, n, C, W, H, 10_000 + i))
    return specs


def mix_workload(spec: MixSpec, n_states: int = 64) -> Workload:
    """One scene of the mix: SH degree 3, rank-2 temporal basis, 4 layers;
    64 prefix-valid states, state s at camera s mod 8 of a radius-4 ring and
    t = (s mod 16)/16; focal 1.2 W.  The training target of each state is the
    complete render of the same scene at its view (held fixed)."""
    sc = make_scene(spec.n, spec.n_clusters, 4, seed=spec.seed, sh_degree=3, fast=True)
    rng = np.random.default_rng(20_000 + spec.index)
    d = prefix_states(n_states, spec.n_clusters, 4, rng)
    t = (np.arange(n_states) % 16) / 16.0
    cams = [ring_camera(k, 8, spec.width, spec.height, 1.2 * spec.width) for k in range(8)]
    st = States(_pack(depths_to_bits(d, 4)), t.astype(np.float32), (np.arange(n_states) % 8).astype(np.int32))
    return Workload("c5_mix_48/%d" % spec.index, sc, cams, st, np.zeros(3, np.float32))


def config(name: str, *, scale: float = 1.0, n_states: int | None = None) -> Workload:
    """The benchmark workloads.  ``scale`` < 1 shrinks Gaussians and image sides
    (for oracle-sized parity cases); ``n_states`` overrides the state count."""
    def nn(n):
        return max(16, int(round(n * scale)))

    def px(w):
        return max(16, int(round(w * np.sqrt(scale)))) if scale < 1.0 else w

    if name == "c1_plain_4k":
        sc = make_scene(4096, 8, 2, seed=1001, temporal_rank=0, residual_attrs="colour_opacity")
        rng = np.random.default_rng(2001)
        S = n_states or 1
        bits = bernoulli_states(S, 8, 2, rng)
        st = States(_pack(bits), np.zeros(S, np.float32), np.zeros(S, np.int32))
        cams = [ring_camera(0, 1, 128, 128, 150.0)]
        return Workload(name, sc, cams, st, np.zeros(3, np.float32))
    if name == "c2_dynamic_250k":
        sc = make_scene(nn(250_000), 32, 4, seed=1002)
        rng = np.random.default_rng(2002)
        S = n_states or 256
        d = prefix_states(S, 32, 4, rng)
        t = (np.arange(S) % 16) / 16.0
        W = px(800)
        cams = [ring_camera(0, 1, W, W, 960.0 * W / 800)]
        st = States(_pack(depths_to_bits(d, 4)), t.astype(np.float32), np.zeros(S, np.int32))
        return Workload(name, sc, cams, st, np.zeros(3, np.float32))
    if name == "c3_fwdbwd_250k":
        sc = make_scene(nn(250_000), 64, 4, seed=1003)
        teacher = make_scene(nn(250_000), 64, 4, seed=4003)
        rng = np.random.default_rng(2003)
        S = n_states or 64
        d = prefix_states(S, 64, 4, rng)
        bits = erase_one_packet(depths_to_bits(d, 4), 0.10, rng)
        rng_t = np.random.default_rng(3003)
        t = rng_t.integers(0, 16, size=S) / 16.0
        W = px(512)
        cams = [ring_camera(k, 8, W, W, 600.0 * W / 512) for k in range(8)]
        st = States(_pack(bits), t.astype(np.float32), (np.arange(S) % 8).astype(np.int32))
        return Workload(name, sc, cams, st, np.zeros(3, np.float32), target_scene=teacher)
    if name == "c4_utility_2p7m":
        sc = make_scene(nn(2_700_000), 64, 4, seed=1004)
        rng = np.random.default_rng(2004)
        S = n_states or 32768
        d = prefix_states(S, 64, 4, rng, distinct=True)
        W, H = (px(480), px(270))
        cams = [ring_camera(0, 1, W, H, 520.0 * W / 480)]
        st = States(_pack(depths_to_bits(d, 4)), np.full(S, 0.25, np.float32),
                    np.zeros(S, np.int32))
        return Workload(name, sc, cams, st, np.zeros(3, np.float32))
    raise KeyError(name)
