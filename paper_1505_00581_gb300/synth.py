"""Seeded synthetic models and scenes shaped like the paper's workloads.

This module holds input generation only: it draws point positions, frame
indices and descriptors and implants jittered model copies into clutter. It
contains none of the matching arithmetic, so both the CPU oracle (tests) and
the CUDA path (library, benchmark) draw their inputs from here.

Shapes follow the paper's setting (Sec. 4): space-time interest points with
162-d HoG/HoF-like descriptors, models of roughly one second (t in [0, 30)),
scenes with many points per frame. The real KTH features are not available,
so every input is synthetic: cluster-structured Gaussian descriptors, uniform
positions, Poisson or fixed point counts per frame, and implanted model
instances (xy jitter, frame jitter, descriptor noise).
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence, Tuple

import numpy as np


@dataclasses.dataclass
class PointSet:
    """A model or scene: positions (n,2) f32, frame index (n,) i32, descriptors (n,F) f32."""

    xy: np.ndarray
    t: np.ndarray
    f: np.ndarray
    centres: Optional[np.ndarray] = None  # descriptor cluster centres (models only)

    @property
    def n(self) -> int:
        return int(self.t.shape[0])

    @property
    def F(self) -> int:
        return int(self.f.shape[1])


@dataclasses.dataclass
class Implant:
    model: int      # index of the implanted model
    offset: int     # scene frame offset o of the implant
    idx: np.ndarray  # scene indices (caller order) of the implanted points, model order


@dataclasses.dataclass
class Scene(PointSet):
    n_frames: int = 0
    implants: List[Implant] = dataclasses.field(default_factory=list)


def make_model(rng: np.random.Generator, M: int, F: int = 162, frame: Tuple[float, float] = (160.0, 120.0),
               t_span: int = 30, T: int = 10, n_clusters: int = 8, noise: float = 0.3) -> PointSet:
    """One model: M points sorted by frame, descriptors from n_clusters N(0,1) centres + N(0,noise).

    Frames are resampled until every t_i - t_{i-2} < T, so that a noise-free
    implant of the model is feasible under the temporal closeness rule.
    """
    centres = rng.standard_normal((n_clusters, F))
    while True:
        t = np.sort(rng.integers(0, t_span, size=M))
        if M < 3 or np.all(t[2:] - t[:-2] < T):
            break
    xy = rng.uniform((0.0, 0.0), frame, size=(M, 2))
    lab = rng.integers(0, n_clusters, size=M)
    f = centres[lab] + noise * rng.standard_normal((M, F))
    return PointSet(xy.astype(np.float32), t.astype(np.int32), f.astype(np.float32), centres)


def make_scene(rng: np.random.Generator, n_frames: int, frame: Tuple[float, float],
               per_frame, centre_pool: np.ndarray, models: Sequence[PointSet],
               implants: Sequence[Tuple[int, int]], translate: bool = True, noise: float = 0.3,
               xy_jitter: float = 2.0, t_jitter: float = 1.0, f_noise: float = 0.1,
               F_pad: Optional[int] = None) -> Scene:
    """A scene of n_frames frames: uniform clutter plus jittered copies of models.

    per_frame: an int (fixed count) or ("poisson", lam).
    centre_pool: (C,F) descriptor centres; clutter picks one at random + N(0,noise).
    implants: (model index, offset o) pairs; a copy of model m is placed at
        frames t + o + rint(N(0,t_jitter)) clipped to the scene, positions
        xy + N(0,xy_jitter) (+ a random in-frame translation if translate),
        descriptors f + N(0,f_noise).
    Points are emitted clutter first (frame order), implants appended after, so
    the scene is NOT time sorted: the library's stable sort is exercised.
    F_pad: zero-pad descriptors to this width (zeros leave distances unchanged).
    """
    F = centre_pool.shape[1]
    if isinstance(per_frame, tuple):
        counts = rng.poisson(per_frame[1], size=n_frames)
    else:
        counts = np.full(n_frames, int(per_frame))
    n_clutter = int(counts.sum())
    t = np.repeat(np.arange(n_frames, dtype=np.int64), counts)
    xy = rng.uniform((0.0, 0.0), frame, size=(n_clutter, 2))
    ci = rng.integers(0, centre_pool.shape[0], size=n_clutter)
    f = centre_pool[ci] + noise * rng.standard_normal((n_clutter, F))
    xs, ts, fs = [xy], [t], [f]
    recs = []
    base = n_clutter
    for (m, o) in implants:
        mod = models[m]
        mxy = mod.xy.astype(np.float64) + xy_jitter * rng.standard_normal((mod.n, 2))
        if translate:
            lo = -mxy.min(axis=0)
            hi = np.asarray(frame) - mxy.max(axis=0)
            shift = rng.uniform(np.minimum(lo, hi), np.maximum(lo, hi))
            mxy = mxy + shift
        mt = mod.t.astype(np.int64) + o + np.rint(t_jitter * rng.standard_normal(mod.n)).astype(np.int64)
        mt = np.clip(mt, 0, n_frames - 1)
        mf = mod.f.astype(np.float64) + f_noise * rng.standard_normal((mod.n, F))
        xs.append(mxy); ts.append(mt); fs.append(mf)
        recs.append(Implant(m, int(o), np.arange(base, base + mod.n)))
        base += mod.n
    xy = np.concatenate(xs).astype(np.float32)
    t = np.concatenate(ts).astype(np.int32)
    f = np.concatenate(fs).astype(np.float32)
    if F_pad is not None and F_pad > F:
        f = np.concatenate([f, np.zeros((f.shape[0], F_pad - F), np.float32)], axis=1)
    return Scene(xy, t, f, None, n_frames, recs)


def pad_model(m: PointSet, F_pad: int) -> PointSet:
    if F_pad <= m.F:
        return m
    f = np.concatenate([m.f, np.zeros((m.n, F_pad - m.F), np.float32)], axis=1)
    return PointSet(m.xy, m.t, f, m.centres)


@dataclasses.dataclass
class Workload:
    name: str
    models: List[PointSet]
    scenes: List[Scene]
    K: int
    window: int
    lambda1: float = 0.6
    lambda2: float = 0.2
    lambda3: float = 5.0
    T: int = 10
    # optional offset range applied to every pair (hgm_params offset_lo / offset_hi), and the scene frames a
    # pass over the workload stands for (blocks cut from longer scenes: the frames whose offsets they own)
    offset_lo: Optional[int] = None
    offset_hi: Optional[int] = None
    frames_credit: Optional[int] = None

    @property
    def total_frames(self) -> int:
        if self.frames_credit is not None:
            return int(self.frames_credit)
        return int(sum(s.n_frames for s in self.scenes))

    def offset_range(self, m: int, s: int) -> Tuple[int, int]:
        """[first, last] offset of pair (m, s): o in [-t_1, F_s-1-t_M] within the optional offset range."""
        mod, sc = self.models[m], self.scenes[s]
        lo, hi = -int(mod.t.min()), sc.n_frames - 1 - int(mod.t.max())
        if self.offset_lo is not None:
            lo = max(lo, self.offset_lo)
        if self.offset_hi is not None:
            hi = min(hi, self.offset_hi)
        return lo, hi

    def n_offsets(self, m: int, s: int) -> int:
        lo, hi = self.offset_range(m, s)
        return max(0, hi - lo + 1)


def single_match(seed: int = 0) -> Workload:
    """One M=16 model vs a 60-frame, 10 points/frame scene with one implant at o=20; K=32, w=2."""
    rng = np.random.default_rng(seed)
    mod = make_model(rng, 16)
    sc = make_scene(rng, 60, (160.0, 120.0), 10, mod.centres, [mod], [(0, 20)], translate=False)
    return Workload("single_match_M16_F60_K32", [mod], [sc], K=32, window=2)


def batched_scenes(rng: np.random.Generator, models: Sequence[PointSet], n_scenes: int, frames_range=(300, 1500),
                   lam: float = 30.0, implants_per_scene: int = 3, frame=(320.0, 240.0)) -> List[Scene]:
    """Scenes of the batched workload for a given model set: clutter from the models' centres, implants of
    random models at random offsets."""
    pool = np.concatenate([m.centres for m in models])
    scenes = []
    for _ in range(n_scenes):
        nf = int(rng.integers(frames_range[0], frames_range[1] + 1))
        imp = []
        for _ in range(implants_per_scene):
            m = int(rng.integers(0, len(models)))
            span = int(models[m].t.max())
            imp.append((m, int(rng.integers(0, max(1, nf - span)))))
        scenes.append(make_scene(rng, nf, frame, ("poisson", lam), pool, models, imp))
    return scenes


def batched_exact(seed: int = 1, n_models: int = 10, n_scenes: int = 8, M_range=(16, 64),
                  frames_range=(300, 1500), lam: float = 30.0, implants_per_scene: int = 3) -> Workload:
    """10 models (M in 16..64) vs 8 scenes of 300-1500 frames, Poisson(30)/frame at 320x240; K=64, w=3."""
    rng = np.random.default_rng(seed)
    models = [make_model(rng, int(rng.integers(M_range[0], M_range[1] + 1))) for _ in range(n_models)]
    scenes = batched_scenes(rng, models, n_scenes, frames_range, lam, implants_per_scene)
    return Workload(f"batched_exact_{n_models}x{n_scenes}_K64", models, scenes, K=64, window=3)


def training_scenes(wl: Workload, seed: int, n_scenes: int = 3) -> Workload:
    """The same models with separately seeded scenes (the proposal network's training data)."""
    rng = np.random.default_rng(seed)
    scenes = batched_scenes(rng, wl.models, n_scenes)
    return Workload(wl.name + f"_train{seed}", wl.models, scenes, K=wl.K, window=wl.window, T=wl.T)


def precision_long(seed: int = 2, n_models: int = 50, n_frames: int = 30000, M_range=(32, 128),
                   lam: float = 60.0, F_pad: int = 176, n_implants: int = 50) -> Workload:
    """50 models (M in 32..128) vs one 30,000-frame 640x480 Poisson(60)/frame scene, F padded to 176; K=64, w=3."""
    rng = np.random.default_rng(seed)
    models = [make_model(rng, int(rng.integers(M_range[0], M_range[1] + 1))) for _ in range(n_models)]
    pool = np.concatenate([m.centres for m in models])
    imp = []
    for k in range(n_implants):
        m = k % n_models
        imp.append((m, int(rng.integers(0, n_frames - 30))))
    sc = make_scene(rng, n_frames, (640.0, 480.0), ("poisson", lam), pool, models, imp, F_pad=F_pad)
    models = [pad_model(m, F_pad) for m in models]
    return Workload(f"precision_long_{n_models}x1x{n_frames}_K64", models, [sc], K=64, window=3)


class CombinedScenes:
    """The full combined workload, its scenes generated on demand: models of M in 16..256 points (drawn as by
    make_model) against n_scenes scenes of 10k-100k frames at 640x480 with Poisson(lam) clutter points per
    frame, implants of random models at about implant_frac of the offsets (each implant is seen by the 2w+1
    offsets around it); K = 64, w = 3.

    Sixteen scenes of up to 100k frames hold about 70 M points (46 GB of FP32 descriptors), so a scene is
    never built whole unless asked for: the clutter of every 64-frame chunk of scene s is drawn from its own
    seeded stream (seed, s, chunk), and every implant from its own stream (seed, s, 10^6 + k), so any run of
    frames [f0, f1) of a scene is generated alone (block), point for point the same as in the whole scene.
    Within a block the clutter comes first in frame order, then the implant points that fall in it, implant
    by implant (not time sorted, as make_scene)."""

    CHUNK = 64

    def __init__(self, seed: int = 3, n_models: int = 100, n_scenes: int = 16, M_range=(16, 256),
                 frames_range=(10_000, 100_000), lam: float = 80.0, implant_frac: float = 0.05,
                 frame=(640.0, 480.0), window: int = 3, K: int = 64, F: int = 162):
        rng = np.random.default_rng(seed)
        self.seed, self.lam, self.frame, self.window, self.K, self.F = seed, lam, frame, window, K, F
        self.models = [make_model(rng, int(rng.integers(M_range[0], M_range[1] + 1)), F=F) for _ in range(n_models)]
        self.pool = np.concatenate([m.centres for m in self.models])
        self.n_frames: List[int] = []
        self.implants: List[List[Tuple[int, int]]] = []
        for _ in range(n_scenes):
            nf = int(rng.integers(frames_range[0], frames_range[1] + 1))
            n_imp = max(1, int(round(implant_frac * nf / (2 * window + 1))))
            imp = []
            for _ in range(n_imp):
                m = int(rng.integers(0, n_models))
                span = int(self.models[m].t.max())
                imp.append((m, int(rng.integers(0, max(1, nf - span)))))
            self.n_frames.append(nf)
            self.implants.append(imp)

    @property
    def total_frames(self) -> int:
        return int(sum(self.n_frames))

    def _chunk(self, s: int, c: int):
        rng = np.random.default_rng([self.seed, s, c])
        counts = rng.poisson(self.lam, size=self.CHUNK)
        n = int(counts.sum())
        t = c * self.CHUNK + np.repeat(np.arange(self.CHUNK, dtype=np.int64), counts)
        xy = rng.uniform((0.0, 0.0), self.frame, size=(n, 2))
        ci = rng.integers(0, self.pool.shape[0], size=n)
        f = (self.pool[ci] + 0.3 * rng.standard_normal((n, self.F))).astype(np.float32)
        return xy.astype(np.float32), t, f

    def _implant(self, s: int, k: int):
        m, o = self.implants[s][k]
        mod, nf = self.models[m], self.n_frames[s]
        rng = np.random.default_rng([self.seed, s, 1_000_000 + k])
        mxy = mod.xy.astype(np.float64) + 2.0 * rng.standard_normal((mod.n, 2))
        lo = -mxy.min(axis=0)
        hi = np.asarray(self.frame) - mxy.max(axis=0)
        mxy = mxy + rng.uniform(np.minimum(lo, hi), np.maximum(lo, hi))
        mt = np.clip(mod.t.astype(np.int64) + o + np.rint(rng.standard_normal(mod.n)).astype(np.int64), 0, nf - 1)
        mf = (mod.f.astype(np.float64) + 0.1 * rng.standard_normal((mod.n, self.F))).astype(np.float32)
        return mxy.astype(np.float32), mt, mf

    def block(self, s: int, f0: int, f1: int) -> Scene:
        """Frames [f0, f1) of scene s as a scene of f1 - f0 frames (frame f0 becomes 0)."""
        nf = self.n_frames[s]
        if not (0 <= f0 < f1 <= nf):
            raise ValueError(f"block [{f0}, {f1}) outside scene {s} of {nf} frames")
        xs, ts, fs = [], [], []
        for c in range(f0 // self.CHUNK, (f1 - 1) // self.CHUNK + 1):
            xy, t, f = self._chunk(s, c)
            sel = (t >= f0) & (t < f1)
            xs.append(xy[sel]); ts.append(t[sel]); fs.append(f[sel])
        recs = []
        base = int(sum(len(t) for t in ts))
        for k, (m, o) in enumerate(self.implants[s]):
            if o + int(self.models[m].t.max()) + 8 < f0 or o - 8 >= f1:
                continue            # frame jitter moves a point by a few frames at most
            xy, t, f = self._implant(s, k)
            sel = (t >= f0) & (t < f1)
            if not sel.any():
                continue
            xs.append(xy[sel]); ts.append(t[sel]); fs.append(f[sel])
            n = int(sel.sum())
            recs.append(Implant(m, o - f0, np.arange(base, base + n)))
            base += n
        return Scene(np.concatenate(xs).astype(np.float32), (np.concatenate(ts) - f0).astype(np.int32),
                     np.concatenate(fs).astype(np.float32), None, f1 - f0, recs)

    def scene(self, s: int) -> Scene:
        return self.block(s, 0, self.n_frames[s])

    def training_scenes(self, seed: int, n_scenes: int = 3, n_frames: int = 300) -> Workload:
        """The same models against separately seeded scenes of the same shape (Poisson(lam) clutter at
        640x480, implants at about 5% of the offsets): the proposal network's training data."""
        rng = np.random.default_rng(seed)
        w = self.window
        scenes = []
        for _ in range(n_scenes):
            n_imp = max(1, int(round(0.05 * n_frames / (2 * w + 1))))
            imp = []
            for _ in range(n_imp):
                m = int(rng.integers(0, len(self.models)))
                imp.append((m, int(rng.integers(0, max(1, n_frames - int(self.models[m].t.max()))))))
            scenes.append(make_scene(rng, n_frames, self.frame, ("poisson", self.lam), self.pool, self.models, imp))
        return Workload(f"combined_train{seed}", self.models, scenes, K=self.K, window=w)

    def step(self, hop: int = 256, seed: int = 0, span: int = 29) -> Workload:
        """One pass over a sample of the job: every model against one block of each scene. Block s covers
        frames [f0 - w, f0 + hop + span + w) of scene s, f0 a seeded multiple of hop, and every pair is
        restricted to the block's offsets w .. w + hop - 1: those are the full scene's offsets f0 .. f0+hop-1,
        whose windows (model frames 0..span, +-w) lie inside the block, so their candidate lists and results
        are the full scene's. Tiling a scene with such blocks (hop apart) evaluates every offset once; a
        pass therefore stands for n_scenes x hop scene frames (frames_credit)."""
        w = self.window
        rng = np.random.default_rng([self.seed, 7_000_000 + seed])
        blocks = []
        for s, nf in enumerate(self.n_frames):
            n_pos = (nf - span - 2 * w) // hop
            f0 = w + hop * int(rng.integers(0, max(1, n_pos)))
            blocks.append(self.block(s, f0 - w, min(nf, f0 + hop + span + w)))
        return Workload(f"combined_{len(self.models)}x{len(self.n_frames)}_K{self.K}_hop{hop}", self.models, blocks,
                        K=self.K, window=w, offset_lo=w, offset_hi=w + hop - 1, frames_credit=len(blocks) * hop)


def combined(seed: int = 3, n_models: int = 100, n_scenes: int = 16, M_range=(16, 256),
             frames_range=(10_000, 100_000), lam: float = 80.0, implant_frac: float = 0.05,
             frame=(640.0, 480.0)) -> Workload:
    """The combined workload with its scenes built whole (CombinedScenes.scene); meant for scaled-down
    instances (fewer models and scenes, shorter scenes) of the same shape."""
    cs = CombinedScenes(seed, n_models, n_scenes, M_range, frames_range, lam, implant_frac, frame)
    return Workload(f"combined_{n_models}x{n_scenes}_K64", cs.models, [cs.scene(s) for s in range(n_scenes)],
                    K=64, window=3)


def paper_model(rng: np.random.Generator, M: int = 30, F: int = 162, frame: Tuple[float, float] = (160.0, 120.0),
                n_clusters: int = 8, noise: float = 0.3) -> PointSet:
    """A model shaped like the paper's: one point per frame over M consecutive frames (Sec. 4: models of
    20-30 frames after saliency selection), descriptors as make_model."""
    centres = rng.standard_normal((n_clusters, F))
    t = np.arange(M)
    xy = rng.uniform((0.0, 0.0), frame, size=(M, 2))
    f = centres[rng.integers(0, n_clusters, size=M)] + noise * rng.standard_normal((M, F))
    return PointSet(xy.astype(np.float32), t.astype(np.int32), f.astype(np.float32), centres)


def paper_blocks(seed: int = 4, n_models: int = 50, M: int = 30, n_blocks: int = 4, block_frames: int = 60,
                 lam: float = 1.0, implant_frac: float = 0.5, frame=(160.0, 120.0)) -> Workload:
    """The paper's real-time scenario (Sec. 4, Table 2): 50 models of 30 one-per-frame points against scene
    blocks of 60 frames with about one point per frame (Poisson(lam) clutter), matched as whole blocks;
    about implant_frac of the blocks hold a jittered copy of a random model at a random offset."""
    rng = np.random.default_rng(seed)
    models = [paper_model(rng, M) for _ in range(n_models)]
    pool = np.concatenate([m.centres for m in models])
    scenes = []
    for _ in range(n_blocks):
        imps = []
        if rng.random() < implant_frac:
            imps = [(int(rng.integers(n_models)), int(rng.integers(0, block_frames - M + 1)))]
        scenes.append(make_scene(rng, block_frames, frame, ("poisson", lam), pool, models, imps))
    return Workload(f"paper_blocks_{n_models}x{n_blocks}_M{M}_F{block_frames}", models, scenes, K=64, window=3)


def paper_stream(seed: int = 5, n_models: int = 50, M: int = 30, n_frames: int = 1800, lam: float = 1.0,
                 implant_every: int = 120, frame=(160.0, 120.0)) -> Workload:
    """The paper's continuous-video scenario (Sec. 4): 50 one-per-frame models of 30 points and one long scene
    of about one point per frame (a minute at 30 frames/s), with a jittered copy of a random model every
    implant_every frames; streamed as 60-frame blocks."""
    rng = np.random.default_rng(seed)
    models = [paper_model(rng, M) for _ in range(n_models)]
    pool = np.concatenate([m.centres for m in models])
    imps = [(int(rng.integers(n_models)), int(o)) for o in range(15, n_frames - M, implant_every)]
    sc = make_scene(rng, n_frames, frame, ("poisson", lam), pool, models, imps)
    return Workload(f"paper_stream_{n_models}x1_M{M}_F{n_frames}", models, [sc], K=64, window=3)


def paper_whole(seed: int = 6, n_models: int = 50, M: int = 30, n_frames: int = 723, nodes: int = 754,
                frame=(160.0, 120.0)) -> Workload:
    """Table 2's scene: a 723-frame video with about 754 interest points (one implant), matched whole."""
    rng = np.random.default_rng(seed)
    models = [paper_model(rng, M) for _ in range(n_models)]
    pool = np.concatenate([m.centres for m in models])
    sc = make_scene(rng, n_frames, frame, ("poisson", (nodes - M) / n_frames), pool, models,
                    [(int(rng.integers(n_models)), n_frames // 2)])
    return Workload(f"paper_whole_{n_models}x1_M{M}_F{n_frames}", models, [sc], K=64, window=3)


def tiny_case(seed: int, M: int = 5, n_frames: int = 12, per_frame: int = 3, K: int = 5, window: int = 1,
              F: int = 8, T: int = 10, frame=(20.0, 20.0)) -> Workload:
    """Very small random instance for brute-force enumeration."""
    rng = np.random.default_rng(seed)
    mod = make_model(rng, M, F=F, frame=frame, t_span=min(8, n_frames), T=T, n_clusters=3)
    sc = make_scene(rng, n_frames, frame, per_frame, mod.centres, [mod],
                    [(0, int(rng.integers(0, max(1, n_frames - int(mod.t.max())))))], translate=False)
    return Workload(f"tiny_{seed}", [mod], [sc], K=K, window=window, T=T)
