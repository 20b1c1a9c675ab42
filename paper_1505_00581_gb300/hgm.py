"""Thin Python binding of libhgm (include/hgm.h): argument marshalling only.

Every step of the matching runs inside libhgm's CUDA kernels; this module
converts numpy arrays / torch tensors into pointers, passes torch's current
CUDA stream, and raises on a non-zero status. There is no CPU fallback: if
``_build/libhgm.so`` is missing or cannot be loaded, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhgm.so")

HGM_OK, HGM_EINVAL, HGM_ENOMEM, HGM_ECUDA, HGM_ETIMEOUT, HGM_EUNSUPPORTED = range(6)
KERNELS = ("unary", "select", "recurse", "backtrack", "prune")

# Every function declared in include/hgm.h, with (restype, argtypes).
_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_f32 = ctypes.c_float
_p32 = ctypes.POINTER(ctypes.c_int32)
_p64 = ctypes.POINTER(ctypes.c_int64)
_pf = ctypes.POINTER(ctypes.c_float)
_pd = ctypes.POINTER(ctypes.c_double)


class Params(ctypes.Structure):
    """hgm_params (include/hgm.h)."""
    _fields_ = [("lambda1", ctypes.c_float), ("lambda2", ctypes.c_float), ("lambda3", ctypes.c_float),
                ("T", ctypes.c_int32), ("window", ctypes.c_int32), ("K", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("offset_lo", ctypes.c_int32), ("offset_hi", ctypes.c_int32),
                ("prune", ctypes.c_void_p), ("keep", ctypes.c_int32), ("refine", ctypes.c_int32),
                ("dummy_cost", ctypes.c_float)]


_PP = ctypes.POINTER(Params)
SIGNATURES = {
    "hgm_default_params": (None, [_PP]),
    "hgm_create_model": (_i32, [_vp, _vp, _vp, _i32, _i32, _vp, ctypes.POINTER(_vp)]),
    "hgm_create_scene": (_i32, [_vp, _vp, _vp, _i32, _i32, _i32, _vp, ctypes.POINTER(_vp)]),
    "hgm_destroy": (None, [_vp]),
    "hgm_last_error": (ctypes.c_char_p, []),
    "hgm_offsets": (_i32, [_vp, _vp, _PP, _p32, _p32]),
    "hgm_match": (_i32, [_vp, _vp, _PP, _vp, _p32, _p32, _vp, _vp]),
    "hgm_batch_layout": (_i32, [ctypes.POINTER(_vp), _i32, ctypes.POINTER(_vp), _i32, _PP, _p32, _p64, _p64]),
    "hgm_match_batch": (_i32, [ctypes.POINTER(_vp), _i32, ctypes.POINTER(_vp), _i32, _PP, _vp, _vp, _vp]),
    "hgm_match_noalloc": (_i32, [_vp, _vp, _PP, _vp, _vp, _vp]),
    "hgm_prop_create": (_i32, [_i32, _vp, ctypes.c_uint64, ctypes.POINTER(_vp)]),
    "hgm_prop_size": (_i64, [_i32]),
    "hgm_prop_get": (_i32, [_vp, _vp, _p64]),
    "hgm_prop_set": (_i32, [_vp, _vp, _i64]),
    "hgm_prop_forward": (_i32, [_vp, _vp, _i32, _vp, _vp]),
    "hgm_prop_gradients": (_i32, [_vp, _vp, _vp, _i32, _vp, _vp, _vp]),
    "hgm_prop_train_step": (_i32, [_vp, _vp, _vp, _i32, _f32, _vp, _vp]),
    "hgm_autotune": (_i32, [ctypes.POINTER(_vp), _i32, ctypes.POINTER(_vp), _i32, _PP, _vp, _i32, _p32, _pf]),
    "hgm_set_recurse_variant": (_i32, [_i32]),
    "hgm_get_recurse_variant": (_i32, []),
    "hgm_set_workspace_budget": (_i32, [_i64]),
    "hgm_plan_create": (_i32, [_vp, _i32, _vp, _i32, _vp, _vp, _vp, _vp, _vp]),
    "hgm_plan_run": (_i32, [_vp, _vp]),
    "hgm_plan_check": (_i32, [_vp, _vp]),
    "hgm_prop_scores": (_i32, [_vp, _vp, _vp, _vp, _i32, _i32, _vp, _vp]),
    "hgm_match_chains": (_i32, [_vp, _vp, _PP, _i32, _vp, _p32, _p32, _vp, _vp]),
    "hgm_stream_create": (_i32, [ctypes.POINTER(_vp), _i32, _PP, _i32, _i32, _vp, ctypes.POINTER(_vp)]),
    "hgm_stream_match": (_i32, [_vp, _vp, _vp, _vp, _i32, _vp, _vp, _vp]),
    "hgm_match_block": (_i32, [ctypes.POINTER(_vp), _i32, ctypes.POINTER(_vp), _i32, _PP, _vp, _vp, _vp]),
    "hgm_match_chains_batch": (_i32, [ctypes.POINTER(_vp), _i32, ctypes.POINTER(_vp), _i32, _PP, _i32, _vp, _vp,
                                      _vp]),
    "hgm_model_order": (_i32, [_vp, _p32]),
    "hgm_scene_order": (_i32, [_vp, _p32]),
    "hgm_unary": (_i32, [_vp, _vp, _f32, _vp, _vp]),
    "hgm_unary_bf16": (_i32, [_vp, _vp, _f32, _vp, _vp]),
    "hgm_candidates": (_i32, [_vp, _vp, _PP, _i32, _i32, _vp, _vp, _vp, _vp]),
    "hgm_count_triples": (_i32, [_vp, _vp, _PP, _i32, _i32, _vp, _vp]),
    "hgm_atan2_f32": (_i32, [_vp, _vp, _i64, _vp, _vp]),
    "hgm_debug_timeout": (_i32, [ctypes.c_uint32, _vp, _vp]),
    "hgm_gemm_bf16": (_i32, [_vp, _vp, _i32, _i32, _i32, _vp, _vp, _vp]),
    "hgm_profile_enable": (_i32, [_i32]),
    "hgm_profile_read": (_i32, [_pd, _p64, _i32]),
    "hgm_profile_evaluated": (_i32, [_p64, _i32]),
    "hgm_prune_counters": (_i32, [_p64, _p64, _i32]),
    "hgm_refine_counter": (_i32, [_p64, _i32]),
    "hgm_profile_reset": (_i32, []),
}

_lib = None


class HgmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"hgm status {status}: {msg}")
        self.status = status


def load(path: str = LIB_PATH):
    """Loads libhgm.so (built by __graft_entry__.build() / paper_1505_00581_gb300.build). No fallback."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libhgm.so not found at {path}: build it first (python -c 'import __graft_entry__ as g; "
                          f"g.build()'); there is no CPU fallback")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int):
    if status != HGM_OK:
        msg = _lib.hgm_last_error()
        raise HgmError(status, msg.decode() if msg else "")


def default_params(**over) -> Params:
    lib = load()
    p = Params()
    lib.hgm_default_params(ctypes.byref(p))
    for k, v in over.items():
        if k == "prune" and v is not None and hasattr(v, "handle"):
            v = v.handle.value    # a Proposal object
        setattr(p, k, v)
    return p


def _stream(stream=None) -> int:
    """cudaStream_t handle: an int, a torch.cuda.Stream (its cuda_stream), or None for torch's current stream."""
    if stream is not None:
        return int(getattr(stream, "cuda_stream", stream))
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            return int(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return 0


def _ptr(a):
    """(pointer, keepalive) for a torch tensor (CPU/CUDA) or numpy array, contiguous."""
    if a is None:
        return None, None
    try:
        import torch
        if isinstance(a, torch.Tensor):
            a = a.contiguous()
            return a.data_ptr(), a
    except ImportError:
        pass
    a = np.ascontiguousarray(a)
    return a.ctypes.data, a


class Model:
    """A model handle: M points (xy float32 [M,2], t int32 [M], f float32 [M,F]), host or device."""

    def __init__(self, xy, t, f, stream=None):
        self.lib = load()
        xy = _as(xy, np.float32)
        t = _as(t, np.int32)
        f = _as(f, np.float32)
        (pxy, kxy), (pt, kt), (pf, kf) = _ptr(xy), _ptr(t), _ptr(f)
        h = ctypes.c_void_p()
        M, F = int(f.shape[0]), int(f.shape[1])
        _check(self.lib.hgm_create_model(pxy, pt, pf, M, F, _stream(stream), ctypes.byref(h)))
        self.handle, self.M, self.F = h, M, F

    def order(self) -> np.ndarray:
        out = np.zeros(self.M, np.int32)
        _check(self.lib.hgm_model_order(self.handle, out.ctypes.data_as(_p32)))
        return out

    def close(self):
        if getattr(self, "handle", None):
            self.lib.hgm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Scene:
    """A scene handle: S points (xy [S,2], t [S], f [S,F]) over n_frames frames, host or device."""

    def __init__(self, xy, t, f, n_frames: int = 0, stream=None):
        self.lib = load()
        xy = _as(xy, np.float32)
        t = _as(t, np.int32)
        f = _as(f, np.float32)
        (pxy, kxy), (pt, kt), (pf, kf) = _ptr(xy), _ptr(t), _ptr(f)
        h = ctypes.c_void_p()
        S, F = int(f.shape[0]), int(f.shape[1])
        _check(self.lib.hgm_create_scene(pxy, pt, pf, S, F, int(n_frames), _stream(stream), ctypes.byref(h)))
        self.handle, self.S, self.F, self.n_frames = h, S, F, int(n_frames)

    def order(self) -> np.ndarray:
        out = np.zeros(self.S, np.int32)
        _check(self.lib.hgm_scene_order(self.handle, out.ctypes.data_as(_p32)))
        return out

    def close(self):
        if getattr(self, "handle", None):
            self.lib.hgm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _as(a, dtype):
    try:
        import torch
        if isinstance(a, torch.Tensor):
            tdt = {np.float32: torch.float32, np.int32: torch.int32}[dtype]
            return a.to(tdt).contiguous()
    except ImportError:
        pass
    return np.ascontiguousarray(a, dtype=dtype)


class Proposal:
    """Candidate-proposal network handle (hgm_prop_*). weights: flat FP32 host array in the ABI order."""

    def __init__(self, F: int, weights=None, seed: int = 0):
        self.lib = load()
        self.F = int(F)
        self.size = int(self.lib.hgm_prop_size(self.F))
        h = ctypes.c_void_p()
        w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float32)
        if w is not None and w.size != self.size:
            raise ValueError(f"expected {self.size} weights, got {w.size}")
        _check(self.lib.hgm_prop_create(self.F, None if w is None else w.ctypes.data, int(seed), ctypes.byref(h)))
        self.handle = h

    @property
    def d_in(self):
        return 2 * self.F + 3

    def get(self):
        w = np.zeros(self.size, np.float32)
        st = ctypes.c_int64()
        _check(self.lib.hgm_prop_get(self.handle, w.ctypes.data, ctypes.byref(st)))
        return w, int(st.value)

    def set(self, weights, step: int = 0):
        w = np.ascontiguousarray(weights, dtype=np.float32)
        _check(self.lib.hgm_prop_set(self.handle, w.ctypes.data, int(step)))

    def unflatten(self, w):
        H, d = 128, self.d_in
        o = 0
        out = {}
        for name, shape in (("W1", (H, d)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("w3", (H,)), ("b3", (1,))):
            n = int(np.prod(shape))
            out[name] = np.asarray(w[o:o + n]).reshape(shape)
            o += n
        return out

    def forward(self, X, out, stream=None):
        _check(self.lib.hgm_prop_forward(self.handle, _ptr(X)[0], int(X.shape[0]), _stream(stream), _ptr(out)[0]))
        return out

    def gradients(self, X, y, stream=None):
        g = np.zeros(self.size, np.float32)
        loss = ctypes.c_float()
        _check(self.lib.hgm_prop_gradients(self.handle, _ptr(X)[0], _ptr(y)[0], int(X.shape[0]), _stream(stream),
                                           ctypes.byref(loss), g.ctypes.data))
        return float(loss.value), g

    def train_step(self, X, y, lr: float, loss_out=None, stream=None):
        _check(self.lib.hgm_prop_train_step(self.handle, _ptr(X)[0], _ptr(y)[0], int(X.shape[0]), float(lr),
                                            _stream(stream), None if loss_out is None else _ptr(loss_out)[0]))

    def close(self):
        if getattr(self, "handle", None):
            self.lib.hgm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def offsets(model: Model, scene: Scene, params: Params):
    n, f = ctypes.c_int32(), ctypes.c_int32()
    _check(load().hgm_offsets(model.handle, scene.handle, ctypes.byref(params), ctypes.byref(n), ctypes.byref(f)))
    return int(f.value), int(n.value)


def match(model: Model, scene: Scene, params: Params, energy=None, assign=None, stream=None):
    """Solves all offsets of one pair. energy/assign: preallocated outputs (torch CUDA tensors or numpy), or
    None to get numpy arrays back. Returns (first_offset, energy, assign)."""
    lib = load()
    first, n = offsets(model, scene, params)
    if energy is None and assign is None:
        energy = np.zeros(n, np.float32)
        assign = np.zeros((n, model.M), np.int32)
    (pe, ke), (pa, ka) = _ptr(energy), _ptr(assign)
    nn, ff = ctypes.c_int32(), ctypes.c_int32()
    _check(lib.hgm_match(model.handle, scene.handle, ctypes.byref(params), _stream(stream), ctypes.byref(nn),
                         ctypes.byref(ff), pe, pa))
    return first, ke if energy is not None else None, ka if assign is not None else None


def match_chains(model: Model, scene: Scene, params: Params, n_chains: int, energy=None, assign=None, stream=None):
    """hgm_match_chains: the mean energy of the model's single-point chains per offset and the union of their
    assignments. Returns (first_offset, energy, assign) like match()."""
    lib = load()
    first, n = offsets(model, scene, params)
    if energy is None and assign is None:
        energy = np.zeros(n, np.float32)
        assign = np.zeros((n, model.M), np.int32)
    (pe, ke), (pa, ka) = _ptr(energy), _ptr(assign)
    nn, ff = ctypes.c_int32(), ctypes.c_int32()
    _check(lib.hgm_match_chains(model.handle, scene.handle, ctypes.byref(params), int(n_chains), _stream(stream),
                                ctypes.byref(nn), ctypes.byref(ff), pe, pa))
    return first, ke if energy is not None else None, ka if assign is not None else None


def match_noalloc(model: Model, scene: Scene, params: Params, energy, assign, stream=None):
    """hgm_match_noalloc: like match() with device outputs, but allocates no device memory (fixed scratch)."""
    (pe, ke), (pa, ka) = _ptr(energy), _ptr(assign)
    _check(load().hgm_match_noalloc(model.handle, scene.handle, ctypes.byref(params), _stream(stream), pe, pa))
    return ke, ka


N_VARIANTS = 3


def _tune_cache_path():
    return os.environ.get("HGM_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "hgm_autotune.json"))


def _tune_key(params: Params) -> str:
    try:
        import torch
        dev = torch.cuda.get_device_name() if torch.cuda.is_available() else "none"
    except ImportError:
        dev = "unknown"
    return f"{dev}|K{'<=32' if params.K <= 32 else '<=64'}|precision{params.precision}"


def autotune(models: Sequence[Model], scenes: Sequence[Scene], params: Params, sample_offsets: int = 128,
             use_cache: bool = True, stream=None):
    """Picks the fastest recursion tile variant for this workload (hgm_autotune) and caches the choice
    in a JSON file keyed by device name and K bucket. Returns (variant, {variant: ms} or None)."""
    import json
    lib = load()
    key, path = _tune_key(params), _tune_cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            cache = json.load(open(path))
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            _check(lib.hgm_set_recurse_variant(int(cache[key]["variant"])))
            return int(cache[key]["variant"]), None
    nm, ns = len(models), len(scenes)
    mh = (ctypes.c_void_p * nm)(*[m.handle for m in models])
    sh = (ctypes.c_void_p * ns)(*[s.handle for s in scenes])
    best = ctypes.c_int32()
    ms = np.zeros(N_VARIANTS, np.float32)
    _check(lib.hgm_autotune(mh, nm, sh, ns, ctypes.byref(params), _stream(stream), int(sample_offsets),
                            ctypes.byref(best), ms.ctypes.data_as(_pf)))
    times = {v: float(ms[v]) for v in range(N_VARIANTS)}
    if use_cache:
        cache[key] = {"variant": int(best.value), "ms": times, "sample_offsets": int(sample_offsets)}
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            with open(path, "w") as fh:
                json.dump(cache, fh, indent=1)
        except OSError:
            pass
    return int(best.value), times


class Plan:
    """hgm_plan: a batch laid out once and replayed as a CUDA graph. energy / assign: device tensors in the
    batch_layout order (kept alive by the plan)."""

    def __init__(self, models, scenes, params: Params, energy=None, assign=None, stream=None):
        self.lib = load()
        mh = (ctypes.c_void_p * len(models))(*[m.handle for m in models])
        sh = (ctypes.c_void_p * len(scenes))(*[s.handle for s in scenes])
        (pe, ke), (pa, ka) = _ptr(energy), _ptr(assign)
        self._keep = (models, scenes, params, ke, ka)
        h = ctypes.c_void_p()
        _check(self.lib.hgm_plan_create(mh, len(models), sh, len(scenes), ctypes.byref(params), pe, pa,
                                        _stream(stream), ctypes.byref(h)))
        self.handle = h

    def run(self, stream=None):
        _check(self.lib.hgm_plan_run(self.handle, _stream(stream)))

    def check(self, stream=None):
        _check(self.lib.hgm_plan_check(self.handle, _stream(stream)))

    def close(self):
        if getattr(self, "handle", None):
            self.lib.hgm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def set_workspace_budget(nbytes: int):
    """Bytes for a segment group's unary table and a chunk's lists/argmin tables (0 = automatic)."""
    _check(load().hgm_set_workspace_budget(int(nbytes)))


def set_recurse_variant(v: int):
    _check(load().hgm_set_recurse_variant(int(v)))


def batch_layout(models: Sequence[Model], scenes: Sequence[Scene], params: Params):
    lib = load()
    nm, ns = len(models), len(scenes)
    mh = (ctypes.c_void_p * max(nm, 1))(*[m.handle for m in models])
    sh = (ctypes.c_void_p * max(ns, 1))(*[s.handle for s in scenes])
    first = np.zeros(max(nm * ns, 1), np.int32)
    es = np.zeros(nm * ns + 1, np.int64)
    as_ = np.zeros(nm * ns + 1, np.int64)
    _check(lib.hgm_batch_layout(mh, nm, sh, ns, ctypes.byref(params), first.ctypes.data_as(_p32),
                                es.ctypes.data_as(_p64), as_.ctypes.data_as(_p64)))
    return first[:nm * ns], es, as_


def match_batch(models: Sequence[Model], scenes: Sequence[Scene], params: Params, energy=None, assign=None,
                stream=None):
    """All offsets of all (model, scene) pairs in one pass; outputs in the batch_layout order."""
    lib = load()
    nm, ns = len(models), len(scenes)
    mh = (ctypes.c_void_p * max(nm, 1))(*[m.handle for m in models])
    sh = (ctypes.c_void_p * max(ns, 1))(*[s.handle for s in scenes])
    (pe, ke), (pa, ka) = _ptr(energy), _ptr(assign)
    _check(lib.hgm_match_batch(mh, nm, sh, ns, ctypes.byref(params), _stream(stream), pe, pa))
    return ke, ka


def block_layout(models: Sequence[Model], n_scenes: int):
    """First assignment element of every (model, scene) pair of match_block (pair q = m * n_scenes + s)."""
    sizes = np.repeat(np.array([m.M for m in models], np.int64), n_scenes)
    return np.concatenate([[0], np.cumsum(sizes)])


def match_block(models: Sequence[Model], scenes: Sequence[Scene], params: Params, energy=None, assign=None,
                stream=None):
    """The whole-block problem (every scene point a candidate, no offsets): one energy per (model, scene) pair
    and the pairs' assignments laid out as block_layout. None outputs are returned as numpy arrays."""
    lib = load()
    nm, ns = len(models), len(scenes)
    starts = block_layout(models, ns)
    if energy is None and assign is None:
        energy = np.zeros(nm * ns, np.float32)
        assign = np.zeros(int(starts[-1]), np.int32)
    mh = (ctypes.c_void_p * max(nm, 1))(*[m.handle for m in models])
    sh = (ctypes.c_void_p * max(ns, 1))(*[s.handle for s in scenes])
    (pe, ke), (pa, ka) = _ptr(energy), _ptr(assign)
    _check(lib.hgm_match_block(mh, nm, sh, ns, ctypes.byref(params), _stream(stream), pe, pa))
    return ke, ka


class Stream:
    """hgm_stream_*: blocks of block_frames frames matched whole against fixed models as they arrive. Every
    buffer is sized at creation for blocks of up to max_points points (larger blocks are refused)."""

    def __init__(self, models: Sequence[Model], params: Params, block_frames: int, stream=None,
                 max_points: int = 256):
        self.lib = load()
        self.models = list(models)     # the handles must outlive the stream
        self.params = params
        self.block_frames = int(block_frames)
        self.max_points = int(max_points)
        self.starts = block_layout(self.models, 1)
        mh = (ctypes.c_void_p * len(self.models))(*[m.handle for m in self.models])
        h = ctypes.c_void_p()
        _check(self.lib.hgm_stream_create(mh, len(self.models), ctypes.byref(params), self.block_frames,
                                          self.max_points, _stream(stream), ctypes.byref(h)))
        self.handle = h

    def match(self, xy, t, f, energy=None, assign=None, stream=None):
        """One block: frames t in [0, block_frames). Returns (energy [n_models], assign [sum M])."""
        if energy is None and assign is None:
            energy = np.zeros(len(self.models), np.float32)
            assign = np.zeros(int(self.starts[-1]), np.int32)
        xy, t, f = _as(xy, np.float32), _as(t, np.int32), _as(f, np.float32)
        n = int(t.shape[0])
        (pxy, kxy), (pt, kt), (pf, kf) = _ptr(xy), _ptr(t), _ptr(f)
        (pe, ke), (pa, ka) = _ptr(energy), _ptr(assign)
        _check(self.lib.hgm_stream_match(self.handle, pxy, pt, pf, n, _stream(stream), pe, pa))
        return ke, ka

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            self.lib.hgm_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def stream_blocks(xy, t, f, n_frames: int, block_frames: int = 60, hop: int = 30):
    """Cuts a scene into blocks of block_frames frames starting every hop frames (the last block ends at the
    scene's end; a scene shorter than a block is one block). With hop > block_frames the frames between
    blocks are skipped. Yields (first_frame, xy, t - first_frame, f, caller indices) per block."""
    if block_frames < 1 or hop < 1:
        raise ValueError(f"block_frames and hop must be >= 1 (got {block_frames}, {hop})")
    t = np.asarray(t)
    starts = list(range(0, max(1, n_frames - block_frames + 1), hop))
    if starts[-1] + block_frames < n_frames:
        starts.append(n_frames - block_frames)
    for s0 in starts:
        idx = np.nonzero((t >= s0) & (t < s0 + block_frames))[0]
        yield s0, xy[idx], (t[idx] - s0).astype(np.int32), f[idx], idx


def match_chains_batch(models: Sequence[Model], scenes: Sequence[Scene], params: Params, n_chains: int,
                       energy=None, assign=None, stream=None):
    """match_chains for every (model, scene) pair in one pass; outputs in the batch_layout order."""
    lib = load()
    nm, ns = len(models), len(scenes)
    mh = (ctypes.c_void_p * max(nm, 1))(*[m.handle for m in models])
    sh = (ctypes.c_void_p * max(ns, 1))(*[s.handle for s in scenes])
    (pe, ke), (pa, ka) = _ptr(energy), _ptr(assign)
    _check(lib.hgm_match_chains_batch(mh, nm, sh, ns, ctypes.byref(params), int(n_chains), _stream(stream), pe, pa))
    return ke, ka


def unary(model: Model, scene: Scene, lambda1: float, out, stream=None):
    (po, ko) = _ptr(out)
    _check(load().hgm_unary(model.handle, scene.handle, float(lambda1), _stream(stream), po))
    return ko


def unary_bf16(model: Model, scene: Scene, lambda1: float, out, stream=None):
    (po, ko) = _ptr(out)
    _check(load().hgm_unary_bf16(model.handle, scene.handle, float(lambda1), _stream(stream), po))
    return ko


def candidates(model: Model, scene: Scene, params: Params, first: int, n: int, idx, cnt, stream=None, cost=None):
    (pi, ki), (pc, kc) = _ptr(idx), _ptr(cnt)
    pu = None if cost is None else _ptr(cost)[0]
    _check(load().hgm_candidates(model.handle, scene.handle, ctypes.byref(params), int(first), int(n),
                                 _stream(stream), pi, pc, pu))
    return ki, kc


def prop_scores(prop: "Proposal", model: Model, scene: Scene, params: Params, first: int, n: int, out, stream=None):
    """The pruning pass's logit of every candidate (out: device float [n, M, K]; -inf for empty slots)."""
    (po, ko) = _ptr(out)
    _check(load().hgm_prop_scores(prop.handle, model.handle, scene.handle, ctypes.byref(params), int(first), int(n),
                                  _stream(stream), po))
    return ko


def count_triples(model: Model, scene: Scene, params: Params, first: int, n: int, out, stream=None):
    (po, ko) = _ptr(out)
    _check(load().hgm_count_triples(model.handle, scene.handle, ctypes.byref(params), int(first), int(n),
                                    _stream(stream), po))
    return ko


def debug_timeout(polls: int, status, stream=None):
    """hgm_debug_timeout: a bounded wait that runs out; status (device int32 tensor) becomes 1."""
    (ps, ks) = _ptr(status)
    _check(load().hgm_debug_timeout(int(polls), _stream(stream), ps))
    return ks


def atan2_f32(y, x, out, stream=None):
    """The recursion kernel's FP32 atan2 applied elementwise (device tensors)."""
    (py, ky), (px, kx), (po, ko) = _ptr(y), _ptr(x), _ptr(out)
    _check(load().hgm_atan2_f32(py, px, int(ko.numel() if hasattr(ko, "numel") else ko.size), _stream(stream), po))
    return ko


def gemm_bf16(A, B, C, status, stream=None):
    """C = bf16(A) @ bf16(B).T on the tensor cores (test hook); all device tensors, status int32[1] zeroed."""
    M, K = A.shape
    N = B.shape[0]
    _check(load().hgm_gemm_bf16(_ptr(A)[0], _ptr(B)[0], int(M), int(N), int(K), _stream(stream), _ptr(C)[0],
                                _ptr(status)[0]))
    return C


def profile_enable(on=True):
    """True/1: CUDA-event timing of the kernels; 2: accounting variant of the recursion; False/0: off."""
    _check(load().hgm_profile_enable(int(on)))


def prune_counters(reset: bool = False):
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(load().hgm_prune_counters(ctypes.byref(a), ctypes.byref(b), 1 if reset else 0))
    return int(a.value), int(b.value)


def refine_counter(reset: bool = False) -> int:
    v = ctypes.c_int64()
    _check(load().hgm_refine_counter(ctypes.byref(v), 1 if reset else 0))
    return int(v.value)


def profile_evaluated(reset: bool = False) -> int:
    v = ctypes.c_int64()
    _check(load().hgm_profile_evaluated(ctypes.byref(v), 1 if reset else 0))
    return int(v.value)


def profile_reset():
    _check(load().hgm_profile_reset())


def profile_read():
    """{kernel: (total ms, launches)} since the last reset."""
    ms = np.zeros(len(KERNELS), np.float64)
    n = np.zeros(len(KERNELS), np.int64)
    _check(load().hgm_profile_read(ms.ctypes.data_as(_pd), n.ctypes.data_as(_p64), len(KERNELS)))
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNELS)}
