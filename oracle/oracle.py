"""Python front of the FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Loads ``hgm_oracle.c`` (compiled with the host C compiler by ``build()``),
sorts models and scenes stably by frame with numpy, and maps results back to
the caller's point order. Only the test-suite, the smoke check and the
benchmark's CPU-baseline / reference leg may import this module; the CUDA
library never does.

The arithmetic (energy of Eqs. 1-6/9, recursion of Eqs. 10-13, candidate
lists) lives in the C file; this module only marshals arguments and runs
independent offsets on a thread pool (ctypes releases the GIL during calls).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hgm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so with gcc (no fast-math, no contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lp = ctypes.POINTER(ctypes.c_int64)
        lib.or_ctx_create.restype = ctypes.c_void_p
        lib.or_ctx_create.argtypes = [ctypes.c_int, dp, dp, ip, dp, ctypes.c_int, dp, dp, ip, dp,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.or_ctx_destroy.argtypes = [ctypes.c_void_p]
        lib.or_ctx_set_dummy.argtypes = [ctypes.c_void_p, ctypes.c_double]
        lib.or_unary.restype = ctypes.c_double
        lib.or_unary.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
        lib.or_rank_key.restype = ctypes.c_float
        lib.or_rank_key.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int]
        lib.or_geo.restype = ctypes.c_double
        lib.or_geo.argtypes = [ctypes.c_void_p] + [ctypes.c_int] * 4
        lib.or_triple.restype = ctypes.c_double
        lib.or_triple.argtypes = [ctypes.c_void_p] + [ctypes.c_int] * 4
        lib.or_feasible.restype = ctypes.c_int
        lib.or_feasible.argtypes = [ctypes.c_void_p] + [ctypes.c_int] * 3
        lib.or_energy.restype = ctypes.c_double
        lib.or_energy.argtypes = [ctypes.c_void_p, ip]
        lib.or_candidates.restype = ctypes.c_int
        lib.or_candidates.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ip, dp]
        lib.or_match_offset.restype = ctypes.c_int
        lib.or_match_offset.argtypes = [ctypes.c_void_p, ctypes.c_int, dp, ip, lp]
        lib.or_match_offsets.restype = ctypes.c_int
        lib.or_match_offsets.argtypes = [ctypes.c_void_p, ip, ctypes.c_int, dp, ip, lp]
        lib.or_bruteforce.restype = ctypes.c_int
        lib.or_bruteforce.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64,
                                      dp, ip, lp]
        lib.or_match_block.restype = ctypes.c_int
        lib.or_match_block.argtypes = [ctypes.c_void_p, dp, ip, lp]
        lib.or_bruteforce_block.restype = ctypes.c_int
        lib.or_bruteforce_block.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int64, dp, ip, lp]
        _lib = lib
        return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _lp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


class Oracle:
    """One (model, scene) pair with its parameters, in FP64.

    model_xy (M,2), model_t (M,), model_f (M,F); scene_xy (S,2), scene_t (S,),
    scene_f (S,F); any point order (sorted stably by frame here). Results are
    returned in the caller's order: assignment[i] is the caller index of the
    scene point given to the caller's model point i, or -1.
    """

    def __init__(self, model_xy, model_t, model_f, scene_xy, scene_t, scene_f, n_frames: int,
                 K: int, window: int, lambda1: float = 0.6, lambda2: float = 0.2, lambda3: float = 5.0,
                 T: int = 10, dummy_cost: Optional[float] = None):
        self.lib = _load()
        mt = np.asarray(model_t).astype(np.int64)
        st = np.asarray(scene_t).astype(np.int64)
        self.mperm = np.argsort(mt, kind="stable")
        self.sperm = np.argsort(st, kind="stable")
        self.M, self.S = len(mt), len(st)
        self.F = int(np.asarray(model_f).shape[1])
        self.n_frames = int(n_frames)
        self.K, self.window, self.T = int(K), int(window), int(T)
        self.lambdas = (float(lambda1), float(lambda2), float(lambda3))
        mxy = np.asarray(model_xy, dtype=np.float64)[self.mperm]
        sxy = np.asarray(scene_xy, dtype=np.float64)[self.sperm]
        self._mx = np.ascontiguousarray(mxy[:, 0]); self._my = np.ascontiguousarray(mxy[:, 1])
        self._sx = np.ascontiguousarray(sxy[:, 0]); self._sy = np.ascontiguousarray(sxy[:, 1])
        self._mt = np.ascontiguousarray(mt[self.mperm].astype(np.int32))
        self._st = np.ascontiguousarray(st[self.sperm].astype(np.int32))
        self._mf = np.ascontiguousarray(np.asarray(model_f, dtype=np.float64)[self.mperm])
        self._sf = np.ascontiguousarray(np.asarray(scene_f, dtype=np.float64)[self.sperm])
        if self.S and (self._st.min() < 0 or self._st.max() >= self.n_frames):
            raise ValueError("scene frame outside [0, n_frames)")
        self.ctx = self.lib.or_ctx_create(self.M, _dp(self._mx), _dp(self._my), _ip(self._mt), _dp(self._mf),
                                          self.S, _dp(self._sx), _dp(self._sy), _ip(self._st), _dp(self._sf),
                                          self.F, self.n_frames, *self.lambdas, self.T, self.window, self.K)
        if not self.ctx:
            raise MemoryError("oracle context allocation failed")
        # the dummy assignment of Eq. 2 (reading R5): an extra candidate eps per list, cost W^d
        self.dummy_cost = dummy_cost
        if dummy_cost is not None:
            self.lib.or_ctx_set_dummy(self.ctx, float(dummy_cost))

    @classmethod
    def from_workload(cls, wl, m: int = 0, s: int = 0, **over):
        mod, sc = wl.models[m], wl.scenes[s]
        kw = dict(K=wl.K, window=wl.window, lambda1=wl.lambda1, lambda2=wl.lambda2, lambda3=wl.lambda3, T=wl.T)
        kw.update(over)
        return cls(mod.xy, mod.t, mod.f, sc.xy, sc.t, sc.f, sc.n_frames, **kw)

    def __del__(self):
        ctx = getattr(self, "ctx", None)
        if ctx:
            self.lib.or_ctx_destroy(ctx)
            self.ctx = None

    # ---- offsets ---------------------------------------------------------
    @property
    def first_offset(self) -> int:
        return -int(self._mt[0])

    @property
    def n_offsets(self) -> int:
        return max(0, self.n_frames - int(self._mt[-1] - self._mt[0]))

    def offsets(self):
        return np.arange(self.first_offset, self.first_offset + self.n_offsets, dtype=np.int64)

    # ---- per-term access (sorted indices) ---------------------------------
    EPS = -2   # the dummy assignment in assignment arrays

    def _to_sorted_z(self, z_caller):
        """Caller-order assignment -> sorted-order scene indices in chain order (eps stays -2)."""
        inv = np.empty(max(self.S, 1), np.int64)
        inv[self.sperm] = np.arange(self.S)
        z = np.asarray(z_caller, dtype=np.int64)[self.mperm]
        return np.where(z >= 0, inv[np.maximum(z, 0)], np.where(z == self.EPS, self.EPS, -1)).astype(np.int32)

    def _to_caller_z(self, z_sorted):
        z_sorted = np.asarray(z_sorted, dtype=np.int64)
        out = np.full(self.M, -1, np.int64)
        ok = z_sorted >= 0
        out[self.mperm[ok]] = self.sperm[z_sorted[ok]]
        out[self.mperm[z_sorted == self.EPS]] = self.EPS
        return out

    def energy(self, z_caller) -> float:
        """E(z) (Eq. 9) of a caller-order assignment (-2 = the dummy eps); +inf if infeasible."""
        z = np.ascontiguousarray(self._to_sorted_z(z_caller))
        if np.any(z == -1) or (self.dummy_cost is None and np.any(z < 0)):
            return float("inf")
        return float(self.lib.or_energy(self.ctx, _ip(z)))

    def candidates(self, i_sorted: int, o: int):
        """C_i(o) for the i-th model point in chain order: (caller scene indices, FP64 U)."""
        idx = np.zeros(self.K, np.int32)
        u = np.zeros(self.K, np.float64)
        n = self.lib.or_candidates(self.ctx, int(i_sorted), int(o), _ip(idx), _dp(u))
        return self.sperm[idx[:n]].astype(np.int64), u[:n].copy()

    def candidates_sorted(self, i_sorted: int, o: int):
        idx = np.zeros(self.K, np.int32)
        u = np.zeros(self.K, np.float64)
        n = self.lib.or_candidates(self.ctx, int(i_sorted), int(o), _ip(idx), _dp(u))
        return idx[:n].copy(), u[:n].copy()

    def unary(self, i_sorted: int, j_sorted: int) -> float:
        return float(self.lib.or_unary(self.ctx, int(i_sorted), int(j_sorted)))

    def rank_key(self, i_sorted: int, j_sorted: int) -> float:
        return float(self.lib.or_rank_key(self.ctx, int(i_sorted), int(j_sorted)))

    # ---- solving -----------------------------------------------------------
    def match(self, o: int):
        """(energy, caller-order assignment, feasible-triple count) at offset o (Eqs. 10-13)."""
        e = np.zeros(1, np.float64)
        z = np.zeros(self.M, np.int32)
        nt = np.zeros(1, np.int64)
        rc = self.lib.or_match_offset(self.ctx, int(o), _dp(e), _ip(z), _lp(nt))
        if rc:
            raise MemoryError("oracle allocation failed")
        return float(e[0]), self._to_caller_z(z), int(nt[0])

    def match_many(self, offsets: Optional[Sequence[int]] = None, threads: Optional[int] = None,
                   chunk: int = 4):
        """All (or the given) offsets on a thread pool. Returns (offsets, energy[n], assign[n,M], triples[n])."""
        offs = self.offsets() if offsets is None else np.asarray(offsets, dtype=np.int64)
        n = len(offs)
        energy = np.zeros(n, np.float64)
        zs = np.zeros((n, self.M), np.int32)
        nt = np.zeros(n, np.int64)
        offs32 = np.ascontiguousarray(offs.astype(np.int32))

        def run(lo):
            hi = min(n, lo + chunk)
            rc = self.lib.or_match_offsets(self.ctx, _ip(offs32[lo:hi]), hi - lo, _dp(energy[lo:hi]),
                                           _ip(zs[lo:hi]), _lp(nt[lo:hi]))
            if rc:
                raise MemoryError("oracle allocation failed")

        threads = threads or os.cpu_count() or 1
        if threads <= 1 or n <= chunk:
            for lo in range(0, n, chunk):
                run(lo)
        else:
            with ThreadPoolExecutor(max_workers=threads) as ex:
                list(ex.map(run, range(0, n, chunk)))
        assign = np.stack([self._to_caller_z(zs[k]) for k in range(n)]) if n else np.zeros((0, self.M), np.int64)
        return offs, energy, assign, nt

    def bruteforce(self, o: int, tol: float = 1e-9, max_assignments: int = 2_000_000):
        """(min energy, caller-order first minimiser, number of near-ties) by enumeration."""
        e = np.zeros(1, np.float64)
        z = np.zeros(self.M, np.int32)
        nt = np.zeros(1, np.int64)
        rc = self.lib.or_bruteforce(self.ctx, int(o), float(tol), int(max_assignments), _dp(e), _ip(z), _lp(nt))
        if rc:
            raise ValueError("too many assignments for brute force")
        return float(e[0]), self._to_caller_z(z), int(nt[0])


    # ---- the whole-block problem (Sec. 2.2 and Sec. 3: every scene node a candidate, no offsets) ----------
    def match_block(self):
        """(energy, caller-order assignment, feasible-triple count) of the whole-block problem: z_i ranges over
        all S scene points, restricted only by causality, temporal closeness and distinctness (Eqs. 7-8)."""
        e = np.zeros(1, np.float64)
        z = np.zeros(self.M, np.int32)
        nt = np.zeros(1, np.int64)
        if self.lib.or_match_block(self.ctx, _dp(e), _ip(z), _lp(nt)):
            raise MemoryError("oracle allocation failed")
        return float(e[0]), self._to_caller_z(z), int(nt[0])

    def bruteforce_block(self, tol: float = 1e-9, max_assignments: int = 2_000_000):
        """(min energy, caller-order first minimiser, near-ties) of the whole-block problem by enumeration."""
        e = np.zeros(1, np.float64)
        z = np.zeros(self.M, np.int32)
        nt = np.zeros(1, np.int64)
        rc = self.lib.or_bruteforce_block(self.ctx, float(tol), int(max_assignments), _dp(e), _ip(z), _lp(nt))
        if rc:
            raise ValueError("too many assignments for brute force")
        return float(e[0]), self._to_caller_z(z), int(nt[0])


class ChainOracle:
    """The "independent chains" variant (Sec. 4, multiple points per frame, method 2), FP64: the model's
    points are grouped by frame; within a frame they are ranked by their index in the caller's arrays, and
    chain k is the sequence of rank-k points in frame order. Every chain with at least 3 points is an
    ordinary model for Oracle; the distance at offset o is the mean of the chains' optimal energies
    (+inf if any chain is infeasible at o), and each model point takes its chain's optimal scene point
    (-1 for points of chains shorter than 3)."""

    def __init__(self, model_xy, model_t, model_f, scene_xy, scene_t, scene_f, n_frames: int, n_chains: int,
                 **kw):
        mt = np.asarray(model_t).astype(np.int64)
        self.M = len(mt)
        rank = np.zeros(self.M, np.int64)
        for fr in np.unique(mt):
            idx = np.nonzero(mt == fr)[0]            # caller indices of the frame, ascending
            rank[idx] = np.arange(len(idx))
        self.members = []
        for k in range(int(n_chains)):
            idx = np.nonzero(rank == k)[0]
            idx = idx[np.argsort(mt[idx], kind="stable")]
            if len(idx) >= 3:
                self.members.append(idx)
        if not self.members:
            raise ValueError("no chain has 3 points")
        mxy = np.asarray(model_xy)
        mf = np.asarray(model_f)
        self.chains = [Oracle(mxy[idx], mt[idx], mf[idx], scene_xy, scene_t, scene_f, n_frames, **kw)
                       for idx in self.members]
        self.first_offset = -int(mt.min())
        self.n_offsets = max(0, int(n_frames) - int(mt.max() - mt.min()))

    def match(self, o: int):
        """(mean energy, caller-order assignment of all model points) at offset o."""
        energies, z = [], np.full(self.M, -1, np.int32)
        for idx, orc in zip(self.members, self.chains):
            e, zc, _ = orc.match(o)
            energies.append(e)
            z[idx] = zc
        e = float(np.mean(energies)) if all(np.isfinite(energies)) else float("inf")
        return e, z
