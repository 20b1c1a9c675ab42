"""Training and evaluation of the candidate-proposal network (learned pruning layered on the exact method).

Labels come from the exact recursion itself: on separately seeded batched workloads, every (offset,
model point) candidate list is labelled 1 for the candidate the exact optimum assigns and 0 for the
others. The network is trained by libhgm's own kernels (hgm_prop_train_step: BF16 tensor-core forward
and backward, FP32 Adam). torch only gathers the training rows (device memory plumbing).

Evaluation compares the pruned form with the exact path on the same units: point recall (fraction of
model points whose exact-optimal scene point the pruned optimum also picks), unit match rate, and the
mean relative energy gap (E_pruned - E_exact) / E_exact over feasible units.
"""
from __future__ import annotations

import json
import os
import time
from typing import Dict, Optional

import numpy as np

from . import hgm, synth


def _handles(torch, dev, wl):
    models = [hgm.Model(*(torch.from_numpy(a).to(dev) for a in (m.xy, m.t, m.f))) for m in wl.models]
    scenes = [hgm.Scene(*(torch.from_numpy(a).to(dev) for a in (s.xy, s.t, s.f)), s.n_frames) for s in wl.scenes]
    return models, scenes


def training_pairs(torch, wl, n_pairs: int = 1 << 20, seed: int = 0, device=None) -> Dict:
    """(X [N x (2F+3)], y [N]) device tensors from exact optima on workload wl; about n_pairs rows
    (whole candidate lists, so every list keeps its single positive)."""
    dev = device or torch.device("cuda")
    rng = np.random.default_rng(seed)
    models, scenes = _handles(torch, dev, wl)
    p = hgm.default_params(K=wl.K, window=wl.window, T=wl.T)
    first, es, as_ = hgm.batch_layout(models, scenes, p)
    assign = torch.empty(int(as_[-1]), dtype=torch.int32, device=dev)
    energy = torch.empty(int(es[-1]), dtype=torch.float32, device=dev)
    hgm.match_batch(models, scenes, p, energy, assign)
    torch.cuda.synchronize()
    n_lists_want = max(1, n_pairs // wl.K)
    pairs = [(mi, si) for mi in range(len(models)) for si in range(len(scenes))]
    lists_per_pair = int(np.ceil(n_lists_want / len(pairs)))
    Xs, ys = [], []
    for mi, si in pairs:
        mod, sc = wl.models[mi], wl.scenes[si]
        q = mi * len(scenes) + si
        n = int(es[q + 1] - es[q])
        if n == 0:
            continue
        M = mod.n
        # sample lists (offset k, sorted model point i), keep those whose exact optimum is feasible
        ks = rng.integers(0, n, size=lists_per_pair)
        idx = torch.empty((n, M, wl.K), dtype=torch.int32, device=dev)
        cnt = torch.empty((n, M), dtype=torch.int32, device=dev)
        hgm.candidates(models[mi], scenes[si], p, int(first[q]), n, idx, cnt)
        mperm = torch.from_numpy(models[mi].order().astype(np.int64)).to(dev)
        sperm = torch.from_numpy(scenes[si].order().astype(np.int64)).to(dev)
        a = assign[int(as_[q]):int(as_[q + 1])].view(n, M).long()
        e = energy[int(es[q]):int(es[q + 1])]
        ks_t = torch.from_numpy(ks).to(dev)
        ok = torch.isfinite(e[ks_t])
        ks_t = ks_t[ok]
        if ks_t.numel() == 0:
            continue
        i_t = torch.from_numpy(rng.integers(0, M, size=ks_t.numel())).to(dev)
        cand = idx[ks_t, i_t].long()                          # [L, K] sorted scene indices, -1 pad
        valid = cand >= 0
        j_caller = sperm[cand.clamp(min=0)]                   # caller scene index of each candidate
        i_caller = mperm[i_t]                                 # caller model index
        target = a[ks_t, i_caller]                            # exact optimum's caller scene index
        y = ((j_caller == target[:, None]) & valid).float()
        mf = torch.from_numpy(mod.f).to(dev)
        sf = torch.from_numpy(sc.f).to(dev)
        mxy = torch.from_numpy(mod.xy).to(dev)
        sxy = torch.from_numpy(sc.xy).to(dev)
        mt = torch.from_numpy(mod.t).to(dev).float()
        st = torch.from_numpy(sc.t).to(dev).float()
        o = (ks_t + int(first[q])).float()
        L, K = cand.shape
        ic = i_caller[:, None].expand(L, K)
        d = torch.stack([(sxy[j_caller, 0] - mxy[ic, 0]) / 100.0, (sxy[j_caller, 1] - mxy[ic, 1]) / 100.0,
                         (st[j_caller] - (mt[ic] + o[:, None])) / float(max(wl.window, 1))], dim=-1)
        X = torch.cat([mf[ic], sf[j_caller], d], dim=-1)
        Xs.append(X[valid])
        ys.append(y[valid])
    for h in models + scenes:
        h.close()
    X = torch.cat(Xs).contiguous()
    y = torch.cat(ys).contiguous()
    return {"X": X, "y": y, "lists": int(y.sum().item())}


def train(torch, data: Dict, F: int, steps: int = 2000, batch: int = 4096, lr: float = 1e-3, seed: int = 0,
          prop: Optional["hgm.Proposal"] = None, log_every: int = 0):
    """Trains (or continues training) a Proposal on data; returns (prop, loss history)."""
    gen = torch.Generator(device=data["X"].device).manual_seed(seed)
    prop = prop or hgm.Proposal(F, seed=seed)
    N = data["X"].shape[0]
    loss = torch.zeros(1, device=data["X"].device)
    hist = []
    for step in range(steps):
        sel = torch.randint(0, N, (batch,), generator=gen, device=data["X"].device)
        Xb = data["X"].index_select(0, sel).contiguous()
        yb = data["y"].index_select(0, sel).contiguous()
        prop.train_step(Xb, yb, lr, loss)
        if log_every and (step % log_every == 0 or step == steps - 1):
            hist.append((step, float(loss.item())))
    torch.cuda.synchronize()
    return prop, hist


def save_checkpoint(path: str, prop: "hgm.Proposal", meta: Optional[Dict] = None):
    """Flat FP32 weights (<path>.bin, ABI order) plus a JSON header (<path>.json)."""
    w, step = prop.get()
    w.astype(np.float32).tofile(path + ".bin")
    head = {"F": prop.F, "d_in": prop.d_in, "hidden": 128, "step": step, "count": int(w.size)}
    head.update(meta or {})
    with open(path + ".json", "w") as fh:
        json.dump(head, fh, indent=1)


def load_checkpoint(path: str) -> "hgm.Proposal":
    head = json.load(open(path + ".json"))
    w = np.fromfile(path + ".bin", dtype=np.float32)
    if w.size != head["count"]:
        raise ValueError("checkpoint size mismatch")
    prop = hgm.Proposal(int(head["F"]), weights=w)
    prop.set(w, int(head["step"]))
    return prop


def _stats(e_ref, a_ref, e, a, M_rows, sel=None):
    pts = hits = units = match = 0
    for q, (start, n, M) in enumerate(M_rows):
        A = a[start:start + n * M].reshape(n, M)
        R = a_ref[start:start + n * M].reshape(n, M)
        ok = R[:, 0] >= 0
        if sel is not None:
            ok = ok & sel[q]
        pts += int(ok.sum()) * M
        hits += int((A[ok] == R[ok]).sum())
        units += int(ok.sum())
        match += int(np.all(A[ok] == R[ok], axis=1).sum())
    return hits / max(pts, 1), match / max(units, 1), units


def pair_stats(e_ref, a_ref, e, a, M_rows, e_rows):
    """Quality at the level recognition uses: per (model, scene) pair the matching distance is the
    minimum energy over offsets. Over the pairs with a finite exact minimum: how often the pruned
    minimum sits at the same offset, the point recall of the pruned assignment at the exact best offset,
    and the mean relative gap of the pruned minimum."""
    n = same = pts = hits = 0
    gaps = []
    for q, (start, nu, M) in enumerate(M_rows):
        es = e_rows[q]
        er, ep = e_ref[es:es + nu], e[es:es + nu]
        if nu == 0 or not np.isfinite(er).any():
            continue
        k = int(np.argmin(er))
        n += 1
        same += int(np.isfinite(ep).any() and int(np.argmin(ep)) == k)
        R = a_ref[start + k * M:start + (k + 1) * M]
        A = a[start + k * M:start + (k + 1) * M]
        pts += M
        hits += int((A == R).sum())
        gaps.append((float(np.min(ep)) - float(er[k])) / max(float(er[k]), 1e-12))
    return {"pairs": n, "best_offset_match": same / max(n, 1), "point_recall_at_best": hits / max(pts, 1),
            "mean_rel_gap": float(np.mean(gaps)) if gaps else 0.0}


def compare(e_ref, a_ref, e, a, M_rows, e_rows=None, implant_mask=None):
    """Recall / unit match / energy gap of (e, a) against the exact (e_ref, a_ref).
    a, a_ref: flat assignment arrays; M_rows: (assign start, n_units, M) per (model, scene) pair;
    e_rows: energy start per pair; implant_mask: per pair a boolean array marking the offsets whose
    windows can see an implanted copy of that model (reported separately from pure clutter)."""
    rec, um, n_units = _stats(e_ref, a_ref, e, a, M_rows)
    fin = np.isfinite(e_ref) & np.isfinite(e)
    gaps = (e[fin] - e_ref[fin]) / np.maximum(e_ref[fin], 1e-12)
    out = {"point_recall": rec, "unit_match": um,
           "mean_rel_gap": float(np.mean(gaps)) if gaps.size else 0.0,
           "mean_abs_rel_gap": float(np.mean(np.abs(gaps))) if gaps.size else 0.0,
           "feasible_mismatch": int(np.sum(np.isfinite(e_ref) != np.isfinite(e)))}
    if e_rows is not None:
        out["pairs"] = pair_stats(e_ref, a_ref, e, a, M_rows, e_rows)
    if implant_mask is not None and e_rows is not None:
        for name, pick in (("implant", implant_mask), ("clutter", [~m for m in implant_mask])):
            r, u, nu = _stats(e_ref, a_ref, e, a, M_rows, pick)
            g = []
            for q, (start, n, M) in enumerate(M_rows):
                es = e_rows[q]
                er, ep = e_ref[es:es + n], e[es:es + n]
                ok = pick[q] & np.isfinite(er) & np.isfinite(ep)
                g.append((ep[ok] - er[ok]) / np.maximum(er[ok], 1e-12))
            g = np.concatenate(g) if g else np.zeros(0)
            out[name] = {"units": nu, "point_recall": r, "unit_match": u,
                         "mean_rel_gap": float(np.mean(g)) if g.size else 0.0}
    return out


def implant_masks(wl, first, es):
    """Per (model, scene) pair: offsets within +-w of an implant of that model in that scene."""
    masks = []
    for mi in range(len(wl.models)):
        for si, sc in enumerate(wl.scenes):
            q = mi * len(wl.scenes) + si
            n = int(es[q + 1] - es[q])
            offs = int(first[q]) + np.arange(n)
            m = np.zeros(n, bool)
            for imp in sc.implants:
                if imp.model == mi:
                    m |= np.abs(offs - imp.offset) <= wl.window
            masks.append(m)
    return masks


def train_default(torch, wl, steps: int = 2000, batch: int = 4096, n_pairs: int = 1 << 20, seed: int = 101,
                  lr: float = 1e-3, train_wl=None):
    """Trains on the workload's own models matched against separately seeded scenes: train_wl if given,
    else 3 scenes shaped like the batched workload's (synth.training_scenes)."""
    t0 = time.time()
    F = wl.models[0].F
    wl = train_wl if train_wl is not None else synth.training_scenes(wl, seed)
    data = training_pairs(torch, wl, n_pairs=n_pairs, seed=seed)
    t1 = time.time()
    prop, hist = train(torch, data, F, steps=steps, batch=batch, lr=lr, seed=seed, log_every=max(1, steps // 10))
    t2 = time.time()
    info = {"pairs": int(data["X"].shape[0]), "positives": data["lists"], "steps": steps, "batch": batch, "lr": lr,
            "seed": seed, "loss": hist, "data_s": t1 - t0, "train_s": t2 - t1}
    del data
    return prop, info
