"""Helpers shared by the GPU parity tests: handles from synthetic workloads and the parity rule.

Parity rule (energies and assignments of the exact path):
  |E_gpu - E*| <= 1e-5 |E*| (+1e-5 absolute when |E*| < 1), E* from the FP64 oracle;
  the GPU assignment equals the oracle's, or its FP64 energy is within
  E* (1 + 1e-5) + 1e-6 (a near-tie resolved differently in FP32).
Candidate lists (integer work) must match bit for bit.
"""
import numpy as np

REL = 1e-5


def handles(hgm, model, scene, torch=None, device=None):
    if torch is not None:
        dev = device or torch.device("cuda:0")
        m = hgm.Model(torch.from_numpy(model.xy).to(dev), torch.from_numpy(model.t).to(dev),
                      torch.from_numpy(model.f).to(dev))
        s = hgm.Scene(torch.from_numpy(scene.xy).to(dev), torch.from_numpy(scene.t).to(dev),
                      torch.from_numpy(scene.f).to(dev), scene.n_frames)
    else:
        m = hgm.Model(model.xy, model.t, model.f)
        s = hgm.Scene(scene.xy, scene.t, scene.f, scene.n_frames)
    return m, s


def energy_ok(e_gpu, e_or):
    if not np.isfinite(e_or):
        return not np.isfinite(e_gpu)
    if not np.isfinite(e_gpu):
        return False
    tol = REL * abs(e_or) + (1e-5 if abs(e_or) < 1.0 else 0.0)
    return abs(float(e_gpu) - e_or) <= tol


def check_offset(orc, o, e_gpu, a_gpu, e_or=None, z_or=None):
    """Returns (ok, tie) for one offset under the parity rule."""
    if e_or is None:
        e_or, z_or, _ = orc.match(int(o))
    if not energy_ok(e_gpu, e_or):
        return False, False, f"energy {e_gpu} vs {e_or}"
    if not np.isfinite(e_or):
        return bool(np.all(np.asarray(a_gpu) == -1)), False, "infeasible row not -1"
    a_gpu = np.asarray(a_gpu).astype(np.int64)
    if np.array_equal(a_gpu, np.asarray(z_or)):
        return True, False, ""
    e_alt = orc.energy(a_gpu)
    ok = e_alt <= e_or * (1 + REL) + 1e-6
    return ok, True, f"assignment differs, E64(gpu)={e_alt} vs E*={e_or}"
