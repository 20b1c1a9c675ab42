"""Energy error of the GPU forms against the FP64 oracle on a dumped sample of units (not a pytest module).

`bench.py --fp64-dump sample.npz` writes, for a seeded fraction of the batch's units (1% by default), the
energies of the plain exact FP32 path and of the BF16-distance + FP32 re-score path. This script rebuilds
the same seeded workload, solves every sampled unit with the FP64 oracle on the host cores (each on the
scene frames its windows reach, the same candidate lists and energies as the whole scene), and prints the
relative energy error of both forms.

  python tests/fp64_sample_report.py sample.npz [threads]
"""
import json
import os
import sys
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def main(path, threads):
    import bench
    d = np.load(path)
    wl, _ = bench.workload(str(d["workload"]), 0, int(d["hop"]))
    units = [tuple(int(x) for x in u) for u in d["units"]]
    with ThreadPoolExecutor(max_workers=threads) as ex:
        e64 = np.array([r[0] for r in ex.map(lambda u: bench._solve_unit(wl, *u), units)])
    out = {"workload": wl.name, "units": len(units)}
    fin = np.isfinite(e64)
    for name in ("e_exact", "e_bf16"):
        eg = d[name].astype(np.float64)
        mism = int(np.sum(np.isfinite(eg) != fin))
        ok = fin & np.isfinite(eg)
        rel = (eg[ok] - e64[ok]) / np.abs(e64[ok])
        out[name] = {"finite": int(ok.sum()), "feasibility_mismatch": mism,
                     "max_abs_rel_err": float(np.abs(rel).max()) if rel.size else None,
                     "mean_abs_rel_err": float(np.abs(rel).mean()) if rel.size else None,
                     "mean_rel_err": float(rel.mean()) if rel.size else None,
                     "within_1e-5": float(np.mean(np.abs(rel) <= 1e-5)) if rel.size else None}
    print(json.dumps(out))


if __name__ == "__main__":
    main(sys.argv[1], int(sys.argv[2]) if len(sys.argv) > 2 else (os.cpu_count() or 1))
