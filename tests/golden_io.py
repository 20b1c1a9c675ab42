"""Reader for the small text fixtures under tests/golden/."""
import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_examples(name="hand_examples.txt"):
    """Returns {example: dict(model_xy, model_t, model_f, scene_xy, scene_t, scene_f, energy)}."""
    out, cur = {}, None
    with open(os.path.join(GOLDEN, name)) as fh:
        for raw in fh:
            line = raw.split("#", 1)[0].strip()
            if not line:
                continue
            if line.startswith("["):
                cur = {"model": [], "scene": []}
                out[line.strip("[]")] = cur
                continue
            key, rest = line.split(None, 1)
            if key in ("model", "scene"):
                cur[key].append([float(v) for v in rest.split()])
            elif key == "energy":
                cur["energy"] = float(eval(rest, {"__builtins__": {}}, {k: getattr(math, k) for k in
                                                                       ("atan", "sqrt", "pi")}))
    res = {}
    for k, v in out.items():
        m = np.array(v["model"], dtype=np.float64)
        s = np.array(v["scene"], dtype=np.float64)
        res[k] = dict(model_xy=m[:, :2], model_t=m[:, 2].astype(np.int32), model_f=m[:, 3:],
                      scene_xy=s[:, :2], scene_t=s[:, 2].astype(np.int32), scene_f=s[:, 3:],
                      energy=v["energy"])
    return res
