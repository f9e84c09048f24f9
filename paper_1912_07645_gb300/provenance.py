"""Result provenance (Sec. 2.3: every output carries the code revision, the library versions, the
parameters and the initial data). ``provenance(desc)`` returns that record; ``save_result`` writes
arrays to ``<path>.npz`` with the record beside them in ``<path>.json``."""
from __future__ import annotations

import json
import os
import platform
import subprocess

from . import _abi as A

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _git_rev():
    try:
        r = subprocess.run(["git", "-C", _ROOT, "rev-parse", "HEAD"], capture_output=True, text=True, timeout=10)
        rev = r.stdout.strip() if r.returncode == 0 else None
        d = subprocess.run(["git", "-C", _ROOT, "status", "--porcelain", "--untracked-files=no"], capture_output=True,
                           text=True, timeout=10)
        return rev, bool(d.stdout.strip()) if d.returncode == 0 else None
    except Exception:
        return None, None


def desc_dict(desc: A.alsv_grid_desc) -> dict:
    out = {}
    for name, _ in desc._fields_:
        v = getattr(desc, name)
        try:
            v = [list(x) if hasattr(x, "__len__") else x for x in v]
        except TypeError:
            pass
        out[name] = v
    return out


def provenance(desc: A.alsv_grid_desc | None = None, initial_data: str | None = None, **extra) -> dict:
    rev, dirty = _git_rev()
    rec = {"library": A.alsv_version(), "git_rev": rev, "git_dirty": dirty, "python": platform.python_version(),
           "machine": platform.machine()}
    try:
        import torch
        rec["torch"] = torch.__version__
        rec["cuda_runtime"] = torch.version.cuda
        if torch.cuda.is_available():
            rec["device"] = torch.cuda.get_device_name(0)
            rec["device_capability"] = list(torch.cuda.get_device_capability(0))
    except Exception:
        pass
    if desc is not None:
        rec["descriptor"] = desc_dict(desc)
    if initial_data is not None:
        rec["initial_data"] = initial_data
    rec.update(extra)
    return rec


def save_result(path: str, arrays: dict, desc: A.alsv_grid_desc | None = None, **extra) -> str:
    import numpy as np
    np.savez(path + ".npz", **{k: np.asarray(v) for k, v in arrays.items()})
    with open(path + ".json", "w") as f:
        json.dump(provenance(desc, **extra), f, indent=1, default=str)
    return path + ".json"
