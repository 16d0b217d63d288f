"""Helpers shared by the tests: building the library on demand, moving arrays."""
import os
import re

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def ensure_built():
    from paper_2001_02765_gb300 import build
    from paper_2001_02765_gb300 import sg
    if not os.path.exists(sg.LIB_PATH):
        build.build()
    return sg.load()


def header_functions():
    """Function names declared in include/sg.h."""
    with open(os.path.join(ROOT, "include", "sg.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"^(?:const\s+)?[a-z_0-9]+\s*\*?\s*(sg_[a-z_0-9]+)\s*\(", text, flags=re.M)))


def to_dev(a, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype).ravel()).cuda()


def concat_dev(arrs, dtype):
    return to_dev(np.concatenate([np.asarray(a, dtype=np.float64).ravel() for a in arrs]), dtype)


def gather_leaves(plan, flat, leaves):
    parts = plan.split(np.asarray(flat, dtype=np.float64))
    return np.array([parts[k][j, i] for k, j, i in zip(leaves["patch"], leaves["j"], leaves["i"])])
