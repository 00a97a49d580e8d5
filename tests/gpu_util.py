"""Helpers shared by the GPU tests (inputs and goldens; no method arithmetic)."""
import json
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
LDC = 129


def golden(name):
    return json.load(open(os.path.join(ROOT, "tests", "golden", f"{name}.json")))


def coeff_tensor(polys, device="cuda"):
    import torch
    arr = np.zeros((len(polys), LDC), dtype=np.int64)
    for i, p in enumerate(polys):
        arr[i, :len(p)] = p
    c = torch.from_numpy(arr).to(device)
    d = torch.tensor([len(p) - 1 for p in polys], dtype=torch.int32, device=device)
    return c, d


def u64_tensor(vals, device="cuda"):
    import torch
    a = np.asarray([int(v) for v in vals], dtype=np.uint64).view(np.int64)
    return torch.from_numpy(a.copy()).to(device)


def to_u64(t):
    return t.cpu().numpy().view(np.uint64)


def plans_numpy(plans_tensor):
    from paper_2410_15880_b300 import PLAN_DTYPE
    return plans_tensor.cpu().numpy().view(PLAN_DTYPE).reshape(-1)
