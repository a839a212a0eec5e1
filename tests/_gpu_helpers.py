"""Helpers shared by the GPU parity tests (run the CUDA path through the C ABI)."""
from __future__ import annotations

import numpy as np
import torch

from paper_2112_01508_gb300 import ShortRange


def rel_rms(a, ref):
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.sqrt(((a - ref) ** 2).sum() / (ref ** 2).sum()))


def gpu_forces(pos, x_s, x_r, G_m, softening="bspline", eps=0.0, precision=32, rung=None, rung_min=0,
               n_sub=2, n_rung=8, return_ctx=False, symmetric=True, box=1.0):
    """Sort + build_pairs + forces on the GPU; accelerations returned in the input order.

    Inactive receivers' rows come back as NaN (the output is pre-filled with NaN
    to check that the kernel leaves them untouched)."""
    n = pos.shape[1]
    dev = torch.device("cuda")
    p = torch.from_numpy(np.ascontiguousarray(pos)).to(dev)
    sr = ShortRange(n, x_s, x_r, G_m, softening=softening, eps=eps, n_sub=n_sub, n_rung=n_rung,
                    symmetric=symmetric, box=box)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    carry = []
    rg = None
    if rung is not None:
        rg = torch.from_numpy(np.ascontiguousarray(rung, dtype=np.int8)).to(dev)
        carry.append(rg)
    sr.sort(p, carry=carry, perm_out=perm)
    sr.build_pairs(rg, rung_min)
    dt = torch.float32 if precision == 32 else torch.float64
    out = torch.full((3, n), float("nan"), dtype=dt, device=dev)
    sr.forces(p, precision, out)
    sr.sync()
    st = sr.stats()
    perm_np = perm.cpu().numpy().astype(np.int64)
    acc = np.empty((3, n), dtype=np.float64)
    acc[:, perm_np] = out.cpu().numpy().astype(np.float64)
    res = dict(acc=acc, pairs=st.pairs_last, stats=st, perm=perm_np, pos_sorted=p.cpu().numpy())
    if return_ctx:
        res["ctx"] = sr
        res["pos_dev"] = p
    else:
        sr.close()
    return res
