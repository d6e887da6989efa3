"""GPU-side helpers for the parity tests (call the CUDA path through the C ABI)."""
from __future__ import annotations

import numpy as np

from paper_2608_21826_gb300 import bfq


def create(g, tune=None, on_device=False):
    import torch
    if on_device:
        t = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (g.row_ptr, g.col, g.w)]
        return bfq.bfq_graph_create(t[0], t[1], t[2], tune)
    return bfq.bfq_graph_create(g.row_ptr, g.col, g.w, tune)


def run(handle, V, src, want_pred=False, want_hops=True):
    """One synchronous query; returns (status, dist, hops, pred) as numpy."""
    import torch
    dist = torch.full((V,), -7, dtype=torch.int32, device="cuda")
    hops = torch.full((V,), -7, dtype=torch.int32, device="cuda") if want_hops else None
    pred = torch.full((V,), -7, dtype=torch.int32, device="cuda") if want_pred else None
    st = bfq.bfq_sssp(handle, int(src), dist, hops, pred)
    out = [st, dist.cpu().numpy()]
    out.append(hops.cpu().numpy() if hops is not None else None)
    out.append(pred.cpu().numpy() if pred is not None else None)
    return tuple(out)


def sssp(g, src, tune=None, want_pred=False, on_device=False):
    h = create(g, tune, on_device)
    try:
        return run(h, g.V, src, want_pred)
    finally:
        bfq.bfq_graph_destroy(h)
