"""Helpers shared by the GPU tests (CUDA path on one side, oracle on the other)."""
import numpy as np


def rel_err(a, b, floor=1e-300):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if a.size == 0:
        return 0.0
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), floor)))


def gpu_sttsvc(hg, x, dtype="f64", layout=None, rank=None, **opts):
    """Build a handle for hg and run one S^3TTVc call through the C ABI; returns numpy FP64."""
    import torch

    import paper_2311_08595_gb300 as s3
    kw = dict(opts)
    if rank is not None:
        kw["rank"] = rank
    if layout == "ccss":
        kw["build_ccss"] = 1
    g = s3.s3_build_format(hg.n, hg.edge_ptr, hg.members, **kw)
    dt = torch.float32 if dtype == "f32" else torch.float64
    df = dtype == "df"   # FP64 vectors, double-float series
    xd = torch.tensor(np.asarray(x), dtype=dt, device="cuda")
    yd = torch.full_like(xd, float("nan"))
    if layout == "ccss":
        s3.s3_sttsvc_layout(g, s3.S3_LAYOUT_CCSS, xd, yd, df=df)
    else:
        s3.s3_sttsvc(g, xd, yd, df=df)
    torch.cuda.synchronize()
    out = yd.double().cpu().numpy()
    s3.s3_destroy(g)
    return out
