"""Shared helpers for the GPU tests: tensor <-> numpy views and the float32
comparison rule (distances within 1e-5 relative; id sets equal except
inside the tie band at the k-th distance)."""
import numpy as np

F32_RTOL = 1e-5


def u64(t):
    """uint64 view of an int64 tensor holding uint64 bit patterns."""
    return t.detach().cpu().contiguous().numpy().view(np.uint64)


def dev(x, device="cuda"):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to(device)


def compare_f32(gids, gdist, oids, odist, rtol=F32_RTOL):
    """Returns a list of problems (empty when the float32 results agree)."""
    probs = []
    nq, k = oids.shape
    for i in range(nq):
        ov, gv = odist[i], gdist[i].astype(np.float64)
        valid_o = oids[i] >= 0
        valid_g = gids[i] >= 0
        if valid_o.sum() != valid_g.sum():
            probs.append((i, "valid count", int(valid_o.sum()), int(valid_g.sum())))
            continue
        nv = int(valid_o.sum())
        if not np.all(np.isinf(gv[nv:])):
            probs.append((i, "padding"))
        # rank-wise distances agree (both lists are sorted)
        a, b = ov[:nv], gv[:nv]
        bad = np.abs(a - b) > rtol * np.maximum(np.abs(a), 1e-30)
        if bad.any():
            probs.append((i, "dist", a[bad][:3], b[bad][:3]))
            continue
        so, sg = set(oids[i, :nv].tolist()), set(gids[i, :nv].tolist())
        if so != sg and nv:
            kth = a[nv - 1]
            band = lambda d: abs(d - kth) <= rtol * max(kth, 1e-30)
            only_o = [j for j in range(nv) if oids[i, j] not in sg]
            only_g = [j for j in range(nv) if gids[i, j] not in so]
            if not all(band(a[j]) for j in only_o) or not all(band(b[j]) for j in only_g):
                probs.append((i, "ids outside tie band"))
    return probs
