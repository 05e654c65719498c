"""Shared helpers of the GPU parity tests (comparison utilities only)."""
import numpy as np


def half_offsets(rs):
    """Half-window offsets in the plane order of the library's weight storage:
    (0, 1..rs), then rows 1..rs with ox = -rs..rs."""
    out = [(0, ox) for ox in range(1, rs + 1)]
    for oy in range(1, rs + 1):
        out += [(oy, ox) for ox in range(-rs, rs + 1)]
    return out


def planes_from_matrix(K1, H, W, rs):
    """Oracle K1 (CSR) rearranged as the [n_h][H][W] planes K1(s, s + o)."""
    K1 = K1.tocsr()
    offs = half_offsets(rs)
    out = np.zeros((len(offs), H, W))
    idx = np.arange(H * W).reshape(H, W)
    for k, (oy, ox) in enumerate(offs):
        i0, i1 = 0, H - oy
        j0, j1 = max(0, -ox), min(W, W - ox)
        if i1 <= i0 or j1 <= j0:
            continue
        s = idx[i0:i1, j0:j1].ravel()
        r = idx[i0 + oy:i1 + oy, j0 + ox:j1 + ox].ravel()
        out[k, i0:i1, j0:j1] = np.asarray(K1[s, r]).reshape(i1 - i0, j1 - j0)
    return out


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def cuda(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def host(t):
    return t.detach().float().cpu().numpy().astype(np.float64) if t.dtype.is_floating_point \
        else t.detach().cpu().numpy()
