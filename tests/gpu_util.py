"""Helpers for the GPU tests: device tensors and brute-force tree checks."""
import numpy as np

import paper_1711_02976_gb300 as rp


def cuda_tensor(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to("cuda")


def matvec(pos, f, a, s, digits, leaf_cap=0, precision=0, parts=3, order_p=0, direct_w=0, direct_x=0, flags=0,
           quad=0):
    """Build a tree on the GPU and apply it once; returns (u (N,3) numpy, tree)."""
    import torch
    P, F = cuda_tensor(pos), cuda_tensor(f)
    U = torch.empty_like(F)
    if order_p or direct_w or direct_x or flags or quad:
        t = rp.rpy_forest_build(P, [0, len(pos)], [a], digits, leaf_cap=leaf_cap, precision=precision,
                                order_p=order_p, direct_w=direct_w, direct_x=direct_x, flags=flags, quad=quad)
    else:
        t = rp.rpy_tree_build(P, len(pos), a, digits, leaf_cap=leaf_cap, precision=precision)
    rp.rpy_matvec_parts(t, F, s, U, parts)
    rp.rpy_tree_sync(t)
    return U.cpu().numpy(), t


def leaf_members(t):
    """For every leaf: its caller-order bead indices."""
    perm = rp.rpy_tree_export(t, "perm")
    rng = rp.rpy_tree_export(t, "box_range")
    leaves = rp.rpy_tree_export(t, "leaves")
    return {int(b): perm[rng[b, 0]:rng[b, 1]] for b in leaves}


def box_members(t):
    perm = rp.rpy_tree_export(t, "perm")
    rng = rp.rpy_tree_export(t, "box_range")
    return [perm[r0:r1] for r0, r1 in rng]


def csr(t, off, idx):
    o = rp.rpy_tree_export(t, off)
    i = rp.rpy_tree_export(t, idx)
    return [i[o[k]:o[k + 1]] for k in range(len(o) - 1)]
