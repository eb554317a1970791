"""FP64 CPU oracle of the learned preconditioner's network (test infrastructure).

Only tests may import this.  It restates the network defined for the flexible
GMRES preconditioner (not part of the paper) step by step in float64, with the
weights rounded to bf16 exactly as the forward uses them; gradients come from
torch autograd (CPU, float64), a library primitive, and are pinned by central
finite differences in the tests.

    f_i   = [Re r_i / s, Im r_i / s, x^_i, y^_i, z^_i, n_i (3), k h],  s = rms(r)
    h0    = relu(W_in^T f + b_in)
    m_l   = mean of h_l over the mesh neighbours of i
    h_l+1 = h_l + relu(Ws_l^T h_l + Wn_l^T m_l + b_l)
    y     = W_out^T h_L + b_out,  z_i = (y_i0 + i y_i1) s / h^3
with x^ the coordinates centred at the vertex mean and divided by the largest
distance from it, n_i the normalised sum of the cross products (B-A)x(C-A) of
the triangles at i, and h the mean length of the triangle edges (each triangle
contributes its three edges).
"""
from __future__ import annotations

import numpy as np
import torch

NIN = 9


def layout(hidden: int = 64, layers: int = 4):
    """Offsets of W_in, b_in, per-layer (Ws, Wn, b), W_out, b_out in the flat vector."""
    H = hidden
    off = {"W_in": (0, (NIN, H))}
    pos = NIN * H
    off["b_in"] = (pos, (H,))
    pos += H
    for l in range(layers):
        off[f"Ws{l}"] = (pos, (H, H))
        pos += H * H
        off[f"Wn{l}"] = (pos, (H, H))
        pos += H * H
        off[f"b{l}"] = (pos, (H,))
        pos += H
    off["W_out"] = (pos, (H, 2))
    pos += 2 * H
    off["b_out"] = (pos, (2,))
    pos += 2
    return off, pos


def bf16_round(x):
    """float32 -> nearest bf16 (ties to even), returned as float64."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def graph(vtx, tri):
    """Neighbour lists over mesh edges, per-vertex features (6), mean edge length."""
    vtx = np.asarray(vtx, dtype=np.float64)
    tri = np.asarray(tri, dtype=np.int64)
    nv = vtx.shape[0]
    nb = [set() for _ in range(nv)]
    nrm = np.zeros((nv, 3))
    edges = []
    for t in tri:
        a, b, c = vtx[t[0]], vtx[t[1]], vtx[t[2]]
        n = np.cross(b - a, c - a)
        for q in range(3):
            nrm[t[q]] += n
            p, r = t[q], t[(q + 1) % 3]
            nb[p].add(r)
            nb[r].add(p)
            edges.append(np.linalg.norm(vtx[p] - vtx[r]))
    cen = vtx.mean(axis=0)
    rad = np.max(np.linalg.norm(vtx - cen, axis=1))
    feat = np.zeros((nv, 6))
    feat[:, :3] = (vtx - cen) / rad
    feat[:, 3:] = nrm / np.linalg.norm(nrm, axis=1, keepdims=True)
    return [sorted(s) for s in nb], feat, float(np.mean(edges))


def _forward_torch(params, nbrs, feat, h, k, R, hidden, layers):
    off, _ = layout(hidden, layers)

    def W(name):
        o, shape = off[name]
        return params[o:o + int(np.prod(shape))].reshape(shape)

    nv, B = R.shape
    s = torch.sqrt((R.real ** 2 + R.imag ** 2).sum(dim=0) / nv)          # rms per column
    inv = torch.where(s > 0, 1.0 / s, torch.zeros_like(s))
    geo = torch.as_tensor(feat)
    out = []
    for b in range(B):
        f = torch.cat([(R.real[:, b] * inv[b])[:, None], (R.imag[:, b] * inv[b])[:, None], geo,
                       torch.full((nv, 1), k * h, dtype=torch.float64)], dim=1)
        hcur = torch.relu(f @ W("W_in") + W("b_in"))
        for l in range(layers):
            m = torch.stack([hcur[nbrs[i]].mean(dim=0) if len(nbrs[i]) else torch.zeros(hidden, dtype=torch.float64)
                             for i in range(nv)])
            hcur = hcur + torch.relu(hcur @ W(f"Ws{l}") + m @ W(f"Wn{l}") + W(f"b{l}"))
        y = hcur @ W("W_out") + W("b_out")
        out.append((y[:, 0] + 1j * y[:, 1]) * s[b] / h ** 3)
    return torch.stack(out, dim=1)


def forward(params, vtx, tri, k, R, hidden=64, layers=4):
    """z = M(R) for R (nv, B) complex; params: flat float32 vector (rounded to bf16 here)."""
    nbrs, feat, h = graph(vtx, tri)
    p = torch.as_tensor(bf16_round(params))
    Rt = torch.as_tensor(np.asarray(R, dtype=np.complex128).reshape(len(nbrs), -1))
    with torch.no_grad():
        return _forward_torch(p, nbrs, feat, h, float(k), Rt, hidden, layers).numpy()


def loss_and_grad(params, vtx, tri, k, R, E, hidden=64, layers=4):
    """mean_b |z_b - e_b|^2 / |e_b|^2 and its gradient with respect to the
    (bf16-rounded) weights used in the forward."""
    nbrs, feat, h = graph(vtx, tri)
    p = torch.tensor(bf16_round(params), requires_grad=True)
    Rt = torch.as_tensor(np.asarray(R, dtype=np.complex128).reshape(len(nbrs), -1))
    Et = torch.as_tensor(np.asarray(E, dtype=np.complex128).reshape(len(nbrs), -1))
    Z = _forward_torch(p, nbrs, feat, h, float(k), Rt, hidden, layers)
    d = Z - Et
    per = (d.real ** 2 + d.imag ** 2).sum(dim=0) / (Et.real ** 2 + Et.imag ** 2).sum(dim=0)
    loss = per.mean()
    loss.backward()
    return float(loss.detach()), p.grad.numpy().copy()


def adam_step(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba), bias-corrected; returns (p, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def loss_from_rounded(w64, vtx, tri, k, R, E, hidden=64, layers=4):
    """The loss as a function of float64 weights used as given (no rounding): for
    finite-difference checks of the gradient."""
    nbrs, feat, h = graph(vtx, tri)
    p = torch.as_tensor(np.asarray(w64, dtype=np.float64))
    Rt = torch.as_tensor(np.asarray(R, dtype=np.complex128).reshape(len(nbrs), -1))
    Et = torch.as_tensor(np.asarray(E, dtype=np.complex128).reshape(len(nbrs), -1))
    with torch.no_grad():
        Z = _forward_torch(p, nbrs, feat, h, float(k), Rt, hidden, layers)
        d = Z - Et
        per = (d.real ** 2 + d.imag ** 2).sum(dim=0) / (Et.real ** 2 + Et.imag ** 2).sum(dim=0)
        return float(per.mean())
