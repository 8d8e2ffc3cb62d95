"""CPU oracle of the learned part's MLP (test infrastructure only).

A plain numpy restatement, in FP64, of the network the GPU trains:
x -> tanh(W0 x + b0) -> (depth-1) x tanh(Wl h + bl) -> Wout h + bout, loss
(1/B) sum_b sum_o wt_o (out - y)^2, and its gradient by backpropagation.
With ``bf16=True`` every operand the GPU feeds to a tensor-core product is
rounded to bfloat16 (nearest even) first, at the same places: the
activations entering layers 1..depth, the weights of those layers, the loss
gradient and the pre-activation gradients entering the weight and input
gradient products. Layer 0 and all elementwise steps stay unrounded, as on
the GPU. Parameters use the flat layout of the C-ABI (W_l row-major, then b_l).
Pinned by central finite differences of its own FP64 loss (tests).
"""
from __future__ import annotations

import numpy as np


def bf16_round(a):
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint32) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(params, nin, width, depth, nout):
    p = np.asarray(params, dtype=np.float64)
    Ws, bs, off = [], [], 0
    for l in range(depth + 1):
        fan_in = nin if l == 0 else width
        rows = nout if l == depth else width
        Ws.append(p[off:off + rows * fan_in].reshape(rows, fan_in))
        off += rows * fan_in
        bs.append(p[off:off + rows])
        off += rows
    assert off == p.size
    return Ws, bs


def forward(params, x, nin, width, depth, nout, bf16=False):
    R = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    Ws, bs = unpack(params, nin, width, depth, nout)
    h = np.tanh(np.asarray(x, np.float64) @ Ws[0].T + bs[0])
    hs = [h]
    for l in range(1, depth):
        h = np.tanh(R(h) @ R(Ws[l]).T + bs[l])
        hs.append(h)
    out = R(h) @ R(Ws[depth]).T + bs[depth]
    return out, hs


def loss_and_grad(params, x, y, wt, nin, width, depth, nout, bf16=False):
    R = bf16_round if bf16 else (lambda a: np.asarray(a, dtype=np.float64))
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    B = x.shape[0]
    wt = np.ones(nout) if wt is None else np.asarray(wt, np.float64)
    Ws, bs = unpack(params, nin, width, depth, nout)
    out, hs = forward(params, x, nin, width, depth, nout, bf16)
    r = out - y
    loss = float(np.sum(wt * r * r) / B)
    dout = 2.0 * wt * r / B
    gW = [None] * (depth + 1)
    gb = [None] * (depth + 1)
    gW[depth] = R(dout).T @ R(hs[depth - 1])
    gb[depth] = dout.sum(axis=0)
    dh = R(dout) @ R(Ws[depth])
    for l in range(depth - 1, -1, -1):
        dz = dh * (1.0 - hs[l] ** 2)
        gb[l] = dz.sum(axis=0)
        if l == 0:
            gW[0] = dz.T @ x
        else:
            gW[l] = R(dz).T @ R(hs[l - 1])
            dh = R(dz) @ R(Ws[l])
    flat = np.concatenate([np.concatenate([gW[l].ravel(), gb[l]]) for l in range(depth + 1)])
    return loss, flat
