"""Oracle for the learned initialiser (Sec. 3.2 B: a regressor from the frame
to the Gaussians' parameters, trained with a Chamfer loss) -- TEST
INFRASTRUCTURE ONLY (see the package docstring).

Plain double-precision numpy: BF16 rounding written from its bit-level
definition, matrix products, convolutions as explicit sums over the 3 x 3
taps, the head's decoding of a network output into Gaussians, and the
Chamfer distance by brute force.
"""

from __future__ import annotations

import numpy as np


def bf16_round(x) -> np.ndarray:
    """Rounds float32 values to the nearest bfloat16 (ties to even), returned as
    float32: keep the upper 16 bits of the IEEE single after adding
    0x7FFF + (bit 16) to the lower half.  NaN stays NaN."""
    a = np.ascontiguousarray(np.asarray(x, np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    out = (r & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32)
    return np.where(np.isnan(a), a, out)


def bf16_bits(x) -> np.ndarray:
    """uint16 bit patterns of bf16_round(x)."""
    return (bf16_round(x).view(np.uint32) >> np.uint32(16)).astype(np.uint16)


def gemm(a, b, bias=None, relu=False) -> np.ndarray:
    """C = A B^T (+ bias, then max(., 0)) in double precision; A [M, K], B [N, K]."""
    c = np.asarray(a, np.float64) @ np.asarray(b, np.float64).T
    if bias is not None:
        c = c + np.asarray(bias, np.float64)[None, :]
    if relu:
        c = np.maximum(c, 0.0)
    return c


def gemm_abs(a, b) -> np.ndarray:
    """sum_k |A[m, k] B[n, k]|: the scale of the rounding error of C[m, n]."""
    return np.abs(np.asarray(a, np.float64)) @ np.abs(np.asarray(b, np.float64)).T


# ---------------------------------------------------------------------------
# Convolutions, NHWC, weights [Co][K] with k = (ky ks + kx) C + ci and the
# bias at k = ks^2 C.

def out_size(n: int, ks: int, stride: int, pad: int) -> int:
    return (n + 2 * pad - ks) // stride + 1


def conv(x, w, ks: int, stride: int, pad: int) -> np.ndarray:
    """Direct convolution by explicit sums over the ks x ks taps:
    out[b, oy, ox, co] = w[co, ks^2 C]
                         + sum_{ky, kx, ci} x[b, iy, ix, ci] w[co, (ky ks + kx) C + ci]
    with iy = oy stride + ky - pad (zero outside the image)."""
    x = np.asarray(x, np.float64)
    w = np.asarray(w, np.float64)
    B, H, W, C = x.shape
    Ho, Wo = out_size(H, ks, stride, pad), out_size(W, ks, stride, pad)
    co = w.shape[0]
    out = np.zeros((B, Ho, Wo, co)) + w[:, ks * ks * C][None, None, None, :]
    xp = np.zeros((B, H + 2 * pad + stride, W + 2 * pad + stride, C))
    xp[:, pad:pad + H, pad:pad + W] = x
    for ky in range(ks):
        for kx in range(ks):
            tap = xp[:, ky:ky + stride * Ho:stride, kx:kx + stride * Wo:stride, :]  # [B,Ho,Wo,C]
            wt = w[:, (ky * ks + kx) * C:(ky * ks + kx + 1) * C]                     # [co, C]
            out += np.einsum("bhwc,oc->bhwo", tap, wt)
    return out


def im2col(x, ks: int, stride: int, pad: int, ldk: int) -> np.ndarray:
    """col[p, (ky ks + kx) C + ci] = x at the tap (0 outside), 1 at ks^2 C."""
    x = np.asarray(x, np.float64)
    B, H, W, C = x.shape
    Ho, Wo = out_size(H, ks, stride, pad), out_size(W, ks, stride, pad)
    col = np.zeros((B, Ho, Wo, ldk))
    for oy in range(Ho):
        for ox in range(Wo):
            for ky in range(ks):
                for kx in range(ks):
                    iy, ix = oy * stride + ky - pad, ox * stride + kx - pad
                    if 0 <= iy < H and 0 <= ix < W:
                        k0 = (ky * ks + kx) * C
                        col[:, oy, ox, k0:k0 + C] = x[:, iy, ix, :]
    col[..., ks * ks * C] = 1.0
    return col.reshape(B * Ho * Wo, ldk)


def col2im(dcol, shape, ks: int, stride: int, pad: int) -> np.ndarray:
    """Adjoint of im2col on the image part: dx[b, iy, ix, ci] = sum of dcol over
    the (output pixel, tap) pairs that read input (iy, ix)."""
    B, H, W, C = shape
    Ho, Wo = out_size(H, ks, stride, pad), out_size(W, ks, stride, pad)
    d = np.asarray(dcol, np.float64).reshape(B, Ho, Wo, -1)
    dx = np.zeros((B, H, W, C))
    for oy in range(Ho):
        for ox in range(Wo):
            for ky in range(ks):
                for kx in range(ks):
                    iy, ix = oy * stride + ky - pad, ox * stride + kx - pad
                    if 0 <= iy < H and 0 <= ix < W:
                        k0 = (ky * ks + kx) * C
                        dx[:, iy, ix, :] += d[:, oy, ox, k0:k0 + C]
    return dx


def conv_backward(x, w, dz, ks: int, stride: int, pad: int, ldk: int):
    """Gradients of conv with respect to w ([Co][ldk], bias column included) and
    x, for the output gradient dz [B, Ho, Wo, Co]: dw = dz^T col(x),
    dx = col2im(dz w)."""
    col = im2col(x, ks, stride, pad, ldk)
    d = np.asarray(dz, np.float64).reshape(col.shape[0], -1)
    dw = d.T @ col
    wfull = np.zeros((w.shape[0], ldk))
    wfull[:, :np.asarray(w).shape[1]] = w
    dx = col2im(d @ wfull, np.asarray(x).shape, ks, stride, pad)
    return dw, dx


# ---------------------------------------------------------------------------
# Head

EXP_LO, EXP_HI = -4.0, 3.0


def head_keys(out, gh: int, gw: int, slots: int) -> np.ndarray:
    """|w| of every slot, computed in float32 like the selection on the GPU:
    fabs(0.25f + o8).  [B, gh gw slots]."""
    o = np.asarray(out, np.float32).reshape(-1, gh * gw, np.asarray(out).shape[-1])
    o8 = o[:, :, 8:9 * slots:9]                       # [B, cells, slots]
    return np.abs(np.float32(0.25) + o8).reshape(o.shape[0], -1)


def head_select(out, gh: int, gw: int, slots: int, n: int) -> np.ndarray:
    """Per frame, the n slots with the largest |w| (ties: lower slot index),
    in slot order.  [B, n] int."""
    keys = head_keys(out, gh, gw, slots)
    sel = []
    for k in keys:
        order = sorted(range(len(k)), key=lambda i: (-float(k[i]), i))[:n]
        sel.append(sorted(order))
    return np.array(sel, dtype=np.int64)


def slot_anchor(s: int, slots: int):
    """Offset of slot s inside its cell, as a fraction of the cell: slots on a
    q x r grid, q = ceil(sqrt(slots)), r = ceil(slots / q)."""
    q = 1
    while q * q < slots:
        q += 1
    r = -(-slots // q)
    return ((s % q) + 0.5) / q, ((s // q) + 0.5) / r


def head_decode(out, gh: int, gw: int, slots: int, cell_px: int, scale: float, n: int):
    """Decoded Gaussians of the selected slots, double precision: params
    [B, 9, n] and sel [B, n]."""
    o = np.asarray(out, np.float64).reshape(-1, gh * gw, np.asarray(out).shape[-1])
    sel = head_select(out, gh, gw, slots, n)
    B = o.shape[0]
    params = np.zeros((B, 9, n))
    half = 0.5 * cell_px
    for b in range(B):
        for j, slot in enumerate(sel[b]):
            cell, s = divmod(int(slot), slots)
            cy, cx = divmod(cell, gw)
            ax, ay = slot_anchor(s, slots)
            v = o[b, cell, 9 * s:9 * s + 9]
            params[b, :, j] = [
                (cx + ax) * cell_px + half * np.tanh(v[0]),
                (cy + ay) * cell_px + half * np.tanh(v[1]),
                scale * np.exp(np.clip(v[2], EXP_LO, EXP_HI)),
                scale * v[3],
                scale * np.exp(np.clip(v[4], EXP_LO, EXP_HI)),
                0.5 + v[5], 0.5 + v[6], 0.5 + v[7], 0.25 + v[8]]
    return params, sel


def head_decode_bwd(out, sel, dparams, gh: int, gw: int, slots: int, cell_px: int,
                    scale: float) -> np.ndarray:
    """d(loss)/d(out) for d(loss)/d(params) (chain rule through head_decode)."""
    out = np.asarray(out, np.float64)
    o = out.reshape(-1, gh * gw, out.shape[-1])
    d = np.zeros_like(o)
    dp = np.asarray(dparams, np.float64)
    half = 0.5 * cell_px
    for b in range(o.shape[0]):
        for j, slot in enumerate(sel[b]):
            cell, s = divmod(int(slot), slots)
            v = o[b, cell, 9 * s:9 * s + 9]
            g = dp[b, :, j]
            inside = lambda t: EXP_LO <= t <= EXP_HI  # noqa: E731
            d[b, cell, 9 * s:9 * s + 9] = [
                g[0] * half * (1 - np.tanh(v[0]) ** 2),
                g[1] * half * (1 - np.tanh(v[1]) ** 2),
                g[2] * scale * np.exp(v[2]) if inside(v[2]) else 0.0,
                g[3] * scale,
                g[4] * scale * np.exp(v[4]) if inside(v[4]) else 0.0,
                g[5], g[6], g[7], g[8]]
    return d.reshape(out.shape)


# ---------------------------------------------------------------------------
# Chamfer distance (Sec. 3.2 B)

def chamfer(p, q):
    """Chamfer distance between point sets p [n, 2] and q [m, 2]:
    mean_i min_j |p_i - q_j|^2 + mean_j min_i |p_i - q_j|^2, and its gradient
    with respect to p (the nearest-neighbour assignment held fixed)."""
    p = np.asarray(p, np.float64)
    q = np.asarray(q, np.float64)
    d = ((p[:, None, :] - q[None, :, :]) ** 2).sum(-1)   # [n, m]
    nn1 = d.argmin(axis=1)
    nn2 = d.argmin(axis=0)
    loss = d[np.arange(len(p)), nn1].mean() + d[nn2, np.arange(len(q))].mean()
    g = 2.0 * (p - q[nn1]) / len(p)
    np.add.at(g, nn2, 2.0 * (p[nn2] - q) / len(q))
    return loss, g
