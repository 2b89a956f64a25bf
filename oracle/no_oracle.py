"""FP64 CPU oracle of the neural operator used for warm starts -- TEST INFRASTRUCTURE ONLY.

A plain PyTorch CPU (float64) restatement of the 3D Fourier neural operator whose parameter
layout and definition are documented with lbm_no_create in include/cmlbm.h:
  h0 = P a + p;  h_{l+1} = act(K_l h_l + W_l h_l + b_l) (GELU, identity on the last layer);
  out = Q h_L + q,
K_l: rfftn over (z, y, x) without scaling, kept modes kz, ky in {0..m-1, D-m..D-1} and kx in
{0..m-1}, a complex W x W matrix per mode, irfftn (1/D^3) of the kept modes.  Gradients come from
torch autograd on this definition.  Only tests/ use it; it shares no code with the CUDA path.
"""
from __future__ import annotations

import numpy as np
import torch


def layout(D, W, m, L, Ci, Co):
    """Offsets and shapes of the flat parameter vector."""
    shapes = [("P", (W, Ci)), ("p", (W,))]
    for l in range(L):
        shapes += [(f"Wm{l}", (m, 2 * m, 2 * m, W, W, 2)), (f"Wc{l}", (W, W)), (f"b{l}", (W,))]
    shapes += [("Q", (Co, W)), ("q", (Co,))]
    out, off = {}, 0
    for name, shp in shapes:
        n = int(np.prod(shp))
        out[name] = (off, shp)
        off += n
    return out, off


def kept(D, m):
    return list(range(m)) + list(range(D - m, D))


def unpack(theta, D, W, m, L, Ci, Co):
    lay, n = layout(D, W, m, L, Ci, Co)
    assert theta.numel() == n
    return {k: theta[o:o + int(np.prod(s))].reshape(s) for k, (o, s) in lay.items()}


def spectral_modes(h, D, m):
    """Kept Fourier coefficients of h [B, C, D, D, D] (z, y, x): rfftn without scaling, kz, ky in
    kept(D, m), kx < m; returns [B, C, 2m(kz), 2m(ky), m(kx)] complex."""
    X = torch.fft.rfftn(h, dim=(2, 3, 4))                      # [B, C, kz, ky, kx]
    idx = torch.tensor(kept(D, m))
    return X[:, :, idx][:, :, :, idx][..., :m]


def spectral_mix(Xk, Wm):
    """Y[b, o, mode] = sum_c W[mode][o][c] X[b, c, mode]; Wm: [m(kx), 2m(ky), 2m(kz), W(o), W(c), 2]."""
    Wc = torch.complex(Wm[..., 0], Wm[..., 1])
    return torch.einsum("xyzoc,bczyx->bozyx", Wc, Xk)


def spectral_synthesis(Y, D, m):
    """irfftn (1/D^3) of the kept modes Y [B, O, 2m, 2m, m], every other mode zero."""
    B, O = Y.shape[:2]
    idx = torch.tensor(kept(D, m))
    Yf = torch.zeros((B, O, D, D, D // 2 + 1), dtype=Y.dtype)
    zz, yy = torch.meshgrid(idx, idx, indexing="ij")
    Yf[:, :, zz, yy, :m] = Y
    return torch.fft.irfftn(Yf, s=(D, D, D), dim=(2, 3, 4))


def spectral_conv(h, Wm, D, m):
    """h: [B, W, D, D, D] (z, y, x); Wm: [m(kx), 2m(ky), 2m(kz), W(o), W(c), 2]."""
    return spectral_synthesis(spectral_mix(spectral_modes(h, D, m), Wm), D, m)


def forward(theta, a, D, W, m, L, Ci, Co, record=None):
    """theta: flat float64 tensor; a: [B, Ci, D, D, D] float64 -> [B, Co, D, D, D].
    record: optional dict that receives the intermediates h0 .. h_L (block inputs, h_L the last
    block's output), X_l (kept modes of h_l), Y_l (mixed modes) and z_l (pre-activations)."""
    pr = unpack(theta, D, W, m, L, Ci, Co)
    h = torch.einsum("ci,bizyx->bczyx", pr["P"], a) + pr["p"][None, :, None, None, None]
    for l in range(L):
        Xk = spectral_modes(h, D, m)
        Y = spectral_mix(Xk, pr[f"Wm{l}"])
        s = spectral_synthesis(Y, D, m)
        z = s + torch.einsum("oc,bczyx->bozyx", pr[f"Wc{l}"], h) + pr[f"b{l}"][None, :, None, None, None]
        if record is not None:
            record.update({f"h{l}": h, f"X{l}": Xk, f"Y{l}": Y, f"z{l}": z})
        h = torch.nn.functional.gelu(z) if l < L - 1 else z
    if record is not None:
        record[f"h{L}"] = h
    return torch.einsum("oc,bczyx->bozyx", pr["Q"], h) + pr["q"][None, :, None, None, None]


def forward_and_grad(theta, a, dout, D, W, m, L, Ci, Co):
    """Output and the gradient of sum(dout * out) with respect to theta (all float64 numpy)."""
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    out = forward(th, torch.tensor(a, dtype=torch.float64), D, W, m, L, Ci, Co)
    (out * torch.tensor(dout, dtype=torch.float64)).sum().backward()
    return out.detach().numpy(), th.grad.numpy()
