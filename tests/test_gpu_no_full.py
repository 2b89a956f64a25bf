"""The neural operator at the configuration the warm start trains (64^3 grid, width 32, 12 modes per
axis, 4 blocks, 4 input and 4 output channels), batch 2, against the FP64 oracle element by element.

Error model behind the bounds.  The GPU path rounds GEMM operands to BF16 (8 significant bits,
round to nearest: relative error |delta| <= u = 2^-8, close to uniform, variance u^2/3) and
accumulates in FP32 (negligible next to that).  One rounding of an operand whose products are
summed incoherently (the DFT stages, the mode mixing, the 1x1 maps) leaves a relative error of
standard deviation u / sqrt(3) in the result, measured against the RMS of the result.  Per block
the forward pass rounds 7 activations (the block input, two partial DFTs, the mixed modes, two
partial inverse DFTs, and the 1x1 map's input is the block input again) and 7 constant operands
(six DFT matrices, the 1x1 weights): n_fwd = 4 x 14 = 56 roundings.  Independent roundings add
in variance: sigma_fwd = u sqrt(n_fwd / 3).  The backward pass rounds about as many on its own
chain, so the factors of a gradient carry at most sigma_bwd = u sqrt(2 n_fwd / 3).

Outputs, per element e of an output channel of one sample:
    |out_gpu(e) - out_oracle(e)| <= 6 sigma_fwd (rms_channel + |out_oracle(e)|)
(6 sigma leaves a Gaussian tail of 2e-9 per element), and the RMS of the error over the channel
stays within 1.5 sigma_fwd rms_channel, which a systematic error (a wrong term, a dropped mode)
exceeds even where it stays under the per-element bound.

Gradients.  Every parameter gradient is a sum of products of two factors that the network
computes (dP = sum dh0 a, dWc_l = sum dz_l h_l, dWm_l = sum_b G_l conj(X_l) per Fourier mode,
dQ = sum dout h_L; the biases sum one factor), taken from the oracle's intermediates by autograd.
If each computed factor v is within 6 sigma_bwd (|v| + rms_v) of its exact value (rms_v over the
factor's channel, or over one Fourier mode), the triangle inequality bounds the gradient element
by 6 sigma_bwd sum_terms (|v1| + rms_v1)(|v2| + rms_v2) (to first order).  This scale follows the
size of the products, not of their sum, so an element whose terms cancel keeps the error its
terms carry.  The RMS of the error over each block must also stay within 1.5 sigma_bwd of the
block's RMS; for the mode matrices, whose elements sum two products each, within 1.5 sigma_bwd of
the RMS of the term scale of each mode.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import no_oracle as no  # noqa: E402
from paper_1905_10182_gb300.neural import NeuralOperator  # noqa: E402
from no_params import host_params  # noqa: E402

CFG = dict(D=64, W=32, m=12, L=4, Ci=4, Co=4)
B = 2
U = 2.0 ** -8
N_FWD = 14 * CFG["L"]
SIGMA_FWD = U * math.sqrt(N_FWD / 3.0)
SIGMA_BWD = U * math.sqrt(2 * N_FWD / 3.0)


def _check_scope(got, ref, sigma, label):
    """Element-wise and RMS checks of one scope; returns (max err / rms, rms err / rms)."""
    rms = float(np.sqrt(np.mean(ref ** 2)))
    if rms == 0.0:
        assert np.abs(got).max() == 0.0, label
        return 0.0, 0.0
    err = np.abs(got - ref)
    bound = 6.0 * sigma * (rms + np.abs(ref))
    worst = int(np.argmax(err - bound))
    assert (err <= bound).all(), (label, float(err.flat[worst]), float(bound.flat[worst]), rms)
    erms = float(np.sqrt(np.mean(err ** 2)))
    assert erms <= 1.5 * sigma * rms, (label, erms, rms)
    return float(err.max()) / rms, erms / rms


def _oracle_intermediates(theta, a, dout):
    """Oracle output, parameter gradient and the factors of every gradient (FP64 autograd)."""
    c = CFG
    th = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    rec = {}
    out = no.forward(th, torch.tensor(a, dtype=torch.float64), c["D"], c["W"], c["m"], c["L"], c["Ci"], c["Co"],
                     record=rec)
    for v in rec.values():
        v.retain_grad()
    (out * torch.tensor(dout, dtype=torch.float64)).sum().backward()
    fac = {"dh0": rec["h0"].grad.numpy(), f"h{c['L']}": rec[f"h{c['L']}"].detach().numpy()}
    for l in range(c["L"]):
        fac[f"h{l}"] = rec[f"h{l}"].detach().numpy()
        fac[f"dz{l}"] = rec[f"z{l}"].grad.numpy()
        fac[f"X{l}"] = np.abs(rec[f"X{l}"].detach().numpy())
        fac[f"G{l}"] = np.abs(rec[f"Y{l}"].grad.numpy())
    return out.detach().numpy(), th.grad.numpy(), fac


def _channel_mag(v):
    """|v| + the RMS of v over each channel (axis 1) of a [B, C, ...] field."""
    r = np.sqrt(np.mean(v ** 2, axis=(0,) + tuple(range(2, v.ndim)), keepdims=True))
    return np.abs(v) + r


def _mode_mag(v):
    """|v| + the RMS of v over batch and channel for each Fourier mode of a [B, C, kz, ky, kx] field."""
    return np.abs(v) + np.sqrt(np.mean(v ** 2, axis=(0, 1), keepdims=True))


def _grad_scales(fac, lay):
    """Per-parameter scale sum_terms (|v1| + rms_v1)(|v2| + rms_v2) in the layout of the flat vector."""
    c = CFG
    flat = lambda v: v.reshape(v.shape[0], v.shape[1], -1)  # noqa: E731
    out = {}
    dh0 = flat(_channel_mag(fac["dh0"]))
    out["P"] = np.einsum("bcs,bis->ci", dh0, np.abs(flat(fac["a"])))
    out["p"] = dh0.sum(axis=(0, 2))
    for l in range(c["L"]):
        dz = flat(_channel_mag(fac[f"dz{l}"]))
        h = flat(_channel_mag(fac[f"h{l}"]))
        out[f"Wc{l}"] = np.einsum("bos,bcs->oc", dz, h)
        out[f"b{l}"] = dz.sum(axis=(0, 2))
        G, X = _mode_mag(fac[f"G{l}"]), _mode_mag(fac[f"X{l}"])      # [B, W, kz, ky, kx]
        sc = np.einsum("bozyx,bczyx->xyzoc", G, X)
        out[f"Wm{l}"] = np.repeat(sc[..., None], 2, axis=-1)
    hL = flat(_channel_mag(fac[f"h{c['L']}"]))
    dout = np.abs(flat(fac["dout"]))
    out["Q"] = np.einsum("bos,bcs->oc", dout, hL)
    out["q"] = dout.sum(axis=(0, 2))
    return {k: out[k].reshape(lay[k][1]) for k in lay}


@pytest.fixture(scope="module")
def case():
    c = CFG
    net = NeuralOperator(D=c["D"], width=c["W"], modes=c["m"], layers=c["L"], in_ch=c["Ci"], out_ch=c["Co"],
                         max_batch=B, seed=11)
    lay = no.layout(c["D"], c["W"], c["m"], c["L"], c["Ci"], c["Co"])
    theta = host_params(lay, c["W"], seed=11)
    net.set_params(theta)
    rng = np.random.default_rng(12)
    D = c["D"]
    a = rng.normal(size=(B, c["Ci"], D, D, D)).astype(np.float32)
    dout = rng.normal(size=(B, c["Co"], D, D, D)).astype(np.float32)
    out = torch.empty((B, c["Co"], D, D, D), device="cuda")
    net.forward(torch.from_numpy(a).cuda(), out)
    net.backward(torch.from_numpy(dout).cuda())
    got_out = out.cpu().numpy().astype(np.float64)
    got_grad = net.get_grads().astype(np.float64)
    net.close()
    ref_out, ref_grad, fac = _oracle_intermediates(theta.astype(np.float64), a.astype(np.float64),
                                                   dout.astype(np.float64))
    fac.update(a=a.astype(np.float64), dout=dout.astype(np.float64))
    return dict(lay=lay[0], got_out=got_out, got_grad=got_grad, ref_out=ref_out, ref_grad=ref_grad,
                scales=_grad_scales(fac, lay[0]))


def test_forward_elementwise_real_config(case):
    worst = []
    for b in range(B):
        for o in range(CFG["Co"]):
            worst.append(_check_scope(case["got_out"][b, o], case["ref_out"][b, o], SIGMA_FWD, f"out[{b},{o}]"))
    w = np.max(worst, axis=0)
    print(f"forward: max |err| / rms = {w[0]:.3e}, rms err / rms = {w[1]:.3e} "
          f"(bounds: per element 6 sigma = {6 * SIGMA_FWD:.3e} x (rms + |x|), rms {1.5 * SIGMA_FWD:.3e})")


def test_gradients_elementwise_real_config(case):
    c = CFG
    for name, (off, shp) in case["lay"].items():
        n = int(np.prod(shp))
        g = case["got_grad"][off:off + n].reshape(shp)
        r = case["ref_grad"][off:off + n].reshape(shp)
        sc = case["scales"][name]
        err = np.abs(g - r)
        bound = 6.0 * SIGMA_BWD * sc
        worst = np.unravel_index(int(np.argmax(err / bound)), shp)
        assert (err <= bound).all(), (name, worst, float(err[worst]), float(bound[worst]), float(r[worst]))
        if name.startswith("Wm"):
            # two products per element (batch 2): the sum may cancel, so the RMS of the error is
            # held against the RMS of the term scale of each mode
            nm = c["m"] * 2 * c["m"] * 2 * c["m"]
            gm, rm, sm = g.reshape(nm, -1), r.reshape(nm, -1), sc.reshape(nm, -1)
            srms = np.sqrt(np.mean(sm ** 2, axis=1))
            erms = np.sqrt(np.mean((gm - rm) ** 2, axis=1))
            assert (erms <= 1.5 * SIGMA_BWD * srms).all(), (name, float((erms / srms).max()))
            rel_rms = float((erms / srms).max())
        else:
            rms = float(np.sqrt(np.mean(r ** 2)))
            rel_rms = float(np.sqrt(np.mean((g - r) ** 2)) / rms)
            assert rel_rms <= 1.5 * SIGMA_BWD, (name, rel_rms)
        print(f"grad {name}: max |err| / element bound = {float((err / bound).max()):.3e}, "
              f"rms err / rms = {rel_rms:.3e}")
    print(f"sigma_bwd = {SIGMA_BWD:.3e}; element bound 6 sigma_bwd x sum (|v1| + rms)(|v2| + rms), "
          f"rms bound {1.5 * SIGMA_BWD:.3e}")
