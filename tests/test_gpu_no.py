"""The GPU neural operator (lbm_no_*) against the FP64 oracle: forward outputs and gradients.

BF16 operands in about ten chained GEMM stages: outputs within 3 % of the output scale,
gradients within 5 % relative (L2 over each parameter block).
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from oracle import no_oracle as no  # noqa: E402
from paper_1905_10182_gb300.neural import NeuralOperator  # noqa: E402
from no_params import host_params  # noqa: E402

CFG = dict(D=16, W=8, m=4, L=2, Ci=4, Co=4)


def _model(seed=3, B=2):
    """The operator with seeded host-side parameters (also returned, as float64, for the oracle)."""
    c = CFG
    net = NeuralOperator(D=c["D"], width=c["W"], modes=c["m"], layers=c["L"], in_ch=c["Ci"], out_ch=c["Co"],
                         max_batch=B, seed=seed)
    theta = host_params(no.layout(c["D"], c["W"], c["m"], c["L"], c["Ci"], c["Co"]), c["W"], seed)
    net.set_params(theta)
    return net, theta.astype(np.float64)


def test_forward_matches_oracle():
    c = CFG
    net, theta = _model()
    rng = np.random.default_rng(4)
    a = rng.normal(size=(2, c["Ci"], c["D"], c["D"], c["D"])).astype(np.float32)
    out = torch.empty((2, c["Co"], c["D"], c["D"], c["D"]), device="cuda")
    net.forward(torch.from_numpy(a).cuda(), out)
    ref = no.forward(torch.tensor(theta), torch.tensor(a.astype(np.float64)), c["D"], c["W"], c["m"], c["L"], c["Ci"],
                     c["Co"]).numpy()
    err = np.abs(out.cpu().numpy() - ref).max()
    assert err <= 0.03 * np.abs(ref).max(), (err, np.abs(ref).max())


def test_gradients_match_oracle():
    c = CFG
    net, theta = _model(seed=5)
    rng = np.random.default_rng(6)
    a = rng.normal(size=(2, c["Ci"], c["D"], c["D"], c["D"])).astype(np.float32)
    dout = rng.normal(size=(2, c["Co"], c["D"], c["D"], c["D"])).astype(np.float32)
    out = torch.empty((2, c["Co"], c["D"], c["D"], c["D"]), device="cuda")
    net.forward(torch.from_numpy(a).cuda(), out)
    net.backward(torch.from_numpy(dout).cuda())
    g = net.get_grads().astype(np.float64)
    _, gref = no.forward_and_grad(theta, a.astype(np.float64), dout.astype(np.float64), c["D"], c["W"], c["m"], c["L"],
                                  c["Ci"], c["Co"])
    lay, _ = no.layout(c["D"], c["W"], c["m"], c["L"], c["Ci"], c["Co"])
    for name, (off, shp) in lay.items():
        n = int(np.prod(shp))
        gg, gr = g[off:off + n], gref[off:off + n]
        rel = np.linalg.norm(gg - gr) / max(np.linalg.norm(gr), 1e-30)
        assert rel <= 0.05, (name, rel)


def test_training_reduces_loss():
    c = CFG
    net, _ = _model(seed=7, B=2)
    rng = np.random.default_rng(8)
    D = c["D"]
    a = rng.normal(size=(2, c["Ci"], D, D, D)).astype(np.float32)
    # a smooth target: the first input channel low-pass filtered, plus a constant
    t = np.zeros((2, c["Co"], D, D, D), np.float32)
    t[:, 0] = 0.5 * a[:, 0] + 0.1
    ad, td = torch.from_numpy(a).cuda(), torch.from_numpy(t).cuda()
    losses = [net.train_step(ad, td, 3e-3) for _ in range(60)]
    assert losses[-1] < 0.3 * losses[0], losses[::10]


def test_graph_replayed_steps_equal_eager_steps():
    """Five training steps replayed from the captured graph (after the first, eager one) leave the
    parameters bit-identical to five eager steps: the graph holds the same kernels in the same
    order.  The batch size then changes (a second capture) and the two stay identical."""
    c = CFG
    rng = np.random.default_rng(21)
    D = c["D"]
    runs = []
    for graphs in (True, False):
        net, _ = _model(seed=11, B=2)
        net.use_graphs(graphs)
        losses = []
        for B in (2, 2, 2, 2, 2, 1, 1):
            r = np.random.default_rng(100 + len(losses))
            a = torch.from_numpy(r.normal(size=(B, c["Ci"], D, D, D)).astype(np.float32)).cuda()
            t = torch.from_numpy(r.normal(size=(B, c["Co"], D, D, D)).astype(np.float32)).cuda()
            losses.append(net.train_step(a, t, 1e-3))
        runs.append((net.get_params(), np.array(losses)))
        net.close()
    assert np.array_equal(runs[0][0], runs[1][0])
    np.testing.assert_allclose(runs[0][1], runs[1][1], rtol=1e-12)
