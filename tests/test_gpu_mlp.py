"""The correction network's CUDA kernels (forward, loss, backward, Adam) against the FP64
oracle network on the same BF16-valued weights."""
import numpy as np
import pytest

import oracle.learned as LN
from gpu_common import bf16_bits, bf16_values

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _params(seed):
    from paper_1911_02366_gb300 import sc
    P = LN.init_params(seed=seed, scale_out=1.0)
    rng = np.random.default_rng(seed + 1)
    for k in ("b1", "b2", "b3"):
        P[k] = rng.standard_normal(P[k].shape) * 0.05
    W = np.concatenate([P["W1"].ravel(), P["W2"].ravel(), P["W3"].ravel()]).astype(np.float32)
    b = np.concatenate([P["b1"], P["b2"], P["b3"]]).astype(np.float32)
    # the oracle sees exactly the values the GPU multiplies with
    Wq = bf16_values(bf16_bits(W)).astype(np.float64)
    n1 = 256 * LN.N_IN
    Pq = {"W1": Wq[:n1].reshape(256, LN.N_IN), "W2": Wq[n1:n1 + 65536].reshape(256, 256),
          "W3": Wq[n1 + 65536:].reshape(25, 256), "b1": b[:256].astype(np.float64),
          "b2": b[256:512].astype(np.float64), "b3": b[512:].astype(np.float64)}
    return W, b, Pq


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-30))


@pytest.mark.parametrize("n", [1, 37, 1000])
def test_forward_matches_oracle(n):
    from paper_1911_02366_gb300 import sc
    W, b, Pq = _params(1)
    X = np.random.default_rng(2).standard_normal((n, LN.N_IN)).astype(np.float32)
    net = sc.MLP(W, b)
    Xd = torch.tensor(X, device="cuda")
    Y = torch.empty(n, 25, device="cuda")
    cache = torch.empty(4 * n * 256, device="cuda")
    net.forward(Xd, Y, cache)
    yref, c = LN.forward(Pq, X.astype(np.float64))
    assert _rel(Y.cpu().numpy(), yref) < 2e-5
    h2 = cache[3 * n * 256:].view(n, 256).cpu().numpy()
    assert _rel(h2, c[4]) < 2e-5
    Y2 = torch.empty(n, 25, device="cuda")
    net.forward(Xd, Y2)  # without a cache
    assert torch.equal(Y, Y2)


def test_loss_and_gradient_match_oracle():
    from paper_1911_02366_gb300 import sc
    rng = np.random.default_rng(3)
    Yh = rng.standard_normal((300, 25)).astype(np.float32)
    Th = rng.standard_normal((300, 25)).astype(np.float32)
    W, b, _ = _params(1)
    net = sc.MLP(W, b)
    Y, T = torch.tensor(Yh, device="cuda"), torch.tensor(Th, device="cuda")
    dY = torch.empty_like(Y)
    acc = torch.zeros(1, device="cuda")
    net.loss(Y, T, dY, acc)
    ref = LN.loss(Yh.astype(np.float64), Th.astype(np.float64))
    assert abs(acc.item() - ref) < 1e-5 * ref
    assert _rel(dY.cpu().numpy(), LN.loss_grad(Yh.astype(np.float64), Th.astype(np.float64))) < 1e-5


@pytest.mark.parametrize("n", [5, 3000])
def test_backward_matches_oracle(n):
    from paper_1911_02366_gb300 import sc
    W, b, Pq = _params(4)
    rng = np.random.default_rng(5)
    X = rng.standard_normal((n, LN.N_IN)).astype(np.float32)
    dYh = rng.standard_normal((n, 25)).astype(np.float32)
    net = sc.MLP(W, b)
    Xd, dY = torch.tensor(X, device="cuda"), torch.tensor(dYh, device="cuda")
    Y = torch.empty(n, 25, device="cuda")
    cache = torch.empty(4 * n * 256, device="cuda")
    work = torch.empty(2 * n * 256, device="cuda")
    net.forward(Xd, Y, cache)
    net.backward(Xd, cache, dY, work)
    _, c = LN.forward(Pq, X.astype(np.float64))
    g = LN.backward(Pq, c, dYh.astype(np.float64))
    gW = net.gW.cpu().numpy()
    gb = net.gb.cpu().numpy()
    n1 = 256 * LN.N_IN
    assert _rel(gW[:n1], g["W1"].ravel()) < 1e-4
    assert _rel(gW[n1:n1 + 65536], g["W2"].ravel()) < 1e-4
    assert _rel(gW[n1 + 65536:], g["W3"].ravel()) < 1e-4
    assert _rel(gb, np.concatenate([g["b1"], g["b2"], g["b3"]])) < 1e-4


def test_adam_matches_oracle_and_refreshes_bf16_copy():
    from paper_1911_02366_gb300 import sc
    W, b, _ = _params(6)
    rng = np.random.default_rng(7)
    net = sc.MLP(W, b)
    P = {"W": W.astype(np.float64), "b": b.astype(np.float64)}
    st = {}
    for _ in range(3):
        gWh = rng.standard_normal(W.size).astype(np.float32)
        gbh = rng.standard_normal(b.size).astype(np.float32)
        net.gW.copy_(torch.tensor(gWh))
        net.gb.copy_(torch.tensor(gbh))
        net.adam(1e-2)
        LN.adam_step(P, {"W": gWh.astype(np.float64), "b": gbh.astype(np.float64)}, st, lr=1e-2)
    assert _rel(net.W.cpu().numpy(), P["W"]) < 1e-5
    assert _rel(net.b.cpu().numpy(), P["b"]) < 1e-5
    assert np.array_equal(net.Wh.cpu().numpy().view(np.uint16), bf16_bits(net.W.cpu().numpy()))
    assert float(net.gW.abs().max()) == 0.0


def test_training_fits_a_teacher_network():
    """Mini-batch Adam through the kernels drives the loss on a learnable target down."""
    from paper_1911_02366_gb300 import sc
    W, b, Pq = _params(8)
    rng = np.random.default_rng(9)
    n = 8192
    X = rng.standard_normal((n, LN.N_IN)).astype(np.float32)
    teacher = LN.init_params(seed=11, scale_out=1.0)
    T, _ = LN.forward(teacher, X.astype(np.float64))
    net = sc.MLP(W, b)
    hist = net.train(torch.tensor(X, device="cuda"), torch.tensor(T.astype(np.float32), device="cuda"),
                     epochs=15, batch=512, lr=2e-3)
    assert hist[-1] < 0.3 * hist[0], hist


def test_initial_bf16_copy_and_save_load_round_trip(tmp_path):
    """The binding's BF16 copy comes from the library (nearest even), and a saved network
    reads back bit for bit, also into a context (sc_load_mlp)."""
    from paper_1911_02366_gb300 import sc
    W, b, _ = _params(12)
    net = sc.MLP(W, b)
    assert np.array_equal(net.Wh.cpu().numpy().view(np.uint16), bf16_bits(np.asarray(W, dtype=np.float32)))
    path = str(tmp_path / "net.scmlp")
    net.save(path)
    back = sc.MLP.load(path)
    assert np.array_equal(back.W.cpu().numpy(), net.W.cpu().numpy())
    assert np.array_equal(back.b.cpu().numpy(), net.b.cpu().numpy())
    assert np.array_equal(back.Wh.cpu().numpy(), net.Wh.cpu().numpy())
    ctx = sc.Context(stream=torch.cuda.current_stream().cuda_stream, precision=sc.SC_PREC_MIXED,
                     precond=sc.SC_PC_LEARNED)
    ctx.sc_set_mesh(2, 2 * np.pi, 2)
    ctx.sc_load_mlp(path)
    with pytest.raises(sc.SCError):
        ctx.sc_load_mlp(str(tmp_path / "missing.scmlp"))
