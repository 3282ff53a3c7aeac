"""Learned correction of the block-Jacobi preconditioner: GPU features and targets against
the FP64 oracle, the corrected preconditioner inside the solve, and a trained network
evaluated on held-out seeds against plain block Jacobi."""
import numpy as np
import pytest

import oracle as O
import oracle.learned as LN
import sc_inputs as I
from gpu_common import TWO_PI, case, gpu_context

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _mixed(n, N, cfl=10.0, seed=0, tc=0, **kw):
    from paper_1911_02366_gb300 import sc
    cfg = dict(precision=sc.SC_PREC_MIXED, rel_tol=1e-8, inner_tol=1e-4, gmres_restart=30, gmres_max_iters=4000,
               max_refine=20, tensor_cores=tc)
    cfg.update(kw)
    Q, dt, p, ctx = case(n, N, cfl=cfl, seed=seed, **cfg)
    ctx.sc_set_state(Q, Q)
    ctx.sc_assemble()
    return Q, dt, p, ctx


def _oracle_ft(Q, dt, p, n, N):
    S = O.condensed_operator(O.jacobian(p, Q), n, N).dense_S()
    return LN.features_and_targets(S, Q, n, N, 0.1, 1600.0, dt)


@pytest.mark.parametrize("N", [2, 3])
def test_features_and_targets_match_oracle(N):
    n = 3
    Q, dt, p, ctx = _mixed(n, N)
    ctx.sc_condense()
    nsmp = n ** 3 * len(LN.boundary_nodes(N))
    F = torch.empty(nsmp, 64, device="cuda")
    sn = torch.empty(nsmp, device="cuda")
    T = torch.empty(nsmp, 25, device="cuda")
    ctx.sc_learned_features(F, sn)
    ctx.sc_learned_targets(T)
    Fo, To, sno = _oracle_ft(Q, dt, p, n, N)
    Fg = F.cpu().numpy()
    assert np.max(np.abs(Fg[:, :5] - Fo[:, :5])) < 1e-6 * np.max(np.abs(Fo[:, :5]))
    assert np.max(np.abs(Fg[:, 5:55] - Fo[:, 5:55])) < 1e-4      # unit-norm blocks
    assert np.max(np.abs(Fg[:, 55:] - Fo[:, 55:])) < 1e-5 * np.max(np.abs(Fo[:, 55:]))
    assert np.max(np.abs(sn.cpu().numpy() - sno) / sno) < 1e-4  # S_ee formed in FP32
    Tg = T.cpu().numpy()
    assert np.max(np.abs(Tg - To)) < 2e-3 * np.max(np.abs(To))


def _net(seed, zero_out=False):
    from paper_1911_02366_gb300 import sc
    P = LN.init_params(seed=seed, scale_out=0.01)
    if zero_out:
        P["W3"][:] = 0.0
    W = np.concatenate([P["W1"].ravel(), P["W2"].ravel(), P["W3"].ravel()])
    b = np.concatenate([P["b1"], P["b2"], P["b3"]])
    return sc.MLP(W, b, stream=torch.cuda.current_stream().cuda_stream)


def _solve(ctx, Q):
    dQ = np.zeros(Q.size)
    st = ctx.sc_solve(dQ)
    return dQ, st


def test_zero_correction_reproduces_block_jacobi_and_a_correction_changes_it():
    from paper_1911_02366_gb300 import sc
    n, N = 3, 3
    Q, dt, p, ctx = _mixed(n, N)
    ctx.sc_condense()
    _, st_bj = _solve(ctx, Q)
    res = {}
    for key, net in (("zero", _net(1, zero_out=True)), ("rand", _net(2))):
        Q, dt, p, cl = _mixed(n, N, precond=sc.SC_PC_LEARNED, learned_min_reduction=1.0)
        cl.sc_set_learned_weights(net)
        cl.sc_condense()
        dQ, st = _solve(cl, Q)
        assert st["rel_residual"] < 1e-8
        res[key] = st
    assert res["zero"]["gmres_iters"] == st_bj["gmres_iters"]
    assert res["rand"]["gmres_iters"] != st_bj["gmres_iters"]


def test_learned_solve_matches_oracle_global_solve():
    from paper_1911_02366_gb300 import sc
    n, N = 2, 3
    Q, dt, p, ctx = _mixed(n, N, precond=sc.SC_PC_LEARNED, rel_tol=1e-12)
    ctx.sc_set_learned_weights(_net(3))
    ctx.sc_condense()
    dQ, st = _solve(ctx, Q)
    A = O.jacobian(p, Q)
    B = -O.residual(p, Q).reshape(-1)
    x = O.global_solve(A, B)
    assert np.linalg.norm(dQ - x) / np.linalg.norm(x) < 1e-9


def test_trained_correction_against_block_jacobi_on_held_out_seeds(capsys):
    """Train on systems the method forms (seeds 100..105, Ma 0.05..0.3), evaluate GMRES
    iterations on held-out seeds 1000..1001 against plain block Jacobi; records both."""
    from paper_1911_02366_gb300 import sc
    n, N = 3, 3
    Fs, Ts = [], []
    for i, seed in enumerate(range(100, 106)):
        Ma = [0.05, 0.1, 0.15, 0.2, 0.25, 0.3][i]
        Q, dt = I.tgv_state(n, N, Ma=Ma, cfl=10.0, seed=seed)
        ctx = gpu_context(precision=sc.SC_PREC_MIXED, Ma=Ma, tensor_cores=0)
        ctx.sc_set_mesh(n, TWO_PI, N)
        ctx.sc_set_timestep(dt, 1)
        ctx.sc_set_state(Q, Q)
        ctx.sc_assemble()
        ctx.sc_condense()
        nsmp = n ** 3 * len(LN.boundary_nodes(N))
        F = torch.empty(nsmp, 64, device="cuda")
        sn = torch.empty(nsmp, device="cuda")
        T = torch.empty(nsmp, 25, device="cuda")
        ctx.sc_learned_features(F, sn)
        ctx.sc_learned_targets(T)
        Fs.append(F)
        Ts.append(T)
    X = torch.cat(Fs).contiguous()
    Y = torch.cat(Ts).contiguous()
    net = _net(7)
    hist = net.train(X, Y, epochs=40, batch=256, lr=1e-3)
    assert hist[-1] < hist[0]
    out = {}
    for seed in (1000, 1001):
        Q, dt, p, ctx = _mixed(n, N, seed=seed)
        ctx.sc_condense()
        _, st_bj = _solve(ctx, Q)
        row = {"block_jacobi": st_bj["gmres_iters"]}
        Q, dt, p, cl = _mixed(n, N, seed=seed, precond=sc.SC_PC_LEARNED, learned_min_reduction=1.0)
        cl.sc_set_learned_weights(net)
        cl.sc_condense()
        _, st_l = _solve(cl, Q)
        assert st_l["rel_residual"] < 1e-8
        row["network"] = st_l["gmres_iters"]
        # what a perfect network would give: the exact targets, full and damped
        nsmp = n ** 3 * len(LN.boundary_nodes(N))
        T = torch.empty(nsmp, 25, device="cuda")
        F = torch.empty(nsmp, 64, device="cuda")
        sn = torch.empty(nsmp, device="cuda")
        cl.sc_learned_targets(T)
        cl.sc_learned_features(F, sn)
        Cexact = (T / sn[:, None]).contiguous()
        for w in (1.0, 0.5):
            cl.sc_set_learned_correction(Cexact, w)
            _, st_x = _solve(cl, Q)
            row[f"exact_x{w}"] = st_x["gmres_iters"]
        out[seed] = row
    with capsys.disabled():
        print(f"\nlearned correction: loss {hist[0]:.3g} -> {hist[-1]:.3g}; GMRES iterations per held-out seed: {out}")
