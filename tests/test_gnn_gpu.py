"""Learned preconditioner (solver 3) on the GPU, through the C ABI, against
the FP64 oracle of oracle/gnn.py: graph inputs, the preconditioner applied to
vectors, loss and gradient at the same weights (matrices rounded to BF16 on
both sides, as the CUDA kernels apply them), and what training gains on
reduced camera systems of the method. Tolerances: features and edge weights
are stored in FP32 (1e-5 relative); network outputs and gradients carry FP32
activations (1e-5 relative for the FP32 application of the factor, 1e-3
for gradients)."""

import numpy as np
import pytest

from oracle import gnn
from paper_1910_08138_gb300 import rpba, synth

pytestmark = pytest.mark.gpu


def _systems(seed=1, sizes=(12, 20, 7), n_probes=3):
    sy = synth.rcs_like_systems(seed, sizes=sizes, n_probes=n_probes)
    return sy, [(gnn.graph(S, S.shape[0] // 6), z) for S, z in sy]


def _as_applied(w):
    """The parameters as the kernels apply them: matrices in BF16, the rest in FP32."""
    out, o = [], 0
    for name, s in gnn.param_shapes():
        n = int(np.prod(s))
        seg = np.asarray(w[o:o + n], dtype=np.float32).astype(np.float64)
        out.append(gnn.to_bf16(seg) if name in gnn.MATRICES else seg)
        o += n
    return np.concatenate(out)


def _trainer(sy, seed=0):
    G = rpba.Gnn(seed=seed)
    for S, z in sy:
        G.add_system(S, z)
    return G


def test_graph_inputs_match_oracle():
    sy, gs = _systems()
    G = _trainer(sy)
    x, ptr, adj, e = G.graph()
    n, ne, ns = G.size()
    assert ns == 3 and n == sum(g["x"].shape[0] for g, _ in gs)
    xo = np.concatenate([g["x"] for g, _ in gs])
    np.testing.assert_allclose(x, xo, rtol=1e-5, atol=2e-6)
    off, po, ao, eo = 0, [0], [], []
    for g, _ in gs:
        po += list(po[-1] + g["ptr"][1:])
        ao += list(g["adj"] + off)
        eo += list(g["e"])
        off += g["x"].shape[0]
    np.testing.assert_array_equal(ptr, po)
    np.testing.assert_array_equal(adj, ao)
    np.testing.assert_allclose(e, eo, rtol=1e-5)


@pytest.mark.parametrize("scale", [0.0, 0.1])
def test_preconditioner_matches_oracle(scale):
    sy, gs = _systems(2)
    G = _trainer(sy)
    rng = np.random.default_rng(4)
    w = G.weights()
    if scale:
        w = (rng.normal(size=w.size) * scale).astype(np.float32)
        G.set_weights(w)
    n = sum(g["n"] for g, _ in gs)
    r = rng.normal(size=6 * n)
    z = G.precondition(r)
    wa = _as_applied(w)
    o = 0
    for (S, _), (g, _) in zip(sy, gs):
        d = 6 * g["n"]
        zo = gnn.precondition(wa, g, r[o:o + d])
        # the factor is formed in FP64 and applied in FP32
        assert np.linalg.norm(z[o:o + d] - zo) <= 1e-5 * np.linalg.norm(zo)
        if scale == 0:  # a new network is block-Jacobi
            A = np.tril(S) + np.tril(S, -1).T
            want = np.concatenate([np.linalg.solve(A[6 * i:6 * i + 6, 6 * i:6 * i + 6], r[o + 6 * i:o + 6 * i + 6])
                                   for i in range(g["n"])])
            assert np.linalg.norm(z[o:o + d] - want) <= 1e-5 * np.linalg.norm(want)
        o += d


def test_loss_and_gradient_match_oracle():
    sy, gs = _systems(3, sizes=(10, 16), n_probes=4)
    G = _trainer(sy)
    rng = np.random.default_rng(8)
    w = (rng.normal(size=G.n_params) * 0.1).astype(np.float32)
    G.set_weights(w)
    loss, grad = G.loss_grad()
    lo, go = gnn.loss_and_grad(_as_applied(w), gs)
    assert loss == pytest.approx(lo, rel=1e-5, abs=1e-5)
    assert np.linalg.norm(grad - go) <= 1e-3 * np.linalg.norm(go)
    o = 0
    for name, s in gnn.param_shapes():
        n = int(np.prod(s))
        gg, gr = grad[o:o + n], go[o:o + n]
        assert np.linalg.norm(gg - gr) <= 1e-3 * np.linalg.norm(go) + 1e-3 * np.linalg.norm(gr), name
        o += n


def test_training_lowers_the_loss():
    sy, _ = _systems(5, sizes=(16, 24, 12), n_probes=4)
    G = _trainer(sy)
    l0 = G.loss_grad()[0]
    hist = G.train(60, lr=3e-3)
    l1 = G.loss_grad()[0]
    assert hist[0] == pytest.approx(l0, rel=1e-6)
    assert l1 < l0 - 0.05 * abs(l0), (l0, l1)


@pytest.fixture(scope="module")
def trained_weights():
    """Trained by the project's own kernels on reduced camera systems of the
    method: every sub-block of configs 1 and 2 after 0 and 1 outer iterations,
    at two dampings, with probes drawn anew at every step."""
    G = rpba.Gnn(seed=0)
    for cfg in (1, 2):
        ctx = rpba.Rpba(synth.config(cfg), precision=0, solver=0, robust=1, robust_from_start=1)
        ctx.intersect()
        for k in range(2):
            for lam in (1e-4, 1e-2):
                G.add_rcs(ctx, lam, n_probes=4, seed=100 * cfg + 10 * k + int(lam * 1e4))
            ctx.iterate(1)
        ctx.close()
    hist = G.train(300, lr=3e-4, probe_seed=7)
    assert hist[-20:].mean() < hist[:20].mean()
    return G.weights()


def _lm_step_solution(prob, solver, w, outer):
    ctx = rpba.Rpba(prob, precision=0, solver=solver, robust=1, robust_from_start=1, pcg_max_iter=3000)
    if solver == 3:
        ctx.set_gnn_weights(w)
    ctx.intersect()
    if outer:
        ctx.iterate(outer)
    _, _, _, dc, _ = ctx.lm_step(1e-4)
    it, rr, fb = None, None, 0
    if solver in (1, 3):
        it, rr = ctx.solver_stats()
    if solver == 3:
        fb = ctx.solver_fallbacks()
    ctx.close()
    return dc, it, rr, fb


@pytest.mark.parametrize("name,make,outer", [
    ("1000-camera block after 3 outer iterations (a state not trained on)", lambda: synth.config(2), 3),
    ("5000-camera strip block (a layout not trained on)", lambda: synth.config(4, scale=0.1), 1),
])
def test_learned_preconditioner_gain(trained_weights, name, make, outer):
    """What the trained network gains over the method without it (block-Jacobi
    PCG, Sec. 5.5): both reach the 1e-8 relative residual, both solutions equal
    the direct Cholesky solution, and the learned one needs fewer iterations."""
    prob = make()
    d0, _, _, _ = _lm_step_solution(prob, 0, None, outer)
    d1, it1, rr1, _ = _lm_step_solution(prob, 1, None, outer)
    d3, it3, rr3, fb = _lm_step_solution(prob, 3, trained_weights, outer)
    assert rr1.max() <= 1e-8 and rr3.max() <= 1e-8 and fb == 0
    for d in (d1, d3):
        assert np.linalg.norm(d - d0) <= 1e-6 * np.linalg.norm(d0)
    gain = 1.0 - it3.sum() / it1.sum()
    print(f"{name}: PCG iterations block-Jacobi {it1.sum()}, learned {it3.sum()}, gain {gain:.0%}")
    assert gain >= 0.2


@pytest.mark.parametrize("precision", [0, 1])
def test_whole_run_with_learned_preconditioner(trained_weights, precision):
    import oracle
    prob = synth.config(1)
    ro = oracle.Oracle(prob).run(robust=1, robust_from_start=1)
    g = rpba.Rpba(prob, precision=precision, solver=3, robust=1, robust_from_start=1)
    g.set_gnn_weights(trained_weights)
    rg = g.iterate()
    assert abs(rg["rms"] - ro["rms"]) <= 1e-3, (rg["rms"], ro["rms"])
    assert g.solver_fallbacks() == 0
