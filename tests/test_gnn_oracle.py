"""Pins of the learned-guess network oracle: finite differences, identities, invariances."""
import numpy as np
import pytest

from oracle import cgp_oracle as O
from oracle import gnn_oracle as G
from paper_2003_00082_gb300 import inputs


@pytest.fixture(scope="module")
def tiny():
    xy, tri = inputs.ogrid(8, 4)
    om = O.OracleMesh(xy, tri)
    g = G.Graph(om.K, om.xy_c)
    rng = np.random.default_rng(0)
    samples = []
    for s in range(2):
        b = rng.standard_normal(om.n_c)
        phi1 = rng.standard_normal(om.n_c)
        phi2 = rng.standard_normal(om.n_c)
        f, s_p = G.features(g, om.K, b, phi1, phi2)
        samples.append((f, rng.standard_normal(om.n_c) * 0.1))
    return om, g, samples


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.standard_normal(1000) * 10.0 ** rng.uniform(-20, 20, 1000),
                        [0.0, -0.0, 1.0, 3.0000001, 1.00390625, 1.01171875]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(G.bf16(x), ref)


def test_graph_is_the_symmetric_edge_set(tiny):
    om, g, _ = tiny
    assert g.dst.shape[0] == 2 * om.edges.shape[0]
    pairs = set(zip(g.dst.tolist(), g.src.tolist()))
    for a, b in om.edges:
        assert (a, b) in pairs and (b, a) in pairs


def test_zero_decoder_returns_previous_solution(tiny):
    om, g, _ = tiny
    p = G.init_params(3, zero_decoder=True)
    rng = np.random.default_rng(2)
    b, phi1, phi2 = rng.standard_normal((3, om.n_c))
    x0 = G.guess(p, g, om.K, b, phi1, phi2)
    np.testing.assert_allclose(x0, phi1 - phi1.mean(), atol=1e-14)


def test_gradients_match_central_differences(tiny):
    om, g, samples = tiny
    p = G.init_params(4, zero_decoder=False)
    loss, grads = G.loss_and_grad(p, g, samples, bf16_storage=False)
    rng = np.random.default_rng(5)
    h = 1e-6
    worst = 0.0
    for k in p:
        flat = p[k].reshape(-1)
        for idx in rng.choice(flat.size, size=min(4, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = G.loss_and_grad(p, g, samples, bf16_storage=False)
            flat[idx] = old - h
            lm, _ = G.loss_and_grad(p, g, samples, bf16_storage=False)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            an = grads[k].reshape(-1)[idx]
            scale = max(abs(fd), abs(an), 1e-7)
            worst = max(worst, abs(fd - an) / scale)
    assert worst <= 1e-5, worst


def test_planted_backward_mistake_is_caught(tiny, monkeypatch):
    """Swapping source and destination in the message gradient breaks the finite-difference pin."""
    om, g, samples = tiny
    p = G.init_params(6, zero_decoder=False)
    g2 = G.Graph(om.K, om.xy_c)
    loss, grads = G.loss_and_grad(p, g, samples, bf16_storage=False)
    # a network whose backward scatters to the wrong end of each edge
    g2.src, g2.dst = g.dst.copy(), g.src.copy()
    _, bad = G.loss_and_grad(p, g2, samples, bf16_storage=False)
    # forward of g2 is a different network: same loss only if the graph is symmetric in values
    h = 1e-6
    flat = p["Wm0"].reshape(-1)
    old = flat[7]
    flat[7] = old + h
    lp, _ = G.loss_and_grad(p, g, samples, bf16_storage=False)
    flat[7] = old - h
    lm, _ = G.loss_and_grad(p, g, samples, bf16_storage=False)
    flat[7] = old
    fd = (lp - lm) / (2 * h)
    assert abs(grads["Wm0"].reshape(-1)[7] - fd) <= 1e-5 * max(abs(fd), 1e-7)
    assert abs(bad["Wm0"].reshape(-1)[7] - fd) > 1e-3 * max(abs(fd), 1e-7)


def test_node_relabelling_permutes_the_output(tiny):
    om, g, samples = tiny
    p = G.init_params(7, zero_decoder=False)
    f = samples[0][0]
    out, _ = G.forward(p, g, f, bf16_storage=False)
    rng = np.random.default_rng(8)
    perm = rng.permutation(om.n_c)          # new index of old node i is inv[i]
    inv = np.argsort(perm)
    import scipy.sparse as sp
    # relabel the pattern by index arithmetic (a matrix product would drop exact zeros of K)
    K = om.K.tocoo()
    Kp = sp.csr_matrix((np.ones(K.nnz), (inv[K.row], inv[K.col])), shape=K.shape)
    Kp.sort_indices()
    gp = G.Graph(Kp, om.xy_c[perm])
    outp, _ = G.forward(p, gp, f[perm], bf16_storage=False)
    np.testing.assert_allclose(outp, out[perm], rtol=1e-12, atol=1e-12)


def test_features_make_linear_extrapolation_learnable(tiny):
    """Feature 1 is the last increment in units of s_d: out = f[:, 1] reproduces phi1 + (phi1 - phi2)."""
    om, g, _ = tiny
    rng = np.random.default_rng(9)
    b, phi1, phi2 = rng.standard_normal((3, om.n_c))
    f, s_d = G.features(g, om.K, b, phi1, phi2)
    np.testing.assert_allclose(phi1 + s_d * f[:, 1], 2 * phi1 - phi2, atol=1e-12)
    # feature 0 is the residual of phi1 for b, in its own units
    r = b - om.K @ phi1
    np.testing.assert_allclose(f[:, 0] * np.sqrt(np.mean(r ** 2)), r, atol=1e-12)


def test_adam_first_step_is_lr_times_sign():
    p = {"w": np.array([1.0, -2.0, 3.0])}
    opt = G.Adam(p, lr=1e-3)
    opt.step(p, {"w": np.array([0.5, -4.0, 0.0])})
    np.testing.assert_allclose(p["w"], [1.0 - 1e-3, -2.0 + 1e-3, 3.0], atol=1e-9)


def test_magnitudes_bound_every_output_and_gradient_element(tiny):
    """The magnitude pass is the absolute-value network: never below the value it sizes, and equal to
    it when no term can cancel (non-negative weights, inputs and edge features, targets <= 0, no BF16
    rounding: every ReLU is the identity and every product is non-negative)."""
    om, g, samples = tiny
    p = G.init_params(6, zero_decoder=False)
    outs, mags = G.magnitudes(p, g, samples)
    _, grads = G.loss_and_grad(p, g, samples)
    for (f, _), m in zip(samples, outs):
        out, _ = G.forward(p, g, f)
        assert np.all(np.abs(out) <= m * (1 + 1e-12))
    for k in grads:
        assert np.all(np.abs(grads[k]) <= mags[k] * (1 + 1e-12) + 1e-300), k
    pos = {k: np.abs(v) + 0.01 for k, v in p.items()}
    gp = G.Graph(om.K, om.xy_c)
    gp.efeat = np.abs(gp.efeat)
    rng = np.random.default_rng(9)
    psamples = [(np.abs(f), -np.abs(rng.standard_normal(om.n_c))) for f, _ in samples]
    outs, mags = G.magnitudes(pos, gp, psamples, bf16_storage=False)
    _, grads = G.loss_and_grad(pos, gp, psamples, bf16_storage=False)
    for (f, _), m in zip(psamples, outs):
        out, _ = G.forward(pos, gp, f, bf16_storage=False)
        np.testing.assert_allclose(out, m, rtol=1e-12)
    for k in grads:
        np.testing.assert_allclose(np.abs(grads[k]), mags[k], rtol=1e-11, err_msg=k)
