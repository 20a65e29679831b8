"""The learned-guess network on the GPU against its FP64 CPU oracle.

Both sides store activations, messages, aggregates and dense weights in BF16
at the same points; the GPU accumulates in FP32 where the oracle uses FP64,
so outputs and gradients agree element by element to a few BF16 steps of
each element's magnitude, and the loss to BF16-level relative error.
"""
import numpy as np
import pytest

from oracle import cgp_oracle as O
from oracle import gnn_oracle as G
from paper_2003_00082_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda:0"


@pytest.fixture(scope="module")
def cgp():
    from paper_2003_00082_gb300 import build, cgp as c
    build.build()
    c.load()
    return c


def pack(p):
    return np.concatenate([p[k].reshape(-1) for k in G.param_shapes()]).astype(np.float32)


def unpack(v):
    out, o = {}, 0
    for k, shp in G.param_shapes().items():
        size = int(np.prod(shp))
        out[k] = np.asarray(v[o:o + size], dtype=np.float64).reshape(shp)
        o += size
    return out


def make_setting(cgp, shape, batch=3):
    xy, tri = inputs.ogrid(*shape)
    m = cgp.Mesh(xy, tri)
    om = O.OracleMesh(xy, tri)
    g = G.Graph(om.K, om.xy_c)
    rng = np.random.default_rng(11)
    data = []
    for s in range(batch):
        u, v = inputs.velocity(om.xy_f, s, 3, vortices=True, noise_std=1e-3)
        Fx, Fy = O.source_field(O.POTENTIAL, om.restrict(u), om.restrict(v), (0.0, 0.0, 1.0))
        b = O.rhs(om.Gx, om.Gy, Fx, Fy)
        phi2 = O.pcg(om.K, om.d, b * 0.97, tol=1e-10)["x"]
        phi1 = O.pcg(om.K, om.d, b * 0.99, tol=1e-10)["x"]
        phit = O.pcg(om.K, om.d, b, tol=1e-10)["x"] + 0.01 * rng.standard_normal(om.n_c)
        data.append((b, phi1, phi2, phit))
    return m, om, g, data


@pytest.fixture(scope="module")
def setting(cgp):
    m, om, g, data = make_setting(cgp, (16, 8))
    yield m, om, g, data
    m.close()


def stacked(data, k):
    return torch.as_tensor(np.concatenate([d[k] for d in data]), dtype=torch.float64, device=DEV)


def test_param_count_matches_the_oracle(cgp):
    assert cgp.cgp_gnn_param_count() == sum(int(np.prod(s)) for s in G.param_shapes().values())


# Elementwise bound, in BF16 units of each element's magnitude (the sum of the absolute
# values of the products behind it, gnn_oracle.magnitudes).  Both sides round to BF16 at
# the same ten points of the forward pass (h0, then m, a and h in each of three layers);
# the GPU's FP32 sums differ from the oracle's exact ones in the last bits, so a value
# near a rounding boundary may land one BF16 step (2^-7 relative) apart, and the backward
# runs on those values.  Ten stages of at most one step each, forward and backward, bound
# every output and gradient element by 20 * 2^-7 * magnitude; the test allows 24 * 2^-8 =
# 12 steps.  A wrong weight row, a transposed operand or a dropped edge changes an element
# by a sizeable fraction of its magnitude.
BF16_STEPS = 24 * 2.0 ** -8


@pytest.mark.parametrize("shape", [(16, 8), (64, 32)])
def test_forward_and_gradients_match_the_oracle_elementwise(cgp, shape):
    """Outputs, loss and every gradient element of a batch of three samples, on the 16x8 mesh
    (one gather chunk per block) and on the 64x32 mesh of the learned-guess workload."""
    m, om, g, data = make_setting(cgp, shape)
    p = G.init_params(5, zero_decoder=False)
    p = unpack(pack(p))                      # the FP32 values the GPU holds
    net = cgp.GNN(m, 4, pack(p))
    B = len(data)
    grads, out, loss = net.gradients(B, stacked(data, 0), stacked(data, 1), stacked(data, 2), stacked(data, 3))
    samples = []
    for s, (b, phi1, phi2, phit) in enumerate(data):
        f, s_p = G.features(g, om.K, b, phi1, phi2)
        samples.append((f, (phit - phi1) / s_p))
    mag_out, mag_grads = G.magnitudes(p, g, samples)
    worst = 0.0
    for s, (f, _) in enumerate(samples):
        ref_out, _ = G.forward(p, g, f, bf16_storage=True)
        err = np.abs(out[s] - ref_out)
        assert np.all(err <= BF16_STEPS * mag_out[s]), (s, float(np.max(err / mag_out[s])))
        worst = max(worst, float(np.max(err / mag_out[s])))
    ref_loss, ref_grads = G.loss_and_grad(p, g, samples, bf16_storage=True)
    assert abs(loss - ref_loss) <= 2e-2 * ref_loss
    gd = unpack(grads)
    for k in ref_grads:
        err = np.abs(gd[k] - ref_grads[k])
        bound = BF16_STEPS * mag_grads[k]
        assert np.all(err <= bound + 1e-30), (k, float(np.max(err / np.maximum(mag_grads[k], 1e-300))))
        worst = max(worst, float(np.max(err / np.maximum(mag_grads[k], 1e-300))))
    print(f"{shape}: largest error {worst / 2.0 ** -8:.2f} BF16 half-steps of the element's magnitude")
    net.close()
    m.close()


def test_zero_decoder_predicts_the_previous_solution(cgp, setting):
    m, om, g, data = setting
    net = cgp.GNN(m, 1, pack(G.init_params(6, zero_decoder=True)))
    b, phi1, phi2, _ = data[0]
    x0 = torch.empty(om.n_c, dtype=torch.float64, device=DEV)
    net.predict(torch.as_tensor(b, device=DEV), torch.as_tensor(phi1, device=DEV), torch.as_tensor(phi2, device=DEV), x0)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(x0.cpu().numpy(), phi1)
    net.close()


def test_training_lowers_the_loss_and_is_deterministic(cgp, setting):
    m, om, g, data = setting
    init = pack(G.init_params(7, zero_decoder=False))
    B = len(data)
    args = [stacked(data, k) for k in range(4)]
    results = []
    for run in range(2):
        net = cgp.GNN(m, 4, init)
        _, _, loss0 = net.gradients(B, *args)
        for it in range(60):
            net.train_step(B, *args, lr=1e-3)
        _, _, loss1 = net.gradients(B, *args)
        results.append((loss0, loss1, net.get_params()))
        net.close()
    assert results[0][1] < 0.5 * results[0][0], results[0][:2]
    np.testing.assert_array_equal(results[0][2], results[1][2])


def test_one_adam_step_matches_the_oracle(cgp, setting):
    m, om, g, data = setting
    p = unpack(pack(G.init_params(8, zero_decoder=False)))
    net = cgp.GNN(m, 4, pack(p))
    B = len(data)
    args = [stacked(data, k) for k in range(4)]
    grads, _, _ = net.gradients(B, *args)
    net.train_step(B, *args, lr=1e-3)
    after = unpack(net.get_params())
    # with the GPU's own gradient, one Adam step moves every weight by lr * g / (|g| + eps)
    opt = G.Adam(p, lr=1e-3, eps=1e-8)
    opt.step(p, unpack(grads))
    for k in p:
        np.testing.assert_allclose(after[k], p[k], rtol=0, atol=2e-6)
    net.close()


@pytest.mark.parametrize("shape", [(16, 8), (33, 17), (64, 32), (128, 64)])
def test_fused_inference_matches_the_batched_forward(cgp, shape):
    """cgp_gnn_predict (one cooperative launch over 16-node chunks, ragged last chunk; the
    batched forward when there are more chunks than co-resident blocks, as at 128x64)
    runs the batched kernels' arithmetic in the same order: the same FP32 outputs."""
    xy, tri = inputs.ogrid(*shape)
    m = cgp.Mesh(xy, tri)
    om = O.OracleMesh(xy, tri)
    u, v = inputs.velocity(om.xy_f, 4, 2, vortices=True, noise_std=1e-3)
    Fx, Fy = O.source_field(O.POTENTIAL, om.restrict(u), om.restrict(v), (0.0, 0.0, 1.0))
    b = O.rhs(om.Gx, om.Gy, Fx, Fy)
    phi2 = O.pcg(om.K, om.d, b * 0.97, tol=1e-10)["x"]
    phi1 = O.pcg(om.K, om.d, b * 0.99, tol=1e-10)["x"]
    net = cgp.GNN(m, 1, pack(G.init_params(9, zero_decoder=False)))
    T = lambda a: torch.as_tensor(a, dtype=torch.float64, device=DEV)  # noqa: E731
    x0 = torch.empty(om.n_c, dtype=torch.float64, device=DEV)
    net.predict(T(b), T(phi1), T(phi2), x0)
    torch.cuda.synchronize()
    _, out, _ = net.gradients(1, T(b), T(phi1), T(phi2), T(phi1))
    s_d = float(np.sqrt(np.mean((phi1 - phi2) ** 2)))
    got = x0.cpu().numpy() - phi1
    want = s_d * out[0].astype(np.float64)
    # identical FP32 outputs leave only the rounding of the scale and of x0 (far below one BF16 step)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))
    f, _ = G.features(G.Graph(om.K, om.xy_c), om.K, b, phi1, phi2)
    p = unpack(pack(G.init_params(9, zero_decoder=False)))
    ref_out, _ = G.forward(p, G.Graph(om.K, om.xy_c), f, bf16_storage=True)
    assert np.linalg.norm(got / s_d - ref_out) <= 2e-2 * np.linalg.norm(ref_out)
    net.close()
    m.close()
