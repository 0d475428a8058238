"""Learned initial guess on the GPU vs the MLP oracle, and what it gains.

Forward pass, loss gradient and one Adam step of the CUDA network are compared
with the FP64 NumPy oracle on the same parameters and data (FP32 kernels:
relative tolerances 1e-5 forward, 1e-4 gradient; BF16-weight inference 3e-2);
node features with the oracle's generic restatement.  Then the network is
trained on solves the AMG-PCG path generates and must cut the iteration count
on a held-out problem, while a useless network is caught by the residual
guard and the solve still converges.
"""
import numpy as np
import pytest

from gpu_util import need_gpu, torch
from oracle import mlp as omlp
from paper_1804_10060_gb300 import meshgen

pytestmark = pytest.mark.gpu


def _net(tam, width=16, depth=2, seed=3):
    net = tam.Mlp(8, width, depth, 3, seed=seed)
    rng = np.random.default_rng(seed)
    shift = rng.standard_normal(8).astype(np.float32) * 0.1
    scale = (1.0 + rng.random(8)).astype(np.float32)
    out_scale = np.array([0.5, 2.0, 1.5], np.float32)
    net.set_normalization(shift, scale, out_scale)
    shapes = omlp.layer_shapes(8, width, depth, 3)
    return net, shapes, shift.astype(np.float64), scale.astype(np.float64), out_scale.astype(np.float64)


@pytest.mark.parametrize("width,depth", [(16, 2), (128, 3)])
def test_forward_and_gradient_match_oracle(width, depth):
    tam = need_gpu()
    net, shapes, shift, scale, out_scale = _net(tam, width, depth)
    rng = np.random.default_rng(0)
    n = 3000
    X = rng.standard_normal((n, 8)).astype(np.float32)
    Y = rng.standard_normal((n, 3)).astype(np.float32)
    theta = net.get_params().astype(np.float64)
    Xg, Yg = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    ref, _ = omlp.forward(theta, shapes, X.astype(np.float64), shift, scale, out_scale)
    got = net.forward(Xg).cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max() + 1e-6
    got16 = net.forward(Xg, bf16=True).cpu().numpy()
    assert np.abs(got16 - ref).max() <= 3e-2 * np.abs(ref).max()
    loss_o, g_o = omlp.loss_and_grad(theta, shapes, X.astype(np.float64), Y.astype(np.float64), shift, scale,
                                     out_scale)
    loss_g, g_g = net.loss_grad(Xg, Yg)
    assert abs(loss_g - loss_o) <= 1e-5 * loss_o
    assert np.linalg.norm(g_g - g_o) <= 1e-4 * np.linalg.norm(g_o)


@pytest.mark.parametrize("width,depth,n", [(16, 2, 3000), (128, 3, 4099), (128, 3, 7)])
def test_fused_bf16_inference_equals_layer_by_layer(width, depth, n):
    """The one-kernel BF16 network (activations kept in registers between
    layers) makes the same roundings, products and sums as the layer-by-layer
    BF16 kernels: bitwise equal outputs, ragged last tile included."""
    tam = need_gpu()
    net, shapes, shift, scale, out_scale = _net(tam, width, depth)
    rng = np.random.default_rng(2)
    Xg = torch.from_numpy(rng.standard_normal((n, 8)).astype(np.float32)).cuda()
    fused = net.forward(Xg, bf16=1).cpu().numpy()
    layered = net.forward(Xg, bf16=2).cpu().numpy()
    assert np.array_equal(fused, layered)
    theta = net.get_params().astype(np.float64)
    ref, _ = omlp.forward(theta, shapes, Xg.cpu().numpy().astype(np.float64), shift, scale, out_scale)
    assert np.abs(fused - ref).max() <= 3e-2 * np.abs(ref).max()


def test_adam_step_matches_oracle():
    tam = need_gpu()
    net, shapes, shift, scale, out_scale = _net(tam)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((4096, 8)).astype(np.float32)
    Y = rng.standard_normal((4096, 3)).astype(np.float32)
    theta = net.get_params().astype(np.float64)
    _, g_o = omlp.loss_and_grad(theta, shapes, X.astype(np.float64), Y.astype(np.float64), shift, scale, out_scale)
    lr = 1e-3
    net.train_step(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), lr)
    t1 = net.get_params().astype(np.float64)
    t1_o, _, _ = omlp.adam_step(theta, g_o, np.zeros_like(theta), np.zeros_like(theta), 1, lr)
    big = np.abs(g_o) > 1e-3 * np.abs(g_o).max()   # first Adam step is lr * sign(g): skip near-zero g
    np.testing.assert_allclose(t1[big], t1_o[big], atol=1e-6)


@pytest.mark.parametrize("degree", [1, 2])
def test_node_features_match_oracle(degree):
    tam = need_gpu()
    pb = meshgen.bladed_disc_problem(n_r=6, n_theta_per_blade=4, n_z=2, n_blades=12, n_r_blade=3, degree=degree)
    d = tam.problem_to_device(pb)
    dist = meshgen.clamp_distance(pb)
    F = tam.tam_node_features(d["coords"], d["cells"], d["T"], torch.from_numpy(dist).cuda()).cpu().numpy()
    ref = omlp.node_features(pb.coords, pb.cells, pb.T, dist)
    scale = np.abs(ref).max(axis=0)
    assert np.all(np.abs(F - ref) <= 1e-5 * scale + 1e-6)


def _disc(seed, blades=24, n_r=10, degree=1):
    return meshgen.bladed_disc_problem(n_r=n_r, n_theta_per_blade=4, n_z=3, n_blades=blades, n_r_blade=4,
                                       degree=degree, seed=seed)


# P1 discs of 16,128 DOF; P2 discs (the element of the benchmark's disc) of 72,576 DOF
@pytest.mark.parametrize("degree,n_r", [(1, 10), (2, 6)])
def test_trained_guess_reduces_iterations_and_guard_catches_bad_guess(degree, n_r):
    tam = need_gpu()
    from paper_1804_10060_gb300 import learned
    train = [_disc(s, n_r=n_r, degree=degree) for s in (1, 2, 3, 4)]
    X, Y = learned.training_set(train)
    net = tam.Mlp(8, 64, 3, 3, seed=7)
    net.set_normalization(*learned.normalization(X, Y))
    hist = learned.train(net, X, Y, steps=600, batch=16384, lr=3e-3)
    assert hist[-1] < 0.2 * hist[0]
    res = learned.evaluate(net, _disc(11, n_r=n_r, degree=degree))
    assert res["guess_used"], res
    assert res["rel_resid_guess"] <= 1e-8 and res["solution_diff"] <= 1e-6, res
    assert res["iters_guess"] < res["iters_zero"], res
    # a network that outputs garbage is refused by the residual guard
    bad = tam.Mlp(8, 16, 1, 3, seed=1)
    bad.set_normalization(np.zeros(8), np.ones(8), np.full(3, 1e6))
    res_bad = learned.evaluate(bad, _disc(12, n_r=n_r, degree=degree))
    assert not res_bad["guess_used"]
    assert res_bad["iters_guess"] == res_bad["iters_zero"] and res_bad["rel_resid_guess"] <= 1e-8
