"""Pins of the fp64 network reference (oracle/mlp.py): BF16 rounding against
torch's own conversion, GELU against closed-form values, the cross-entropy
at zero weights, and the analytic gradient against central finite
differences in float64."""
import math

import numpy as np
import pytest

from oracle import mlp


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000).astype(np.float32),
                        np.float32([0.0, -0.0, 1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8),
                                    3.0e38, 1e-40, 65504.0])])
    ours = mlp.bf16_round(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(ours.view(np.uint32), ref.view(np.uint32))
    # ties go to the even neighbour
    assert mlp.bf16_round(np.float32([1 + 2 ** -8]))[0] == 1.0
    assert mlp.bf16_round(np.float32([1 + 3 * 2 ** -8]))[0] == np.float32(1 + 2 ** -6)


def test_gelu_closed_forms():
    x = np.array([0.0, 1.0, -1.0, 2.0, 12.0, -12.0])
    phi = np.array([0.5, 0.8413447460685429, 0.15865525393145707, 0.9772498680518208, 1.0, 0.0])
    assert np.allclose(mlp.gelu(x), x * phi, rtol=0, atol=1e-15)
    # derivative: Phi(x) + x phi(x); at 0 it is 1/2
    assert mlp.gelu_grad(np.array([0.0]))[0] == 0.5
    h = 1e-6
    xs = np.linspace(-4, 4, 33)
    fd = (mlp.gelu(xs + h) - mlp.gelu(xs - h)) / (2 * h)
    assert np.allclose(mlp.gelu_grad(xs), fd, atol=1e-8)


def test_zero_weights_uniform_softmax():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((9, mlp.IN))
    y = rng.integers(0, mlp.OUT, 9)
    loss, g = mlp.loss_and_grad(np.zeros(mlp.P), X, y)
    assert abs(loss - math.log(mlp.OUT)) < 1e-12
    gb3 = mlp.unpack(g)["b3"]
    expect = np.full(mlp.OUT, 1.0 / mlp.OUT) - np.bincount(y, minlength=mlp.OUT) / len(y)
    assert np.allclose(gb3, expect, atol=1e-15)
    # with zero weights nothing reaches the hidden layers
    assert np.all(mlp.unpack(g)["W1"] == 0)


def test_gradient_vs_central_differences():
    rng = np.random.default_rng(2)
    w = mlp.init_params(3).astype(np.float64)
    w += 0.05 * rng.standard_normal(w.size)  # non-zero biases too
    X = rng.standard_normal((7, mlp.IN))
    y = rng.integers(0, mlp.OUT, 7)
    _, g = mlp.loss_and_grad(w, X, y)
    # every tensor: sampled coordinates
    off = 0
    h = 1e-5
    for name, shape in mlp.SHAPES:
        k = int(np.prod(shape))
        idx = off + rng.choice(k, size=min(k, 24), replace=False)
        for i in idx:
            wp = w.copy(); wp[i] += h
            wm = w.copy(); wm[i] -= h
            fd = (mlp.loss_only(wp, X, y) - mlp.loss_only(wm, X, y)) / (2 * h)
            assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(fd), (name, i, fd, g[i])
        off += k
    # one random direction over all parameters
    u = rng.standard_normal(w.size)
    fd = (mlp.loss_only(w + h * u, X, y) - mlp.loss_only(w - h * u, X, y)) / (2 * h)
    assert abs(fd - g @ u) <= 1e-6 * max(1.0, abs(fd))


def test_features_map_box_to_unit_cube():
    rays = np.array([[0, 0, 0, 0, 1, 0, 0, np.inf], [2, 4, 6, 0, 0, 0, 1, np.inf]], np.float32)
    box = np.array([1, 2, 3, 1, 2, 3], np.float64)
    X = mlp.features(rays, box)
    assert np.array_equal(X, [[-1, -1, -1, 1, 0, 0], [1, 1, 1, 0, 0, 1]])


def test_bf16_operand_gradient_is_the_exact_one_within_rounding():
    """The tensor-core reference (every product operand rounded to BF16)
    stays within the BF16 rounding bound of the exact gradient, which is
    pinned by finite differences above: a dropped term, a sign or a
    transposed operand would move a tensor by far more.  Its loss is the
    loss of the BF16-activation logits."""
    rng = np.random.default_rng(17)
    w = mlp.bf16_round(mlp.init_params(17)).astype(np.float64)
    X = np.concatenate([rng.uniform(-1, 1, (300, 3)), rng.normal(size=(300, 3))], 1)
    X[:, 3:] /= np.linalg.norm(X[:, 3:], axis=1, keepdims=True)
    y = rng.integers(0, 256, 300)
    lb, gb = mlp.loss_and_grad_bf16_operands(w, X, y)
    le, ge = mlp.loss_and_grad(w, X, y)
    z = mlp.logits_bf16_activations(w, X)
    m = z.max(1, keepdims=True)
    ref = float(np.mean(np.log(np.exp(z - m).sum(1)) + m[:, 0] - z[np.arange(300), y]))
    assert abs(lb - ref) <= 1e-12 * abs(ref)
    assert abs(lb - le) <= 1e-2 * abs(le)
    db, de = mlp.unpack(gb), mlp.unpack(ge)
    for name, _ in mlp.SHAPES:
        rel = np.linalg.norm(db[name] - de[name]) / np.linalg.norm(de[name])
        assert 0 < rel <= 2e-2, (name, rel)
