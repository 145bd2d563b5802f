"""The FP64 reference network against what calculus fixes: central finite
differences of the loss, the loss of uniform logits, and probabilities that
sum to one."""
import math

import numpy as np

from oracle import mlp_oracle as M


def _setup(seed=0, n_in=7, hidden=9, classes=5, n=11):
    rng = np.random.default_rng(seed)
    p = rng.standard_normal(M.param_count(n_in, hidden, classes)) * 0.5
    X = rng.standard_normal((n, n_in))
    y = rng.integers(0, classes, size=n)
    return p, X, y, (n_in, hidden, classes)


def test_gradient_matches_finite_differences():
    p, X, y, dims = _setup()
    loss, g = M.loss_and_grad(p, X, y, *dims)
    rng = np.random.default_rng(1)
    idx = rng.choice(p.size, size=60, replace=False)
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (M.loss_and_grad(pp, X, y, *dims)[0] - M.loss_and_grad(pm, X, y, *dims)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_uniform_logits_loss_is_log_classes():
    n_in, hidden, classes = 4, 6, 7
    p = np.zeros(M.param_count(n_in, hidden, classes))
    X = np.random.default_rng(2).standard_normal((5, n_in))
    loss, g = M.loss_and_grad(p, X, np.arange(5) % classes, n_in, hidden, classes)
    assert abs(loss - math.log(classes)) < 1e-12


def test_probabilities_sum_to_one():
    p, X, y, dims = _setup(seed=3)
    P = M.predict_proba(p, X, *dims)
    assert np.allclose(P.sum(axis=1), 1.0) and np.all(P > 0)


def test_probabilities_match_the_loss():
    """The forward pass the tensor-core test compares with is the one whose
    loss the finite differences pin: mean(-log P[i, y_i]) equals the loss."""
    p, X, y, dims = _setup(seed=4)
    P = M.predict_proba(p, X, *dims)
    loss, _ = M.loss_and_grad(p, X, y, *dims)
    assert abs(-np.mean(np.log(P[np.arange(len(y)), y])) - loss) < 1e-12


def test_identity_network_closed_form():
    """W1 = W2 = W3 = I, zero biases: the logits are ReLU(x), so the
    probabilities are softmax(max(x, 0)) -- with the ReLU visible on a
    negative input."""
    n_in = hidden = classes = 3
    eye = np.eye(3)
    p = np.concatenate([eye.ravel(), np.zeros(3), eye.ravel(), np.zeros(3), eye.ravel(),
                        np.zeros(3)])
    X = np.array([[0.5, -2.0, 1.5], [3.0, 1.0, -0.25]])
    z = np.maximum(X, 0.0)
    want = np.exp(z) / np.exp(z).sum(axis=1, keepdims=True)
    assert np.allclose(M.predict_proba(p, X, n_in, hidden, classes), want, rtol=0, atol=1e-15)
