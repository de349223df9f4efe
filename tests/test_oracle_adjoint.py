"""Pins of the oracle's FP64 gradients (CPU only): central finite differences
and the transpose (adjoint) identity."""
import numpy as np

from oracle import adjoint as J


def test_sgemm_grads_match_finite_differences():
    rng = np.random.default_rng(0)
    M, N, K = 5, 4, 6
    A, B, C = rng.standard_normal((M, K)), rng.standard_normal((K, N)), rng.standard_normal((M, N))
    G = rng.standard_normal((M, N))
    alpha, beta = 1.5, -0.5

    def loss(A_, B_, C_):
        return float(np.sum((alpha * A_ @ B_ + beta * C_) * G))

    dA, dB, dC = J.sgemm_grads(A, B, alpha, beta, G)
    h = 1e-6
    for X, dX, which in [(A, dA, 0), (B, dB, 1), (C, dC, 2)]:
        E = rng.standard_normal(X.shape)
        args_p = [A, B, C]
        args_m = [A, B, C]
        args_p[which] = X + h * E
        args_m[which] = X - h * E
        fd = (loss(*args_p) - loss(*args_m)) / (2 * h)
        assert abs(fd - np.sum(dX * E)) <= 1e-7 * max(1.0, abs(fd))


def test_adjoint_identity():
    # <dY, op(A) E> = <op(A)^T dY, E>: the d op(B) formula is the adjoint of X -> op(A) X
    rng = np.random.default_rng(1)
    A, E, dY = rng.standard_normal((6, 3)), rng.standard_normal((3, 5)), rng.standard_normal((6, 5))
    _, dB, _ = J.sgemm_grads(A, E, 1.0, 0.0, dY)
    assert np.isclose(np.sum(dY * (A @ E)), np.sum(dB * E), rtol=1e-13)


def test_chain_grads_match_finite_differences():
    # the 24 x 16 copy of the streamed chain: 4 sgemm leaves, tanh between them
    rng = np.random.default_rng(2)
    rows, w, L = 24, 16, 4
    X = rng.standard_normal((rows, w))
    Ws = [rng.standard_normal((w, w)) / np.sqrt(w) for _ in range(L)]
    G = rng.standard_normal((rows, w))
    dX, dW = J.chain_backward(X, Ws, G)
    h = 1e-6
    E = rng.standard_normal(X.shape)
    fd = (J.chain_loss(X + h * E, Ws, G) - J.chain_loss(X - h * E, Ws, G)) / (2 * h)
    assert abs(fd - np.sum(dX * E)) <= 1e-6 * max(1.0, abs(fd))
    for l in range(L):
        E = rng.standard_normal(Ws[l].shape)
        Wp = [w_.copy() for w_ in Ws]
        Wm = [w_.copy() for w_ in Ws]
        Wp[l] += h * E
        Wm[l] -= h * E
        fd = (J.chain_loss(X, Wp, G) - J.chain_loss(X, Wm, G)) / (2 * h)
        assert abs(fd - np.sum(dW[l] * E)) <= 1e-6 * max(1.0, abs(fd))


def test_chain_without_tanh_is_a_product():
    # with one layer the chain is a plain product and dW = X^T G
    rng = np.random.default_rng(3)
    X, W, G = rng.standard_normal((4, 3)), rng.standard_normal((3, 3)), rng.standard_normal((4, 3))
    _, _, Y = J.chain_forward(X, [W])
    assert np.allclose(Y, X @ W)
    dX, dW = J.chain_backward(X, [W], G)
    assert np.allclose(dW[0], X.T @ G) and np.allclose(dX, G @ W.T)
