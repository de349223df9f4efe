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
    # Each gradient formula is the adjoint of the product in its operand:
    # <dY, A E> = <A^T dY, E> (d op(B)) and <dY, E B> = <dY B^T, E> (d op(A)).
    # Together they give Euler's identity for the bilinear product:
    # <dA, A> + <dB, B> = 2 <dY, A B>.
    rng = np.random.default_rng(1)
    A, E, dY = rng.standard_normal((6, 3)), rng.standard_normal((3, 5)), rng.standard_normal((6, 5))
    _, dB, _ = J.sgemm_grads(A, E, 1.0, 0.0, dY)
    assert np.isclose(np.sum(dY * (A @ E)), np.sum(dB * E), rtol=1e-13)
    F, B = rng.standard_normal((6, 3)), rng.standard_normal((3, 5))
    dA, _, _ = J.sgemm_grads(F, B, 1.0, 0.0, dY)
    assert np.isclose(np.sum(dY * (F @ B)), np.sum(dA * F), rtol=1e-13)
    dA, dB, _ = J.sgemm_grads(A, B, 1.0, 0.0, dY)
    assert np.isclose(np.sum(dA * A) + np.sum(dB * B), 2 * np.sum(dY * (A @ B)), rtol=1e-13)


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


def test_perturbed_chain_backward():
    rng = np.random.default_rng(4)
    rows, w, L = 6, 5, 3
    X = rng.standard_normal((rows, w))
    Ws = [rng.standard_normal((w, w)) / np.sqrt(w) for _ in range(L)]
    G = rng.standard_normal((rows, w))
    dX, dW = J.chain_backward(X, Ws, G)
    # no perturbation: the plain gradients
    pX, pW = J.chain_backward_perturbed(X, Ws, G)
    assert np.array_equal(pX, dX) and all(np.array_equal(a, b) for a, b in zip(pW, dW))
    # an error on the last adjoint product reaches dX unchanged (dX = dH_0)
    D = rng.standard_normal((rows, w))
    qX, _ = J.chain_backward_perturbed(X, Ws, G, dh={0: D})
    assert np.allclose(qX - dX, D, rtol=0, atol=1e-12)
    # an error on dH_1 reaches dX through (1 - H_1^2) and W_0^T
    H, Z, _ = J.chain_forward(X, Ws)
    qX, qW = J.chain_backward_perturbed(X, Ws, G, dh={1: D})
    assert np.allclose(qX - dX, (D * (1 - np.tanh(Z[0]) ** 2)) @ Ws[0].T, rtol=0, atol=1e-12)
    assert np.allclose(qW[0] - dW[0], X.T @ (D * (1 - np.tanh(Z[0]) ** 2)), rtol=0, atol=1e-12)
    # an error on Z_0 is an error on the chain's first tanh input: the same
    # gradients as the unperturbed chain with W_0 changed so that X W_0
    # moves by that error (X square and invertible here)
    Xs = rng.standard_normal((w, w))
    dXs, dWs = J.chain_backward(Xs, Ws, G[:w])
    D2 = 1e-3 * rng.standard_normal((w, w))
    W0 = Ws[0] + np.linalg.solve(Xs, D2)
    _, rW = J.chain_backward(Xs, [W0] + Ws[1:], G[:w])
    _, qW = J.chain_backward_perturbed(Xs, Ws, G[:w], dz={0: D2})
    for a, b in zip(qW[1:], rW[1:]):
        assert np.allclose(a, b, rtol=1e-9, atol=1e-12)


def test_grad_error_bound_holds_for_sampled_errors():
    # The first-order bound must cover product errors of norm eps * ||P||
    # in any direction: sample random and adversarial-looking errors, apply
    # them through chain_backward_perturbed, and compare.
    rng = np.random.default_rng(5)
    rows, w, L = 8, 6, 4
    X = rng.standard_normal((rows, w))
    Ws = [rng.standard_normal((w, w)) / np.sqrt(w) for _ in range(L)]
    G = rng.standard_normal((rows, w))
    eps = 1e-7
    bx, bw = J.chain_grad_error_bound(X, Ws, G, eps)
    dX, dW = J.chain_backward(X, Ws, G)
    H, Z, _ = J.chain_forward(X, Ws)
    dZ = G
    dHs = {}
    for l in range(L - 1, -1, -1):
        dHs[l] = dZ @ Ws[l].T
        if l > 0:
            dZ = dHs[l] * (1 - np.tanh(Z[l - 1]) ** 2)
    worst = 0.0
    for trial in range(50):
        dz = {l: rng.standard_normal(Z[l].shape) for l in range(L - 1)}
        dh = {l: rng.standard_normal(dHs[l].shape) for l in range(L)}
        if trial % 2:  # all errors of one sign pattern, aligned with the results
            dz = {l: np.sign(Z[l]) for l in dz}
            dh = {l: np.sign(dHs[l]) for l in dh}
        dz = {l: v * eps * np.linalg.norm(Z[l]) / np.linalg.norm(v) for l, v in dz.items()}
        dh = {l: v * eps * np.linalg.norm(dHs[l]) / np.linalg.norm(v) for l, v in dh.items()}
        qX, _ = J.chain_backward_perturbed(X, Ws, G, dz=dz, dh=dh)
        worst = max(worst, np.linalg.norm(qX - dX) / np.linalg.norm(dX))
    assert 0 < worst <= bx, (worst, bx)
    assert all(b >= eps for b in bw)


def test_forward_error_bound():
    rng = np.random.default_rng(6)
    rows, w, L = 8, 6, 4
    X = rng.standard_normal((rows, w))
    Ws = [rng.standard_normal((w, w)) / np.sqrt(w) for _ in range(L)]
    H, Z, Y = J.chain_forward(X, Ws)
    assert np.array_equal(J.chain_forward_perturbed(X, Ws), Y)
    # an error on the last product is an error on Y itself
    D = rng.standard_normal(Y.shape)
    assert np.allclose(J.chain_forward_perturbed(X, Ws, {L - 1: D}) - Y, D, rtol=0, atol=1e-12)
    eps = 1e-7
    b = J.chain_forward_error_bound(X, Ws, eps)
    assert b >= eps  # at least the last product's own error
    worst = 0.0
    for _ in range(50):
        dz = {l: rng.standard_normal(Z[l].shape) for l in range(L)}
        dz = {l: v * eps * np.linalg.norm(Z[l]) / np.linalg.norm(v) for l, v in dz.items()}
        worst = max(worst, np.linalg.norm(J.chain_forward_perturbed(X, Ws, dz) - Y) / np.linalg.norm(Y))
    assert 0 < worst <= b
