"""FP64 gradients of the sgemm leaf and of the tanh-separated sgemm chain.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper has no differentiation; these are the plain chain-rule adjoints of
its sgemm leaf (Section 6.1) and of a chain of such leaves joined by
elementwise tanh leaves over streaming edges (Section 2.1 streaming edges;
Section 3.5 pipelining). A matrix product from numpy serves as a step.

sgemm leaf, Y = alpha*op(A)*op(B) + beta*C, upstream gradient dY:
    d op(A) = alpha * dY * op(B)^T,   d op(B) = alpha * op(A)^T * dY,
    dC = beta * dY,
and dA = d op(A) (or its transpose when op(A) = A^T), likewise for B.

chain (row-major items X of shape rows x w, weights W_l of shape w x w):
    Z_0 = X W_0,  Z_l = tanh(Z_{l-1}) W_l (l = 1..L-1),  Y = Z_{L-1},
    loss = sum(Y * G) for a fixed upstream G;
    dZ_{L-1} = G,  dW_l = H_l^T dZ_l with H_0 = X, H_l = tanh(Z_{l-1}),
    dH_l = dZ_l W_l^T,  dZ_{l-1} = dH_l * (1 - tanh(Z_{l-1})^2),  dX = dH_0.
"""
from __future__ import annotations

import numpy as np


def sgemm_grads(opA, opB, alpha, beta, dY):
    """Gradients w.r.t. op(A) (M x K), op(B) (K x N) and C (M x N)."""
    opA = np.asarray(opA, np.float64)
    opB = np.asarray(opB, np.float64)
    dY = np.asarray(dY, np.float64)
    return alpha * (dY @ opB.T), alpha * (opA.T @ dY), beta * dY


def chain_forward(X, Ws):
    """Activations of the chain: returns (H list, Z list, Y)."""
    H = [np.asarray(X, np.float64)]
    Z = []
    for l, W in enumerate(Ws):
        z = H[-1] @ np.asarray(W, np.float64)
        Z.append(z)
        if l + 1 < len(Ws):
            H.append(np.tanh(z))
    return H, Z, Z[-1]


def chain_loss(X, Ws, G) -> float:
    _, _, Y = chain_forward(X, Ws)
    return float(np.sum(Y * np.asarray(G, np.float64)))


def chain_backward(X, Ws, G):
    """Gradients of sum(Y * G) w.r.t. X and every W_l (FP64)."""
    H, Z, _ = chain_forward(X, Ws)
    L = len(Ws)
    dW = [None] * L
    dZ = np.asarray(G, np.float64)
    dX = None
    for l in range(L - 1, -1, -1):
        W = np.asarray(Ws[l], np.float64)
        dW[l] = H[l].T @ dZ
        dH = dZ @ W.T
        if l == 0:
            dX = dH
        else:
            t = np.tanh(Z[l - 1])
            dZ = dH * (1.0 - t * t)
    return dX, dW


def chain_backward_perturbed(X, Ws, G, dz=None, dh=None):
    """chain_backward with an additive error on the result of each product
    that the gradients read: dz[l] is added to Z_l = H_l W_l (l = 0..L-2; the
    product of Y does not reach the gradients, since its adjoint is the
    given G), dh[l] to dH_l = dZ_l W_l^T (l = 0..L-1). Missing entries (or
    None) add nothing. Perturbations may carry leading batch dimensions
    (one gradient per perturbation), which broadcast through every step.
    Returns (dX, [dW_l])."""
    dz = dz or {}
    dh = dh or {}
    Xd = np.asarray(X, np.float64)
    W64 = [np.asarray(W, np.float64) for W in Ws]
    L = len(W64)
    Hs = [Xd]
    Zs = []
    for l in range(L - 1):
        z = Hs[-1] @ W64[l]
        if l in dz:
            z = z + dz[l]
        Zs.append(z)
        Hs.append(np.tanh(z))
    dW = [None] * L
    dZ = np.asarray(G, np.float64)
    dX = None
    for l in range(L - 1, -1, -1):
        dW[l] = np.swapaxes(Hs[l], -1, -2) @ dZ
        dH = dZ @ W64[l].T
        if l in dh:
            dH = dH + dh[l]
        if l == 0:
            dX = dH
        else:
            t = np.tanh(Zs[l - 1])
            dZ = dH * (1.0 - t * t)
    return dX, dW


def chain_grad_error_bound(X, Ws, G, eps: float):
    """First-order normwise bound on the gradients of a chain whose every
    product result P_p carries an error of at most eps * ||P_p||_F (the
    per-product bound a leaf meets): with J_p the Jacobian of a gradient
    with respect to P_p,
        ||error of dX||_F <= eps * sum_p ||J_p||_2 ||P_p||_F,
    and for dW_l the same sum plus eps * ||dW_l||_F (its own product).
    J_p is formed column by column with central differences through
    chain_backward_perturbed (exact for the adjoint products, on which the
    gradients depend linearly) and its 2-norm taken by SVD. Meant for small
    chains (a J_p has (rows*w)^2 entries). Returns (bound for dX, [bound for
    dW_l]), each relative to the gradient's FP64 norm."""
    Xd = np.asarray(X, np.float64)
    W64 = [np.asarray(W, np.float64) for W in Ws]
    L = len(W64)
    dX0, dW0 = chain_backward(Xd, W64, G)
    H, Z, _ = chain_forward(Xd, W64)
    # the products the gradients read, and their exact results
    prods = [("z", l, Z[l]) for l in range(L - 1)]
    dZ = np.asarray(G, np.float64)
    for l in range(L - 1, -1, -1):
        dH = dZ @ W64[l].T
        prods.append(("h", l, dH))
        if l > 0:
            t = np.tanh(Z[l - 1])
            dZ = dH * (1.0 - t * t)
    sx = 0.0
    sw = [0.0] * L
    for kind, l, P in prods:
        n = P.size
        basis = np.eye(n).reshape((n,) + P.shape)
        step = 1e-6 * max(1.0, float(np.sqrt(np.mean(P * P))))
        plus = chain_backward_perturbed(Xd, W64, G, **{("dz" if kind == "z" else "dh"): {l: step * basis}})
        minus = chain_backward_perturbed(Xd, W64, G, **{("dz" if kind == "z" else "dh"): {l: -step * basis}})
        Pn = float(np.linalg.norm(P))
        Jx = ((plus[0] - minus[0]) / (2 * step)).reshape(n, -1).T
        sx += np.linalg.norm(Jx, 2) * Pn
        for k in range(L):
            d = plus[1][k] - minus[1][k]
            if d.ndim < 3:  # a gradient computed before the perturbed product: unchanged
                continue
            Jw = (d / (2 * step)).reshape(n, -1).T
            sw[k] += np.linalg.norm(Jw, 2) * Pn
    bx = eps * sx / float(np.linalg.norm(dX0))
    bw = [eps * (sw[k] + float(np.linalg.norm(dW0[k]))) / float(np.linalg.norm(dW0[k])) for k in range(L)]
    return bx, bw


def chain_forward_perturbed(X, Ws, dz=None):
    """The chain's output Y with dz[l] added to the result of product l,
    Z_l = H_l W_l (l = 0..L-1, Y = Z_{L-1}); perturbations may carry
    leading batch dimensions."""
    dz = dz or {}
    Hm = np.asarray(X, np.float64)
    L = len(Ws)
    for l in range(L):
        z = Hm @ np.asarray(Ws[l], np.float64)
        if l in dz:
            z = z + dz[l]
        if l + 1 == L:
            return z
        Hm = np.tanh(z)


def chain_forward_error_bound(X, Ws, eps: float) -> float:
    """First-order normwise bound on the chain's output Y when each product
    result Z_l carries an error of at most eps * ||Z_l||_F:
    eps * sum_l ||dY/dZ_l||_2 ||Z_l||_F / ||Y||_F, the Jacobians by central
    differences through chain_forward_perturbed (the last one is the
    identity). Meant for small chains."""
    Xd = np.asarray(X, np.float64)
    _, Z, Y = chain_forward(Xd, Ws)
    s = 0.0
    for l, P in enumerate(Z):
        n = P.size
        basis = np.eye(n).reshape((n,) + P.shape)
        step = 1e-6 * max(1.0, float(np.sqrt(np.mean(P * P))))
        d = chain_forward_perturbed(Xd, Ws, {l: step * basis}) - chain_forward_perturbed(Xd, Ws, {l: -step * basis})
        Jl = (d / (2 * step)).reshape(n, -1).T
        s += np.linalg.norm(Jl, 2) * float(np.linalg.norm(P))
    return eps * s / float(np.linalg.norm(Y))
