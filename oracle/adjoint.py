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
