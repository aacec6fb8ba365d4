"""NumPy reference of the learned coarse correction's network: forward, backward, Adam.

TEST INFRASTRUCTURE ONLY (see the package docstring). The paper has no learned component;
this restates, in FP64, the two-hidden-layer ReLU perceptron that the CUDA path trains, so that
its gradients and updates can be checked:

    h1 = relu(W1 x + b1),  h2 = relu(W2 h1 + b2),  y = W3 h2 + b3,
    loss = 1/(2B) sum_b ||y_b - t_b||^2

with weights stored [out][in] and a batch of B samples in rows. Adam follows Kingma & Ba
(2015): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2, step lr m^ / (sqrt(v^) + eps) with the
bias corrections m^ = m / (1 - b1^t), v^ = v / (1 - b2^t).

Per-mode coarse map (the data the network is trained on): for a spectral mode with Jhat
diagonal mu, the coarse operator G = h S_0(mu) = Z_t^T T(mu) Z_t (T = Jhat Jhat^T in time,
Eq 14 and the definition of S_0 after it) is formed densely, and the target is the unit vector
along G^{-1} c for a coarse right-hand side c = Z_t^T r (the restriction R_0 of Eq 14 for one
mode's time series r).

Coarse-residual loss (the quantity the learned correction's guard tests): for a network
output d and a normalised coarse right-hand side c, the correction is alpha d with the
minimal-residual step alpha = (G d)^T c / ||G d||^2, and the loss of the sample is the squared
relative coarse residual ||c - alpha G d||^2 / ||c||^2 = 1 - cos^2(G d, c). With g = G d and
r = c - alpha g its gradient is dL/dd = -2 alpha G r / ||c||^2 (G symmetric).
"""

from __future__ import annotations

import numpy as np

from .schwarz import SchurPreconditioner


def init_params(d_in: int, width: int, d_out: int, seed: int) -> dict:
    """He-normal weights, zero biases (the CUDA side is given the same arrays)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return {
        "W1": rng.standard_normal((width, d_in)) * np.sqrt(2.0 / d_in), "b1": np.zeros(width),
        "W2": rng.standard_normal((width, width)) * np.sqrt(2.0 / width), "b2": np.zeros(width),
        "W3": rng.standard_normal((d_out, width)) * np.sqrt(2.0 / width), "b3": np.zeros(d_out),
    }


def forward(params: dict, X: np.ndarray):
    a1 = X @ params["W1"].T + params["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ params["W2"].T + params["b2"]
    h2 = np.maximum(a2, 0.0)
    Y = h2 @ params["W3"].T + params["b3"]
    return Y, (X, a1, h1, a2, h2)


def loss(Y: np.ndarray, T: np.ndarray) -> float:
    return 0.5 * float(np.sum((Y - T) ** 2)) / Y.shape[0]


def backward(params: dict, cache, Y: np.ndarray, T: np.ndarray) -> dict:
    """Gradients of `loss` with respect to every parameter (chain rule written out)."""
    return backward_from(params, cache, (Y - T) / Y.shape[0])


def backward_from(params: dict, cache, dY: np.ndarray) -> dict:
    """Gradients of any loss with respect to every parameter, given dY = dloss/dY."""
    X, a1, h1, a2, h2 = cache
    g = {"W3": dY.T @ h2, "b3": dY.sum(axis=0)}
    dh2 = (dY @ params["W3"]) * (a2 > 0)
    g["W2"] = dh2.T @ h1
    g["b2"] = dh2.sum(axis=0)
    dh1 = (dh2 @ params["W2"]) * (a1 > 0)
    g["W1"] = dh1.T @ X
    g["b1"] = dh1.sum(axis=0)
    return g


def adam_step(params: dict, grads: dict, state: dict, t: int, lr: float, b1: float = 0.9, b2: float = 0.999,
              eps: float = 1e-8) -> None:
    """One Adam update in place; state holds m and v per parameter (created on first use)."""
    for k in params:
        m = state.setdefault("m_" + k, np.zeros_like(params[k]))
        v = state.setdefault("v_" + k, np.zeros_like(params[k]))
        m *= b1
        m += (1 - b1) * grads[k]
        v *= b2
        v += (1 - b2) * grads[k] ** 2
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        params[k] -= lr * mh / (np.sqrt(vh) + eps)


def coarse_operator(mu: float, Nt: int, n_sub: int, pou: str = "left") -> np.ndarray:
    """h S_0(mu) for one mode: Z_t^T (Jhat Jhat^T) Z_t with Jhat the scalar time-stepping matrix."""
    pre = SchurPreconditioner(np.array([[mu]]), Nt, n_sub, 1.0, pou=pou)
    return pre.coarse_matrix().toarray()


def coarse_restriction(Nt: int, n_sub: int, pou: str = "left") -> np.ndarray:
    """Z_t (Nt x 2 n_sub) for one mode: column 2s is subdomain s's constant, 2s+1 its linear
    function on the nodes it owns (Eq 14), so R_0 r = Z_t^T r for a time series r."""
    pre = SchurPreconditioner(np.array([[1.0]]), Nt, n_sub, 1.0, pou=pou)
    return pre.Z.toarray()


def coarse_data(r: np.ndarray, mu: np.ndarray, Nt: int, n_sub: int) -> tuple[np.ndarray, np.ndarray]:
    """Training pairs of the learned correction: per sample b (a column of r, [Nt][S]),
    c_b = Z_t^T r_b and x_b = G(mu_b)^{-1} c_b (dense solve)."""
    Zt = coarse_restriction(Nt, n_sub)
    C = (Zt.T @ r).T
    X = np.stack([np.linalg.solve(coarse_operator(float(m), Nt, n_sub), c) for m, c in zip(mu, C)])
    return C, X


def coarse_residual_loss(D: np.ndarray, C: np.ndarray, G: list) -> tuple[float, np.ndarray]:
    """Mean over the batch of ||c - alpha G d||^2 / ||c||^2 with the minimal-residual alpha,
    and its gradient with respect to D (rows d_b, c_b; G[b] the sample's coarse operator)."""
    B = D.shape[0]
    total, dD = 0.0, np.zeros_like(D)
    for b in range(B):
        d, c, Gb = D[b], C[b], G[b]
        g = Gb @ d
        cc = c @ c
        gg = g @ g
        if gg == 0.0:
            total += 1.0
            continue
        alpha = (g @ c) / gg
        r = c - alpha * g
        total += (r @ r) / cc
        dD[b] = -2.0 * alpha * (Gb @ r) / cc / B
    return total / B, dD
