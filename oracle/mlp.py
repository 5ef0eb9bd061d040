"""Learned initial guess, FP64 reference (oracle).  TEST INFRASTRUCTURE ONLY.

The paper's initial guess is the KL/gPC surrogate (Algorithm 3, step 6); the
workload adds a learned alternative with the same role: an MLP maps the KL
coefficients xi to the coarse state at all N coarse times, sampled at 64
interior points, and is upsampled to the grid to form U^0.

  architecture  M -> 256 -> 256 -> 256 -> 64 N, ReLU on the hidden layers
  parameters    flat FP32/FP64 vector [W1, b1, W2, b2, W3, b3, W4, b4],
                W_l stored [out][in] row-major
  targets       U*(xi) at x_m = (m+1)/65, m = 0..63, normalized per output
                column: t = (y - mean) / std
  loss          mean of the squared error over batch and outputs
  optimizer     Adam (Kingma & Ba): m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
                w <- w - lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)
  grid maps     linear interpolation with the zero Dirichlet values at x = 0, 1
"""
from __future__ import annotations

import numpy as np

N_POINTS = 64


def layer_sizes(M: int, N: int, width: int = 256):
    return [M, width, width, width, N_POINTS * N]


def n_params(sizes) -> int:
    return sum(o * i + o for i, o in zip(sizes[:-1], sizes[1:]))


def unflatten(theta: np.ndarray, sizes):
    out, k = [], 0
    for i, o in zip(sizes[:-1], sizes[1:]):
        W = theta[k:k + o * i].reshape(o, i)
        k += o * i
        b = theta[k:k + o]
        k += o
        out.append((W, b))
    return out


def init_params(sizes, seed: int) -> np.ndarray:
    """He-normal weights N(0, 2/fan_in), zero biases, as one flat vector."""
    rng = np.random.default_rng(seed)
    parts = []
    for i, o in zip(sizes[:-1], sizes[1:]):
        parts.append(rng.standard_normal(o * i) * np.sqrt(2.0 / i))
        parts.append(np.zeros(o))
    return np.concatenate(parts)


def forward(theta, sizes, X):
    """Returns (pre-activations Z_l, activations A_l with A_0 = X, output)."""
    layers = unflatten(theta, sizes)
    A, Zs, As = np.asarray(X, dtype=np.float64), [], []
    for l, (W, b) in enumerate(layers):
        As.append(A)
        Z = A @ W.T + b
        Zs.append(Z)
        A = np.maximum(Z, 0.0) if l < len(layers) - 1 else Z
    return Zs, As, A


def loss_and_grad(theta, sizes, X, T):
    """Mean squared error and its gradient (flat, same layout as theta)."""
    layers = unflatten(theta, sizes)
    Zs, As, Y = forward(theta, sizes, X)
    R = Y - T
    loss = float(np.mean(R ** 2))
    dA = 2.0 * R / R.size
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        dZ = dA if l == len(layers) - 1 else dA * (Zs[l] > 0)
        W, _ = layers[l]
        grads[l] = (dZ.T @ As[l], dZ.sum(axis=0))
        dA = dZ @ W
    flat = np.concatenate([np.concatenate([g[0].ravel(), g[1]]) for g in grads])
    return loss, flat


class Adam:
    def __init__(self, n, lr, b1=0.9, b2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps

    def step(self, theta, g, lr=None):
        self.t += 1
        lr = self.lr if lr is None else lr
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return theta - lr * mh / (np.sqrt(vh) + self.eps)


def coarse_points() -> np.ndarray:
    return (np.arange(N_POINTS) + 1) / (N_POINTS + 1)


def downsample(U: np.ndarray) -> np.ndarray:
    """[..., nx] grid values (zero at x=0,1) -> [..., 64] at x_m = (m+1)/65."""
    U = np.asarray(U, dtype=np.float64)
    nx = U.shape[-1]
    xg = np.arange(nx + 2) / (nx + 1)
    flat = U.reshape(-1, nx)
    out = np.empty((flat.shape[0], N_POINTS))
    for r in range(flat.shape[0]):
        out[r] = np.interp(coarse_points(), xg, np.concatenate([[0.0], flat[r], [0.0]]))
    return out.reshape(U.shape[:-1] + (N_POINTS,))


def upsample(Y: np.ndarray, nx: int) -> np.ndarray:
    """[..., 64] -> [..., nx] on x_i = i/(nx+1), zero values at x = 0, 1."""
    Y = np.asarray(Y, dtype=np.float64)
    xc = np.concatenate([[0.0], coarse_points(), [1.0]])
    xg = np.arange(1, nx + 1) / (nx + 1)
    flat = Y.reshape(-1, N_POINTS)
    out = np.empty((flat.shape[0], nx))
    for r in range(flat.shape[0]):
        out[r] = np.interp(xg, xc, np.concatenate([[0.0], flat[r], [0.0]]))
    return out.reshape(Y.shape[:-1] + (nx,))
