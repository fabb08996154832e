"""FP64 reference of the warm-start network: forward pass and back-propagated
gradient of the mean squared error, written out with the chain rule.

TEST INFRASTRUCTURE ONLY (checks the library's MLP kernels; see oracle.py).
Network: x (8) -> tanh(W1 x + b1) (64) -> tanh(W2 h1 + b2) (64) -> W3 h2 + b3.
Flat parameter layout: W1[64][8], b1[64], W2[64][64], b2[64], W3[64], b3.
"""
import numpy as np

IN, H = 8, 64
NPARAM = H * IN + H + H * H + H + H + 1


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    i = 0
    W1 = p[i:i + H * IN].reshape(H, IN); i += H * IN
    b1 = p[i:i + H]; i += H
    W2 = p[i:i + H * H].reshape(H, H); i += H * H
    b2 = p[i:i + H]; i += H
    W3 = p[i:i + H]; i += H
    b3 = p[i]
    return W1, b1, W2, b2, W3, b3


def forward(p, X):
    W1, b1, W2, b2, W3, b3 = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return h2 @ W3 + b3


def round_bf16(a):
    """Round to the nearest bfloat16 (8-bit significand), ties to even, by bit
    arithmetic on the float32 representation; returned as float64."""
    b = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward_bf16_hidden(p, X):
    """The network with the hidden layer's operands (tanh(h1) in float32, and
    W2) rounded to bfloat16 and the products summed exactly: what a BF16
    tensor-core product with a wide accumulator computes for that layer."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.tanh((X.astype(np.float32) @ W1.T.astype(np.float32) + b1.astype(np.float32)).astype(np.float64))
    h2 = np.tanh(round_bf16(h1) @ round_bf16(W2).T + b2)
    return h2 @ W3 + b3


def loss_and_grad(p, X, T):
    """L = mean (y - t)^2 and dL/dp by reverse-mode differentiation."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    n = X.shape[0]
    a1 = X @ W1.T + b1
    h1 = np.tanh(a1)
    a2 = h1 @ W2.T + b2
    h2 = np.tanh(a2)
    y = h2 @ W3 + b3
    e = y - T
    L = float(np.mean(e * e))
    dy = 2.0 * e / n                       # dL/dy
    gW3 = h2.T @ dy
    gb3 = dy.sum()
    da2 = np.outer(dy, W3) * (1.0 - h2 * h2)
    gW2 = da2.T @ h1
    gb2 = da2.sum(axis=0)
    da1 = (da2 @ W2) * (1.0 - h1 * h1)
    gW1 = da1.T @ X
    gb1 = da1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, [gb3]])
    return L, g
