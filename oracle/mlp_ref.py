"""FP64 reference of the warm-start network: forward pass and back-propagated
gradient of the mean squared error, written out with the chain rule; the
per-bead features, training targets and the guess built from the network's
output, from the definitions the library's header states.

TEST INFRASTRUCTURE ONLY (checks the library's MLP kernels; see oracle.py).
Network: x (12) -> tanh(W1 x + b1) (64) -> tanh(W2 h1 + b2) (64) -> W3 h2 + b3.
Flat parameter layout: W1[64][IN], b1[64], W2[64][64], b2[64], W3[64], b3.
"""
import math

import numpy as np

IN, H = 12, 64
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


# ---------------------------------------------------------------------------
# Warm-start features and targets, from their definitions (the learned warm start
# is not part of the paper: the definitions are the library's own, restated here
# term by term with plain loops over bodies and beads, in FP64)
# ---------------------------------------------------------------------------

def body_field_of_fixed_charges(x, X, body_offsets, Q, box, a, eps):
    """phi [n] and Es [n,3] at the beads of every multi-bead body b: potential and
    field of the fixed charges (an ion's own charge, Q/N on a bead of another
    multi-bead body) of the beads of OTHER bodies whose minimum image lies within
    R_max + 6R of b's reference point, with the regularised free-space kernel of
    Sec. II, M(r) = 1/(4 pi r) for r >= 2a and (4a - r)/(16 pi a^2) below, over eps.
    Zero on single-bead bodies."""
    from .oracle import body_index, min_image, relative_positions
    x = np.asarray(x, dtype=np.float64)
    off = np.asarray(body_offsets, dtype=np.int64)
    bid = body_index(off)
    counts = np.diff(off)
    qfix = np.asarray(Q, dtype=np.float64)[bid] / counts[bid]
    rel = relative_positions(x, X, off, box)
    Xb = np.asarray(X, dtype=np.float64)
    n = len(x)
    phi = np.zeros(n)
    Es = np.zeros((n, 3))
    for b in range(len(off) - 1):
        s, e = off[b], off[b + 1]
        if e - s < 2:
            continue
        rn = np.linalg.norm(rel[s:e], axis=1)
        cut = rn.max() + 6.0 * rn.mean()
        d = min_image(x - Xb[b], box)                  # sources relative to the reference point
        src = np.nonzero((np.linalg.norm(d, axis=1) < cut) & (bid != b) & (qfix != 0.0))[0]
        qs, ds = qfix[src], d[src]
        for j in range(s, e):
            v = rel[j] - ds                            # x_j - x_beta, one row per source
            r = np.sqrt(np.sum(v * v, axis=1))
            out = r >= 2.0 * a
            # M(r) and -dM/dr: 1/(4 pi r), 1/(4 pi r^2) outside 2a; (4a - r)/(16 pi a^2), 1/(16 pi a^2) inside
            M = np.where(out, 1.0 / (4.0 * math.pi * np.maximum(r, 2.0 * a)), (4.0 * a - r) / (16.0 * math.pi * a * a))
            g = np.where(out, 1.0 / (4.0 * math.pi * np.maximum(r, 2.0 * a) ** 2), 1.0 / (16.0 * math.pi * a * a))
            phi[j] = np.sum(qs * M)
            unit = v / np.where(r > 0.0, r, 1.0)[:, None]
            Es[j] = np.sum((qs * g)[:, None] * unit, axis=0)
    return phi / eps, Es / eps


def warm_start_features(x, X, body_offsets, Q, E0, box, a, eps):
    """Features [n][IN] of every bead (zeros on single-bead bodies) and the body
    scales S [n_bodies] for one field E0, as the header of the library defines
    them (geometry of the body's own beads, E0, the net charges and the
    potential and field of the other bodies' fixed charges near the body)."""
    from .oracle import relative_positions
    x = np.asarray(x, dtype=np.float64)
    E0 = np.asarray(E0, dtype=np.float64).reshape(3)
    off = np.asarray(body_offsets, dtype=np.int64)
    Q = np.asarray(Q, dtype=np.float64)
    rel = relative_positions(x, X, off, box)
    phi, Es = body_field_of_fixed_charges(x, X, off, Q, box, a, eps)
    n = len(x)
    F = np.zeros((n, IN))
    S_body = np.zeros(len(off) - 1)
    for b in range(len(off) - 1):
        s, e = off[b], off[b + 1]
        N = e - s
        if N < 2:
            continue
        rb = rel[s:e]
        rn = np.sqrt(np.sum(rb * rb, axis=1))
        R = rn.mean()
        A = 4.0 * math.pi * R * R / N
        h = math.sqrt(A)
        pb = phi[s:e]
        pm = pb.mean()
        Eb = Es[s:e]
        rE = rb @ E0
        rEm = rE.mean()
        S = eps * A * (np.linalg.norm(E0) + math.sqrt(np.mean(np.sum(Eb * Eb, axis=1))))
        S_body[b] = S
        if not S > 0.0:
            continue
        k = min(6, N - 1)
        for i in range(N):
            d = np.delete(rb - rb[i], i, axis=0)        # x_k - x_j over the body's other beads
            d2 = np.sum(d * d, axis=1)
            dist = np.sort(np.sqrt(d2))
            d1, dk = dist[0], dist[k - 1]
            w = np.exp(-d2 / (h * h))
            W = w.sum()
            m = (w[:, None] * d).sum(axis=0) / W
            s2 = (w * d2).sum() / W
            Cw = (w[:, None, None] * d[:, :, None] * d[:, None, :]).sum(axis=0) / W
            nv = np.linalg.eigh(Cw)[1][:, 0]                  # smallest eigenvalue's vector
            if nv @ rb[i] < 0.0:
                nv = -nv
            kappa = -2.0 * (m @ nv) / s2
            En = E0 @ nv
            Sn = Eb[i] @ nv
            f = F[s + i]
            f[0] = eps * A * En / S
            f[1] = eps * A * np.linalg.norm(E0 - En * nv) / S
            f[2] = eps * A * (rE[i] - rEm) / (R * S)
            f[3] = eps * A * (pb[i] - pm) / (R * S)
            f[4] = eps * A * Sn / S
            f[5] = eps * A * np.linalg.norm(Eb[i] - Sn * nv) / S
            f[6] = kappa * R
            f[7] = rn[i] / R - 1.0
            f[8] = min(10.0, max(-10.0, Q[b] / (N * S)))
            f[9] = 10.0 * a / R
            f[10] = d1 / h
            f[11] = (dk - d1) / h
    return F, S_body


def warm_start_targets(q, body_offsets, Q, S_body):
    """y = (q - Q/N) / S on beads of multi-bead bodies with S > 0, else 0."""
    off = np.asarray(body_offsets, dtype=np.int64)
    y = np.zeros(len(q))
    for b in range(len(off) - 1):
        s, e = off[b], off[b + 1]
        if e - s > 1 and S_body[b] > 0.0:
            y[s:e] = (np.asarray(q[s:e], dtype=np.float64) - Q[b] / (e - s)) / S_body[b]
    return y


def warm_start_guess(y, body_offsets, Q, S_body):
    """q = Q/N + S y on multi-bead bodies (Q itself on single beads), then a uniform
    shift per body so that its charges sum to Q."""
    off = np.asarray(body_offsets, dtype=np.int64)
    q = np.zeros(len(y))
    for b in range(len(off) - 1):
        s, e = off[b], off[b + 1]
        N = e - s
        v = np.full(N, Q[b] / N)
        if N > 1 and S_body[b] > 0.0:
            v = v + S_body[b] * np.asarray(y[s:e], dtype=np.float64)
        q[s:e] = v + (Q[b] - v.sum()) / N
    return q
