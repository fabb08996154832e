"""Training of the learned warm start on solves made by the method itself.

Host orchestration around the C ABI: each training configuration is solved from
the zero guess (``induced_charge_solve``), its features and targets are formed on
the device (``ibpme_features``) and the rows of beads on multi-bead bodies are
kept; the network is then fitted with ``ibpme_mlp_train``.  Every step of the
arithmetic runs in the library's kernels; torch holds the device buffers.

The features need no mesh evaluation (body geometry, E0, the net charges and the
real-space potential of the other bodies' fixed charges), so a solve started from
the learned guess makes the same evaluations as one started from zero.
"""
from __future__ import annotations

import numpy as np


def _dev(torch, a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a)).to(dtype).to("cuda")


def collect(ib, ctx, systems, rtol: float = 1e-6, max_rows: int | None = None):
    """Solve every system (all sharing ctx's box, mesh, bead radius and
    permittivity; one right-hand side each) from zero and return the training
    rows of their body beads as device tensors (features [m][IBPME_MLP_IN] float32,
    targets [m] float32) with the solve statistics.  Stops early once max_rows
    rows are gathered."""
    import torch
    feats, targs, stats = [], [], []
    rows = 0
    for s in systems:
        n = s.n
        off = _dev(torch, s.body_offsets, torch.int32)
        bodies = ib.Bodies(off, _dev(torch, s.X, torch.float64), _dev(torch, s.Q, torch.float64))
        x = _dev(torch, s.x, torch.float64)
        E0 = _dev(torch, s.E0[:1], torch.float64)
        q = torch.zeros((1, n), dtype=torch.float64, device="cuda")
        status, st = ib.induced_charge_solve(ctx, n, x, bodies, E0, 1, ib.make_opts(rtol=rtol), q)
        if status != ib.IBPME_OK:
            raise RuntimeError(f"training solve of {s.name} did not converge ({st.rel_residual:.2e})")
        f = torch.empty((1, n, ib.IBPME_MLP_IN), dtype=torch.float32, device="cuda")
        t = torch.empty((1, n), dtype=torch.float32, device="cuda")
        ib.ibpme_features(ctx, n, x, bodies, E0, 1, f, q, t)
        sizes = np.diff(s.body_offsets)
        keep = torch.as_tensor(np.repeat(sizes > 1, sizes), device="cuda")
        feats.append(f[0][keep])
        targs.append(t[0][keep])
        stats.append(st)
        rows += int(feats[-1].shape[0])
        if max_rows is not None and rows >= max_rows:
            break
    return torch.cat(feats).contiguous(), torch.cat(targs).contiguous(), stats


def train(ib, feat, target, seed: int = 5, epochs: int = 20, batch: int = 4096, lr: float = 2e-3,
          lr_final: float = 2e-4, stages: int = 4):
    """A new network fitted to (feat, target): Adam over shuffled mini-batches, the
    learning rate stepped down geometrically from lr to lr_final over ``stages``
    equal parts of the epochs.  Returns (mlp handle, last loss)."""
    m = ib.ibpme_mlp_create(seed=seed)
    loss = float("nan")
    per = max(1, epochs // stages)
    for k in range(stages):
        rate = lr * (lr_final / lr) ** (k / max(1, stages - 1))
        loss = ib.ibpme_mlp_train(m, int(feat.shape[0]), feat, target, batch=batch, epochs=per, lr=rate,
                                  seed=seed * 131 + k)
    return m, loss
