"""Shared test helpers: contexts from workload systems and error measures."""
import numpy as np

FP64_RTOL = 1e-5     # GPU FP64 path vs the FP64 oracle (stated target)
MIXED_RTOL = 1e-3    # GPU mixed precision vs the FP64 oracle (stated target)


def rel_err(got, ref):
    """max_i |got_i - ref_i| / max_i |ref_i|: element-wise difference on the vector's scale."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.max(np.abs(ref)) if ref.size else 0.0
    if scale == 0.0:
        return float(np.max(np.abs(got))) if got.size else 0.0
    return float(np.max(np.abs(got - ref)) / scale)


def context(ib, s, precision=None, max_rhs=3, stream=None, **over):
    prec = {"fp64": ib.IBPME_FP64, "mixed": ib.IBPME_MIXED}[precision or s.precision]
    kw = dict(box=s.box, mesh=s.mesh, tol=s.tol, bead_radius=s.a, eps_f=s.eps, precision=prec, max_rhs=max_rhs)
    kw.update(over)
    return ib.pme_setup(ib.make_params(**kw), stream)


def cuda(a, dtype=None):
    import torch
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda().contiguous()


def random_neutral_charges(n, seed=0):
    rng = np.random.default_rng(seed)
    q = rng.normal(size=n)
    return q - q.mean()
