"""Helpers shared by the GPU parity tests: build the same seeded problem on both sides."""
import numpy as np

from oracle import krylov, mac


def problem(w, rho=1.0, mu=0.5, b=(1.0, 0.0, 0.0), dt=0.0, n_dilate=1, n_tag=1):
    return krylov.Problem(w.mask, w.labels, mac.Params(rho, mu, b, dt), w.periodic, n_dilate, n_tag)


def solver(w, rho=1.0, mu=0.5, b=(1.0, 0.0, 0.0), dt=0.0, **kw):
    from paper_2510_22077_gb300 import pns
    return pns.Solver(w.mask, w.labels, rho, mu, b, dt, periodic=w.periodic, **kw)


def to_dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64)).cuda()


def random_state(pb, seed=0, scale=1.0):
    """Physical-looking state: Stokes solution plus noise on the unknowns (zeros elsewhere)."""
    g = pb.g
    rng = np.random.default_rng(seed)
    xs = krylov.stokes_solution(pb)
    x = xs.copy()
    x[g.unknown] += 0.2 * scale * np.abs(xs).max() * rng.standard_normal(len(g.unknown))
    return x


def random_vector(pb, seed=1):
    g = pb.g
    rng = np.random.default_rng(seed)
    v = np.zeros(g.nfull)
    v[g.unknown] = rng.standard_normal(len(g.unknown))
    return v


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def oracle_converged(pb, x0, tol=1e-14, steps=30):
    x = x0.copy()
    for _ in range(steps):
        dx = pb.direct_step(x)
        x = x + dx
        if np.linalg.norm(dx) <= tol * np.linalg.norm(x):
            break
    return x
