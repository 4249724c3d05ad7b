"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers and assembles test matrices; it holds
none of the LU or Newton arithmetic, and it is the one module that both the
CPU oracle's tests and the CUDA path's tests and benchmark take inputs from.

Host generators use numpy's counter-based Philox bit generator; device
generators (for the full-size benchmark batches) use a seeded
torch.Generator on the device.  The same seed does not give the same numbers
on host and device: parity tests always copy ONE generated batch to both
sides.

Recipes (paper Sec. 4.2 and 4.3 workloads, at the batch sizes of the
benchmark configurations):
  * uniform   -- entries i.i.d. U[-1, 1] (the paper's LINPACK-like default
                 draws U[-0.5, 0.5]; its "stress" set U[-5e-10, 5e-10]).
  * kappa     -- A = U diag(s) V^T with Haar-random orthogonal U, V (QR of a
                 Gaussian matrix with the sign of diag(R) folded into Q) and
                 singular values s_i = kappa^(-i/(n-1)), i = 0..n-1, shuffled,
                 kappa log-uniform in [kappa_lo, kappa_hi].
  * sweep     -- first half uniform, second half kappa; b = A x_true with
                 x_true i.i.d. U[-1, 1] for both halves.
  * norton    -- sig0: 6 Mandel components U[-150, 150] MPa with the mean of
                 the three normal components removed (deviatoric); deps: 6
                 Mandel components U[-1e-3, 1e-3].
  * tanh      -- A = n I + U[-1, 1] (per entry), c U[0.5, 2], b U[-3, 3] * n.
"""
import numpy as np

SEED_BASE = 1234


def config_seed(config_id: int, n: int = 0) -> int:
    """Seed of a workload: 1234 + config id, then seed*1000 + n per size."""
    s = SEED_BASE + config_id
    return s * 1000 + n if n else s


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


def uniform_systems(n, batch, seed, lo=-1.0, hi=1.0):
    """A (batch, n, n) with A[s, i, j] = a_ij, b (batch, n); i.i.d. U[lo, hi]."""
    g = rng(seed)
    A = g.uniform(lo, hi, size=(batch, n, n))
    b = g.uniform(lo, hi, size=(batch, n))
    return A, b


def haar_orthogonal(g, batch, n):
    """Haar-distributed orthogonal matrices (QR of Gaussian, sign-fixed)."""
    Z = g.standard_normal(size=(batch, n, n))
    Q, R = np.linalg.qr(Z)
    d = np.sign(np.diagonal(R, axis1=1, axis2=2))
    d[d == 0] = 1.0
    return Q * d[:, None, :]


def kappa_systems(n, batch, seed, kappa_lo=1e2, kappa_hi=1e8):
    """A = U diag(s) V^T with prescribed 2-norm condition number.

    Returns A, x_true, b = A x_true and the kappa of each system."""
    g = rng(seed)
    U = haar_orthogonal(g, batch, n)
    V = haar_orthogonal(g, batch, n)
    kappa = np.exp(g.uniform(np.log(kappa_lo), np.log(kappa_hi), size=batch))
    if n > 1:
        expo = np.arange(n) / (n - 1)
        s = kappa[:, None] ** (-expo[None, :])
        s = np.take_along_axis(s, np.argsort(g.random(size=(batch, n)), axis=1), axis=1)
    else:
        s = np.ones((batch, 1))
        kappa = np.ones(batch)
    A = np.einsum("bij,bj,bkj->bik", U, s, V)
    x_true = g.uniform(-1.0, 1.0, size=(batch, n))
    b = np.einsum("bij,bj->bi", A, x_true)
    return A, x_true, b, kappa


def sweep_systems(n, batch, seed):
    """The standalone-sweep recipe: half uniform, half kappa-controlled,
    b = A x_true throughout.  Returns A, b, x_true, kappa (nan for the
    uniform half)."""
    h = batch // 2
    g = rng(seed)
    A1 = g.uniform(-1.0, 1.0, size=(h, n, n))
    x1 = g.uniform(-1.0, 1.0, size=(h, n))
    b1 = np.einsum("bij,bj->bi", A1, x1)
    A2, x2, b2, k2 = kappa_systems(n, batch - h, seed + 7919)
    A = np.concatenate([A1, A2])
    b = np.concatenate([b1, b2])
    x = np.concatenate([x1, x2])
    kappa = np.concatenate([np.full(h, np.nan), k2])
    return A, b, x, kappa


def norton_points(npoints, seed, sig_amp=150.0, eps_amp=1e-3):
    """sig0 (npoints, 6) deviatoric Mandel stresses, deps (npoints, 6)."""
    g = rng(seed)
    sig0 = g.uniform(-sig_amp, sig_amp, size=(npoints, 6))
    sig0[:, :3] -= sig0[:, :3].mean(axis=1, keepdims=True)
    deps = g.uniform(-eps_amp, eps_amp, size=(npoints, 6))
    return sig0, deps


def tanh_points(n, npoints, seed):
    """A (npoints, n, n) = n I + U[-1,1], c U[0.5,2], b U[-3,3]*n."""
    g = rng(seed)
    A = g.uniform(-1.0, 1.0, size=(npoints, n, n)) + n * np.eye(n)[None]
    c = g.uniform(0.5, 2.0, size=(npoints, n))
    b = g.uniform(-3.0, 3.0, size=(npoints, n)) * n
    return A, c, b


# ---------------------------------------------------------------------------
# Device generators (full-size benchmark batches).  torch is imported lazily
# so that the host generators work without it.
# ---------------------------------------------------------------------------

def _tgen(seed, device):
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    return g


def uniform_systems_torch(n, batch, seed, device, lo=-1.0, hi=1.0):
    import torch
    g = _tgen(seed, device)
    A = torch.empty((batch, n, n), dtype=torch.float64, device=device).uniform_(lo, hi, generator=g)
    b = torch.empty((batch, n), dtype=torch.float64, device=device).uniform_(lo, hi, generator=g)
    return A, b


def _haar_torch(g, batch, n, device, chunk=1 << 16):
    """Haar-distributed orthogonal matrices on the device: Householder QR of
    a Gaussian matrix, Q rebuilt from the reflectors and multiplied by the
    signs of diag(R) (Mezzadri 2007), all as batched tensor operations."""
    import torch
    out = torch.empty((batch, n, n), dtype=torch.float64, device=device)
    for c0 in range(0, batch, chunk):
        c1 = min(batch, c0 + chunk)
        m = c1 - c0
        Z = torch.randn((m, n, n), dtype=torch.float64, device=device, generator=g)
        vs = []
        rsign = torch.empty((m, n), dtype=torch.float64, device=device)
        for k in range(n):
            x = Z[:, k:, k]
            nx = torch.linalg.vector_norm(x, dim=1)
            s0 = torch.where(x[:, 0] >= 0, 1.0, -1.0).to(torch.float64)
            alpha = -s0 * nx                      # R[k, k]
            v = x.clone()
            v[:, 0] -= alpha
            nv = torch.linalg.vector_norm(v, dim=1, keepdim=True)
            v = torch.where(nv > 0, v / torch.where(nv > 0, nv, 1.0), v)
            Z[:, k:, k:] -= 2.0 * v[:, :, None] * torch.einsum("bi,bij->bj", v, Z[:, k:, k:])[:, None, :]
            vs.append(v)
            rsign[:, k] = torch.where(alpha >= 0, 1.0, -1.0)
        Q = torch.eye(n, dtype=torch.float64, device=device).expand(m, n, n).clone()
        for k in range(n - 1, -1, -1):
            v = vs[k]
            Q[:, k:, :] -= 2.0 * v[:, :, None] * torch.einsum("bi,bij->bj", v, Q[:, k:, :])[:, None, :]
        out[c0:c1] = Q * rsign[:, None, :]
        del Z, Q, vs
    return out


def sweep_systems_torch(n, batch, seed, device, chunk=1 << 17):
    """Device version of sweep_systems: returns A (batch, n, n) math-indexed,
    b, x_true (all float64 on `device`)."""
    import torch
    g = _tgen(seed, device)
    h = batch // 2
    A = torch.empty((batch, n, n), dtype=torch.float64, device=device)
    A[:h].uniform_(-1.0, 1.0, generator=g)
    x = torch.empty((batch, n), dtype=torch.float64, device=device).uniform_(-1.0, 1.0, generator=g)
    m = batch - h
    if m > 0:
        lk = torch.empty(m, dtype=torch.float64, device=device).uniform_(np.log(1e2), np.log(1e8), generator=g)
        kappa = torch.exp(lk)
        if n > 1:
            expo = torch.arange(n, dtype=torch.float64, device=device) / (n - 1)
            s = kappa[:, None] ** (-expo[None, :])
            perm = torch.argsort(torch.rand((m, n), device=device, generator=g), dim=1)
            s = torch.gather(s, 1, perm)
        else:
            s = torch.ones((m, 1), dtype=torch.float64, device=device)
        for c0 in range(0, m, chunk):
            c1 = min(m, c0 + chunk)
            U = _haar_torch(g, c1 - c0, n, device)
            V = _haar_torch(g, c1 - c0, n, device)
            A[h + c0:h + c1] = torch.matmul(U * s[c0:c1, None, :], V.transpose(1, 2))
            del U, V
    b = torch.matmul(A, x[:, :, None])[:, :, 0]
    return A, b, x


def norton_points_torch(npoints, seed, device, sig_amp=150.0, eps_amp=1e-3):
    import torch
    g = _tgen(seed, device)
    sig0 = torch.empty((npoints, 6), dtype=torch.float64, device=device).uniform_(-sig_amp, sig_amp, generator=g)
    sig0[:, :3] -= sig0[:, :3].mean(dim=1, keepdim=True)
    deps = torch.empty((npoints, 6), dtype=torch.float64, device=device).uniform_(-eps_amp, eps_amp, generator=g)
    return sig0, deps


def tanh_points_torch(n, npoints, seed, device):
    """The tanh-law points of tanh_points on the device, as the field-major
    input of tl_newton_integrate: rows j*n + i hold a_ij, then c_i, then b_i
    (npoints columns)."""
    import torch
    g = _tgen(seed, device)
    A = torch.empty((npoints, n, n), dtype=torch.float64, device=device).uniform_(-1.0, 1.0, generator=g)
    A += n * torch.eye(n, dtype=torch.float64, device=device)
    c = torch.empty((npoints, n), dtype=torch.float64, device=device).uniform_(0.5, 2.0, generator=g)
    b = torch.empty((npoints, n), dtype=torch.float64, device=device).uniform_(-3.0, 3.0, generator=g) * n
    fields = torch.cat([A.transpose(1, 2).reshape(npoints, n * n).t(), c.t(), b.t()], dim=0).contiguous()
    return fields

