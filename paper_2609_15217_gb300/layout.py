"""Host-side packing between math-indexed batches and the two device layouts
of the C ABI (pure data movement with torch; no arithmetic).

Math indexing: A[s, i, j] = a_ij of system s, b[s, i] = b_i.
  per-system  : flat buffer, A[s*n*n + j*n + i]  (column-major per system)
  interleaved : flat buffer, A[(j*n + i)*ld + s] (batch-minor), ld >= batch
"""
import torch


def pad_ld(batch, align=32):
    """Batch stride of the interleaved layout: batch rounded up to a multiple
    of 32 elements (256 bytes of float64), so every row starts aligned."""
    return max(align, (batch + align - 1) // align * align)


def matrices_to_layout(A, layout, ld=None):
    """(batch, n, n) -> flat tensor in the given layout (0 per-system, 1 interleaved)."""
    batch, n, _ = A.shape
    if layout == 0:
        return A.transpose(1, 2).contiguous().reshape(-1)
    ld = ld or pad_ld(batch)
    out = torch.zeros((n * n, ld), dtype=A.dtype, device=A.device)
    out[:, :batch] = A.permute(2, 1, 0).reshape(n * n, batch)
    return out.reshape(-1)


def matrices_from_layout(flat, batch, n, layout, ld=None):
    if layout == 0:
        return flat.reshape(batch, n, n).transpose(1, 2).contiguous()
    ld = ld or pad_ld(batch)
    return flat.reshape(n * n, ld)[:, :batch].reshape(n, n, batch).permute(2, 1, 0).contiguous()


def vectors_to_layout(v, layout, ld=None):
    """(batch, n) -> flat tensor in the given layout (also int32 pivots)."""
    batch, n = v.shape
    if layout == 0:
        return v.contiguous().reshape(-1)
    ld = ld or pad_ld(batch)
    out = torch.zeros((n, ld), dtype=v.dtype, device=v.device)
    out[:, :batch] = v.t()
    return out.reshape(-1)


def vectors_from_layout(flat, batch, n, layout, ld=None):
    if layout == 0:
        return flat.reshape(batch, n).contiguous()
    ld = ld or pad_ld(batch)
    return flat.reshape(n, ld)[:, :batch].t().contiguous()


def multi_rhs_to_layout(B, layout, ld=None):
    """(batch, nrhs, n) right-hand sides -> flat (per-system: n x nrhs
    column-major per system; interleaved: [(r*n + i)*ld + s])."""
    batch, nrhs, n = B.shape
    if layout == 0:
        return B.contiguous().reshape(-1)
    ld = ld or pad_ld(batch)
    out = torch.zeros((nrhs * n, ld), dtype=B.dtype, device=B.device)
    out[:, :batch] = B.reshape(batch, nrhs * n).t()
    return out.reshape(-1)


def multi_rhs_from_layout(flat, batch, nrhs, n, layout, ld=None):
    if layout == 0:
        return flat.reshape(batch, nrhs, n).contiguous()
    ld = ld or pad_ld(batch)
    return flat.reshape(nrhs * n, ld)[:, :batch].t().reshape(batch, nrhs, n).contiguous()
