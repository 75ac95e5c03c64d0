"""Direct NDFT and adjoint NDFT in FP64 (TEST INFRASTRUCTURE ONLY).

Sec. 2.1 of arXiv 2208.00049:
  * Eq. NDFT  (type 2):  fhat_j = sum_{n in I_N} f_n exp(-2 pi i n.k_j)
  * Eq. NDFTH (type 1):  y_n    = sum_j fhat_j exp(+2 pi i n.k_j)
with I_N = prod_d {-floor(N_d/2), ..., ceil(N_d/2) - 1} and k_j in [-1/2, 1/2)^D.

Arrays are row-major: f has shape (N_1, ..., N_D) with array index
i_d = n_d + floor(N_d/2); nodes k have shape (M, D).

The phase n.k_j is reduced modulo 1 in FP64 before multiplying by 2 pi, so
that the exponential's argument stays in [0, 2 pi).  Nodes are processed in
chunks only to bound memory; each output is the plain sum of the definition
(a library matrix-vector product serves as the summation step).
"""
import numpy as np

from .window import index_set


def _all_indices(N):
    """All n in I_N as an (|I_N|, D) FP64 array, in row-major order of f."""
    axes = [index_set(n).astype(np.float64) for n in N]
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack([a.ravel() for a in mesh], axis=1)


def _chunk(total, per_row, budget=1 << 22):
    return max(1, min(total, budget // max(1, per_row)))


def ndft(k, f):
    """Type-2 NDFT (Eq. NDFT).  k: (M, D) real, f: complex array of shape N."""
    k = np.asarray(k, dtype=np.float64)
    f = np.asarray(f, dtype=np.complex128)
    N = f.shape
    if k.ndim != 2 or k.shape[1] != len(N):
        raise ValueError("k must have shape (M, D)")
    n = _all_indices(N)
    fv = f.ravel()
    M = k.shape[0]
    out = np.empty(M, dtype=np.complex128)
    step = _chunk(M, n.shape[0])
    for s in range(0, M, step):
        ph = k[s:s + step] @ n.T
        ph -= np.floor(ph)
        out[s:s + step] = np.exp(-2j * np.pi * ph) @ fv
    return out


def ndft_adjoint(k, fhat, N):
    """Type-1 adjoint NDFT (Eq. NDFTH).  Returns a complex array of shape N."""
    k = np.asarray(k, dtype=np.float64)
    fhat = np.asarray(fhat, dtype=np.complex128).ravel()
    N = tuple(int(v) for v in N)
    n = _all_indices(N)
    out = np.empty(n.shape[0], dtype=np.complex128)
    step = _chunk(n.shape[0], k.shape[0])
    for s in range(0, n.shape[0], step):
        ph = n[s:s + step] @ k.T
        ph -= np.floor(ph)
        out[s:s + step] = np.exp(2j * np.pi * ph) @ fhat
    return out.reshape(N)


def ndft_adjoint_at(k, fhat, N, idx):
    """Eq. NDFTH at selected outputs only: y at the array indices idx (a tuple
    of D integer arrays, as from np.unravel_index), for checks at sizes where
    the full adjoint is out of reach.  Nodes are summed in chunks."""
    k = np.asarray(k, dtype=np.float64)
    fhat = np.asarray(fhat, dtype=np.complex128).ravel()
    n = np.stack([np.asarray(idx[d], dtype=np.float64) - (int(N[d]) // 2) for d in range(len(N))], axis=1)
    out = np.zeros(n.shape[0], dtype=np.complex128)
    step = _chunk(k.shape[0], n.shape[0])
    for s in range(0, k.shape[0], step):
        ph = n @ k[s:s + step].T
        ph -= np.floor(ph)
        out += np.exp(2j * np.pi * ph) @ fhat[s:s + step]
    return out


def ndft_node_derivative(k, f):
    """d fhat_j / d k_{j,d} of the exact NDFT: sum_n f_n (-2 pi i n_d) exp(-2 pi i n.k_j).

    Returns a complex (M, D) array.  It is the NDFT applied to the D
    coefficient arrays (-2 pi i n_d) f_n, by differentiating Eq. NDFT.
    """
    f = np.asarray(f, dtype=np.complex128)
    N = f.shape
    D = len(N)
    out = np.empty((np.asarray(k).shape[0], D), dtype=np.complex128)
    for d in range(D):
        shape = [1] * D
        shape[d] = N[d]
        nd = index_set(N[d]).reshape(shape).astype(np.float64)
        out[:, d] = ndft(k, -2j * np.pi * nd * f)
    return out


def ndft_node_grad(k, f, cot):
    """Node gradient of a real loss through fhat = A f (PyTorch convention):
    g[j, d] = Re(conj(cot_j) * d fhat_j / d k_{j,d})."""
    dk = ndft_node_derivative(k, f)
    return np.real(np.conj(np.asarray(cot, dtype=np.complex128))[:, None] * dk)
