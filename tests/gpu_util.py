"""Helpers shared by the GPU parity tests (host-side conversions only)."""
import numpy as np
import pytest
import scipy.sparse as sp

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1804_10060_gb300 import thermoamg  # raises if the library is missing
    return thermoamg


def bsr_to_csr(rp, ci, vals, n_cols_blocks=None):
    """Device block-CSR (torch) -> scipy CSR in scalar indices."""
    rp = rp.cpu().numpy().astype(np.int64)
    ci = ci.cpu().numpy().astype(np.int64)
    v = vals.cpu().numpy()
    n = rp.size - 1
    br, bc = v.shape[1], v.shape[2]
    nc = (ci.max() + 1 if ci.size else 0) if n_cols_blocks is None else n_cols_blocks
    B = sp.bsr_matrix((v, ci, rp), shape=(n * br, nc * bc))
    return B.tocsr()


def max_rel(a, b):
    a = a.toarray() if sp.issparse(a) else np.asarray(a)
    b = b.toarray() if sp.issparse(b) else np.asarray(b)
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def sparse_rel(A, B):
    D = (A - B).tocsr()
    m = abs(B).max()
    return (abs(D).max() if D.nnz else 0.0) / m


def _veltkamp(a):
    """a = hi + lo with 26-bit halves (Veltkamp's splitting; exact for |a| < 2^996)."""
    c = 134217729.0 * a          # 2^27 + 1
    hi = c - (c - a)
    return hi, a - hi


def exact_spmv(A, x):
    """Correctly rounded y = A x and s = sum_j |A_ij x_j| per row (A scipy CSR, x float64).

    Every product is made exact with Dekker's TwoProduct (p + e = a x exactly),
    then each row's 2 nnz terms are summed exactly by math.fsum.
    """
    import math
    A = A.tocsr()
    a = A.data
    xv = x[A.indices]
    p = a * xv
    ah, al = _veltkamp(a)
    xh, xl = _veltkamp(xv)
    e = ((ah * xh - p) + ah * xl + al * xh) + al * xl
    y = np.empty(A.shape[0])
    s = np.empty(A.shape[0])
    ab = np.abs(p)
    for i in range(A.shape[0]):
        lo, hi = A.indptr[i], A.indptr[i + 1]
        y[i] = math.fsum(np.concatenate([p[lo:hi], e[lo:hi]]))
        s[i] = math.fsum(ab[lo:hi])
    return y, s
