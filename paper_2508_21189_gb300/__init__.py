"""GB300-native structured random sketching (arxiv 2508.21189): Python binding of librsk.

Each function has the name of the C entry point it calls and does argument marshalling only
(torch tensors -> device pointers, dtypes -> rsk_dtype, the current CUDA stream).  Every step
of the computation runs in librsk's CUDA kernels; there is no CPU path.
"""
import ctypes

import torch

from ._lib import LsqInfo, LsqOpts, LsqProblem, RskError, STATUS, load

RSK_F64, RSK_F32, RSK_BF16, RSK_F32X2 = 0, 1, 2, 3
_DT = {torch.float64: RSK_F64, torch.float32: RSK_F32, torch.bfloat16: RSK_BF16, "f32x2": RSK_F32X2}

_handles = {}


def lib():
    return load()


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def handle(device=None):
    """Per-device rsk_handle (created on first use with that device current)."""
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else torch.device(device).index or 0)
    h = _handles.get(dev.index)
    if h is None:
        with torch.cuda.device(dev):
            out = ctypes.c_void_p()
            st = load().rsk_create(ctypes.byref(out))
            if st:
                raise RskError(st, "rsk_create failed")
            h = out
        _handles[dev.index] = h
    return h


def _check(st, h):
    if st:
        msg = load().rsk_last_error(h) if h is not None else b""
        raise RskError(st, (msg or b"").decode())


def _dt(t):
    try:
        return _DT[t.dtype]
    except KeyError:
        raise TypeError(f"unsupported dtype {t.dtype}") from None


def _matrix(A, name):
    if not A.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if A.dim() != 2 or A.stride(1) != 1 or A.stride(0) < A.shape[1]:
        raise ValueError(f"{name} must be 2-D row-major with unit column stride")
    return A


def rsk_sync_status(stream=None, device=None):
    h = handle(device)
    _check(load().rsk_sync_status(h, _stream(stream)), h)


def rsk_set_wait_limit(spins, device=None):
    """Iteration limit of the handle's bounded polls on global-memory flags (0 = default)."""
    h = handle(device)
    _check(load().rsk_set_wait_limit(h, spins), h)


def rsk_sparse_sign_generate(n, d, zeta, seed, device=None, stream=None):
    """Draw S: returns (rows int32 [n, zeta], sign_bits int32 view of uint32 [n]) on the device."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    rows = torch.empty(n, zeta, dtype=torch.int32, device=dev)
    bits = torch.empty(n, dtype=torch.int32, device=dev)
    h = handle(dev)
    _check(load().rsk_sparse_sign_generate(h, n, d, zeta, seed, rows.data_ptr(), bits.data_ptr(), _stream(stream)), h)
    return rows, bits


def rsk_sparse_sign_index_dims(n, d, zeta):
    """(chunk_rows, n_chunks, offsets_pitch) of the chunked inverted index."""
    c = ctypes.c_int64()
    m = ctypes.c_int64()
    p = ctypes.c_int64()
    _check(load().rsk_sparse_sign_index_dims(n, d, zeta, ctypes.byref(c), ctypes.byref(m), ctypes.byref(p)), None)
    return c.value, m.value, p.value


def rsk_sparse_sign_index(n, d, zeta, seed, device=None, stream=None):
    """Chunked inverted index of S: (offsets uint16-as-int16 [n_chunks, pitch], entries [n*zeta])."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    _, nch, pitch = rsk_sparse_sign_index_dims(n, d, zeta)
    offs = torch.empty(nch, pitch, dtype=torch.int16, device=dev)
    ents = torch.empty(n * zeta + 8, dtype=torch.int16, device=dev)
    h = handle(dev)
    _check(load().rsk_sparse_sign_index(h, n, d, zeta, seed, offs.data_ptr(), ents.data_ptr(), _stream(stream)), h)
    return offs, ents[: n * zeta]


def rsk_sparse_sign_apply(A, d, zeta, seed, out_dtype=torch.float32, out=None, stream=None):
    """SA = S @ A for a CUDA tensor A (n x k, row-major; F64/F32/BF16)."""
    _matrix(A, "A")
    n, k = A.shape
    if out is None:
        out = torch.empty(d, k, dtype=out_dtype, device=A.device)
    _matrix(out, "out")
    h = handle(A.device)
    st = load().rsk_sparse_sign_apply(h, A.data_ptr(), _dt(A), n, k, A.stride(0), d, zeta, seed,
                                      out.data_ptr(), _dt(out), out.stride(0), _stream(stream))
    _check(st, h)
    return out


def rsk_sparse_sign_apply_host(A, d, zeta, seed, out_dtype=torch.float32, out=None, device=None, stream=None):
    """SA = S @ A for a HOST tensor A (n x k row-major, pinned for overlap); SA on the device."""
    if A.is_cuda or A.dim() != 2 or A.stride(1) != 1 or A.stride(0) < A.shape[1]:
        raise ValueError("A must be a 2-D row-major host tensor with unit column stride")
    n, k = A.shape
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    if out is None:
        out = torch.empty(d, k, dtype=out_dtype, device=dev)
    _matrix(out, "out")
    h = handle(out.device)
    st = load().rsk_sparse_sign_apply_host(h, A.data_ptr(), _dt(A), n, k, A.stride(0), d, zeta, seed,
                                           out.data_ptr(), _dt(out), out.stride(0), _stream(stream))
    _check(st, h)
    return out


def rsk_split_pairs(A, stream=None):
    """Interleaved double-float form of a CUDA FP64 matrix: float32 tensor (n, k, 2) = (hi, lo)."""
    _matrix(A, "A")
    if A.dtype != torch.float64:
        raise TypeError("rsk_split_pairs takes FP64 A")
    n, k = A.shape
    P = torch.empty(n, k, 2, dtype=torch.float32, device=A.device)
    h = handle(A.device)
    _check(load().rsk_split_pairs(h, A.data_ptr(), n, k, A.stride(0), P.data_ptr(), _stream(stream)), h)
    return P


def rsk_sparse_sign_apply_pairs(P, d, zeta, seed, out_dtype=torch.float64, out=None, stream=None):
    """SA = S @ (hi + lo) for interleaved pairs P (float32, n x k x 2), double-float accumulation."""
    if not P.is_cuda or P.dtype != torch.float32 or P.dim() != 3 or P.shape[2] != 2 or P.stride(2) != 1 \
            or P.stride(1) != 2:
        raise ValueError("P must be a CUDA float32 tensor (n, k, 2) with packed pairs")
    n, k = P.shape[0], P.shape[1]
    if out is None:
        out = torch.empty(d, k, dtype=out_dtype, device=P.device)
    _matrix(out, "out")
    h = handle(P.device)
    st = load().rsk_sparse_sign_apply(h, P.data_ptr(), RSK_F32X2, n, k, P.stride(0) // 2, d, zeta, seed,
                                      out.data_ptr(), _dt(out), out.stride(0), _stream(stream))
    _check(st, h)
    return out


class SparseSignPlan:
    """rsk_sparse_sign_plan_*: keeps one S's inverted index on the device for reuse."""

    def __init__(self, n, d, zeta, seed, device=None, stream=None):
        self.n, self.d, self.zeta, self.seed = n, d, zeta, seed
        self.h = handle(device)
        p = ctypes.c_void_p()
        _check(load().rsk_sparse_sign_plan_create(self.h, n, d, zeta, seed, ctypes.byref(p), _stream(stream)), self.h)
        self.p = p

    def apply(self, A, out_dtype=torch.float32, out=None, stream=None):
        _matrix(A, "A")
        if A.shape[0] != self.n:
            raise ValueError("row count does not match the plan")
        k = A.shape[1]
        if out is None:
            out = torch.empty(self.d, k, dtype=out_dtype, device=A.device)
        st = load().rsk_sparse_sign_plan_apply(self.h, self.p, A.data_ptr(), _dt(A), k, A.stride(0),
                                               out.data_ptr(), _dt(out), out.stride(0), _stream(stream))
        _check(st, self.h)
        return out

    def close(self, stream=None):
        if self.p:
            load().rsk_sparse_sign_plan_destroy(self.h, self.p, _stream(stream))
            self.p = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def rsk_sparse_sign_plan_create(n, d, zeta, seed, device=None, stream=None):
    return SparseSignPlan(n, d, zeta, seed, device, stream)


def rsk_srtt_draw(n, d, seed, device=None, stream=None):
    """P (int64 [d], draw order) and D bits (int32 view of uint32 [ceil(n/32)]) of the SRTT."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    rows = torch.empty(d, dtype=torch.int64, device=dev)
    bits = torch.empty((n + 31) // 32, dtype=torch.int32, device=dev)
    h = handle(dev)
    _check(load().rsk_srtt_draw(h, n, d, seed, rows.data_ptr(), bits.data_ptr(), _stream(stream)), h)
    return rows, bits


def rsk_srtt_apply(A, d, seed, out_dtype=torch.float32, out=None, stream=None):
    """Y = d^{-1/2} P H_n D A for a CUDA tensor A (n x k, n a power of two; F32/BF16)."""
    _matrix(A, "A")
    n, k = A.shape
    if out is None:
        out = torch.empty(d, k, dtype=out_dtype, device=A.device)
    _matrix(out, "out")
    h = handle(A.device)
    st = load().rsk_srtt_apply(h, A.data_ptr(), _dt(A), n, k, A.stride(0), d, seed, out.data_ptr(), _dt(out),
                               out.stride(0), _stream(stream))
    _check(st, h)
    return out


def rsk_sparse_stack_generate(n, d, zeta, seed, device=None, stream=None):
    """Draw a SparseStack S: (rows int32 [n, zeta], sign_bits int32 view of uint32 [n]) on the device."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    rows = torch.empty(n, zeta, dtype=torch.int32, device=dev)
    bits = torch.empty(n, dtype=torch.int32, device=dev)
    h = handle(dev)
    _check(load().rsk_sparse_stack_generate(h, n, d, zeta, seed, rows.data_ptr(), bits.data_ptr(), _stream(stream)), h)
    return rows, bits


def rsk_sparse_stack_apply(A, d, zeta, seed, out_dtype=torch.float32, out=None, stream=None):
    """SA = S @ A with S a SparseStack (d = b * zeta)."""
    _matrix(A, "A")
    n, k = A.shape
    if out is None:
        out = torch.empty(d, k, dtype=out_dtype, device=A.device)
    _matrix(out, "out")
    h = handle(A.device)
    st = load().rsk_sparse_stack_apply(h, A.data_ptr(), _dt(A), n, k, A.stride(0), d, zeta, seed,
                                       out.data_ptr(), _dt(out), out.stride(0), _stream(stream))
    _check(st, h)
    return out


def rsk_sparse_sign_apply_right(A, k, zeta, seed, kind=0, philox_stream=-1, out=None, stream=None):
    """Y = A @ S.T (n x k, returned as a column-major view) for S the k x dc sparse sign of `kind`
    (0 SparseUniform, 1 SparseStack) on Philox stream `philox_stream` (-1: the kind's own)."""
    _matrix(A, "A")
    if A.dtype != torch.float32:
        raise TypeError("the right sketch takes FP32 A")
    n, dc = A.shape
    if out is None:
        out = torch.empty(k, n, dtype=torch.float32, device=A.device).t()
    if out.shape != (n, k) or out.stride(0) != 1 or out.dtype != torch.float32:
        raise ValueError("out must be an FP32 n x k column-major view")
    h = handle(A.device)
    st = load().rsk_sparse_sign_apply_right(h, kind, A.data_ptr(), n, dc, A.stride(0), k, zeta, seed, philox_stream,
                                            out.data_ptr(), out.stride(1), _stream(stream))
    _check(st, h)
    return out


def rsk_sparse_sign_apply_rows(A, row0, d, zeta, seed, out_dtype=torch.float32, out=None, stream=None):
    """Partial sketch S[:, row0:row0+n] @ A of a row block A (n x k) of a row-sharded matrix."""
    _matrix(A, "A")
    n, k = A.shape
    if out is None:
        out = torch.empty(d, k, dtype=out_dtype, device=A.device)
    _matrix(out, "out")
    h = handle(A.device)
    st = load().rsk_sparse_sign_apply_rows(h, A.data_ptr(), _dt(A), n, k, A.stride(0), row0, d, zeta, seed,
                                           out.data_ptr(), _dt(out), out.stride(0), _stream(stream))
    _check(st, h)
    return out


def rsk_srtt_apply_rows(A, row0, n_total, d, seed, out_dtype=torch.float32, out=None, stream=None):
    """Partial SRTT d^{-1/2} P H[:, row0:row0+n] D A of a row block A (n x k, row0 % 2048 == 0)."""
    _matrix(A, "A")
    n, k = A.shape
    if out is None:
        out = torch.empty(d, k, dtype=out_dtype, device=A.device)
    _matrix(out, "out")
    h = handle(A.device)
    st = load().rsk_srtt_apply_rows(h, A.data_ptr(), _dt(A), n, k, A.stride(0), row0, n_total, d, seed,
                                    out.data_ptr(), _dt(out), out.stride(0), _stream(stream))
    _check(st, h)
    return out


def rsk_sketch_sum_partials(parts, out=None, stream=None):
    """out = parts[0] + parts[1] + ... in that order; parts is a CUDA tensor [count, d, k] (F32/F64)."""
    if not parts.is_cuda or parts.dim() != 3 or not parts.is_contiguous():
        raise ValueError("parts must be a contiguous CUDA tensor [count, d, k]")
    count, d, k = parts.shape
    if out is None:
        out = torch.empty(d, k, dtype=parts.dtype, device=parts.device)
    _matrix(out, "out")
    h = handle(parts.device)
    st = load().rsk_sketch_sum_partials(h, parts.data_ptr(), _dt(parts), count, d * k, d, k, out.data_ptr(),
                                        out.stride(0), _stream(stream))
    _check(st, h)
    return out


def rsk_sparse_rtt_default_xi(d):
    return int(load().rsk_sparse_rtt_default_xi(d))


def rsk_sparse_rtt_draw(n, d, seed, xi=0, device=None, stream=None):
    """SparseCol positions of a SparseRTT: (positions int32 [d, xi], sign_bits int32 view of uint32 [d])."""
    xi = xi or rsk_sparse_rtt_default_xi(d)
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    pos = torch.empty(d, xi, dtype=torch.int32, device=dev)
    bits = torch.empty(d, dtype=torch.int32, device=dev)
    h = handle(dev)
    _check(load().rsk_sparse_rtt_draw(h, n, d, xi, seed, pos.data_ptr(), bits.data_ptr(), _stream(stream)), h)
    return pos, bits


def rsk_sparse_rtt_apply(A, d, seed, xi=0, out_dtype=torch.float32, out=None, stream=None):
    """Y = Omega^T A with Omega = D F S a SparseRTT (WHT, xi positions per output row; 0 = default)."""
    _matrix(A, "A")
    n, k = A.shape
    if out is None:
        out = torch.empty(d, k, dtype=out_dtype, device=A.device)
    _matrix(out, "out")
    h = handle(A.device)
    st = load().rsk_sparse_rtt_apply(h, A.data_ptr(), _dt(A), n, k, A.stride(0), d, xi, seed, out.data_ptr(),
                                     _dt(out), out.stride(0), _stream(stream))
    _check(st, h)
    return out


def rsk_lstsq_sketch_precond(A, b, d, zeta=8, seed=0, sketch_dtype=torch.bfloat16, inner_dtype=torch.float32,
                             tol=1e-10, max_refine=20, max_inner=50, inner_tol=1e-6, x=None, stream=None,
                             raise_on_nonconvergence=True):
    """x = argmin ||A x - b|| by sketch-and-precondition; returns (x FP64 [k], info dict).

    A: CUDA tensor n x k (F64 or F32, row-major); b: CUDA FP64 [n]."""
    _matrix(A, "A")
    n, k = A.shape
    if b.dtype != torch.float64 or not b.is_cuda or b.numel() != n or not b.is_contiguous():
        raise ValueError("b must be a contiguous CUDA float64 vector of length n")
    if x is None:
        x = torch.empty(k, dtype=torch.float64, device=A.device)
    opts = LsqOpts(d, zeta, seed, _DT[sketch_dtype], _DT[inner_dtype], tol, max_refine, max_inner, inner_tol)
    info = LsqInfo()
    h = handle(A.device)
    st = load().rsk_lstsq_sketch_precond(h, A.data_ptr(), _dt(A), n, k, A.stride(0), b.data_ptr(), x.data_ptr(),
                                         ctypes.byref(opts), ctypes.byref(info), _stream(stream))
    out = {"backward_err": info.backward_err, "residual_norm": info.residual_norm,
           "frobenius_norm": info.frobenius_norm, "refine_steps": info.refine_steps,
           "inner_iters": info.inner_iters, "status": STATUS.get(info.status, info.status)}
    if st == 4 and not raise_on_nonconvergence:
        return x, out
    _check(st, h)
    return x, out


def rsk_lstsq_sketch_precond_batched(As, bs, ds=None, zeta=8, seed=0, sketch_dtype=torch.float32,
                                     inner_dtype=torch.float32, tol=1e-10, max_refine=20, max_inner=50,
                                     inner_tol=1e-6, xs=None, stream=None, raise_on_nonconvergence=True,
                                     qr_dtype=torch.float64):
    """Batched sketch-and-precondition: lists of CUDA A_i (n_i x k_i) and b_i (FP64); returns
    (list of x_i, list of info dicts).  Problem i uses seed + i and d_i = ds[i] (default 4 k_i).
    qr_dtype: precision of the sketch's Householder QR (float64 default, or float32)."""
    count = len(As)
    if xs is None:
        xs = [torch.empty(A.shape[1], dtype=torch.float64, device=A.device) for A in As]
    arr = (LsqProblem * count)()
    for i, (A, b, x) in enumerate(zip(As, bs, xs)):
        _matrix(A, "A")
        if b.dtype != torch.float64 or not b.is_contiguous() or b.numel() != A.shape[0]:
            raise ValueError("each b must be a contiguous float64 vector of length n")
        d = 0 if ds is None else int(ds[i])
        arr[i] = LsqProblem(A.data_ptr(), _dt(A), A.shape[0], A.shape[1], A.stride(0), d, b.data_ptr(), x.data_ptr())
    opts = LsqOpts(0, zeta, seed, _DT[sketch_dtype], _DT[inner_dtype], tol, max_refine, max_inner, inner_tol,
                   _DT[qr_dtype])
    infos = (LsqInfo * count)()
    h = handle(As[0].device)
    st = load().rsk_lstsq_sketch_precond_batched(h, count, arr, ctypes.byref(opts), infos, _stream(stream))
    out = [{"backward_err": f.backward_err, "residual_norm": f.residual_norm, "frobenius_norm": f.frobenius_norm,
            "refine_steps": f.refine_steps, "inner_iters": f.inner_iters, "status": STATUS.get(f.status, f.status)}
           for f in infos]
    if st == 4 and not raise_on_nonconvergence:
        return xs, out
    _check(st, h)
    return xs, out


def _colmajor(X, name):
    """A CUDA FP32 matrix viewed column-major: X must be the transpose of a row-major tensor
    (stride (1, ld)), i.e. X.t() contiguous."""
    if not X.is_cuda or X.dtype != torch.float32 or X.dim() != 2 or X.stride(0) != 1 or X.stride(1) < X.shape[0]:
        raise ValueError(f"{name} must be a column-major CUDA float32 matrix (stride (1, ld))")
    return X


def rsk_svd_econ(A, stream=None):
    """Thin SVD of a column-major CUDA FP32 matrix A (m x q, m >= q): returns (U, s, V), U and V
    column-major (A = U diag(s) V^T)."""
    _colmajor(A, "A")
    m, q = A.shape
    U = torch.empty(q, m, device=A.device).t()
    V = torch.empty(q, q, device=A.device).t()
    s = torch.empty(q, device=A.device)
    h = handle(A.device)
    _check(load().rsk_svd_econ(h, A.data_ptr(), m, q, A.stride(1), U.data_ptr(), U.stride(1), s.data_ptr(),
                               V.data_ptr(), V.stride(1), _stream(stream)), h)
    return U, s, V


def rsk_cholesky(G, shift_coeff=0.0, stream=None):
    """Upper Cholesky factor R of sym(G) + shift_coeff * trace(G) I for a column-major CUDA FP32 G."""
    _colmajor(G, "G")
    q = G.shape[0]
    R = torch.empty(q, q, device=G.device).t()
    h = handle(G.device)
    _check(load().rsk_cholesky(h, G.data_ptr(), q, G.stride(1), float(shift_coeff), R.data_ptr(), R.stride(1),
                               _stream(stream)), h)
    return R


def rsk_trinv(R, stream=None):
    """R^{-1} of an upper triangular column-major CUDA FP32 R."""
    _colmajor(R, "R")
    q = R.shape[0]
    Ri = torch.empty(q, q, device=R.device).t()
    h = handle(R.device)
    _check(load().rsk_trinv(h, R.data_ptr(), q, R.stride(1), Ri.data_ptr(), _stream(stream)), h)
    return Ri


def rsk_qr_econ(X, stream=None):
    """Thin QR of a column-major CUDA FP32 matrix X (m x q): returns (Q column-major, R upper q x q)."""
    _colmajor(X, "X")
    m, q = X.shape
    Q = torch.empty(q, m, device=X.device).t()
    R = torch.empty(q, q, device=X.device).t()
    h = handle(X.device)
    _check(load().rsk_qr_econ(h, X.data_ptr(), m, q, X.stride(1), Q.data_ptr(), Q.stride(1), R.data_ptr(),
                              _stream(stream)), h)
    return Q, R


def rsk_nystrom_psd(A, k, rank=None, zeta=4, seed=0, kind="stack", stream=None):
    """Nystrom approximation of a psd CUDA FP32 matrix A (n x n, row-major): (U [n, rank] column-major,
    lambda [rank]) with A ~ U diag(lambda) U^T; kind "stack" (SparseStack) or "uniform"."""
    _matrix(A, "A")
    if A.dtype != torch.float32 or A.shape[0] != A.shape[1]:
        raise ValueError("A must be a square float32 matrix")
    n = A.shape[0]
    rank = k if rank is None else rank
    U = torch.empty(rank, n, device=A.device).t()
    lam = torch.empty(rank, device=A.device)
    h = handle(A.device)
    _check(load().rsk_nystrom_psd(h, A.data_ptr(), n, A.stride(0), k, rank, zeta, seed,
                                  {"uniform": 0, "stack": 1}[kind], U.data_ptr(), U.stride(1), lam.data_ptr(),
                                  _stream(stream)), h)
    return U, lam


def rsk_gen_nystrom(A, k, p=None, zeta=4, seed=0, kind="stack", form="svd", stream=None):
    """Generalized Nystrom approximation of a CUDA FP32 matrix A (n x d, row-major).
    form "outer" (Alg. 4): returns (F [n, k], G [d, k], r) with A ~ F G^T;
    form "svd" (Alg. 5): returns (U [n, k], sigma [k], V [d, k], r) with A ~ U diag(sigma) V^T.
    Matrices are column-major; r is the numerical rank.  p defaults to ceil(1.5 k) (rounded up to a
    multiple of zeta for SparseStack)."""
    _matrix(A, "A")
    if A.dtype != torch.float32:
        raise TypeError("A must be float32")
    n, d = A.shape
    if p is None:
        p = -(-3 * k // 2)
        if kind == "stack":
            p = -(-p // zeta) * zeta
    out1 = torch.empty(k, n, device=A.device).t()
    out2 = torch.empty(k, d, device=A.device).t()
    sig = torch.empty(k, device=A.device)
    r = torch.zeros(1, dtype=torch.int32, device=A.device)
    h = handle(A.device)
    fm = {"outer": 0, "svd": 1}[form]
    _check(load().rsk_gen_nystrom(h, A.data_ptr(), n, d, A.stride(0), k, p, zeta, seed, {"uniform": 0, "stack": 1}[kind],
                                  fm, out1.data_ptr(), out1.stride(1), sig.data_ptr(), out2.data_ptr(), out2.stride(1),
                                  r.data_ptr(), _stream(stream)), h)
    if fm == 0:
        return out1, out2, int(r.item())
    return out1, sig, out2, int(r.item())


def rsk_osi_estimate(r, k=None, zeta=8, seed=0, kind="stack", iters=300, device=None, stream=None):
    """(alpha, beta): injectivity and dilation estimates of the sketch on Q = [e_1 ... e_r] (k = 2r by default)."""
    k = 2 * r if k is None else k
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    a, b = ctypes.c_double(), ctypes.c_double()
    h = handle(dev)
    _check(load().rsk_osi_estimate(h, r, k, zeta, seed, {"uniform": 0, "stack": 1}[kind], iters, ctypes.byref(a),
                                   ctypes.byref(b), _stream(stream)), h)
    return a.value, b.value


def rsk_autotune_sketch(kernel, dtype, n, k, d, zeta=8, device=None, stream=None):
    """Time candidate launch parameters of kernel 0 (sparse gather apply) or 1 (SRTT) for this shape and
    keep the fastest in the tuning table; returns the chosen value (0 = the default rule)."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    chosen, ms = ctypes.c_int32(), ctypes.c_double()
    h = handle(dev)
    _check(load().rsk_autotune_sketch(h, kernel, _DT[dtype], n, k, d, zeta, ctypes.byref(chosen), ctypes.byref(ms),
                                      _stream(stream)), h)
    return chosen.value


def rsk_gemm_bf16(A, B, nsplit=1, stream=None):
    """D = A @ B.T on the tensor cores: A (M x K) and B (N x K) row-major CUDA BF16; D FP32 (M x N)
    returned column-major.  nsplit > 1 splits K that many ways; 0 lets the library choose (splits
    that fill the SMs, and a short last round of row tiles split over K)."""
    _matrix(A, "A")
    _matrix(B, "B")
    if A.dtype != torch.bfloat16 or B.dtype != torch.bfloat16 or A.shape[1] != B.shape[1]:
        raise ValueError("A and B must be bfloat16 with the same number of columns")
    M, K = A.shape
    N = B.shape[0]
    D = torch.empty(N, M, device=A.device).t()
    h = handle(A.device)
    _check(load().rsk_gemm_bf16(h, A.data_ptr(), M, K, A.stride(0), B.data_ptr(), N, B.stride(0), D.data_ptr(),
                                D.stride(1), nsplit, _stream(stream)), h)
    return D


def _gemm_operands(A, B, a_mn, dtype):
    _matrix(A, "A")
    _matrix(B, "B")
    if A.dtype != dtype or B.dtype != dtype:
        raise ValueError(f"A and B must be {dtype}")
    # a_mn: the product's A operand is A.T (A given K x M row-major, read MN-major in place)
    M, K = (A.shape[1], A.shape[0]) if a_mn else (A.shape[0], A.shape[1])
    if B.shape[1] != K:
        raise ValueError("B must have K columns")
    return M, K, B.shape[0]


def _gemm_out(M, N, row_major_out, device):
    return torch.empty(M, N, device=device) if row_major_out else torch.empty(N, M, device=device).t()


def rsk_gemm_bf16_ex(A, B, a_mn=False, row_major_out=False, nsplit=1, cluster=0, stream=None):
    """D = op(A) @ B.T on the tensor cores, BF16 operands, FP32 D (M x N).  op(A) = A.T when a_mn (A is
    K x M row-major, read in place as an MN-major operand), else A (M x K).  D row-major when
    row_major_out, else a column-major view.  cluster: row tiles sharing the B tile (0 automatic);
    nsplit as rsk_gemm_bf16."""
    M, K, N = _gemm_operands(A, B, a_mn, torch.bfloat16)
    D = _gemm_out(M, N, row_major_out, A.device)
    h = handle(A.device)
    _check(load().rsk_gemm_bf16_ex(h, int(a_mn), A.data_ptr(), M, K, A.stride(0), B.data_ptr(), N, B.stride(0),
                                   D.data_ptr(), D.stride(0) if row_major_out else D.stride(1), int(row_major_out),
                                   nsplit, cluster, _stream(stream)), h)
    return D


def rsk_gemm_f32(A, B, a_mn=False, row_major_out=False, nsplit=1, stream=None):
    """D = op(A) @ B.T for FP32 operands at FP32 accuracy (three-term BF16 splits on the tensor cores);
    layouts as rsk_gemm_bf16_ex."""
    M, K, N = _gemm_operands(A, B, a_mn, torch.float32)
    D = _gemm_out(M, N, row_major_out, A.device)
    h = handle(A.device)
    _check(load().rsk_gemm_f32(h, int(a_mn), A.data_ptr(), M, K, A.stride(0), B.data_ptr(), N, B.stride(0),
                               D.data_ptr(), D.stride(0) if row_major_out else D.stride(1), int(row_major_out), nsplit,
                               _stream(stream)), h)
    return D


def rsk_rsvd(A, r, power_iters=2, zeta=8, seed=0, stream=None):
    """Randomized SVD of a CUDA FP32 tensor A (m x n): returns (U [m, r] FP32, s [r] FP64, Vt [r, n] FP32)."""
    _matrix(A, "A")
    if A.dtype != torch.float32:
        raise TypeError("rsk_rsvd takes FP32 A")
    m, n = A.shape
    U = torch.empty(m, r, dtype=torch.float32, device=A.device)
    s = torch.empty(r, dtype=torch.float64, device=A.device)
    Vt = torch.empty(r, n, dtype=torch.float32, device=A.device)
    h = handle(A.device)
    st = load().rsk_rsvd(h, A.data_ptr(), m, n, A.stride(0), r, power_iters, zeta, seed, U.data_ptr(), s.data_ptr(),
                         Vt.data_ptr(), _stream(stream))
    _check(st, h)
    return U, s, Vt


# Kernel ids of rsk_profile_read (rsk_kernel_id in rsk.h).
KERNEL_IDS = {"sketch_index": 0, "sketch_apply": 1, "sketch_reduce": 2, "sketch_generate": 3,
              "srtt_apply": 4, "srtt_reduce": 5, "dense": 6, "gemm": 7, "factor": 8, "small_svd": 9,
              "convert": 10, "gemm_split": 11, "batch_sketch": 12, "batch_qr": 13, "batch_resid": 14,
              "batch_cg": 15}


def rsk_profile_enable(on=True, device=None):
    h = handle(device)
    _check(load().rsk_profile_enable(h, 1 if on else 0), h)


def rsk_profile_read(kernel, device=None):
    """(total device ms, launches) recorded for one kernel id since profiling was enabled."""
    h = handle(device)
    ms = ctypes.c_double()
    cnt = ctypes.c_int64()
    kid = KERNEL_IDS[kernel] if isinstance(kernel, str) else int(kernel)
    _check(load().rsk_profile_read(h, kid, ctypes.byref(ms), ctypes.byref(cnt)), h)
    return ms.value, cnt.value
