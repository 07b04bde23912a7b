"""Python names for the C ABI entry points (argument marshalling only)."""
from __future__ import annotations

import ctypes

import numpy as np

from ._lib import FFSPMVError, Options, check, lib, options_default


def _torch():
    import torch
    return torch


def stream_ptr(stream=None):
    """The cudaStream_t of a torch stream (default: torch's current one)."""
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(a):
    """Raw pointer of a torch tensor, a numpy array or an int."""
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        return a.ctypes.data if a.size else None
    return a.data_ptr() if a.numel() else None


def _as_u32_tensor(a, device):
    """A 4-byte integer tensor on `device` with the bits of `a` (numpy uint32,
    int32 or a torch tensor)."""
    torch = _torch()
    if isinstance(a, np.ndarray):
        a = torch.from_numpy(np.ascontiguousarray(a).view(np.int32))
    if a.dtype not in (torch.int32, torch.uint32):
        raise TypeError("residues must be 32-bit integers")
    return a.to(device).contiguous()


def spmv_create_hybrid(nrows, ncols, row_ptr, col, values, modulus, options=None,
                       stream=None):
    """Build a plan; arrays may be numpy (host) or torch (host or device)."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64) if isinstance(row_ptr, (list, np.ndarray)) else row_ptr
    col = np.ascontiguousarray(col, dtype=np.int32) if isinstance(col, (list, np.ndarray)) else col
    values = np.ascontiguousarray(values, dtype=np.uint32) if isinstance(values, (list, np.ndarray)) else values
    nnz = int(row_ptr[-1]) if len(row_ptr) else 0
    h = ctypes.c_void_p()
    opt = options if options is not None else options_default()
    st = lib().spmv_create_hybrid(ctypes.byref(h), int(nrows), int(ncols), nnz,
                                  _ptr(row_ptr), _ptr(col), _ptr(values),
                                  int(modulus), ctypes.byref(opt),
                                  stream_ptr(stream) if stream is not None else None)
    check(st, "spmv_create_hybrid")
    return h


def spmv_apply(h, x, ldx, y, ldy, nvec, alpha=1, beta=0, stream=None):
    check(lib().spmv_apply(h, _ptr(x), int(ldx), _ptr(y), int(ldy), int(nvec),
                           int(alpha), int(beta), stream_ptr(stream)), "spmv_apply")


def spmv_apply_transpose(h, x, ldx, y, ldy, nvec, alpha=1, beta=0, stream=None):
    check(lib().spmv_apply_transpose(h, _ptr(x), int(ldx), _ptr(y), int(ldy), int(nvec),
                                     int(alpha), int(beta), stream_ptr(stream)),
          "spmv_apply_transpose")


def spmv_apply_transpose_noalloc(h, x, ldx, y, ldy, nvec, alpha=1, beta=0, stream=None):
    check(lib().spmv_apply_transpose_noalloc(h, _ptr(x), int(ldx), _ptr(y), int(ldy), int(nvec),
                                             int(alpha), int(beta), stream_ptr(stream)),
          "spmv_apply_transpose_noalloc")


def spmv_block_sequence(h, X, Y, s, start_step, nsteps, S, V_state=None, stream=None):
    check(lib().spmv_block_sequence(h, _ptr(X), _ptr(Y), int(s), int(start_step), int(nsteps),
                                    _ptr(S), _ptr(V_state), stream_ptr(stream)),
          "spmv_block_sequence")


def spmv_block_project(p, n, s, X, V, Sacc, stream=None):
    check(lib().spmv_block_project(int(p), int(n), int(s), _ptr(X), _ptr(V), _ptr(Sacc), stream_ptr(stream)),
          "spmv_block_project")


def spmv_block_project_finish(p, s, Sacc, S, stream=None):
    check(lib().spmv_block_project_finish(int(p), int(s), _ptr(Sacc), _ptr(S), stream_ptr(stream)),
          "spmv_block_project_finish")


def spmv_batch_apply(handles, xs, ys, nvec, stream=None):
    n = len(handles)
    H = (ctypes.c_void_p * n)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    X = (ctypes.c_void_p * n)(*[_ptr(x) for x in xs])
    Y = (ctypes.c_void_p * n)(*[_ptr(y) for y in ys])
    NV = (ctypes.c_int32 * n)(*[int(v) for v in nvec])
    check(lib().spmv_batch_apply(n, H, X, Y, NV, stream_ptr(stream)), "spmv_batch_apply")


def spmv_destroy(h):
    if h:
        lib().spmv_destroy(h)


def spmv_describe_plan(h):
    buf = ctypes.create_string_buffer(1 << 16)
    check(lib().spmv_describe_plan(h, buf, len(buf)), "spmv_describe_plan")
    return buf.value.decode()


def spmv_get_info(h):
    v = [ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_uint32(), ctypes.c_int64()]
    check(lib().spmv_get_info(h, *[ctypes.byref(t) for t in v]), "spmv_get_info")
    return dict(nrows=v[0].value, ncols=v[1].value, nnz=v[2].value, modulus=v[3].value,
                device_bytes=v[4].value)


def spmv_count_launches(h, transpose, nvec):
    n = ctypes.c_int64()
    check(lib().spmv_count_launches(h, int(transpose), int(nvec), ctypes.byref(n)),
          "spmv_count_launches")
    return n.value


def spmv_apply_gf2(h, transpose, x, y, words, accumulate=False, stream=None):
    """Y = A X (or A^T X; Y ^= ... when accumulate) over GF(2), 64 components
    per 64-bit word; x, y: device tensors of 64-bit words."""
    check(lib().spmv_apply_gf2(h, int(transpose), _ptr(x), _ptr(y), int(words), int(bool(accumulate)),
                               stream_ptr(stream)), "spmv_apply_gf2")


def polymat_mul(p, A, B, stream=None):
    """C = A B mod p for polynomial matrices, coefficient-major (d+1, s, s)
    arrays of residues (numpy uint32 or torch int32 on the device); returns a
    device tensor of shape (da + db + 1, s, s)."""
    torch = _torch()
    dev = torch.device("cuda", torch.cuda.current_device())
    A = _as_u32_tensor(A, dev)
    B = _as_u32_tensor(B, dev)
    da, db, s = A.shape[0] - 1, B.shape[0] - 1, A.shape[1]
    need = ctypes.c_int64()
    check(lib().polymat_mul_workspace(s, da, db, ctypes.byref(need)), "polymat_mul_workspace")
    work = torch.empty(need.value, dtype=torch.uint8, device=dev)
    C = torch.empty((da + db + 1, s, s), dtype=torch.int32, device=dev)
    check(lib().polymat_mul(int(p), s, da, db, _ptr(A), _ptr(B), _ptr(C), _ptr(work), need.value,
                            stream_ptr(stream)), "polymat_mul")
    return C


def sigma_basis(p, F, shift=None, base=0, stream=None):
    """Order-d sigma-basis of F, a coefficient-major (d, m, n) array of
    residues (numpy uint32 or torch int32 on the device), d the order, for
    the row shift `shift` (m integers, default 0); `base` is the largest
    order handed to M-Basis (0 = the library's default).  Returns (P, delta,
    degree): P a device tensor (d + 1, m, m), delta the m shifted row
    degrees, degree an upper bound on deg P."""
    torch = _torch()
    dev = torch.device("cuda", torch.cuda.current_device())
    F = _as_u32_tensor(F, dev)
    d, m, n = F.shape
    need = ctypes.c_int64()
    check(lib().sigma_basis_workspace(m, n, d, int(base), ctypes.byref(need)), "sigma_basis_workspace")
    work = torch.empty(need.value, dtype=torch.uint8, device=dev)
    P = torch.empty((d + 1, m, m), dtype=torch.int32, device=dev)
    sh = None if shift is None else np.ascontiguousarray(shift, dtype=np.int32)
    delta = np.zeros(m, dtype=np.int32)
    deg = ctypes.c_int64()
    check(lib().sigma_basis(int(p), m, n, d, int(base), _ptr(F), _ptr(sh), _ptr(P), _ptr(delta),
                            ctypes.byref(deg), _ptr(work), need.value, stream_ptr(stream)), "sigma_basis")
    return P, [int(v) for v in delta], int(deg.value)


def sigma_generator_degrees(p, P, delta, n, max_precision=0, stream=None):
    """(deg det U, codeg det U) of the generator U of a sigma-basis: the n
    rows of P (a (d + 1, m, m) array, device or numpy) with the least
    (delta_i, i), first n columns.  deg - codeg is block Wiedemann's rank."""
    torch = _torch()
    dev = torch.device("cuda", torch.cuda.current_device())
    P = _as_u32_tensor(P, dev)
    d1, m = P.shape[0], P.shape[1]
    dl = np.ascontiguousarray(delta, dtype=np.int32)
    if dl.size != m:
        raise ValueError("delta needs one degree per row of P")
    deg, codeg = ctypes.c_int64(), ctypes.c_int64()
    check(lib().sigma_generator_degrees(int(p), m, int(n), d1 - 1, _ptr(P), _ptr(dl), int(max_precision),
                                        ctypes.byref(deg), ctypes.byref(codeg), stream_ptr(stream)),
          "sigma_generator_degrees")
    return int(deg.value), int(codeg.value)


def sigma_wiedemann_input(p, S, stream=None):
    """[S(x); -I] as a (L, 2s, s) device tensor, from the (L, s, s) block
    sequence S (device or numpy)."""
    torch = _torch()
    dev = torch.device("cuda", torch.cuda.current_device())
    S = _as_u32_tensor(S, dev)
    L, s = S.shape[0], S.shape[1]
    F = torch.empty((L, 2 * s, s), dtype=torch.int32, device=dev)
    check(lib().sigma_wiedemann_input(int(p), s, L, _ptr(S), _ptr(F), stream_ptr(stream)),
          "sigma_wiedemann_input")
    return F


def spmv_check_status(h, stream=None):
    """Synchronise the stream; raise FFSPMVError (FFSPMV_ERR_TIMEOUT) if a
    bounded device wait of an earlier apply on h ran out."""
    check(lib().spmv_check_status(h, stream_ptr(stream)), "spmv_check_status")


class Matrix:
    """An n x m sparse matrix over Z/mZ resident on the current CUDA device."""

    def __init__(self, nrows, ncols, row_ptr, col, values, modulus, options=None, **opts):
        if options is None:
            options = options_default(**opts)
        self.nrows, self.ncols, self.modulus = int(nrows), int(ncols), int(modulus)
        self.options = options
        self.handle = spmv_create_hybrid(nrows, ncols, row_ptr, col, values, modulus, options)

    @classmethod
    def from_csr(cls, A, **kw):
        """From an object with nrows, ncols, row_ptr, col, val, modulus."""
        return cls(A.nrows, A.ncols, A.row_ptr, A.col, A.val, kw.pop("modulus", A.modulus), **kw)

    def close(self):
        if getattr(self, "handle", None):
            spmv_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def describe(self):
        return spmv_describe_plan(self.handle)

    def info(self):
        return spmv_get_info(self.handle)

    def launches(self, transpose=False, nvec=1):
        return spmv_count_launches(self.handle, transpose, nvec)

    def check_status(self, stream=None):
        spmv_check_status(self.handle, stream)

    def _run(self, fn, x, y, out_rows, alpha, beta, stream):
        torch = _torch()
        dev = torch.device("cuda", torch.cuda.current_device())
        x = _as_u32_tensor(x, dev)
        nvec = 1 if x.dim() == 1 else x.shape[1]
        if y is None:
            shape = (out_rows,) if x.dim() == 1 else (out_rows, nvec)
            y = torch.empty(shape, dtype=torch.int32, device=dev)
            beta = 0
        fn(self.handle, x, nvec, y, nvec, nvec, alpha, beta, stream)
        return y

    def apply(self, x, y=None, alpha=1, beta=0, stream=None):
        """y <- alpha*A*x + beta*y (mod m); x: ncols or ncols x nvec."""
        return self._run(spmv_apply, x, y, self.nrows, alpha, beta, stream)

    def apply_transpose(self, x, y=None, alpha=1, beta=0, stream=None):
        """y <- alpha*A^T*x + beta*y (mod m); x: nrows or nrows x nvec."""
        return self._run(spmv_apply_transpose, x, y, self.ncols, alpha, beta, stream)

    def apply_gf2(self, x, y=None, transpose=False, accumulate=False, stream=None):
        """Y = A X (or A^T X) over GF(2), or Y ^= ... when accumulate; x: an
        in_rows x words array of 64-bit words (numpy uint64 or a torch int64
        tensor), bit b of word k = component 64 k + b."""
        torch = _torch()
        dev = torch.device("cuda", torch.cuda.current_device())
        if isinstance(x, np.ndarray):
            x = torch.from_numpy(np.ascontiguousarray(x).view(np.int64))
        x = x.to(dev).contiguous()
        words = x.shape[1] if x.dim() == 2 else 1
        out_rows = self.ncols if transpose else self.nrows
        if y is None:
            y = torch.zeros((out_rows, words) if x.dim() == 2 else (out_rows,), dtype=torch.int64, device=dev)
        spmv_apply_gf2(self.handle, transpose, x, y, words, accumulate, stream)
        return y

    def block_sequence(self, X, Y, nsteps, want_next=False, stream=None):
        """S_i = X^T A^i Y (mod m), 0 <= i < nsteps; X, Y: n x s.  With
        want_next, also returns V_nsteps = A^nsteps Y (the state from which
        `resume_sequence` continues)."""
        torch = _torch()
        dev = torch.device("cuda", torch.cuda.current_device())
        X = _as_u32_tensor(X, dev)
        Y = _as_u32_tensor(Y, dev)
        s = X.shape[1] if X.dim() == 2 else 1
        S = torch.empty((max(int(nsteps), 0), s, s), dtype=torch.int32, device=dev)
        Vn = torch.empty((self.nrows, s), dtype=torch.int32, device=dev) if want_next else None
        spmv_block_sequence(self.handle, X, Y, s, 0, nsteps, S, Vn, stream)
        return (S, Vn) if want_next else S

    def resume_sequence(self, X, V_state, start_step, nsteps, stream=None):
        """S_start_step .. S_{start_step+nsteps-1}, continuing from V_state =
        V_start_step (a device tensor, n x s), which is advanced in place to
        V_{start_step+nsteps}."""
        torch = _torch()
        dev = torch.device("cuda", torch.cuda.current_device())
        X = _as_u32_tensor(X, dev)
        s = X.shape[1] if X.dim() == 2 else 1
        S = torch.empty((max(int(nsteps), 0), s, s), dtype=torch.int32, device=dev)
        spmv_block_sequence(self.handle, X, None, s, start_step, nsteps, S, V_state, stream)
        return S


def to_numpy_u32(t):
    """Host numpy uint32 copy of a 4-byte integer tensor."""
    return t.detach().cpu().numpy().view(np.uint32)


__all__ = ["Matrix", "spmv_create_hybrid", "spmv_apply", "spmv_apply_transpose",
           "spmv_apply_transpose_noalloc",
           "spmv_block_sequence", "spmv_block_project", "spmv_block_project_finish",
           "spmv_batch_apply", "spmv_destroy",
           "spmv_describe_plan", "spmv_get_info", "spmv_count_launches", "spmv_check_status",
           "spmv_apply_gf2", "polymat_mul", "sigma_basis", "sigma_wiedemann_input", "stream_ptr",
           "to_numpy_u32",
           "FFSPMVError", "Options"]
