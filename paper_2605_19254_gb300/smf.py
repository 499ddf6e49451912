"""Thin ctypes binding of the C ABI in include/smf.h (argument marshalling only).

Every computation runs in libsmf.so's CUDA kernels.  Device buffers are torch
tensors (torch is used for device memory and streams only); big-integer
matrices are int64 tensors of shape [rows, cols, W] holding the two's
complement words.  If libsmf.so is missing the first call raises: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsmf.so")

SMF_OK = 0
SMF_E_INVALID = 1
SMF_E_SINGULAR = 2
SMF_E_NOMEM = 3
SMF_E_CUDA = 4
SMF_E_BOUND = 5
SMF_E_TIMEOUT = 6
SMF_E_RETRY_EXHAUSTED = 7
SMF_E_UNSUPPORTED = 8
SMF_FORM_FP64 = 0
SMF_FORM_INT8LIMB = 1
SMF_PROF_KINDS = 5
SMF_INJECT_STALL_LOADS = 1
SMF_INJECT_WRONG_SMITH = 2
SMF_INJECT_WRONG_SMITH_ALWAYS = 4
SMF_PLAN_AUTOTUNE = 1
SMF_PLAN_PAD_ALL = 2
SMF_PLAN_ORDER_WORK = 4
SMF_PLAN_PREFETCH = 8
SMF_PLAN_ONE_DIGIT = 16
PROF_NAMES = ("reduce", "digits", "residue_gemm", "crt", "copies")

# every symbol include/smf.h declares
EXPORTS = (
    "smf_create", "smf_destroy", "smf_last_error", "smf_basis_create", "smf_basis_destroy",
    "smf_basis_info", "smf_rns_reduce", "smf_residue_gemm", "smf_residue_gemm_workspace",
    "smf_crt_reconstruct", "smf_rns_matmul", "smf_rns_matmul_workspace", "smf_status_sync",
    "smf_profile_enable", "smf_profile_read", "smf_version", "smf_residue_gemm_noalloc", "smf_debug_inject",
    "smf_rns_matmul_grouped", "smf_rns_matmul_grouped_workspace", "smf_base_convert",
    "smf_server_create", "smf_server_submit", "smf_server_step", "smf_server_job", "smf_server_stats",
    "smf_server_drain", "smf_server_destroy", "smf_server_admit", "smf_padic_lift", "smf_padic_lift_workspace",
    "smf_inverse_mod_p", "smf_inverse_mod_p_workspace", "smf_largest_invariant_factor", "smf_rational_reconstruct",
    "smf_smith_form", "smf_det_mod", "smf_smith_local", "smf_fp64_peak",
    "smf_smith_server_create", "smf_smith_server_submit", "smf_smith_server_job", "smf_smith_server_result",
    "smf_smith_server_stats", "smf_smith_server_drain", "smf_smith_server_destroy", "smf_smith_server_message",
    "smf_group_plan_create", "smf_group_plan_launch", "smf_group_plan_info", "smf_group_plan_report",
    "smf_group_plan_destroy", "smf_set_fused_crt", "smf_set_elim_panels",
)


class SmfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"smf error {code}: {msg}")
        self.code = code


class Bigmat(ctypes.Structure):
    _fields_ = [
        ("rows", ctypes.c_int64), ("cols", ctypes.c_int64), ("ld", ctypes.c_int64),
        ("words", ctypes.c_int32), ("bits", ctypes.c_int32), ("data", ctypes.c_void_p),
        ("on_device", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


_lib = None
_lock = threading.Lock()


def lib():
    """Load libsmf.so (raises when it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libsmf.so is not built ({LIB_PATH}); run __graft_entry__.build()")
            L = ctypes.CDLL(LIB_PATH)
            P, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
            L.smf_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, ctypes.c_int, sz]
            L.smf_destroy.argtypes = [P]
            L.smf_last_error.argtypes = [P]
            L.smf_last_error.restype = ctypes.c_char_p
            L.smf_basis_create.argtypes = [P, i32, ctypes.c_uint32, ctypes.POINTER(P)]
            L.smf_basis_destroy.argtypes = [P]
            L.smf_basis_info.argtypes = [P, ctypes.POINTER(i32), ctypes.POINTER(ctypes.POINTER(ctypes.c_uint32))]
            L.smf_rns_reduce.argtypes = [P, P, ctypes.POINTER(Bigmat), P, P]
            L.smf_residue_gemm.argtypes = [P, P, P, i64, P, P, i64, i64, i64, P, sz, P]
            L.smf_residue_gemm_noalloc.argtypes = [P, P, P, i64, P, P, i64, i64, i64, P]
            L.smf_residue_gemm_workspace.argtypes = [P, P, i64, i64, i64, ctypes.c_int, ctypes.POINTER(sz)]
            L.smf_crt_reconstruct.argtypes = [P, P, P, ctypes.POINTER(Bigmat), P]
            L.smf_base_convert.argtypes = [P, P, P, P, P, ctypes.c_int64, P]
            L.smf_padic_lift_workspace.argtypes = [P, P, ctypes.POINTER(Bigmat), ctypes.POINTER(Bigmat),
                                                   ctypes.POINTER(sz)]
            L.smf_padic_lift.argtypes = [P, P, ctypes.POINTER(Bigmat), P, ctypes.POINTER(Bigmat), ctypes.c_int32, P,
                                         ctypes.POINTER(Bigmat), P, sz, P]
            L.smf_inverse_mod_p_workspace.argtypes = [P, i64, ctypes.POINTER(sz)]
            L.smf_inverse_mod_p.argtypes = [P, P, ctypes.POINTER(Bigmat), P, P, sz, P]
            L.smf_largest_invariant_factor.argtypes = [P, ctypes.POINTER(Bigmat), i32, ctypes.c_uint64, P, i32,
                                                       ctypes.POINTER(i32), P, P]
            L.smf_smith_form.argtypes = [P, ctypes.POINTER(Bigmat), ctypes.c_uint64, P, i64, P, P,
                                         ctypes.POINTER(i32), P]
            L.smf_fp64_peak.argtypes = [P, ctypes.POINTER(ctypes.c_double), P]
            L.smf_smith_server_create.argtypes = [ctypes.c_int, ctypes.c_int, sz, ctypes.c_int, ctypes.POINTER(P)]
            L.smf_smith_server_submit.argtypes = [P, ctypes.POINTER(Bigmat), ctypes.c_uint64,
                                                  ctypes.POINTER(ctypes.c_int64)]
            L.smf_smith_server_job.argtypes = [P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int),
                                               ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
            L.smf_smith_server_result.argtypes = [P, ctypes.c_int64, P, i64, P]
            L.smf_smith_server_stats.argtypes = [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                                 ctypes.POINTER(sz)]
            L.smf_smith_server_drain.argtypes = [P]
            L.smf_smith_server_message.argtypes = [P, ctypes.c_int64, ctypes.c_char_p, i64]
            L.smf_smith_server_destroy.argtypes = [P]
            L.smf_det_mod.argtypes = [P, ctypes.POINTER(Bigmat), P, i32, P, P]
            L.smf_smith_local.argtypes = [P, ctypes.POINTER(Bigmat), P, P, i32, P, P]
            L.smf_rational_reconstruct.argtypes = [P, i32, P, i32, i64, i64, P, ctypes.POINTER(i32),
                                                   ctypes.POINTER(i32), P, ctypes.POINTER(i32), i32]
            L.smf_server_create.argtypes = [P, sz, ctypes.c_int, ctypes.POINTER(P)]
            L.smf_server_submit.argtypes = [P, ctypes.POINTER(Bigmat), ctypes.POINTER(Bigmat), ctypes.POINTER(Bigmat),
                                            ctypes.POINTER(ctypes.c_int64)]
            L.smf_server_step.argtypes = [P, ctypes.POINTER(ctypes.c_int)]
            L.smf_server_job.argtypes = [P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_double)]
            L.smf_server_stats.argtypes = [P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(sz)]
            L.smf_server_drain.argtypes = [P]
            L.smf_server_destroy.argtypes = [P]
            L.smf_server_admit.argtypes = [sz, ctypes.c_int, ctypes.POINTER(sz), ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_int)]
            L.smf_rns_matmul.argtypes = [P, ctypes.POINTER(Bigmat), ctypes.POINTER(Bigmat), ctypes.POINTER(Bigmat),
                                         P, sz, P]
            L.smf_rns_matmul_workspace.argtypes = [P, ctypes.POINTER(Bigmat), ctypes.POINTER(Bigmat),
                                                   ctypes.POINTER(Bigmat), ctypes.POINTER(sz)]
            L.smf_rns_matmul_grouped.argtypes = [P, ctypes.c_int, ctypes.POINTER(Bigmat), ctypes.POINTER(Bigmat),
                                                 ctypes.POINTER(Bigmat), P, sz, P]
            L.smf_rns_matmul_grouped_workspace.argtypes = [P, ctypes.c_int, ctypes.POINTER(Bigmat),
                                                           ctypes.POINTER(Bigmat), ctypes.POINTER(Bigmat),
                                                           ctypes.POINTER(sz)]
            L.smf_group_plan_create.argtypes = [P, ctypes.c_int, ctypes.POINTER(Bigmat), ctypes.POINTER(Bigmat),
                                                ctypes.POINTER(Bigmat), ctypes.c_int, ctypes.POINTER(P), P]
            L.smf_group_plan_launch.argtypes = [P, P]
            L.smf_group_plan_info.argtypes = [P, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                              ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                              ctypes.POINTER(i32),
                                              ctypes.POINTER(ctypes.c_double), ctypes.POINTER(sz)]
            L.smf_group_plan_report.argtypes = [P, ctypes.c_char_p, i64]
            L.smf_group_plan_destroy.argtypes = [P]
            L.smf_set_fused_crt.argtypes = [P, ctypes.c_int]
            L.smf_set_elim_panels.argtypes = [P, ctypes.c_int64]
            L.smf_status_sync.argtypes = [P, P]
            L.smf_debug_inject.argtypes = [P, ctypes.c_int]
            L.smf_profile_enable.argtypes = [P, ctypes.c_int]
            L.smf_profile_read.argtypes = [P, P, P]
            L.smf_version.restype = ctypes.c_char_p
            _lib = L
    return _lib


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def bigmat(t, bits: int = 0) -> Bigmat:
    """Descriptor of an int64 tensor [rows, cols, W] (device or host)."""
    if t.dim() != 3:
        raise ValueError("big-integer matrix tensors are [rows, cols, W]")
    rows, cols, W = t.shape
    if t.numel() == 0:  # no entries: strides carry no layout
        return Bigmat(rows, cols, cols, W, bits, ctypes.c_void_p(t.data_ptr()), 1 if t.is_cuda else 0, 0)
    # a dimension of size one carries no layout, whatever its stride
    if (W > 1 and t.stride(2) != 1) or (cols > 1 and t.stride(1) != W):
        raise ValueError("entries must be contiguous words")
    if rows > 1 and t.stride(0) % W:
        raise ValueError("rows must start on an entry boundary")
    ld = t.stride(0) // W if rows > 1 else cols
    return Bigmat(rows, cols, ld, W, bits, ctypes.c_void_p(t.data_ptr()), 1 if t.is_cuda else 0, 0)


def _to_limbs(x: int):
    """Non-negative int -> little-endian 32-bit limbs (ctypes array) and their count."""
    limbs = []
    while x:
        limbs.append(x & 0xFFFFFFFF)
        x >>= 32
    arr = (ctypes.c_uint32 * max(1, len(limbs)))(*limbs)
    return arr, len(limbs)


def _from_limbs(arr, count: int) -> int:
    return sum(int(arr[i]) << (32 * i) for i in range(count))


def rational_reconstruct(u: int, P: int, nb: int, db: int):
    """(a, b) with a = b u mod P, |a| < 2^nb, 0 < b < 2^db, in lowest terms (host only)."""
    ua, ul = _to_limbs(u)
    pa, pl = _to_limbs(P)
    cap = pl + 2
    num, den = (ctypes.c_uint32 * cap)(), (ctypes.c_uint32 * cap)()
    nl, neg, dl = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    rc = lib().smf_rational_reconstruct(ua, ul, pa, pl, nb, db, num, ctypes.byref(nl), ctypes.byref(neg), den,
                                        ctypes.byref(dl), cap)
    if rc != SMF_OK:
        raise SmfError(rc, "rational reconstruction: no fraction within the bounds")
    a = _from_limbs(num, nl.value)
    return (-a if neg.value else a), _from_limbs(den, dl.value)


class Basis:
    def __init__(self, ctx: "Context", handle):
        self.ctx = ctx
        self.handle = handle

    @property
    def primes(self):
        n = ctypes.c_int32()
        p = ctypes.POINTER(ctypes.c_uint32)()
        lib().smf_basis_info(self.handle, ctypes.byref(n), ctypes.byref(p))
        return [int(p[i]) for i in range(n.value)]

    def destroy(self):
        if self.handle:
            lib().smf_basis_destroy(self.handle)
            self.handle = None


class Context:
    """One smf_ctx (device + residue-product form)."""

    def __init__(self, device: int = 0, form: int = SMF_FORM_INT8LIMB, hbm_budget_bytes: int = 0):
        h = ctypes.c_void_p()
        rc = lib().smf_create(ctypes.byref(h), device, form, hbm_budget_bytes)
        if rc != SMF_OK:
            raise SmfError(rc, "smf_create failed")
        self.handle = h
        self.device = device
        self.form = form

    def _check(self, rc):
        if rc != SMF_OK:
            raise SmfError(rc, lib().smf_last_error(self.handle).decode())

    def destroy(self):
        if self.handle:
            lib().smf_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass

    # ---- ABI calls -------------------------------------------------------
    def basis_create(self, bound_bits: int, p_max: int = 0) -> Basis:
        h = ctypes.c_void_p()
        self._check(lib().smf_basis_create(self.handle, bound_bits, p_max, ctypes.byref(h)))
        return Basis(self, h)

    def rns_reduce(self, basis: Basis, X, residues, bits: int = 0, stream=None):
        d = bigmat(X, bits)
        self._check(lib().smf_rns_reduce(self.handle, basis.handle, ctypes.byref(d),
                                         ctypes.c_void_p(residues.data_ptr()), _stream_ptr(stream)))

    def residue_gemm_workspace(self, basis: Basis, M: int, N: int, K: int, a_shared: bool) -> int:
        n = ctypes.c_size_t()
        self._check(lib().smf_residue_gemm_workspace(self.handle, basis.handle, M, N, K, int(a_shared),
                                                     ctypes.byref(n)))
        return n.value

    @staticmethod
    def _check_residue_operands(basis: Basis, A, a_prime_stride: int, B, C, M: int, N: int, K: int):
        """The residue product's operands must be contiguous int32 CUDA tensors holding at
        least the entries the sizes imply (the C side cannot check device buffers)."""
        L = len(basis.primes)
        if min(M, N, K, a_prime_stride) < 0:
            raise ValueError("negative size or stride")
        a_need = (M * K if a_prime_stride == 0 else (L - 1) * a_prime_stride + M * K) if M * K else 0
        for name, t, need in (("A", A, a_need), ("B", B, L * K * N), ("C", C, L * M * N)):
            if not t.is_cuda or t.dtype.itemsize != 4 or t.dtype.is_floating_point or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous int32 CUDA tensor")
            if t.numel() < need:
                raise ValueError(f"{name} holds {t.numel()} entries; the sizes need {need}")

    def residue_gemm(self, basis: Basis, A, a_prime_stride: int, B, C, M: int, N: int, K: int,
                     workspace=None, stream=None):
        self._check_residue_operands(basis, A, a_prime_stride, B, C, M, N, K)
        ws = ctypes.c_void_p(workspace.data_ptr()) if workspace is not None else ctypes.c_void_p()
        nbytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
        self._check(lib().smf_residue_gemm(self.handle, basis.handle, ctypes.c_void_p(A.data_ptr()),
                                           a_prime_stride, ctypes.c_void_p(B.data_ptr()),
                                           ctypes.c_void_p(C.data_ptr()), M, N, K, ws, nbytes,
                                           _stream_ptr(stream)))

    def residue_gemm_noalloc(self, basis: Basis, A, a_prime_stride: int, B, C, M: int, N: int, K: int,
                             stream=None):
        self._check_residue_operands(basis, A, a_prime_stride, B, C, M, N, K)
        self._check(lib().smf_residue_gemm_noalloc(self.handle, basis.handle, ctypes.c_void_p(A.data_ptr()),
                                                   a_prime_stride, ctypes.c_void_p(B.data_ptr()),
                                                   ctypes.c_void_p(C.data_ptr()), M, N, K, _stream_ptr(stream)))

    def crt_reconstruct(self, basis: Basis, residues, X_out, stream=None):
        d = bigmat(X_out)
        self._check(lib().smf_crt_reconstruct(self.handle, basis.handle, ctypes.c_void_p(residues.data_ptr()),
                                              ctypes.byref(d), _stream_ptr(stream)))

    def padic_lift(self, p_basis: Basis, A, A_inv_mod_p, B, steps: int, X_digits, R, a_bits: int = 0,
                   b_bits: int = 0, workspace=None, stream=None):
        """Dixon lifting: X_digits [steps, n, m] and R (n x m words) with A sum X_i p^i + p^steps R = B."""
        da, db, dr = bigmat(A, a_bits), bigmat(B, b_bits), bigmat(R)
        ws = ctypes.c_void_p(workspace.data_ptr()) if workspace is not None else ctypes.c_void_p()
        nbytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
        self._check(lib().smf_padic_lift(self.handle, p_basis.handle, ctypes.byref(da),
                                         ctypes.c_void_p(A_inv_mod_p.data_ptr()), ctypes.byref(db), steps,
                                         ctypes.c_void_p(X_digits.data_ptr()), ctypes.byref(dr), ws, nbytes,
                                         _stream_ptr(stream)))

    def padic_lift_workspace(self, p_basis: Basis, A, B, a_bits: int = 0, b_bits: int = 0) -> int:
        n = ctypes.c_size_t()
        da, db = bigmat(A, a_bits), bigmat(B, b_bits)
        self._check(lib().smf_padic_lift_workspace(self.handle, p_basis.handle, ctypes.byref(da), ctypes.byref(db),
                                                   ctypes.byref(n)))
        return n.value

    def inverse_mod_p_workspace(self, n: int) -> int:
        b = ctypes.c_size_t()
        self._check(lib().smf_inverse_mod_p_workspace(self.handle, n, ctypes.byref(b)))
        return b.value

    def inverse_mod_p(self, p_basis: Basis, A, A_inv, a_bits: int = 0, workspace=None, stream=None):
        """A^-1 mod p (int32 [n, n], canonical) into A_inv; SMF_E_SINGULAR at the next status_sync if p | det A."""
        da = bigmat(A, a_bits)
        if A_inv.dtype.itemsize != 4 or not A_inv.is_contiguous() or A_inv.numel() != da.rows * da.cols:
            raise ValueError("A_inv must be a contiguous int32 [n, n] tensor")
        ws = ctypes.c_void_p(workspace.data_ptr()) if workspace is not None else ctypes.c_void_p()
        nbytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
        self._check(lib().smf_inverse_mod_p(self.handle, p_basis.handle, ctypes.byref(da),
                                            ctypes.c_void_p(A_inv.data_ptr()), ws, nbytes, _stream_ptr(stream)))

    def largest_invariant_factor(self, A, m: int = 32, seed: int = 0, a_bits: int = 0, stream=None):
        """s_n of A ([n, n, 1] int64, host or device) and the seconds of its phases
        (A^-1 mod p, lifting, reconstruction, total)."""
        da = bigmat(A, a_bits)
        cap = 3 * da.rows + 64  # |det A| has at most about 2.3 n limbs for entries below 2^40
        while True:
            limbs = (ctypes.c_uint32 * cap)()
            n_limbs = ctypes.c_int32()
            secs = (ctypes.c_double * 4)()
            rc = lib().smf_largest_invariant_factor(self.handle, ctypes.byref(da), m, seed, limbs, cap,
                                                    ctypes.byref(n_limbs), secs, _stream_ptr(stream))
            if rc == SMF_E_NOMEM and n_limbs.value > cap:
                cap = n_limbs.value
                continue
            self._check(rc)
            return _from_limbs(limbs, n_limbs.value), tuple(secs)

    def smith_form(self, A, seed: int = 0, a_bits: int = 0, stream=None):
        """The Smith form of a nonsingular A ([n, n, 1] int64, host or device):
        (the invariant factors s_1 | ... | s_n as Python ints, the seconds of
        Phase 1, Phase 2, Phase 3 and the total, the attempts run)."""
        da = bigmat(A, a_bits)
        n = da.rows
        cap = n + (n * (max(a_bits, 1) + n.bit_length())) // 32 + 64
        offs = (ctypes.c_int64 * (n + 1))()
        secs = (ctypes.c_double * 4)()
        att = ctypes.c_int32()
        while True:
            limbs = (ctypes.c_uint32 * max(1, cap))()
            rc = lib().smf_smith_form(self.handle, ctypes.byref(da), seed, limbs, cap, offs, secs, ctypes.byref(att),
                                      _stream_ptr(stream))
            if rc == SMF_E_NOMEM and offs[n] > cap:
                cap = offs[n]
                continue
            self._check(rc)
            s = []
            for i in range(n):
                v = 0
                for j in range(offs[i + 1] - 1, offs[i] - 1, -1):
                    v = (v << 32) | int(limbs[j])
                s.append(v)
            return s, tuple(secs), att.value

    def fp64_peak(self, stream=None) -> float:
        """Measured FP64 FMA throughput of the device (TFLOP/s): the FP64 form's roofline."""
        t = ctypes.c_double()
        self._check(lib().smf_fp64_peak(self.handle, ctypes.byref(t), _stream_ptr(stream)))
        return t.value

    def det_mod(self, A, q, a_bits: int = 0, stream=None):
        """det A mod a prime q < 2^62 ([n, n, 1] int64, host or device), on the device; with a
        list of primes, the list of determinants (up to four per column loop)."""
        qs = list(q) if isinstance(q, (list, tuple)) else [q]
        qa = (ctypes.c_uint64 * len(qs))(*qs)
        d = (ctypes.c_uint64 * len(qs))()
        self._check(lib().smf_det_mod(self.handle, ctypes.byref(bigmat(A, a_bits)), qa, len(qs), d,
                                      _stream_ptr(stream)))
        out = [int(v) for v in d]
        return out if isinstance(q, (list, tuple)) else out[0]

    def smith_local(self, A, q, e, a_bits: int = 0, stream=None):
        """[counts[t] for t = 0 .. e]: the number of invariant factors of A divisible by q^t; with
        lists of primes and exponents, one such list per prime (one joint column loop)."""
        many = isinstance(q, (list, tuple))
        qs, es = (list(q), list(e)) if many else ([q], [e])
        counts = (ctypes.c_int64 * sum(x + 1 for x in es))()
        self._check(lib().smf_smith_local(self.handle, ctypes.byref(bigmat(A, a_bits)),
                                          (ctypes.c_uint64 * len(qs))(*qs), (ctypes.c_int32 * len(es))(*es),
                                          len(qs), counts, _stream_ptr(stream)))
        out, off = [], 0
        for x in es:
            out.append([int(c) for c in counts[off:off + x + 1]])
            off += x + 1
        return out if many else out[0]

    def base_convert(self, src: Basis, dst: Basis, residues_in, residues_out, stream=None):
        """Residues [L_src, ...] of integers in basis `src` -> their residues [L_dst, ...] in `dst`."""
        count = residues_in.numel() // max(1, residues_in.shape[0]) if residues_in.dim() else 0
        if residues_out.numel() != count * len(dst.primes) or residues_in.numel() != count * len(src.primes):
            raise ValueError("residue tensors do not match the bases")
        if not (residues_in.is_contiguous() and residues_out.is_contiguous()):
            raise ValueError("residue tensors must be contiguous")
        self._check(lib().smf_base_convert(self.handle, src.handle, dst.handle,
                                           ctypes.c_void_p(residues_in.data_ptr()),
                                           ctypes.c_void_p(residues_out.data_ptr()), count, _stream_ptr(stream)))

    def rns_matmul_workspace(self, A, B, C, a_bits: int = 0, b_bits: int = 0) -> int:
        n = ctypes.c_size_t()
        da, db, dc = bigmat(A, a_bits), bigmat(B, b_bits), bigmat(C)
        self._check(lib().smf_rns_matmul_workspace(self.handle, ctypes.byref(da), ctypes.byref(db),
                                                   ctypes.byref(dc), ctypes.byref(n)))
        return n.value

    def rns_matmul(self, A, B, C, a_bits: int = 0, b_bits: int = 0, workspace=None, stream=None):
        da, db, dc = bigmat(A, a_bits), bigmat(B, b_bits), bigmat(C)
        ws = ctypes.c_void_p(workspace.data_ptr()) if workspace is not None else ctypes.c_void_p()
        nbytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
        self._check(lib().smf_rns_matmul(self.handle, ctypes.byref(da), ctypes.byref(db), ctypes.byref(dc), ws,
                                         nbytes, _stream_ptr(stream)))

    @staticmethod
    def _bigmats(ts, bits=0):
        """Descriptors of a list of tensors; `bits` is one bound for all or one per tensor."""
        per = list(bits) if isinstance(bits, (list, tuple)) else [bits] * len(ts)
        if len(per) != len(ts):
            raise ValueError("one bit bound per matrix")
        arr = (Bigmat * max(1, len(ts)))()
        for i, t in enumerate(ts):
            arr[i] = bigmat(t, per[i])
        return arr

    def rns_matmul_grouped_workspace(self, As, Bs, Cs, a_bits=0, b_bits=0) -> int:
        n = ctypes.c_size_t()
        self._check(lib().smf_rns_matmul_grouped_workspace(
            self.handle, len(As), self._bigmats(As, a_bits), self._bigmats(Bs, b_bits), self._bigmats(Cs),
            ctypes.byref(n)))
        return n.value

    def rns_matmul_grouped(self, As, Bs, Cs, a_bits=0, b_bits=0, workspace=None, stream=None):
        """C_i = A_i B_i exactly for every i, the residue products in one launch.

        a_bits / b_bits: one entry-size bound for every matrix, or one per matrix
        (0: the full word width)."""
        if not (len(As) == len(Bs) == len(Cs)):
            raise ValueError("As, Bs and Cs differ in length")
        ws = ctypes.c_void_p(workspace.data_ptr()) if workspace is not None else ctypes.c_void_p()
        nbytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
        self._check(lib().smf_rns_matmul_grouped(
            self.handle, len(As), self._bigmats(As, a_bits), self._bigmats(Bs, b_bits), self._bigmats(Cs), ws, nbytes,
            _stream_ptr(stream)))

    def group_plan(self, As, Bs, Cs, a_bits=0, b_bits=0, flags: int = 0, stream=None) -> "GroupPlan":
        """A grouped product prepared once and replayed as a CUDA graph (see smf.h)."""
        return GroupPlan(self, As, Bs, Cs, a_bits, b_bits, flags, stream)

    def set_fused_crt(self, enable: bool = True):
        """Residue product and CRT in one kernel where the product allows it (see smf.h)."""
        self._check(lib().smf_set_fused_crt(self.handle, int(enable)))

    def set_elim_panels(self, min_n: int = 0):
        """Eliminations over Z/(m) of at least min_n columns by panels of 16 (0: the defaults,
        2560 for determinants and 1536 for local Smith forms)."""
        self._check(lib().smf_set_elim_panels(self.handle, int(min_n)))

    def status_sync(self, stream=None):
        self._check(lib().smf_status_sync(self.handle, _stream_ptr(stream)))

    def debug_inject(self, flags: int):
        self._check(lib().smf_debug_inject(self.handle, flags))

    def profile_enable(self, on: bool = True):
        self._check(lib().smf_profile_enable(self.handle, int(on)))

    def profile_read(self):
        counts = (ctypes.c_int32 * SMF_PROF_KINDS)()
        ms = (ctypes.c_double * SMF_PROF_KINDS)()
        self._check(lib().smf_profile_read(self.handle, counts, ms))
        return {PROF_NAMES[k]: (counts[k], ms[k]) for k in range(SMF_PROF_KINDS)}


class GroupPlan:
    """smf_group_plan: the products C_i = A_i B_i on fixed buffers, launched by graph replay."""

    def __init__(self, ctx: "Context", As, Bs, Cs, a_bits=0, b_bits=0, flags: int = 0, stream=None):
        if not (len(As) == len(Bs) == len(Cs)):
            raise ValueError("As, Bs and Cs differ in length")
        for t in list(As) + list(Bs) + list(Cs):
            if not t.is_cuda:
                raise ValueError("plan operands must be on the device")
        self.ctx = ctx
        self._keep = (list(As), list(Bs), list(Cs))  # the plan reads and writes these buffers
        h = ctypes.c_void_p()
        ctx._check(lib().smf_group_plan_create(ctx.handle, len(As), Context._bigmats(As, a_bits),
                                               Context._bigmats(Bs, b_bits), Context._bigmats(Cs), flags,
                                               ctypes.byref(h), _stream_ptr(stream)))
        self.handle = h

    def launch(self, stream=None):
        self.ctx._check(lib().smf_group_plan_launch(self.handle, _stream_ptr(stream)))

    def info(self) -> dict:
        i32 = ctypes.c_int32
        g, pad, pf, one, order, tuned, cached = i32(), i32(), i32(), i32(), i32(), i32(), i32()
        ms, ws = ctypes.c_double(), ctypes.c_size_t()
        self.ctx._check(lib().smf_group_plan_info(self.handle, ctypes.byref(g), ctypes.byref(pad), ctypes.byref(pf),
                                                  ctypes.byref(one), ctypes.byref(order), ctypes.byref(tuned),
                                                  ctypes.byref(cached), ctypes.byref(ms), ctypes.byref(ws)))
        return {"graph": bool(g.value), "padded": pad.value, "prefetched": pf.value, "one_digit": one.value,
                "tile_order": order.value,
                "classes_tuned": tuned.value, "classes_cached": cached.value, "tune_ms": ms.value,
                "workspace_bytes": ws.value}

    def report(self) -> str:
        buf = ctypes.create_string_buffer(1 << 16)
        self.ctx._check(lib().smf_group_plan_report(self.handle, buf, len(buf)))
        return buf.value.decode()

    def destroy(self):
        if getattr(self, "handle", None):
            lib().smf_group_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


SMF_JOB_QUEUED, SMF_JOB_RUNNING, SMF_JOB_DONE, SMF_JOB_FAILED = 0, 1, 2, 3


def server_admit(budget_left: int, bytes_list, max_batch: int):
    """The server's admission rule on its own (host only): which queued jobs a step admits."""
    n = len(bytes_list)
    b = (ctypes.c_size_t * max(1, n))(*bytes_list)
    a = (ctypes.c_int * max(1, n))()
    k = lib().smf_server_admit(budget_left, n, b, max_batch, a)
    if k < 0:
        raise ValueError("bad arguments")
    return [int(a[i]) for i in range(n)]


class Server:
    """Continuous batching of exact products over the grouped launch (see smf.h)."""

    def __init__(self, ctx: "Context", budget_bytes: int, max_batch: int = 64):
        self.ctx = ctx
        h = ctypes.c_void_p()
        ctx._check(lib().smf_server_create(ctx.handle, budget_bytes, max_batch, ctypes.byref(h)))
        self.handle = h
        self._keep = {}  # the tensors of jobs not yet done stay referenced

    def submit(self, A, B, C, a_bits: int = 0, b_bits: int = 0) -> int:
        da, db, dc = bigmat(A, a_bits), bigmat(B, b_bits), bigmat(C)
        jid = ctypes.c_int64()
        self.ctx._check(lib().smf_server_submit(self.handle, ctypes.byref(da), ctypes.byref(db), ctypes.byref(dc),
                                                ctypes.byref(jid)))
        self._keep[jid.value] = (A, B, C)
        return jid.value

    def step(self) -> int:
        n = ctypes.c_int()
        self.ctx._check(lib().smf_server_step(self.handle, ctypes.byref(n)))
        return n.value

    def job(self, jid: int):
        """(state, status, (t_submit, t_start, t_done))"""
        st, code = ctypes.c_int(), ctypes.c_int()
        t = (ctypes.c_double * 3)()
        self.ctx._check(lib().smf_server_job(self.handle, jid, ctypes.byref(st), ctypes.byref(code), t))
        if st.value in (SMF_JOB_DONE, SMF_JOB_FAILED):
            self._keep.pop(jid, None)
        return st.value, code.value, (t[0], t[1], t[2])

    def message(self, jid: int) -> str:
        """A failed job's error message ("" for a job that did not fail)."""
        buf = ctypes.create_string_buffer(512)
        rc = lib().smf_smith_server_message(self.handle, jid, buf, 512)
        if rc != SMF_OK:
            raise SmfError(rc, "smith_server_message failed")
        return buf.value.decode(errors="replace")

    def stats(self):
        q, r = ctypes.c_int(), ctypes.c_int()
        b = ctypes.c_size_t()
        self.ctx._check(lib().smf_server_stats(self.handle, ctypes.byref(q), ctypes.byref(r), ctypes.byref(b)))
        return q.value, r.value, b.value

    def drain(self):
        self.ctx._check(lib().smf_server_drain(self.handle))

    def destroy(self):
        if self.handle:
            lib().smf_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()


def version() -> str:
    return lib().smf_version().decode()


class SmithServer:
    """Continuous batching of Smith-form jobs (see smf.h): worker threads with their own
    contexts and streams, admission by device footprint, per-job latency."""

    def __init__(self, device: int = 0, form: int = SMF_FORM_INT8LIMB, budget_bytes: int = 0, workers: int = 4):
        h = ctypes.c_void_p()
        rc = lib().smf_smith_server_create(device, form, budget_bytes, workers, ctypes.byref(h))
        if rc != SMF_OK:
            raise SmfError(rc, "smf_smith_server_create failed")
        self.handle = h

    def submit(self, A, a_bits: int, seed: int = 0) -> int:
        """Queue the Smith form of A ([n, n, 1] int64 host tensor or [n, n] int64 array)."""
        import numpy as np
        import torch
        if not isinstance(A, torch.Tensor):
            A = torch.from_numpy(np.ascontiguousarray(np.asarray(A, dtype=np.int64))[..., None].copy())
        d = bigmat(A, a_bits)
        jid = ctypes.c_int64()
        rc = lib().smf_smith_server_submit(self.handle, ctypes.byref(d), seed, ctypes.byref(jid))
        if rc != SMF_OK:
            raise SmfError(rc, "smith_server_submit failed")
        return jid.value

    def job(self, jid: int):
        """(state, status, (t_submit, t_start, t_done))"""
        st, code = ctypes.c_int(), ctypes.c_int()
        t = (ctypes.c_double * 3)()
        rc = lib().smf_smith_server_job(self.handle, jid, ctypes.byref(st), ctypes.byref(code), t)
        if rc != SMF_OK:
            raise SmfError(rc, "smith_server_job failed")
        return st.value, code.value, (t[0], t[1], t[2])

    def result(self, jid: int, n: int):
        """The invariant factors s_1 | ... | s_n of a finished job."""
        offs = (ctypes.c_int64 * (n + 1))()
        cap = 4 * n + 64
        while True:
            limbs = (ctypes.c_uint32 * cap)()
            rc = lib().smf_smith_server_result(self.handle, jid, limbs, cap, offs)
            if rc == SMF_E_NOMEM and offs[n] > cap:
                cap = offs[n]
                continue
            if rc != SMF_OK:
                raise SmfError(rc, "smith_server_result failed: " + self.message(jid))
            out = []
            for i in range(n):
                v = 0
                for j in range(offs[i + 1] - 1, offs[i] - 1, -1):
                    v = (v << 32) | int(limbs[j])
                out.append(v)
            return out

    def message(self, jid: int) -> str:
        """A failed job's error message ("" for a job that did not fail)."""
        buf = ctypes.create_string_buffer(512)
        rc = lib().smf_smith_server_message(self.handle, jid, buf, 512)
        if rc != SMF_OK:
            raise SmfError(rc, "smith_server_message failed")
        return buf.value.decode(errors="replace")

    def stats(self):
        q, r = ctypes.c_int(), ctypes.c_int()
        b = ctypes.c_size_t()
        lib().smf_smith_server_stats(self.handle, ctypes.byref(q), ctypes.byref(r), ctypes.byref(b))
        return q.value, r.value, b.value

    def drain(self):
        lib().smf_smith_server_drain(self.handle)

    def destroy(self):
        if self.handle:
            lib().smf_smith_server_destroy(self.handle)
            self.handle = None
