"""Python binding of the NQS local-energy library (C ABI in include/nqs.h).

Argument marshalling only: every step of the hot path runs in the library's CUDA kernels.
Torch is used for device memory and streams.  The module raises ImportError at import time if
the compiled library (_nqs.so) is missing -- there is no CPU fallback.

Function names mirror the C ABI (nqs_ham_create, nqs_sample, nqs_logpsi, nqs_local_energy,
nqs_logpsi_backward, ...); `Hamiltonian` and `Model` are thin owners of the C handles.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_nqs.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build the CUDA library first "
        "(python paper_2208_05637_b300/build.py); there is no CPU fallback")

_lib = ctypes.CDLL(LIB_PATH)

# ----------------------------------------------------------------- constants (include/nqs.h)
NQS_OK = 0
NQS_ERR_INVALID_ARG, NQS_ERR_NQUBITS, NQS_ERR_CAPACITY, NQS_ERR_WORKSPACE = -1, -2, -3, -4
NQS_ERR_CUDA, NQS_ERR_TIMEOUT, NQS_ERR_NAN, NQS_ERR_ALLOC, NQS_ERR_UNSUPPORTED = -5, -6, -7, -8, -9
ARCH = {"product": 0, "made": 1, "transformer": 2}
PREC = {"fp32": 0, "bf16": 1}
OP_SAMPLE, OP_LOGPSI, OP_LOCAL_ENERGY, OP_BACKWARD, OP_TERM_SWEEP = 0, 1, 2, 3, 4

EXPORTED = [
    "nqs_ham_create", "nqs_ham_info", "nqs_ham_export", "nqs_ham_destroy", "nqs_model_create",
    "nqs_model_param_count", "nqs_model_param_tensors", "nqs_model_param_info",
    "nqs_model_bind_params", "nqs_model_destroy", "nqs_workspace_size", "nqs_sample",
    "nqs_logpsi", "nqs_term_sweep", "nqs_local_energy", "nqs_logpsi_backward", "nqs_logpsi_backward_phase",
    "nqs_energy_stats", "nqs_adam_step", "nqs_strerror", "nqs_last_error", "nqs_profile_enable",
    "nqs_profile_reset", "nqs_profile_read", "nqs_launch_count", "nqs_local_energy_noalloc", "nqs_gemm_bf16", "nqs_profile_work", "nqs_probe_pipes", "nqs_model_set_prefix_reuse", "nqs_model_set_pass_bytes",
    "nqs_energy_sums",
]


class ModelDesc(ctypes.Structure):
    _fields_ = [("arch", ctypes.c_int), ("n_qubits", ctypes.c_int), ("n_up", ctypes.c_int),
                ("n_dn", ctypes.c_int), ("hidden", ctypes.c_int), ("layers", ctypes.c_int),
                ("heads", ctypes.c_int), ("precision", ctypes.c_int),
                ("compensated", ctypes.c_int), ("order", ctypes.c_int * 128)]


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_sig = {
    "nqs_ham_create": [ctypes.c_int, _I64, _P, _P, _P, ctypes.POINTER(_P)],
    "nqs_ham_info": [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64)],
    "nqs_ham_export": [_P, _P, _P, _P, _P, _P],
    "nqs_ham_destroy": [_P],
    "nqs_model_create": [ctypes.POINTER(ModelDesc), ctypes.POINTER(_P)],
    "nqs_model_param_count": [_P, ctypes.POINTER(_I64)],
    "nqs_model_param_tensors": [_P, ctypes.POINTER(ctypes.c_int)],
    "nqs_model_param_info": [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p),
                             ctypes.POINTER(_I64), ctypes.POINTER(_I64)],
    "nqs_model_bind_params": [_P, _P],
    "nqs_model_destroy": [_P],
    "nqs_workspace_size": [_P, _P, ctypes.c_int, _I64, ctypes.POINTER(ctypes.c_size_t)],
    "nqs_sample": [_P, _I64, _I64, ctypes.c_uint64, _P, _P, _I64, ctypes.POINTER(_I64), _P, _I64,
                   _P, ctypes.c_size_t, _P],
    "nqs_logpsi": [_P, _P, _I64, _P, _P, _P, ctypes.c_size_t, _P],
    "nqs_term_sweep": [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _I64, _P, _P, _P, _P, _I64,
                       ctypes.POINTER(_I64), _P, ctypes.c_size_t, _P],
    "nqs_local_energy": [_P, _P, _P, _I64, _P, _P, ctypes.c_size_t, _P],
    "nqs_logpsi_backward": [_P, _P, _I64, _P, _P, _P, _P, ctypes.c_size_t, _P],
    "nqs_logpsi_backward_phase": [_P, ctypes.c_int, _P, _I64, _P, _P, _P, _P, ctypes.c_size_t, _P],
    "nqs_energy_stats": [_P, _P, _I64, _P, _P, _P, _P],
    "nqs_adam_step": [_P, _P, _P, _P, _I64, ctypes.c_int, ctypes.c_float, ctypes.c_float,
                      ctypes.c_float, ctypes.c_float, _P],
    "nqs_strerror": [ctypes.c_int],
    "nqs_last_error": [],
    "nqs_profile_enable": [ctypes.c_int],
    "nqs_profile_reset": [],
    "nqs_profile_read": [ctypes.c_char_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I64)],
    "nqs_launch_count": [],
    "nqs_local_energy_noalloc": [_P, _P, _P, _I64, _P, _P],
    "nqs_gemm_bf16": [_P, _P, _P, _P, _I64, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P],
    "nqs_profile_work": [ctypes.c_char_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
    "nqs_probe_pipes": [_P],
    "nqs_model_set_prefix_reuse": [_P, ctypes.c_int],
    "nqs_model_set_pass_bytes": [_P, ctypes.c_int64],
    "nqs_energy_sums": [_P, _P, _I64, _P, _P, _P, _P, _P],
}
for _name, _args in _sig.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int
_lib.nqs_ham_destroy.restype = None
_lib.nqs_model_destroy.restype = None
_lib.nqs_strerror.restype = ctypes.c_char_p
_lib.nqs_last_error.restype = ctypes.c_char_p
_lib.nqs_launch_count.restype = ctypes.c_int64


class NQSError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = _lib.nqs_strerror(status).decode()
        detail = _lib.nqs_last_error().decode()
        super().__init__(f"{where}: {msg} ({status}): {detail}")


def _check(status, where):
    if status != NQS_OK:
        raise NQSError(status, where)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def launch_count() -> int:
    return int(_lib.nqs_launch_count())


def profile_enable(on: bool = True):
    _check(_lib.nqs_profile_enable(int(on)), "nqs_profile_enable")


def profile_reset():
    _check(_lib.nqs_profile_reset(), "nqs_profile_reset")


def profile_read(kernel: str):
    ms = ctypes.c_double(); n = _I64()
    _check(_lib.nqs_profile_read(kernel.encode(), ctypes.byref(ms), ctypes.byref(n)), "nqs_profile_read")
    return ms.value, n.value


def profile_work(kernel: str):
    """(FLOPs, bytes) recorded with the timed launches of `kernel`."""
    w = ctypes.c_double(); b = ctypes.c_double()
    _check(_lib.nqs_profile_work(kernel.encode(), ctypes.byref(w), ctypes.byref(b)), "nqs_profile_work")
    return w.value, b.value


def probe_pipes():
    """Measured SM pipe rates (instructions per SM per clock): dict with popc, lop3, iadd, ffma."""
    out = (ctypes.c_double * 4)()
    _check(_lib.nqs_probe_pipes(ctypes.cast(out, _P)), "nqs_probe_pipes")
    return dict(popc=out[0], lop3=out[1], iadd=out[2], ffma=out[3])


# ----------------------------------------------------------------- Hamiltonian
def words_of(n_qubits: int) -> int:
    """uint64 words per configuration or mask: 1 for n <= 64 qubits, 2 for n <= 128."""
    return (int(n_qubits) + 63) // 64


def _nconf(bits):
    """Number of configurations in a bits tensor ([B] one-word or [B, 2] two-word)."""
    return bits.shape[0] if bits.dim() == 2 else bits.numel()


class Hamiltonian:
    """Owner of an nqs_ham_t built by nqs_ham_create from host masks and coefficients.  Masks are
    uint64 arrays of shape [K] (n <= 64 qubits) or [K, 2] (n <= 128; word 0 holds qubits 0..63)."""

    def __init__(self, n_qubits, x_mask, z_mask, coeff):
        W = words_of(n_qubits)
        xm = np.ascontiguousarray(x_mask, dtype=np.uint64)
        zm = np.ascontiguousarray(z_mask, dtype=np.uint64)
        c = np.ascontiguousarray(coeff, dtype=np.float64)
        if W > 1 and (xm.ndim != 2 or xm.shape[1] != W or zm.shape != xm.shape):
            raise ValueError(f"{n_qubits} qubits need masks of shape [K, {W}]")
        if W == 1 and (xm.ndim != 1 or zm.ndim != 1):
            raise ValueError("masks of n <= 64 qubits are 1-D uint64 arrays")
        if not (len(xm) == len(zm) == len(c)):
            raise ValueError("x_mask, z_mask and coeff must have equal length")
        self.words = W
        h = _P()
        _check(_lib.nqs_ham_create(int(n_qubits), len(c), xm.ctypes.data_as(_P), zm.ctypes.data_as(_P),
                                   c.ctypes.data_as(_P), ctypes.byref(h)), "nqs_ham_create")
        self.handle = h
        self.n_qubits = int(n_qubits)

    def info(self):
        k = _I64(); g = _I64()
        _check(_lib.nqs_ham_info(self.handle, ctypes.byref(k), ctypes.byref(g)), "nqs_ham_info")
        return k.value, g.value

    def export(self):
        K, G = self.info()
        W = self.words
        shp = (lambda k: (k,)) if W == 1 else (lambda k: (k, W))
        out = dict(group_mask=np.zeros(shp(G), np.uint64), group_offset=np.zeros(G + 1, np.int64),
                   term_z=np.zeros(shp(K), np.uint64), term_c_re=np.zeros(K), term_c_im=np.zeros(K))
        _check(_lib.nqs_ham_export(self.handle, *(out[k].ctypes.data_as(_P) for k in
                                                  ("group_mask", "group_offset", "term_z",
                                                   "term_c_re", "term_c_im"))), "nqs_ham_export")
        return out

    def __del__(self):
        if getattr(self, "handle", None):
            _lib.nqs_ham_destroy(self.handle)
            self.handle = None


# ----------------------------------------------------------------- model
class Model:
    """Owner of an nqs_model_t; `params` is a flat fp32 CUDA tensor bound to it."""

    def __init__(self, arch, n_qubits, n_up, n_dn, hidden=0, layers=0, heads=0, precision="fp32",
                 compensated=True, order=None):
        d = ModelDesc()
        d.arch = ARCH[arch]; d.n_qubits = n_qubits; d.n_up = n_up; d.n_dn = n_dn
        d.hidden = hidden; d.layers = layers; d.heads = heads; d.precision = PREC[precision]
        d.compensated = int(bool(compensated))
        order = list(range(n_qubits - 1, -1, -1)) if order is None else [int(q) for q in order]
        for t, q in enumerate(order):
            d.order[t] = q
        h = _P()
        _check(_lib.nqs_model_create(ctypes.byref(d), ctypes.byref(h)), "nqs_model_create")
        self.handle = h
        self.arch, self.n_qubits, self.n_up, self.n_dn = arch, n_qubits, n_up, n_dn
        self.order = order
        self.params = None

    @property
    def param_count(self) -> int:
        n = _I64()
        _check(_lib.nqs_model_param_count(self.handle, ctypes.byref(n)), "nqs_model_param_count")
        return n.value

    def param_layout(self):
        cnt = ctypes.c_int()
        _check(_lib.nqs_model_param_tensors(self.handle, ctypes.byref(cnt)), "nqs_model_param_tensors")
        out = []
        for i in range(cnt.value):
            name = ctypes.c_char_p(); off = _I64(); numel = _I64()
            _check(_lib.nqs_model_param_info(self.handle, i, ctypes.byref(name), ctypes.byref(off),
                                             ctypes.byref(numel)), "nqs_model_param_info")
            out.append((name.value.decode(), off.value, numel.value))
        return out

    def pack(self, named: dict, device="cuda"):
        """Flat fp32 tensor from named arrays (row-major [out][in] weights)."""
        import torch
        flat = np.zeros(self.param_count, dtype=np.float32)
        for name, off, numel in self.param_layout():
            v = np.asarray(named[name], dtype=np.float32).ravel()
            if v.size != numel:
                raise ValueError(f"{name}: {v.size} values, expected {numel}")
            flat[off: off + numel] = v
        return torch.tensor(flat, device=device)

    def unpack(self, flat) -> dict:
        arr = flat.detach().cpu().numpy() if hasattr(flat, "detach") else np.asarray(flat)
        return {name: arr[off: off + numel].copy() for name, off, numel in self.param_layout()}

    def bind(self, params):
        """Borrow a flat fp32 CUDA tensor (kept alive by this object)."""
        if params.dtype.itemsize != 4 or not params.is_cuda or not params.is_contiguous():
            raise ValueError("params must be a contiguous fp32 CUDA tensor")
        _check(_lib.nqs_model_bind_params(self.handle, _ptr(params)), "nqs_model_bind_params")
        self.params = params

    def set_prefix_reuse(self, depth: int):
        """Prefix reuse depth of the transformer local energy (-1 automatic, 0..3; include/nqs.h)."""
        _check(_lib.nqs_model_set_prefix_reuse(self.handle, int(depth)), "nqs_model_set_prefix_reuse")

    def set_pass_bytes(self, nbytes: int):
        """Activation bytes of one prefix-sharing sub-pass (0: the default, 16 GiB)."""
        _check(_lib.nqs_model_set_pass_bytes(self.handle, int(nbytes)), "nqs_model_set_pass_bytes")

    def workspace(self, op, batch, ham=None):
        import torch
        n = ctypes.c_size_t()
        _check(_lib.nqs_workspace_size(self.handle, ham.handle if ham is not None else None, op,
                                       int(batch), ctypes.byref(n)), "nqs_workspace_size")
        return torch.empty(n.value, dtype=torch.uint8, device="cuda")

    def __del__(self):
        if getattr(self, "handle", None):
            _lib.nqs_model_destroy(self.handle)
            self.handle = None


# ----------------------------------------------------------------- hot path
def _ws(ws):
    return (_ptr(ws), ws.numel()) if ws is not None else (None, 0)


def nqs_sample(model, n_samples, max_unique, seed, ws=None, trace=False, stream=None):
    """Returns (bits uint64 -> torch.int64 view, counts int64, p_trace or None) on the device."""
    import torch
    ws = model.workspace(OP_SAMPLE, n_samples) if ws is None else ws
    cap = int(min(n_samples, 2 * max_unique))
    W = words_of(model.n_qubits)
    bits = torch.empty((max(cap, 1),) if W == 1 else (max(cap, 1), W), dtype=torch.int64, device="cuda")
    counts = torch.empty(max(cap, 1), dtype=torch.int64, device="cuda")
    ptrace = torch.zeros((model.n_qubits, cap), dtype=torch.float32, device="cuda") if trace else None
    nu = _I64()
    wp, wn = _ws(ws)
    _check(_lib.nqs_sample(model.handle, int(n_samples), int(max_unique), ctypes.c_uint64(seed & (2**64 - 1)),
                           _ptr(bits), _ptr(counts), cap, ctypes.byref(nu), _ptr(ptrace),
                           cap if trace else 0, wp, wn, _stream(stream)), "nqs_sample")
    U = nu.value
    return bits[:U], counts[:U], ptrace


def nqs_logpsi(model, bits, ws=None, stream=None):
    import torch
    B = _nconf(bits)
    la = torch.empty(B, dtype=torch.float32, device="cuda")
    ph = torch.empty(B, dtype=torch.float32, device="cuda")
    ws = model.workspace(OP_LOGPSI, B) if ws is None else ws
    wp, wn = _ws(ws)
    _check(_lib.nqs_logpsi(model.handle, _ptr(bits), B, _ptr(la), _ptr(ph), wp, wn, _stream(stream)),
           "nqs_logpsi")
    return la, ph


def nqs_term_sweep(ham, n_up, n_dn, bits, compensated=True, capacity=None, stream=None):
    """Returns (row_offset[B+1], xprime[rows] (or [rows, 2] for two-word registers), s_re[rows],
    s_im[rows]) on the device."""
    import torch
    B = _nconf(bits)
    K, G = ham.info()
    cap = B * G if capacity is None else int(capacity)
    size = ctypes.c_size_t()
    # workspace: counts, offsets, the count pass's validity words (one per group and 32-sample
    # batch) and the compensated sums of every feasible row
    T = (G + 255) // 256
    wsz = 4 * B * T + 8 * (B * T + 1) + 4 * max(1, -(-B // 32)) * T * 256 + 16 * B * G + 4 * 256
    ws = torch.empty(wsz, dtype=torch.uint8, device="cuda")
    row_offset = torch.empty(B + 1, dtype=torch.int64, device="cuda")
    W = ham.words
    xp = torch.empty((max(cap, 1),) if W == 1 else (max(cap, 1), W), dtype=torch.int64, device="cuda")
    sre = torch.empty(max(cap, 1), dtype=torch.float32, device="cuda")
    sim = torch.empty(max(cap, 1), dtype=torch.float32, device="cuda")
    nr = _I64()
    _check(_lib.nqs_term_sweep(ham.handle, int(n_up), int(n_dn), int(bool(compensated)), _ptr(bits), B,
                               _ptr(row_offset), _ptr(xp), _ptr(sre), _ptr(sim), cap,
                               ctypes.byref(nr), _ptr(ws), ws.numel(), _stream(stream)),
           "nqs_term_sweep")
    R = nr.value
    return row_offset, xp[:R], sre[:R], sim[:R]


def nqs_local_energy(ham, model, bits, ws=None, out=None, stream=None):
    """Complex local energies as a [B, 2] fp32 tensor (Re, Im)."""
    import torch
    B = _nconf(bits)
    out = torch.empty((B, 2), dtype=torch.float32, device="cuda") if out is None else out
    ws = model.workspace(OP_LOCAL_ENERGY, B, ham) if ws is None else ws
    wp, wn = _ws(ws)
    _check(_lib.nqs_local_energy(ham.handle, model.handle, _ptr(bits), B, _ptr(out), wp, wn,
                                 _stream(stream)), "nqs_local_energy")
    return out


def nqs_local_energy_noalloc(ham, model, bits, out=None, stream=None):
    """nqs_local_energy without a workspace (static library scratch; see include/nqs.h)."""
    import torch
    B = bits.numel()
    out = torch.empty((B, 2), dtype=torch.float32, device="cuda") if out is None else out
    _check(_lib.nqs_local_energy_noalloc(ham.handle, model.handle, _ptr(bits), B, _ptr(out),
                                         _stream(stream)), "nqs_local_energy_noalloc")
    return out


def nqs_gemm_bf16(A, W, bias, C, epilogue=0, stream=None):
    """Diagnostic: C = A W^T + bias on the tensor cores (A [M,K], W [N,K] bf16; see nqs.h)."""
    M, K = A.shape
    N = W.shape[0]
    _check(_lib.nqs_gemm_bf16(_ptr(A), _ptr(W), _ptr(bias), _ptr(C), M, N, K, int(epilogue),
                              _stream(stream)), "nqs_gemm_bf16")
    return C


def nqs_logpsi_backward(model, bits, g_log_abs, g_phase, grad_accum, ws=None, stream=None):
    B = _nconf(bits)
    ws = model.workspace(OP_BACKWARD, B) if ws is None else ws
    wp, wn = _ws(ws)
    _check(_lib.nqs_logpsi_backward(model.handle, _ptr(bits), B, _ptr(g_log_abs), _ptr(g_phase),
                                    _ptr(grad_accum), wp, wn, _stream(stream)), "nqs_logpsi_backward")
    return grad_accum


def nqs_logpsi_backward_phase(model, phase, bits, g_log_abs=None, g_phase=None, grad_accum=None, ws=None,
                              stream=None):
    """nqs_logpsi_backward in two calls: phase 1 recomputes the forward (bits only), phase 2 runs
    the backward from it with the same bits and workspace."""
    B = _nconf(bits)
    ws = model.workspace(OP_BACKWARD, B) if ws is None else ws
    wp, wn = _ws(ws)
    _check(_lib.nqs_logpsi_backward_phase(model.handle, int(phase), _ptr(bits), B, _ptr(g_log_abs), _ptr(g_phase),
                                          _ptr(grad_accum), wp, wn, _stream(stream)), "nqs_logpsi_backward_phase")
    return grad_accum


def nqs_energy_stats(eloc, counts, with_weights=True, stream=None):
    """Returns (stats fp64[4] = Re E, Im E, Var, W, g_abs, g_phase) on the device."""
    import torch
    B = counts.numel()
    stats = torch.empty(4, dtype=torch.float64, device="cuda")
    ga = torch.empty(B, dtype=torch.float32, device="cuda") if with_weights else None
    gp = torch.empty(B, dtype=torch.float32, device="cuda") if with_weights else None
    _check(_lib.nqs_energy_stats(_ptr(eloc), _ptr(counts), B, _ptr(stats), _ptr(ga), _ptr(gp),
                                 _stream(stream)), "nqs_energy_stats")
    return stats, ga, gp


def nqs_energy_sums(eloc, counts, with_weights=True, stream=None):
    """(sums fp64[4] = sum w Re E, sum w Im E, sum w |E|^2, W; g_abs_e, g_phase_e, g_abs_w) on the
    device: the per-rank pieces of the data-parallel gradient (include/nqs.h)."""
    import torch
    B = counts.numel()
    sums = torch.empty(4, dtype=torch.float64, device="cuda")
    ws = [torch.empty(B, dtype=torch.float32, device="cuda") for _ in range(3)] if with_weights else [None] * 3
    _check(_lib.nqs_energy_sums(_ptr(eloc), _ptr(counts), B, _ptr(sums), *(_ptr(w) for w in ws), _stream(stream)),
           "nqs_energy_sums")
    return (sums, *ws)


def nqs_adam_step(params, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.99, eps=1e-8, stream=None):
    _check(_lib.nqs_adam_step(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), params.numel(), int(step),
                              lr, beta1, beta2, eps, _stream(stream)), "nqs_adam_step")


from .vmc import LogPsi, VMC  # noqa: E402  (needs the names above)
