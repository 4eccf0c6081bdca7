"""ctypes binding of include/elbm.h: same names, argument marshalling only.

Arrays may be torch tensors (CUDA or CPU) or numpy arrays; they are passed to
the library as raw pointers (device or host), which the library tells apart.
Every call raises :class:`ElbmError` on a non-OK status.  Nothing here
computes any part of the method.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB

ELBM_F64, ELBM_F32, ELBM_F32_F16DEV, ELBM_F32_BF16DEV = 0, 1, 2, 3
ELBM_DTYPE_F64, ELBM_DTYPE_F32 = 0, 1
PRECISIONS = {"f64": ELBM_F64, "f32": ELBM_F32, "f16dev": ELBM_F32_F16DEV, "bf16dev": ELBM_F32_BF16DEV}

STATUS = ["ELBM_OK", "ELBM_ERR_ARG", "ELBM_ERR_NOT_SPD", "ELBM_ERR_MACH", "ELBM_ERR_OOM", "ELBM_ERR_CUDA",
          "ELBM_ERR_NONFINITE", "ELBM_ERR_TIMEOUT", "ELBM_ERR_STATE", "ELBM_ERR_UNSUPPORTED"]


class ElbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS[status] if 0 <= status < len(STATUS) else status}: {msg}")
        self.status = status


class elbm_bc(C.Structure):
    _fields_ = [("dirichlet_x", C.c_int32), ("phi_lo", C.c_double), ("phi_hi", C.c_double)]


class elbm_params(C.Structure):
    _fields_ = [("theta", C.c_double), ("eps", C.c_double), ("fallback", C.c_int32)]


_lib = None


def lib() -> C.CDLL:
    """Load libelbm.so (built by paper_2605_01774_gb300.build); raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = os.environ.get("ELBM_LIBRARY", LIB)     # a custom build of the same ABI
    if not os.path.exists(path):
        raise ImportError(f"{path} is not built; run `python -m paper_2605_01774_gb300.build` "
                          "(the CUDA library is required, there is no CPU path)")
    L = C.CDLL(path)
    H, S, P, I64 = C.c_void_p, C.c_int, C.c_void_p, C.c_int64
    D = C.POINTER(C.c_double)
    sig = {
        "elbm_create": (S, [C.POINTER(C.c_int64), S, C.POINTER(elbm_bc), P, C.POINTER(H)]),
        "elbm_destroy": (None, [H]),
        "elbm_last_error": (C.c_char_p, [H]),
        "elbm_status_string": (C.c_char_p, [S]),
        "elbm_set_params": (S, [H, C.POINTER(elbm_params)]),
        "elbm_set_tensor_uniform": (S, [H, D]),
        "elbm_set_tensor_field": (S, [H, P]),
        "elbm_set_tensor_params_field": (S, [H, P]),
        "elbm_set_velocity_uniform": (S, [H, D]),
        "elbm_set_velocity_field": (S, [H, P]),
        "elbm_set_source": (S, [H, P]),
        "elbm_set_source_amplitude": (S, [H, C.c_double]),
        "elbm_set_lambda_mode": (S, [H, C.c_int32]),
        "elbm_set_step_kernel": (S, [H, C.c_int32]),
        "elbm_set_wait_limit": (S, [H, I64]),
        "elbm_set_wait_test": (S, [H, C.c_int32]),
        "elbm_get_step_kernel": (S, [H, C.POINTER(C.c_int32)]),
        "elbm_set_exact_mass": (S, [H, C.c_int32]),
        "elbm_storage_projections": (S, [H, C.POINTER(C.c_int64)]),
        "elbm_step_source_schedule": (S, [H, D, I64]),
        "elbm_init_equilibrium": (S, [H, P, S]),
        "elbm_write_populations": (S, [H, P, S]),
        "elbm_read_populations": (S, [H, P, S]),
        "elbm_read_moments": (S, [H, P, P, S]),
        "elbm_step": (S, [H, I64]),
        "elbm_reduce": (S, [H, D, D, D, C.POINTER(C.c_int64)]),
        "elbm_get_step": (S, [H, C.POINTER(C.c_int64)]),
        "elbm_synchronize": (S, [H]),
        "elbm_checkpoint_size": (S, [H, C.POINTER(C.c_size_t)]),
        "elbm_checkpoint_save": (S, [H, P, C.c_size_t]),
        "elbm_checkpoint_load": (S, [H, P, C.c_size_t]),
        "elbm_state_pointers": (S, [H, C.POINTER(P), C.POINTER(P)]),
        "elbm_reduce_noalloc": (S, [P, P, C.POINTER(C.c_int64), S, D, C.POINTER(elbm_bc), P, P, P]),
        "elbm_check_tensor": (S, [D]),
        "elbm_check_velocity": (S, [D]),
        "elbm_relaxation_complement": (S, [D, D]),
        "elbm_fma_peak": (S, [C.c_int32, C.POINTER(C.c_double)]),
        "elbm_bulk_copy_rate": (S, [C.c_int32, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    }
    I32, PI32, PI64 = C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int64)
    sig.update({
        "elbm_batch_create": (S, [I32, P, P, P, C.POINTER(H)]),
        "elbm_batch_destroy": (None, [H]),
        "elbm_batch_last_error": (C.c_char_p, [H]),
        "elbm_batch_info": (S, [H, PI64, PI32, PI32, PI32]),
        "elbm_batch_set_params": (S, [H, C.c_double, I32]),
        "elbm_batch_set_wait_limit": (S, [H, I64, I32]),
        "elbm_batch_init_equilibrium": (S, [H, P]),
        "elbm_batch_step": (S, [H, I64, I32]),
        "elbm_batch_synchronize": (S, [H]),
        "elbm_batch_autotune": (S, [H, I32, PI32, PI32]),
        "elbm_batch_read_phi": (S, [H, P]),
        "elbm_batch_read_populations": (S, [H, I32, P]),
        "elbm_batch_fallback_count": (S, [H, PI64]),
    })
    sig.update({
        "elbm_adjoint_create": (S, [C.POINTER(C.c_int64), S, P, C.POINTER(H)]),
        "elbm_adjoint_destroy": (None, [H]),
        "elbm_adjoint_last_error": (C.c_char_p, [H]),
        "elbm_adjoint_configure": (S, [H, D, C.c_double, I32]),
        "elbm_adjoint_misfit": (S, [H, P, P, I64, I32, PI64, P, D, P, PI64]),
        "elbm_adjoint_step": (S, [H, P, P, P, P, P, P]),
    })
    sig.update({
        "elbm2d_create": (S, [C.POINTER(C.c_int64), S, P, C.POINTER(H)]),
        "elbm2d_destroy": (None, [H]),
        "elbm2d_last_error": (C.c_char_p, [H]),
        "elbm2d_set_params": (S, [H, C.POINTER(elbm_params)]),
        "elbm2d_set_tensor_uniform": (S, [H, D]),
        "elbm2d_set_tensor_field": (S, [H, P]),
        "elbm2d_set_velocity_uniform": (S, [H, D]),
        "elbm2d_set_velocity_field": (S, [H, P]),
        "elbm2d_init_equilibrium": (S, [H, P, S]),
        "elbm2d_write_populations": (S, [H, P, S]),
        "elbm2d_read_populations": (S, [H, P, S]),
        "elbm2d_read_moments": (S, [H, P, S]),
        "elbm2d_step": (S, [H, I64]),
        "elbm2d_reduce": (S, [H, D, D, D, C.POINTER(C.c_int64)]),
        "elbm2d_synchronize": (S, [H]),
        "elbm2d_check_velocity": (S, [D]),
        "elbm2d_relaxation_complement": (S, [D, D]),
    })
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _ptr(a) -> C.c_void_p:
    """Raw pointer of a contiguous torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return C.c_void_p(0)
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return C.c_void_p(a.ctypes.data)
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr())
    raise TypeError(f"unsupported array type {type(a)}")


def _dtype_code(a) -> int:
    name = str(a.dtype)
    if name.endswith("float64"):
        return ELBM_DTYPE_F64
    if name.endswith("float32"):
        return ELBM_DTYPE_F32
    raise TypeError(f"dtype {a.dtype} not supported (float64 or float32)")


def _d(vals, n) -> C.Array:
    vals = [float(v) for v in np.asarray(vals, dtype=np.float64).ravel()]
    if len(vals) != n:
        raise ValueError(f"expected {n} values")
    return (C.c_double * n)(*vals)


def _check(status: int, h=None):
    if status != 0:
        msg = lib().elbm_last_error(h).decode() if h else ""
        raise ElbmError(status, msg)


def _stream_ptr(stream) -> C.c_void_p:
    if stream is None:
        return C.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


# --------------------------------------------------------------------- API
def elbm_create(dims, prec="f32", bc=None, stream=None):
    d = (C.c_int64 * 3)(*[int(v) for v in dims])
    p = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    b = None
    if bc is not None:
        b = C.byref(elbm_bc(1, float(bc[0]), float(bc[1])))
    h = C.c_void_p()
    _check(lib().elbm_create(d, p, b, _stream_ptr(stream), C.byref(h)))
    return h


def elbm_destroy(h):
    lib().elbm_destroy(h)


def elbm_set_params(h, theta, eps=0.0, fallback=True):
    _check(lib().elbm_set_params(h, C.byref(elbm_params(float(theta), float(eps), int(bool(fallback))))), h)


def elbm_set_tensor_uniform(h, D6):
    _check(lib().elbm_set_tensor_uniform(h, _d(D6, 6)), h)


def elbm_set_tensor_field(h, D6):
    _check(lib().elbm_set_tensor_field(h, _ptr(D6)), h)


def elbm_set_tensor_params_field(h, theta6):
    _check(lib().elbm_set_tensor_params_field(h, _ptr(theta6)), h)


def elbm_set_velocity_uniform(h, u):
    _check(lib().elbm_set_velocity_uniform(h, _d(u, 3)), h)


def elbm_set_velocity_field(h, u3):
    _check(lib().elbm_set_velocity_field(h, _ptr(u3)), h)


def elbm_set_source(h, R):
    _check(lib().elbm_set_source(h, _ptr(R)), h)


def elbm_set_lambda_mode(h, mode):
    _check(lib().elbm_set_lambda_mode(h, int(mode)), h)


def elbm_set_step_kernel(h, variant):
    _check(lib().elbm_set_step_kernel(h, int(variant)), h)


def elbm_set_wait_limit(h, cycles):
    _check(lib().elbm_set_wait_limit(h, int(cycles)), h)


def elbm_set_wait_test(h, withheld):
    _check(lib().elbm_set_wait_test(h, int(withheld)), h)


def elbm_set_exact_mass(h, on):
    _check(lib().elbm_set_exact_mass(h, int(on)), h)


def elbm_get_step_kernel(h) -> int:
    v = C.c_int32(0)
    _check(lib().elbm_get_step_kernel(h, C.byref(v)), h)
    return int(v.value)


def elbm_storage_projections(h) -> int:
    n = C.c_int64(0)
    _check(lib().elbm_storage_projections(h, C.byref(n)), h)
    return int(n.value)


def elbm_set_source_amplitude(h, a):
    _check(lib().elbm_set_source_amplitude(h, float(a)), h)


def elbm_step_source_schedule(h, amplitudes):
    a = np.ascontiguousarray(amplitudes, dtype=np.float64)
    _check(lib().elbm_step_source_schedule(h, a.ctypes.data_as(C.POINTER(C.c_double)), len(a)), h)


def elbm_init_equilibrium(h, phi0):
    _check(lib().elbm_init_equilibrium(h, _ptr(phi0), _dtype_code(phi0)), h)


def elbm_write_populations(h, g):
    _check(lib().elbm_write_populations(h, _ptr(g), _dtype_code(g)), h)


def elbm_read_populations(h, out):
    _check(lib().elbm_read_populations(h, _ptr(out), _dtype_code(out)), h)
    return out


def elbm_read_moments(h, phi_out, q_out=None):
    _check(lib().elbm_read_moments(h, _ptr(phi_out), _ptr(q_out), _dtype_code(phi_out)), h)
    return phi_out, q_out


def elbm_step(h, nsteps=1):
    _check(lib().elbm_step(h, int(nsteps)), h)


def elbm_reduce(h, allow_nonfinite=False):
    m, e, g = C.c_double(), C.c_double(), C.c_double()
    n = C.c_int64()
    s = lib().elbm_reduce(h, C.byref(m), C.byref(e), C.byref(g), C.byref(n))
    if s != 0 and not (allow_nonfinite and s == 6):
        _check(s, h)
    return dict(mass=m.value, entropy=e.value, gmin=g.value, n_fallback=n.value, status=s)


def elbm_get_step(h):
    v = C.c_int64()
    _check(lib().elbm_get_step(h, C.byref(v)), h)
    return v.value


def elbm_synchronize(h):
    _check(lib().elbm_synchronize(h), h)


def elbm_checkpoint_size(h):
    v = C.c_size_t()
    _check(lib().elbm_checkpoint_size(h, C.byref(v)), h)
    return v.value


def elbm_checkpoint_save(h, buf):
    _check(lib().elbm_checkpoint_save(h, _ptr(buf), buf.numel() * buf.element_size() if hasattr(buf, "numel")
                                      else buf.nbytes), h)


def elbm_checkpoint_load(h, buf):
    _check(lib().elbm_checkpoint_load(h, _ptr(buf), buf.numel() * buf.element_size() if hasattr(buf, "numel")
                                      else buf.nbytes), h)


def elbm_state_pointers(h):
    p, s = C.c_void_p(), C.c_void_p()
    _check(lib().elbm_state_pointers(h, C.byref(p), C.byref(s)), h)
    return p.value, s.value


def elbm_reduce_noalloc(pops_ptr, scale_ptr, dims, prec, u, bc=None, source=None, stream=None, out=None):
    """Diagnostics of a caller-held state without device allocation (see include/elbm.h).

    pops_ptr / scale_ptr are raw device addresses (ints); out is a host numpy array of
    4 float64 (created if None) or a device tensor.  Returns out."""
    d = (C.c_int64 * 3)(*[int(v) for v in dims])
    p = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    b = C.byref(elbm_bc(1, float(bc[0]), float(bc[1]))) if bc is not None else None
    if out is None:
        out = np.zeros(4, dtype=np.float64)
    _check(lib().elbm_reduce_noalloc(C.c_void_p(pops_ptr), C.c_void_p(scale_ptr or 0), d, p, _d(u, 3), b,
                                     _ptr(source), _stream_ptr(stream), _ptr(out)))
    return out


def elbm_check_tensor(D6) -> int:
    return lib().elbm_check_tensor(_d(D6, 6))


def elbm_check_velocity(u) -> int:
    return lib().elbm_check_velocity(_d(u, 3))


def elbm_relaxation_complement(D6):
    out = (C.c_double * 6)()
    _check(lib().elbm_relaxation_complement(_d(D6, 6), out))
    return np.array(list(out))


# ------------------------------------------------------------- batched domains
def _bcheck(status, h):
    if status != 0:
        raise ElbmError(status, lib().elbm_batch_last_error(h).decode() if h else "")


def elbm_batch_create(edges, D6, stream=None):
    edges = np.ascontiguousarray(edges, dtype=np.int32)
    D6 = np.ascontiguousarray(D6, dtype=np.float64).reshape(len(edges), 6)
    h = C.c_void_p()
    _check(lib().elbm_batch_create(len(edges), _ptr(edges), _ptr(D6), _stream_ptr(stream), C.byref(h)))
    return h


def elbm_batch_destroy(h):
    lib().elbm_batch_destroy(h)


def elbm_batch_info(h):
    n, t, b, g = C.c_int64(), C.c_int32(), C.c_int32(), C.c_int32()
    _bcheck(lib().elbm_batch_info(h, C.byref(n), C.byref(t), C.byref(b), C.byref(g)), h)
    return dict(total_nodes=n.value, tile=t.value, blocks_per_sm=b.value, persistent_in_graph=g.value)


def elbm_batch_set_params(h, eps=0.0, fallback=True):
    _bcheck(lib().elbm_batch_set_params(h, float(eps), int(bool(fallback))), h)


def elbm_batch_set_wait_limit(h, cycles, extra_arrivals=0):
    _bcheck(lib().elbm_batch_set_wait_limit(h, int(cycles), int(extra_arrivals)), h)


def elbm_batch_init_equilibrium(h, phi0):
    _bcheck(lib().elbm_batch_init_equilibrium(h, _ptr(phi0)), h)


def elbm_batch_step(h, nsteps, mode=0):
    _bcheck(lib().elbm_batch_step(h, int(nsteps), int(mode)), h)


def elbm_batch_synchronize(h):
    _bcheck(lib().elbm_batch_synchronize(h), h)


def elbm_batch_autotune(h, steps_per_trial=3):
    t, b = C.c_int32(), C.c_int32()
    _bcheck(lib().elbm_batch_autotune(h, int(steps_per_trial), C.byref(t), C.byref(b)), h)
    return t.value, b.value


def elbm_batch_read_phi(h, out):
    _bcheck(lib().elbm_batch_read_phi(h, _ptr(out)), h)
    return out


def elbm_batch_read_populations(h, domain, out):
    _bcheck(lib().elbm_batch_read_populations(h, int(domain), _ptr(out)), h)
    return out


def elbm_batch_fallback_count(h):
    v = C.c_int64()
    _bcheck(lib().elbm_batch_fallback_count(h, C.byref(v)), h)
    return v.value


# ------------------------------------------------------------------- adjoint
def _acheck(status, h):
    if status != 0:
        raise ElbmError(status, lib().elbm_adjoint_last_error(h).decode() if h else "")


def elbm_adjoint_create(dims, prec="f64", stream=None):
    d = (C.c_int64 * 3)(*[int(v) for v in dims])
    p = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    h = C.c_void_p()
    _check(lib().elbm_adjoint_create(d, p, _stream_ptr(stream), C.byref(h)))
    return h


def elbm_adjoint_destroy(h):
    lib().elbm_adjoint_destroy(h)


def elbm_adjoint_configure(h, u, theta=1e-8, checkpoint_every=50):
    _acheck(lib().elbm_adjoint_configure(h, _d(u, 3), float(theta), int(checkpoint_every)), h)


def elbm_adjoint_misfit(h, theta6, phi0, nsteps, obs_steps, targets, grad6=None):
    """Returns (J, n_fallback); fills grad6 (device tensor) when given."""
    obs = np.ascontiguousarray(obs_steps, dtype=np.int64)
    J = C.c_double()
    nfb = C.c_int64()
    _acheck(lib().elbm_adjoint_misfit(h, _ptr(theta6), _ptr(phi0), int(nsteps), len(obs),
                                      obs.ctypes.data_as(C.POINTER(C.c_int64)), _ptr(targets), C.byref(J),
                                      _ptr(grad6), C.byref(nfb)), h)
    return J.value, nfb.value


def elbm_adjoint_step(h, theta6, g, gbar_next=None, g_next=None, gbar=None, grad6=None):
    _acheck(lib().elbm_adjoint_step(h, _ptr(theta6), _ptr(g), _ptr(gbar_next), _ptr(g_next), _ptr(gbar),
                                    _ptr(grad6)), h)


def tensor_misfit_function():
    """torch.autograd.Function whose forward is J(theta) and whose backward is the
    hand-written adjoint.  Where theta needs a gradient, one elbm_adjoint_misfit call runs the
    forward sweep and the checkpointed reverse sweep and backward only scales the stored
    gradient; otherwise (no_grad, or theta without requires_grad) only the forward sweep runs."""
    import torch

    class TensorMisfit(torch.autograd.Function):
        @staticmethod
        def forward(ctx, theta, handle, phi0, nsteps, obs_steps, targets):
            grad = torch.empty_like(theta) if ctx.needs_input_grad[0] else None
            J, nfb = elbm_adjoint_misfit(handle, theta.detach().contiguous(), phi0, nsteps, obs_steps, targets,
                                         grad6=grad)
            if grad is not None:
                ctx.save_for_backward(grad)
            ctx.n_fallback = nfb
            return torch.tensor(J, dtype=torch.float64, device=theta.device)

        @staticmethod
        def backward(ctx, gJ):
            (grad,) = ctx.saved_tensors
            return gJ.to(grad.dtype) * grad, None, None, None, None, None

    return TensorMisfit


# ------------------------------------------------------------ convenience
class Lattice:
    """Owning wrapper over one handle (marshalling only)."""

    def __init__(self, dims, prec="f32", bc=None, stream=None):
        self.dims = tuple(int(v) for v in dims)
        self.N = self.dims[0] * self.dims[1] * self.dims[2]
        self.prec = prec
        self.h = elbm_create(self.dims, prec, bc, stream)

    def close(self):
        if self.h is not None:
            elbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def elbm_fma_peak(prec="f64") -> float:
    """CUDA-core FMA throughput of the current device in flop/s ("f64" or "f32")."""
    v = C.c_double(0.0)
    _check(lib().elbm_fma_peak(PRECISIONS[prec], C.byref(v)))
    return float(v.value)


def elbm_bulk_copy_rate(copy_bytes, blocks_per_sm=2):
    """(bytes/s, copies/s) of bulk asynchronous global -> shared copies issued by one warp per block."""
    b, c = C.c_double(0), C.c_double(0)
    _check(lib().elbm_bulk_copy_rate(int(copy_bytes), int(blocks_per_sm), C.byref(b), C.byref(c)))
    return b.value, c.value


# ------------------------------------------------------------------- D2Q9 (include/elbm2d.h)
def _check2(status: int, h=None):
    if status != 0:
        msg = lib().elbm2d_last_error(h).decode() if h else ""
        raise ElbmError(status, msg)


def elbm2d_create(dims, prec="f32", stream=None):
    d = (C.c_int64 * 2)(*[int(v) for v in dims])
    h = C.c_void_p()
    _check2(lib().elbm2d_create(d, PRECISIONS[prec] if isinstance(prec, str) else int(prec), _stream_ptr(stream),
                                C.byref(h)))
    return h


def elbm2d_destroy(h):
    lib().elbm2d_destroy(h)


def elbm2d_set_params(h, theta, eps=0.0, fallback=True):
    p = elbm_params(float(theta), float(eps), 1 if fallback else 0)
    _check2(lib().elbm2d_set_params(h, C.byref(p)), h)


def elbm2d_set_tensor_uniform(h, D3):
    _check2(lib().elbm2d_set_tensor_uniform(h, _d(D3, 3)), h)


def elbm2d_set_tensor_field(h, D3):
    _check2(lib().elbm2d_set_tensor_field(h, _ptr(D3)), h)


def elbm2d_set_velocity_uniform(h, u):
    _check2(lib().elbm2d_set_velocity_uniform(h, _d(u, 2)), h)


def elbm2d_set_velocity_field(h, u2):
    _check2(lib().elbm2d_set_velocity_field(h, _ptr(u2)), h)


def elbm2d_init_equilibrium(h, phi0):
    _check2(lib().elbm2d_init_equilibrium(h, _ptr(phi0), _dtype_code(phi0)), h)


def elbm2d_write_populations(h, g):
    _check2(lib().elbm2d_write_populations(h, _ptr(g), _dtype_code(g)), h)


def elbm2d_read_populations(h, out):
    _check2(lib().elbm2d_read_populations(h, _ptr(out), _dtype_code(out)), h)
    return out


def elbm2d_read_moments(h, phi_out):
    _check2(lib().elbm2d_read_moments(h, _ptr(phi_out), _dtype_code(phi_out)), h)
    return phi_out


def elbm2d_step(h, nsteps=1):
    _check2(lib().elbm2d_step(h, int(nsteps)), h)


def elbm2d_reduce(h, allow_nonfinite=False):
    m, e, g = C.c_double(), C.c_double(), C.c_double()
    fb = C.c_int64()
    st = lib().elbm2d_reduce(h, C.byref(m), C.byref(e), C.byref(g), C.byref(fb))
    if st != 0 and not (allow_nonfinite and st == 6):
        _check2(st, h)
    return dict(mass=m.value, entropy=e.value, gmin=g.value, n_fallback=fb.value, status=st)


def elbm2d_synchronize(h):
    _check2(lib().elbm2d_synchronize(h), h)


def elbm2d_check_velocity(u) -> int:
    return int(lib().elbm2d_check_velocity(_d(u, 2)))


def elbm2d_relaxation_complement(D3):
    out = (C.c_double * 3)()
    _check2(lib().elbm2d_relaxation_complement(_d(D3, 3), out))
    return np.array(out[:])


class Lattice2D:
    """Owning wrapper over one D2Q9 handle (marshalling only)."""

    def __init__(self, dims, prec="f32", stream=None):
        self.dims = tuple(int(v) for v in dims)
        self.N = self.dims[0] * self.dims[1]
        self.prec = prec
        self.h = elbm2d_create(self.dims, prec, stream)

    def close(self):
        if self.h is not None:
            elbm2d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
