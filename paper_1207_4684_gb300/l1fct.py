"""Python binding of libl1fct.so (ctypes): argument marshalling only.

Every function here has the name of the C entry point it wraps (see
include/l1fct.h), takes torch tensors for device arrays, passes their data
pointers, sizes and the current CUDA stream, and raises L1SError when the
library reports an error.  No step of the method runs in Python; if the
shared library is missing the import fails instead of falling back to
anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libl1fct.so")

L1S_OK = 0
ERRORS = {1: "INVALID_ARG", 2: "WORKSPACE", 3: "CUDA", 4: "RANK_DEFICIENT", 5: "NONFINITE",
          6: "ZERO_MASS", 7: "CAPACITY", 8: "NOT_CONVERGED", 9: "TIMEOUT"}
F32, BF16 = 0, 1


def flag(code: int) -> int:
    return 1 << (code - 1)


class L1SError(RuntimeError):
    def __init__(self, code: int, where: str, text: str):
        self.code = code
        super().__init__(f"{where}: {ERRORS.get(code, code)}: {text}")


class Params(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("problem_id", C.c_uint32), ("s", C.c_int32),
                ("r1", C.c_int32), ("r2", C.c_int32), ("coreset_size", C.c_double),
                ("global_row_offset", C.c_int64), ("sign_flip", C.c_int32), ("variant", C.c_int32),
                ("sample_scale", C.c_double), ("transform", C.c_int32), ("fjlt_rows", C.c_int32)]


def make_params(s: int, r1: int, r2: int, coreset: float, seed: int = 0, problem_id: int = 0,
                global_row_offset: int = 0, sign_flip: bool = True, variant: int = 0,
                sample_scale: float = 0.0, transform: int = 0, fjlt_rows: int = 0) -> Params:
    """variant 0: FastCauchyRegression; variant 1: OptimizedFastCauchyRegression with
    p̂ = min(1, sample_scale·λ̂) (coreset then only bounds the expected coreset size);
    variant 2: draws with replacement.  transform 0: FCT1; 1: the slow Cauchy transform;
    2: FCT2 with blocks of t = s rows, fjlt_rows of them kept (0: ⌈2·d·ln d⌉)."""
    return Params(seed, problem_id, s, r1, r2, float(coreset), global_row_offset, int(bool(sign_flip)),
                  int(variant), float(sample_scale), int(transform), int(fjlt_rows))


class Schedule(C.Structure):
    _fields_ = [("fct_variant", C.c_int32), ("fct_ctas_per_sm", C.c_int32), ("lam_ctas_per_sm", C.c_int32),
                ("smp_chunks_per_sm", C.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class Problem(C.Structure):
    _fields_ = [("A_dev", C.c_void_p), ("b_dev", C.c_void_p), ("lda", C.c_int64), ("n", C.c_int64),
                ("d", C.c_int32), ("dtype", C.c_int32), ("params", Params), ("capacity", C.c_int64),
                ("idx_dev", C.c_void_p), ("w_dev", C.c_void_p), ("coreset_dev", C.c_void_p),
                ("count_dev", C.c_void_p), ("x_dev", C.c_void_p), ("objective_dev", C.c_void_p)]


_lib = None
_P = C.c_void_p
_I64 = C.c_int64
_I32 = C.c_int32
_SZ = C.c_size_t
_PP = C.POINTER(Params)

_SIGS = {
    "l1s_last_error": (C.c_char_p, []),
    "l1s_version": (C.c_char_p, []),
    "l1s_kernel_launches": (C.c_uint64, []),
    "l1s_workspace_size": (C.c_int, [_PP, _I64, _I32, C.c_int, _I32, C.POINTER(_SZ)]),
    "l1s_status_reset": (C.c_int, [_P, _SZ, _P]),
    "l1s_status_read": (C.c_int, [_P, _SZ, _P, C.POINTER(C.c_uint32)]),
    "fct_embed": (C.c_int, [_P, _I64, C.c_int, _P, _I64, _I32, _PP, _P, _P, _SZ, _P]),
    "l1_condition": (C.c_int, [_P, _I32, _I32, _PP, _P, _P, _P, _SZ, _P]),
    "l1_lambda": (C.c_int, [_P, _I64, C.c_int, _P, _I64, _I32, _P, _PP, _P, _P, _P, _SZ, _P]),
    "l1_basis": (C.c_int, [_P, _I64, C.c_int, _P, _I64, _I32, _P, _P, _P, _P, _P, _SZ, _P]),
    "l1_sample": (C.c_int, [_P, _I64, C.c_int, _P, _I64, _I32, _P, _PP, _I64, _P, _P, _P, _P, _P, _P,
                            _SZ, _P]),
    "l1_sample_from_p": (C.c_int, [_P, _I64, _PP, _I64, _P, _P, _P, _SZ, _P]),
    "l1_sample_lambda": (C.c_int, [_P, _I64, C.c_int, _P, _I64, _I32, _P, _P, _PP, _I32, _I64, _P, _P, _P, _P, _P,
                                   _SZ, _P]),
    "l1s_sample_lambda_workspace_size": (C.c_int, [_PP, _I64, _I32, C.c_int, _I32, C.POINTER(_SZ)]),
    "l1_solve_many": (C.c_int, [_P, _P, _P, _I64, _I32, _I32, _I32, _P, _P, _P, _P, _SZ, _P]),
    "l1s_solve_many_workspace_size": (C.c_int, [_I64, _I32, _I32, C.POINTER(_SZ)]),
    "l1_coreset": (C.c_int, [_P, _I64, C.c_int, _P, _I64, _I32, _PP, _I64, _P, _P, _P, _P, _P, _SZ, _P]),
    "l1_coreset_host": (C.c_int, [_P, _I64, C.c_int, _P, _I64, _I32, _PP, _I64, _P, _P, _P, _P, _SZ, _P]),
    "l1_solve": (C.c_int, [_P, _P, _P, _I64, _I32, _I32, _P, _P, _P, _SZ, _P]),
    "l1_objective": (C.c_int, [_P, _I64, C.c_int, _P, _I64, _I32, _P, _P, _P, _SZ, _P]),
    "l1_regress": (C.c_int, [_P, _I64, C.c_int, _P, _I64, _I32, _PP, _I32, _P, _P, _P, _P, _SZ, _P]),
    "l1s_debug_variates": (C.c_int, [_PP, _I64, _I64, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "l1s_debug_pi2": (C.c_int, [_PP, _I32, _P, _P]),
    "l1_lambda_noalloc": (C.c_int, [_P, _I64, C.c_int, _P, _I64, _I32, _P, _PP, _P, _P, _P]),
    "l1s_schedule_set": (C.c_int, [_I32, C.c_int, _I32, C.POINTER(Schedule)]),
    "l1s_schedule_get": (C.c_int, [_I32, C.c_int, _I32, C.POINTER(Schedule)]),
    "l1s_autotune": (C.c_int, [C.POINTER(Problem), _I32, C.POINTER(Schedule), C.POINTER(C.c_double), _P, _SZ,
                               _P]),
    "l1s_batched_workspace_size": (C.c_int, [C.POINTER(Problem), _I32, C.POINTER(_SZ)]),
    "l1_regress_batched": (C.c_int, [C.POINTER(Problem), _I32, _P, _P, _SZ, _P]),
    "l1s_debug_wait_timeout": (C.c_int, [_P, _SZ, _I64, _P]),
    "l1s_multi_workspace_size": (C.c_int, [_PP, _I64, _I32, _I32, C.c_int, C.POINTER(_SZ)]),
    "l1_coreset_multi": (C.c_int, [_P, _I64, C.c_int, _I64, _I32, _I32, _PP, _I64, _P, _P, _P, _P, _P, _SZ,
                                   _P]),
    "l1_regress_multi": (C.c_int, [_P, _I64, C.c_int, _I64, _I32, _I32, _PP, _I32, _P, _P, _P, _P, _SZ, _P]),
}
EXPORTS = tuple(_SIGS)


def load() -> C.CDLL:
    """Load libl1fct.so (built by paper_1207_4684_gb300.build); raise if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libl1fct.so is not built ({LIB_PATH}); run paper_1207_4684_gb300.build.build()")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(rc: int, where: str) -> None:
    if rc != L1S_OK:
        raise L1SError(rc, where, load().l1s_last_error().decode())


def _ptr(t, contiguous: bool = True) -> int | None:
    """Data pointer of a tensor (None → NULL); arrays other than A must be contiguous."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if contiguous and not t.is_contiguous():
        raise ValueError("array arguments must be contiguous (row-major)")
    return t.data_ptr()


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _dtype_code(A: torch.Tensor) -> int:
    if A.dtype == torch.float32:
        return F32
    if A.dtype in (torch.bfloat16, torch.uint16, torch.int16):
        return BF16
    raise TypeError(f"A must be float32 or bfloat16, not {A.dtype}")


def _matrix(A: torch.Tensor):
    if A.dim() != 2 or A.stride(1) != 1:
        raise ValueError("A must be a 2-D row-major tensor (unit column stride)")
    return A.shape[0], A.shape[1], A.stride(0), _dtype_code(A)


def version() -> str:
    return load().l1s_version().decode()


def l1s_kernel_launches() -> int:
    return int(load().l1s_kernel_launches())


def l1s_workspace_size(params: Params, n: int, d: int, dtype: int = F32, host_staging: bool = False) -> int:
    out = _SZ(0)
    _check(load().l1s_workspace_size(C.byref(params), n, d, dtype, int(host_staging), C.byref(out)),
           "l1s_workspace_size")
    return out.value


def workspace(params: Params, n: int, d: int, dtype: int = F32, host_staging: bool = False,
              device=None) -> torch.Tensor:
    """A device byte tensor of the size l1s_workspace_size asks for (torch's allocator is 256-B aligned)."""
    nbytes = l1s_workspace_size(params, n, d, dtype, host_staging)
    return torch.empty(nbytes, dtype=torch.uint8, device=device or "cuda")


def l1s_status_reset(ws: torch.Tensor, stream=None) -> None:
    _check(load().l1s_status_reset(_ptr(ws), ws.numel(), _stream(stream)), "l1s_status_reset")


def l1s_status_read(ws: torch.Tensor, stream=None) -> int:
    v = C.c_uint32(0)
    _check(load().l1s_status_read(_ptr(ws), ws.numel(), _stream(stream), C.byref(v)), "l1s_status_read")
    return v.value


def fct_embed(A, b, params: Params, PiX, ws, stream=None) -> None:
    n, d, lda, dt = _matrix(A)
    _check(load().fct_embed(_ptr(A, False), lda, dt, _ptr(b), n, d, C.byref(params), _ptr(PiX), _ptr(ws),
                            ws.numel(), _stream(stream)), "fct_embed")


def l1_condition(PiX, params: Params, R, M, ws, stream=None) -> None:
    r1, q = PiX.shape
    _check(load().l1_condition(_ptr(PiX), r1, q, C.byref(params), _ptr(R), _ptr(M), _ptr(ws), ws.numel(),
                               _stream(stream)), "l1_condition")


def l1_lambda(A, b, M, params: Params, lam, lam_sum, ws, stream=None) -> None:
    n, d, lda, dt = _matrix(A)
    _check(load().l1_lambda(_ptr(A, False), lda, dt, _ptr(b), n, d, _ptr(M), C.byref(params), _ptr(lam),
                            _ptr(lam_sum), _ptr(ws), ws.numel(), _stream(stream)), "l1_lambda")


def l1_sample(A, b, M, params: Params, capacity: int, idx, w, coreset, count, lam, ws, stream=None) -> None:
    n, d, lda, dt = _matrix(A)
    _check(load().l1_sample(_ptr(A, False), lda, dt, _ptr(b), n, d, _ptr(M), C.byref(params), capacity, _ptr(idx),
                            _ptr(w), _ptr(coreset), _ptr(count), _ptr(lam), _ptr(ws), ws.numel(),
                            _stream(stream)), "l1_sample")


def l1_sample_from_p(p, params: Params, capacity: int, idx, count, ws, stream=None) -> None:
    _check(load().l1_sample_from_p(_ptr(p), p.numel(), C.byref(params), capacity, _ptr(idx), _ptr(count),
                                   _ptr(ws), ws.numel(), _stream(stream)), "l1_sample_from_p")


def sample_lambda_workspace_size(params: Params, n: int, d: int, dtype: int, k: int) -> int:
    v = C.c_size_t(0)
    _check(load().l1s_sample_lambda_workspace_size(C.byref(params), n, d, dtype, k, C.byref(v)),
           "l1s_sample_lambda_workspace_size")
    return v.value


def l1_sample_lambda(A, b, lam, lam_total, params: Params, k: int, capacity: int, idx, w, coreset, count, ws,
                     stream=None) -> None:
    """k coresets from a given λ and Σλ (device tensors); idx/w are (k, capacity), coreset (k, capacity, q) or
    None, count (k,)."""
    n, d, lda, dt = _matrix(A)
    _check(load().l1_sample_lambda(_ptr(A, False), lda, dt, _ptr(b), n, d, _ptr(lam), _ptr(lam_total),
                                   C.byref(params), k, capacity, _ptr(idx), _ptr(w), _ptr(coreset), _ptr(count),
                                   _ptr(ws), ws.numel(), _stream(stream)), "l1_sample_lambda")


def solve_many_workspace_size(capacity: int, d: int, k: int) -> int:
    v = C.c_size_t(0)
    _check(load().l1s_solve_many_workspace_size(capacity, d, k, C.byref(v)), "l1s_solve_many_workspace_size")
    return v.value


def l1_solve_many(coreset, w, count, capacity: int, d: int, k: int, max_iter: int, x, objective, flags, ws,
                  stream=None) -> None:
    _check(load().l1_solve_many(_ptr(coreset), _ptr(w), _ptr(count), capacity, d, k, max_iter, _ptr(x),
                                _ptr(objective), _ptr(flags), _ptr(ws), ws.numel(), _stream(stream)),
           "l1_solve_many")


def l1_coreset(A, b, params: Params, capacity: int, idx, w, coreset, count, ws, stream=None) -> None:
    n, d, lda, dt = _matrix(A)
    _check(load().l1_coreset(_ptr(A, False), lda, dt, _ptr(b), n, d, C.byref(params), capacity, _ptr(idx), _ptr(w),
                             _ptr(coreset), _ptr(count), _ptr(ws), ws.numel(), _stream(stream)), "l1_coreset")


def l1_coreset_host(A, b, params: Params, capacity: int, idx, w, count, ws, stream=None) -> int:
    """A, b, idx, w, count are CPU tensors (pin them for asynchronous copies); returns the status code."""
    n, d, lda, dt = _matrix(A)
    return load().l1_coreset_host(_ptr(A, False), lda, dt, _ptr(b), n, d, C.byref(params), capacity, _ptr(idx),
                                  _ptr(w), _ptr(count), _ptr(ws), ws.numel(), _stream(stream))


def l1_basis(A, b, R, U=None, rownorm=None, total=None, ws=None, stream=None) -> None:
    """U = [A, −b]·R⁻¹ (FP64), its exact ℓ1 row norms and ‖U‖₁ (device tensors, each may be None)."""
    n, d, lda, dt = _matrix(A)
    if ws is None:
        ws = torch.empty(256 + 8 * 1024, dtype=torch.uint8, device=A.device)
    _check(load().l1_basis(_ptr(A, False), lda, dt, _ptr(b), n, d, _ptr(R), _ptr(U), _ptr(rownorm), _ptr(total),
                           _ptr(ws), ws.numel(), _stream(stream)), "l1_basis")


def l1_solve(coreset, w, count, capacity: int, d: int, max_iter: int, x, objective, ws, stream=None) -> None:
    _check(load().l1_solve(_ptr(coreset), _ptr(w), _ptr(count), capacity, d, max_iter, _ptr(x), _ptr(objective),
                           _ptr(ws), ws.numel(), _stream(stream)), "l1_solve")


def l1_objective(A, b, x, objective, ws, stream=None) -> None:
    n, d, lda, dt = _matrix(A)
    _check(load().l1_objective(_ptr(A, False), lda, dt, _ptr(b), n, d, _ptr(x), _ptr(objective), _ptr(ws), ws.numel(),
                               _stream(stream)), "l1_objective")


def l1_regress(A, b, params: Params, ws, inputs_on_host: bool = False, stream=None):
    """Returns (x̂ as a float64 CPU tensor, objective, coreset rows, status code)."""
    n, d, lda, dt = _matrix(A)
    x = torch.empty(d, dtype=torch.float64)
    obj = C.c_double(0.0)
    rows = C.c_int64(0)
    rc = load().l1_regress(_ptr(A, False), lda, dt, _ptr(b), n, d, C.byref(params), int(inputs_on_host), _ptr(x),
                           C.addressof(obj), C.addressof(rows), _ptr(ws), ws.numel(), _stream(stream))
    if rc in (1, 2, 3):
        _check(rc, "l1_regress")
    return x, obj.value, rows.value, rc


def l1s_debug_wait_timeout(ws, max_cycles: int, stream=None) -> None:
    _check(load().l1s_debug_wait_timeout(_ptr(ws), ws.numel(), int(max_cycles), _stream(stream)),
           "l1s_debug_wait_timeout")


def l1s_multi_workspace_size(params: Params, n: int, d: int, k: int, dtype: int = F32) -> int:
    out = C.c_size_t(0)
    _check(load().l1s_multi_workspace_size(C.byref(params), n, d, k, dtype, C.byref(out)),
           "l1s_multi_workspace_size")
    return out.value


def multi_workspace(params: Params, n: int, d: int, k: int, dtype: int = F32, device=None) -> torch.Tensor:
    return torch.empty(l1s_multi_workspace_size(params, n, d, k, dtype), dtype=torch.uint8,
                       device=device or "cuda")


def l1_coreset_multi(X, k: int, params: Params, capacity: int, idx, w, coreset, count, ws, stream=None) -> None:
    """X = [A | B] (n × (d + k) device matrix, rows contiguous); coreset rows are [A_i, −B_i]."""
    n, q, ldx, dt = _matrix(X)
    _check(load().l1_coreset_multi(_ptr(X, False), ldx, dt, n, q - k, k, C.byref(params), capacity, _ptr(idx),
                                   _ptr(w), _ptr(coreset), _ptr(count), _ptr(ws), ws.numel(), _stream(stream)),
           "l1_coreset_multi")


def l1_regress_multi(X, k: int, params: Params, ws, max_iter: int = 100, stream=None):
    """Returns (W as a d × k float64 CPU tensor, objectives (k,), coreset rows, status code)."""
    n, q, ldx, dt = _matrix(X)
    d = q - k
    W = torch.empty((d, k), dtype=torch.float64)
    obj = torch.empty(k, dtype=torch.float64)
    rows = C.c_int64(0)
    rc = load().l1_regress_multi(_ptr(X, False), ldx, dt, n, d, k, C.byref(params), max_iter, _ptr(W), _ptr(obj),
                                 C.addressof(rows), _ptr(ws), ws.numel(), _stream(stream))
    if rc in (1, 2, 3):
        _check(rc, "l1_regress_multi")
    return W, obj, rows.value, rc


def l1s_debug_variates(params: Params, row_start: int, count: int, device="cuda", stream=None) -> dict:
    out = {
        "bucket_h": torch.empty(count, dtype=torch.int32, device=device),
        "bucket_i": torch.empty(count, dtype=torch.int32, device=device),
        "k_h": torch.empty(count, dtype=torch.int32, device=device),
        "k_i": torch.empty(count, dtype=torch.int32, device=device),
        "cauchy_h": torch.empty(count, dtype=torch.float32, device=device),
        "cauchy_i": torch.empty(count, dtype=torch.float32, device=device),
        "sign": torch.empty(count, dtype=torch.int8, device=device),
        "u_bits": torch.empty(count, dtype=torch.int64, device=device),
    }
    o = out
    _check(load().l1s_debug_variates(C.byref(params), row_start, count, _ptr(o["bucket_h"]), _ptr(o["bucket_i"]),
                                     _ptr(o["k_h"]), _ptr(o["k_i"]), _ptr(o["cauchy_h"]), _ptr(o["cauchy_i"]),
                                     _ptr(o["sign"]), _ptr(o["u_bits"]), _stream(stream)), "l1s_debug_variates")
    return out


def l1s_debug_pi2(params: Params, q: int, device="cuda", stream=None) -> torch.Tensor:
    out = torch.empty((q, params.r2), dtype=torch.float64, device=device)
    _check(load().l1s_debug_pi2(C.byref(params), q, _ptr(out), _stream(stream)), "l1s_debug_pi2")
    return out


def l1_lambda_noalloc(A, b, M, params: Params, lam, lam_sum, stream=None) -> None:
    """l1_lambda without a workspace: the library's own per-device scratch array serves
    callers that cannot allocate device memory (see include/l1fct.h)."""
    n, d, lda, dt = _matrix(A)
    _check(load().l1_lambda_noalloc(_ptr(A, False), lda, dt, _ptr(b), n, d, _ptr(M), C.byref(params), _ptr(lam),
                                    _ptr(lam_sum), _stream(stream)), "l1_lambda_noalloc")


def make_problem(A, b, params: Params, capacity: int = 0, idx=None, w=None, coreset=None, count=None, x=None,
                 objective=None) -> Problem:
    """One member of a batch; the caller keeps every tensor alive while the batch runs."""
    n, d, lda, dt = _matrix(A)
    return Problem(_ptr(A, False), _ptr(b), lda, n, d, dt, params, capacity, _ptr(idx), _ptr(w), _ptr(coreset),
                   _ptr(count), _ptr(x), _ptr(objective))


def _problem_array(problems):
    arr = (Problem * len(problems))(*problems)
    return arr


def l1s_batched_workspace_size(problems) -> int:
    out = _SZ(0)
    _check(load().l1s_batched_workspace_size(_problem_array(problems), len(problems), C.byref(out)),
           "l1s_batched_workspace_size")
    return out.value


def batched_workspace(problems, device=None) -> torch.Tensor:
    return torch.empty(l1s_batched_workspace_size(problems), dtype=torch.uint8, device=device or "cuda")


def l1_regress_batched(problems, ws, flags=None, stream=None) -> None:
    _check(load().l1_regress_batched(_problem_array(problems), len(problems), _ptr(flags), _ptr(ws), ws.numel(),
                                     _stream(stream)), "l1_regress_batched")


def l1s_schedule_set(d: int, dtype: int, s: int, schedule: Schedule | dict | None) -> None:
    if isinstance(schedule, dict):
        schedule = Schedule(**schedule)
    _check(load().l1s_schedule_set(d, dtype, s, C.byref(schedule) if schedule is not None else None),
           "l1s_schedule_set")


def l1s_schedule_get(d: int, dtype: int, s: int) -> dict:
    out = Schedule()
    _check(load().l1s_schedule_get(d, dtype, s, C.byref(out)), "l1s_schedule_get")
    return out.as_dict()


def l1s_autotune(problem: Problem, ws, trials: int = 5, stream=None):
    """Returns (the installed schedule as a dict, its median coreset-pass time in ms)."""
    best = Schedule()
    ms = C.c_double(0.0)
    _check(load().l1s_autotune(C.byref(problem), trials, C.byref(best), C.byref(ms), _ptr(ws), ws.numel(),
                               _stream(stream)), "l1s_autotune")
    return best.as_dict(), ms.value
