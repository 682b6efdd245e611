"""ctypes binding of ``libecmg.so`` (the C ABI of ``include/ecmg.h``).

Argument marshalling only: every step of the method runs in the library's CUDA kernels. The
functions keep the C names; ``Solver`` wraps a handle for torch tensors (device memory and the
current stream come from torch, which is plumbing here). Importing this module loads the
library and raises if it has not been built (``python -m paper_1506_02983_gb300.build``).
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libecmg.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libecmg.so is not built: run python -m paper_1506_02983_gb300.build "
                      "(or __graft_entry__.build()); there is no fallback implementation")
_lib = C.CDLL(LIB_PATH)

ECMG_OK, ECMG_ERR_INVALID_ARG, ECMG_ERR_SINGULAR, ECMG_ERR_NO_CONVERGENCE = 0, 1, 2, 3
ECMG_ERR_BREAKDOWN, ECMG_ERR_OOM, ECMG_ERR_CUDA = 4, 5, 6
ECMG_BC_DIRICHLET, ECMG_BC_ROBIN = 0, 1
ECMG_F_NODAL, ECMG_F_LOAD, ECMG_F_SEPARABLE, ECMG_F_GAUSS = 0, 1, 2, 3
ECMG_FP64, ECMG_MIXED = 0, 1
ECMG_APPLY_K1 = 2  # ecmg_apply_operator: the FP32 search-direction kernel itself
ECMG_EXP_SERENDIPITY20, ECMG_EXP_LAGRANGE27 = 0, 1
ECMG_VEC_U, ECMG_VEC_W, ECMG_VEC_UTILDE, ECMG_VEC_B, ECMG_VEC_BETA = 0, 1, 2, 3, 4
ECMG_PREC_JACOBI, ECMG_PREC_NONE = 0, 1
ECMG_SCHED_TOLERANCE, ECMG_SCHED_FIXED = 0, 1
ECMG_CG_TWO_PASS, ECMG_CG_SINGLE_PASS, ECMG_CG_AUTO = 0, 1, 2
ECMG_NOALLOC_MAX_ELEMS = 536870912  # include/ecmg.h
ECMG_AUTO_SINGLE_PASS_NODES = 1 << 22  # include/ecmg.h
ECMG_RING_AUTO = -1


class ecmg_problem(C.Structure):
    _fields_ = [("n0", C.c_int32 * 3), ("levels", C.c_int32),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("face_bc", C.c_int32 * 6), ("robin_alpha", C.c_double * 6),
                ("beta", C.c_void_p), ("f", C.c_void_p), ("g_D", C.c_void_p),
                ("g_R", C.c_void_p), ("f_mode", C.c_int32), ("f_terms", C.c_int32), ("gD_terms", C.c_int32),
                ("beta_const", C.c_double)]


class ecmg_options(C.Structure):
    _fields_ = [("rtol", C.c_double), ("precision", C.c_int32), ("inner_rtol", C.c_double),
                ("max_iters", C.c_int32), ("use_graph", C.c_int32), ("dsolve_rtol", C.c_double),
                ("exp_variant", C.c_int32), ("true_residual", C.c_int32), ("autotune", C.c_int32),
                ("preconditioner", C.c_int32), ("schedule", C.c_int32), ("sched_mL", C.c_int32),
                ("sched_beta", C.c_double), ("cg_form", C.c_int32),
                ("ring_slots", C.c_int32)]


class ecmg_stats(C.Structure):
    _fields_ = [("levels", C.c_int32), ("iters", C.c_int32 * 16), ("updates", C.c_int32 * 16),
                ("rel_res", C.c_double * 16), ("rhs_norm", C.c_double * 16),
                ("status", C.c_int32), ("seconds", C.c_double * 16), ("setup_seconds", C.c_double)]


_P, _I32, _D = C.c_void_p, C.c_int32, C.c_double
_H = C.c_void_p
# caller-supplied device allocator (ecmg_create_with_allocator)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_SIGS = {
    "ecmg_default_options": (None, [C.POINTER(ecmg_options)]),
    "ecmg_create": (_I32, [C.POINTER(ecmg_problem), C.POINTER(ecmg_options), _P, C.POINTER(_H)]),
    "ecmg_create_with_allocator": (_I32, [C.POINTER(ecmg_problem), C.POINTER(ecmg_options), _P, ALLOC_FN, FREE_FN,
                                          _P, C.POINTER(_H)]),
    "ecmg_solve": (_I32, [_H, _P, C.POINTER(ecmg_stats)]),
    "ecmg_solve_from": (_I32, [_H, _I32, _P, C.POINTER(ecmg_stats)]),
    "ecmg_extrapolate": (_I32, [_H, _I32, _P]),
    "ecmg_get_level": (_I32, [_H, _I32, _I32, _P]),
    "ecmg_set_level": (_I32, [_H, _I32, _P]),
    "ecmg_apply_operator": (_I32, [_H, _I32, _I32, _P, _P]),
    "ecmg_error_norms": (_I32, [_H, _I32, _P, _P, C.POINTER(_D), C.POINTER(_D)]),
    "ecmg_destroy": (None, [_H]),
    "ecmg_status_string": (C.c_char_p, [_I32]),
    "ecmg_last_error": (C.c_char_p, []),
    "ecmg_workspace_bytes": (_I32, [C.POINTER(ecmg_problem), C.POINTER(ecmg_options),
                                    C.POINTER(C.c_uint64)]),
    "ecmg_kernel_launches": (_I32, [C.POINTER(C.c_uint64)]),
    "ecmg_error_norms_noalloc": (_I32, [_P, _P, C.c_int64, _P, C.POINTER(_D), C.POINTER(_D)]),
    "ecmg_time_kernel": (_I32, [_H, _I32, _I32, _I32, C.POINTER(_D), C.POINTER(_D)]),
    "ecmg_create_batched": (_I32, [C.POINTER(ecmg_problem), _I32, C.POINTER(ecmg_options), _P, C.POINTER(_H)]),
    "ecmg_solve_batched": (_I32, [_H, C.POINTER(C.c_void_p), C.POINTER(ecmg_stats)]),
    "ecmg_get_level_batched": (_I32, [_H, _I32, _I32, _I32, _P]),
    "ecmg_set_tiles": (_I32, [_H, _I32, _I32, _I32]),
    "ecmg_get_tiles": (_I32, [_H, _I32, C.POINTER(_I32), C.POINTER(_I32)]),
    "ecmg_autotune": (_I32, [_H, _I32]),
    "ecmg_stencil_timer": (_I32, [_H, _I32, _I32, C.POINTER(_D), C.POINTER(C.c_int64)]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f

EXPORTED = sorted(_SIGS)


class EcmgError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = ecmg_last_error()
        super().__init__("%s: %s (%s)" % (where, ecmg_status_string(status).decode(),
                                          msg.decode() if msg else ""))


def check(status: int, where: str) -> int:
    if status != ECMG_OK:
        raise EcmgError(status, where)
    return status


def default_options(**kw) -> ecmg_options:
    o = ecmg_options()
    ecmg_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def torch_allocator():
    """(alloc, free) callbacks for ecmg_create_with_allocator that take device memory from
    PyTorch's caching allocator on the current device. Keep the returned pair alive as long as
    the handle."""
    import torch

    def alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      int(stream) if stream else None)
        except RuntimeError:
            return None

    def free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    return ALLOC_FN(alloc), FREE_FN(free)


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class Solver:
    """One ECMG_jcg problem on the current CUDA device (torch tensors in, torch tensors out).

    beta: finest elements (nz, ny, nx) float64 tensor; f, g_D, g_R: finest nodes
    (nz+1, ny+1, nx+1) float64 tensors (g_D, g_R optional); each on the current CUDA device or
    in pinned host memory (the kernels then read it over the host link). The tensors must
    outlive the solver and stay unchanged while a solve reads them. Options are the fields of
    ecmg_options as keywords; torch_memory=True takes the workspace from PyTorch's caching
    allocator.

    Compact inputs: beta=None with beta_const > 0 (one beta everywhere); f_mode=ECMG_F_SEPARABLE
    with f the Gauss samples of f_terms separable terms (``inputs.separable_samples``); g_D the
    nodal factors of gD_terms separable terms (``inputs.separable_nodal``).
    """

    def __init__(self, n0, levels, lo, hi, face_bc, robin_alpha, beta, f, g_D=None, g_R=None,
                 f_mode=ECMG_F_NODAL, f_terms=0, gD_terms=0, beta_const=0.0, torch_memory=False, **options):
        p = ecmg_problem()
        p.n0[:] = [int(v) for v in n0]
        p.levels = int(levels)
        p.lo[:] = [float(v) for v in lo]
        p.hi[:] = [float(v) for v in hi]
        p.face_bc[:] = [int(v) for v in face_bc]
        p.robin_alpha[:] = [float(v) for v in robin_alpha]
        self._keep = (beta, f, g_D, g_R)
        for t in self._keep:
            if t is not None and (not (t.is_cuda or t.is_pinned()) or not t.is_contiguous()
                                  or str(t.dtype) != "torch.float64"):
                raise ValueError("inputs must be contiguous float64 CUDA or pinned host tensors")
        p.beta, p.f, p.g_D, p.g_R = (None if t is None else t.data_ptr() for t in self._keep)
        p.f_mode = int(f_mode)
        p.f_terms, p.gD_terms, p.beta_const = int(f_terms), int(gD_terms), float(beta_const)
        self.problem = p
        self.options = default_options(**options)
        self.levels = int(levels)
        self.n0 = [int(v) for v in n0]
        h = _H()
        if torch_memory:
            # the workspace comes from PyTorch's caching allocator (counted in its statistics)
            self._allocator = torch_allocator()
            check(ecmg_create_with_allocator(C.byref(p), C.byref(self.options), _stream(), *self._allocator, None,
                                             C.byref(h)), "ecmg_create_with_allocator")
        else:
            check(ecmg_create(C.byref(p), C.byref(self.options), _stream(), C.byref(h)), "ecmg_create")
        self.handle = h

    def workspace_bytes(self, **override):
        """ecmg_workspace_bytes of this solver's problem and options (keywords override options)."""
        o = ecmg_options.from_buffer_copy(self.options)
        for k, v in override.items():
            setattr(o, k, v)
        n = C.c_uint64()
        check(ecmg_workspace_bytes(C.byref(self.problem), C.byref(o), C.byref(n)), "ecmg_workspace_bytes")
        return n.value

    def ring_slots(self):
        """The slots of the ring of search directions ecmg_create gave the two-pass levels
        (ECMG_RING_AUTO resolved), from the workspace byte counts; 0 when no level has one."""
        if self.options.ring_slots != ECMG_RING_AUTO:
            return int(self.options.ring_slots)
        base = self.workspace_bytes(ring_slots=0)
        per_slot = (self.workspace_bytes(ring_slots=4) - base) // 4
        return 0 if per_slot == 0 else (self.workspace_bytes() - base) // per_slot

    def level_shape(self, level=-1):
        l = self.levels - 1 if level < 0 else level
        n = [v << l for v in self.n0]
        return (n[2] + 1, n[1] + 1, n[0] + 1)

    def solve(self, u_out=None, raise_on_error=True):
        st = ecmg_stats()
        s = ecmg_solve(self.handle, _ptr(u_out), C.byref(st))
        if raise_on_error:
            check(s, "ecmg_solve")
        return stats_dict(st), s

    def solve_from(self, first, u_out=None):
        st = ecmg_stats()
        check(ecmg_solve_from(self.handle, int(first), _ptr(u_out), C.byref(st)), "ecmg_solve_from")
        return stats_dict(st)

    def get(self, which, level=-1):
        import torch
        l = self.levels - 1 if level < 0 else level
        if which == ECMG_VEC_BETA:
            n = [v << l for v in self.n0]
            out = torch.empty((n[2], n[1], n[0]), dtype=torch.float64, device="cuda")
        else:
            out = torch.empty(self.level_shape(l), dtype=torch.float64, device="cuda")
        check(ecmg_get_level(self.handle, int(level), int(which), _ptr(out)), "ecmg_get_level")
        return out

    def extrapolate(self, level=-1):
        import torch
        out = torch.empty(self.level_shape(level), dtype=torch.float64, device="cuda")
        check(ecmg_extrapolate(self.handle, int(level), _ptr(out)), "ecmg_extrapolate")
        return out

    def set_level(self, level, u):
        check(ecmg_set_level(self.handle, int(level), _ptr(u)), "ecmg_set_level")

    def apply(self, x, level=-1, precision=ECMG_FP64):
        import torch
        y = torch.empty_like(x)
        check(ecmg_apply_operator(self.handle, int(level), int(precision), _ptr(x), _ptr(y)),
              "ecmg_apply_operator")
        return y

    def norms(self, a, b=None, level=-1):
        mx, rms = C.c_double(), C.c_double()
        check(ecmg_error_norms(self.handle, int(level), _ptr(a), _ptr(b), C.byref(mx), C.byref(rms)),
              "ecmg_error_norms")
        return mx.value, rms.value

    def time_kernel(self, which, level=-1, reps=5):
        """Mean ms of one launch of a solve kernel run alone, and its algorithmic bytes."""
        ms, nb = C.c_double(), C.c_double()
        check(ecmg_time_kernel(self.handle, int(level), int(which), int(reps), C.byref(ms), C.byref(nb)),
              "ecmg_time_kernel")
        return ms.value, nb.value

    def set_tiles(self, ry, kz, level=-1):
        """Force the FP32 stencil tile shape of a level (MIXED handles)."""
        check(ecmg_set_tiles(self.handle, int(level), int(ry), int(kz)), "ecmg_set_tiles")

    def get_tiles(self, level=-1):
        ry, kz = C.c_int32(), C.c_int32()
        check(ecmg_get_tiles(self.handle, int(level), C.byref(ry), C.byref(kz)), "ecmg_get_tiles")
        return ry.value, kz.value

    def stencil_timer(self, level=-1, reset=False):
        """(ms summed over the FP32 stencil launches of a level inside solves, launches)."""
        ms, n = C.c_double(), C.c_int64()
        check(ecmg_stencil_timer(self.handle, int(level), int(bool(reset)), C.byref(ms), C.byref(n)),
              "ecmg_stencil_timer")
        return ms.value, n.value

    def autotune(self, reps=3):
        """Try the candidate stencil tile shapes on every large MIXED level inside whole solves
        (reps solves per shape; overwrites the levels' vectors); each level keeps its fastest."""
        check(ecmg_autotune(self.handle, int(reps)), "ecmg_autotune")

    def close(self):
        if getattr(self, "handle", None):
            ecmg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchSolver:
    """Many independent problems solved together (ecmg_create_batched): one kernel launch per
    step of Alg. 4 over all problems, one CUDA graph per solve, MIXED precision.

    problems: list of dicts with n0, levels, lo, hi, face_bc, alpha and the device tensors
    beta, f and optionally gD, gR (as for Solver), plus f_mode and, for compact inputs, f_terms,
    gD_terms and beta_const (beta None). The tensors must outlive the solver."""

    def __init__(self, problems, **options):
        n = len(problems)
        arr = (ecmg_problem * n)()
        self._keep = []
        self.problems = problems
        for i, q in enumerate(problems):
            p = arr[i]
            p.n0[:] = [int(v) for v in q["n0"]]
            p.levels = int(q["levels"])
            p.lo[:] = [float(v) for v in q["lo"]]
            p.hi[:] = [float(v) for v in q["hi"]]
            p.face_bc[:] = [int(v) for v in q["face_bc"]]
            p.robin_alpha[:] = [float(v) for v in q["alpha"]]
            ts = (q.get("beta"), q["f"], q.get("gD"), q.get("gR"))
            for t in ts:
                if t is not None and (not t.is_cuda or not t.is_contiguous() or str(t.dtype) != "torch.float64"):
                    raise ValueError("inputs must be contiguous float64 CUDA tensors")
            self._keep.append(ts)
            p.beta, p.f, p.g_D, p.g_R = (None if t is None else t.data_ptr() for t in ts)
            p.f_mode = int(q.get("f_mode", ECMG_F_NODAL))
            p.f_terms, p.gD_terms = int(q.get("f_terms", 0)), int(q.get("gD_terms", 0))
            p.beta_const = float(q.get("beta_const", 0.0))
        options.setdefault("precision", ECMG_MIXED)
        self.options = default_options(**options)
        self.n = n
        self._arr = arr
        h = _H()
        check(ecmg_create_batched(arr, n, C.byref(self.options), _stream(), C.byref(h)), "ecmg_create_batched")
        self.handle = h

    def finest_shape(self, i):
        q = self.problems[i]
        n = [int(v) << (int(q["levels"]) - 1) for v in q["n0"]]
        return (n[2] + 1, n[1] + 1, n[0] + 1)

    def solve(self, u_outs=None, raise_on_error=True):
        """Solve all problems; u_outs: None or a list of finest-level output tensors (or None).
        Returns (list of per-problem stats dicts, status)."""
        st = (ecmg_stats * self.n)()
        ptrs = None
        if u_outs is not None:
            ptrs = (C.c_void_p * self.n)(*[None if u is None else u.data_ptr() for u in u_outs])
        s = ecmg_solve_batched(self.handle, ptrs, st)
        if raise_on_error:
            check(s, "ecmg_solve_batched")
        return [stats_dict(st[i]) for i in range(self.n)], s

    def time_kernel(self, which, stage=-1, reps=5):
        """Mean ms of one launch of the stage's batched K1 (0) or K2 (1) alone, and its
        algorithmic bytes."""
        ms, nb = C.c_double(), C.c_double()
        check(ecmg_time_kernel(self.handle, int(stage), int(which), int(reps), C.byref(ms), C.byref(nb)),
              "ecmg_time_kernel")
        return ms.value, nb.value

    def autotune(self, reps=3):
        """Time the batched stencil tile shapes of every stage; keep the fastest."""
        check(ecmg_autotune(self.handle, int(reps)), "ecmg_autotune")

    def get(self, problem, which, level=-1):
        import torch
        q = self.problems[problem]
        L = int(q["levels"])
        l = L - 1 if level < 0 else level
        n = [int(v) << l for v in q["n0"]]
        out = torch.empty((n[2] + 1, n[1] + 1, n[0] + 1), dtype=torch.float64, device="cuda")
        check(ecmg_get_level_batched(self.handle, int(problem), int(level), int(which), _ptr(out)),
              "ecmg_get_level_batched")
        return out

    def close(self):
        if getattr(self, "handle", None):
            ecmg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kernel_launches() -> int:
    v = C.c_uint64()
    check(ecmg_kernel_launches(C.byref(v)), "ecmg_kernel_launches")
    return v.value


def stats_dict(st: ecmg_stats) -> dict:
    L = st.levels
    return dict(levels=L, iters=list(st.iters[:L]), updates=list(st.updates[:L]),
                rel_res=list(st.rel_res[:L]), rhs_norm=list(st.rhs_norm[:L]), status=st.status,
                seconds=list(st.seconds[:L]), setup_seconds=st.setup_seconds)


def solver_from_problem(prob: dict, device="cuda", **options):
    """Build a Solver from a problem dict of ``paper_1506_02983_gb300.inputs`` (copies the
    host arrays to the device)."""
    import torch
    t = lambda a: None if a is None else torch.as_tensor(a, dtype=torch.float64).contiguous().to(device)
    beta, f, gD, gR = t(prob.get("beta")), t(prob["f"]), t(prob.get("gD")), t(prob.get("gR"))
    options.setdefault("rtol", prob.get("rtol", 1e-9))
    s = Solver(prob["n0"], prob["levels"], prob["lo"], prob["hi"], prob["face_bc"], prob["alpha"],
               beta, f, gD, gR, f_mode=prob.get("f_mode", 0), f_terms=prob.get("f_terms", 0),
               gD_terms=prob.get("gD_terms", 0), beta_const=prob.get("beta_const", 0.0), **options)
    return s
