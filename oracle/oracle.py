"""ctypes binding of the plain C oracle (``ecmg_oracle.c``).

TEST INFRASTRUCTURE: used by the tests, by ``__graft_entry__.smoke()`` and by the CPU-baseline
leg of ``bench.py`` only. It shares no code with the CUDA path; it receives the same seeded
inputs (from ``paper_1506_02983_gb300.inputs``, which holds none of the solver's arithmetic;
the LOAD-mode functionals it evaluates are pinned to ``load_functional`` here) and computes
everything itself, in FP64, on one host core.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ecmg_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "_build", "liboracle_omp.so")

DIRICHLET, ROBIN = 0, 1
F_NODAL, F_LOAD = 0, 1
EXP_SERENDIPITY20, EXP_LAGRANGE27 = 0, 1


def _compile(target: str, extra: list, force: bool) -> str:
    os.makedirs(os.path.dirname(target), exist_ok=True)
    hdr = os.path.join(_HERE, "ecmg_oracle.h")
    if force or not os.path.exists(target) or os.path.getmtime(target) < max(os.path.getmtime(_SRC),
                                                                             os.path.getmtime(hdr)):
        tmp = target + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", *extra,
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, target)
    return target


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into ``oracle/_build/liboracle.so`` (one thread).

    ``-ffp-contract=off`` keeps x86 and Arm hosts bit-identical (no fused multiply-add).
    """
    return _compile(_LIB, [], force)


def build_omp(force: bool = False) -> str:
    """The same source with OpenMP (``liboracle_omp.so``): the CSR products and the element-wise
    vector updates of JCG run on several threads, with results equal to the one-thread build."""
    return _compile(_LIB_OMP, ["-fopenmp"], force)


class _Problem(C.Structure):
    _fields_ = [("n0", C.c_int32 * 3), ("levels", C.c_int32),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("face_bc", C.c_int32 * 6), ("alpha", C.c_double * 6),
                ("beta", C.c_void_p), ("f", C.c_void_p), ("gD", C.c_void_p),
                ("gR", C.c_void_p), ("f_mode", C.c_int32)]


class _Stats(C.Structure):
    _fields_ = [("iters", C.c_int32 * 16), ("rel_res", C.c_double * 16),
                ("rhs_norm", C.c_double * 16), ("status", C.c_int32),
                ("seconds_assembly", C.c_double), ("seconds_solve", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = _load(build())
    return _lib


_lib_omp = None


def lib_omp():
    """The OpenMP build (see build_omp)."""
    global _lib_omp
    if _lib_omp is None:
        _lib_omp = _load(build_omp())
    return _lib_omp


def _load(path):
    """Load one build of the oracle and declare its entry points."""
    _lib = C.CDLL(path)
    D, I64, I32 = C.c_double, C.c_int64, C.c_int32
    P = C.c_void_p
    _lib.or_assemble_csr.restype = I64
    _lib.or_assemble_csr.argtypes = [P, P, P, P, P, P, P, P]
    _lib.or_element_matrix.argtypes = [D, D, D, P]
    _lib.or_element_mass.argtypes = [D, D, D, P]
    _lib.or_face_mass.argtypes = [D, D, P]
    _lib.or_dirichlet_mask.argtypes = [P, P, P]
    _lib.or_load_nodal.argtypes = [P, P, P, P, P, P]
    _lib.or_csr_matvec.argtypes = [I64, P, P, P, P, P]
    _lib.or_coarsen_beta.argtypes = [P, P, P]
    _lib.or_inject.argtypes = [P, P, P]
    _lib.or_restrict_load.argtypes = [P, P, P]
    _lib.or_jcg.restype = C.c_int
    _lib.or_jcg.argtypes = [I64, P, P, P, P, P, P, P, D, I32, P, P, P]
    _lib.or_set_threads.restype = I32
    _lib.or_set_threads.argtypes = [I32]
    _lib.or_pcg.restype = C.c_int
    _lib.or_pcg.argtypes = [I64, P, P, P, P, P, P, P, D, I32, I32, I32, P, P, P]
    _lib.or_pcg_single_pass.restype = C.c_int
    _lib.or_pcg_single_pass.argtypes = [I64, P, P, P, P, P, P, P, D, I32, I32, P, P, P]
    _lib.or_dsolve_banded.restype = C.c_int
    _lib.or_dsolve_banded.argtypes = [P, I64, P, P, P, P, P, P]
    _lib.or_serendipity.argtypes = [D, D, D, P]
    _lib.or_serendipity_nodes.argtypes = [P]
    _lib.or_exp_finite.argtypes = [P, P, P, P]
    _lib.or_exp_finite27.argtypes = [P, P, P, P]
    _lib.or_exp_true.argtypes = [P, P, P, P]
    _lib.or_apply_at.restype = D
    _lib.or_apply_at.argtypes = [P, P, P, P, P, P, I64, I64, I64]
    _lib.or_exp_finite_at.restype = D
    _lib.or_exp_finite_at.argtypes = [P, P, P, I64, I64, I64]
    _lib.or_exp_true_at.restype = D
    _lib.or_exp_true_at.argtypes = [P, P, P, I64, I64, I64]
    _lib.or_ecmg_ex.restype = C.c_int
    _lib.or_ecmg_ex.argtypes = [C.POINTER(_Problem), D, I32, I32, I32, I32, I32, D, P, P, P, C.POINTER(_Stats)]
    _lib.or_schedule_steps.restype = I32
    _lib.or_schedule_steps.argtypes = [I32, I32, I32, D]
    _lib.or_ecmg.restype = C.c_int
    _lib.or_ecmg.argtypes = [C.POINTER(_Problem), D, I32, I32, P, P, P, C.POINTER(_Stats)]
    _lib.or_norms.argtypes = [I64, P, P, P, P]
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data


def _i32(v):
    return np.ascontiguousarray(np.asarray(v, dtype=np.int32))


def _f64(v):
    return np.ascontiguousarray(np.asarray(v, dtype=np.float64))


def num_nodes(n):
    return (n[0] + 1) * (n[1] + 1) * (n[2] + 1)


# ---- discretisation --------------------------------------------------------------------
def element_matrix(hx, hy, hz):
    K = np.zeros(64)
    lib().or_element_matrix(hx, hy, hz, _p(K))
    return K.reshape(8, 8)


def element_mass(hx, hy, hz):
    M = np.zeros(64)
    lib().or_element_mass(hx, hy, hz, _p(M))
    return M.reshape(8, 8)


def face_mass(ha, hb):
    M = np.zeros(16)
    lib().or_face_mass(ha, hb, _p(M))
    return M.reshape(4, 4)


def dirichlet_mask(n, face_bc):
    """1 = free node, 0 = Dirichlet node (flat, x fastest)."""
    m = np.zeros(num_nodes(n), dtype=np.uint8)
    nn, bc = _i32(n), _i32(face_bc)
    lib().or_dirichlet_mask(_p(nn), _p(bc), _p(m))
    return m


@dataclass
class CSR:
    N: int
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    def matvec(self, x):
        x = _f64(x)
        y = np.zeros(self.N)
        lib().or_csr_matvec(self.N, _p(self.rowptr), _p(self.col), _p(self.val), _p(x), _p(y))
        return y

    def dense(self):
        A = np.zeros((self.N, self.N))
        for r in range(self.N):
            s, e = self.rowptr[r], self.rowptr[r + 1]
            A[r, self.col[s:e]] = self.val[s:e]
        return A


def assemble(n, h, beta, face_bc, alpha):
    N = num_nodes(n)
    rowptr = np.zeros(N + 1, dtype=np.int64)
    col = np.zeros(27 * N, dtype=np.int64)
    val = np.zeros(27 * N)
    beta = _f64(beta)
    nn, hh, bc, al = _i32(n), _f64(h), _i32(face_bc), _f64(alpha)
    nnz = lib().or_assemble_csr(_p(nn), _p(hh), _p(beta), _p(bc), _p(al), _p(rowptr),
                                _p(col), _p(val))
    if nnz < 0:
        raise MemoryError("oracle assembly failed")
    return CSR(N, rowptr, col[:nnz].copy(), val[:nnz].copy())


def load_nodal(n, h, f, face_bc, gR=None):
    b = np.zeros(num_nodes(n))
    f = _f64(f)
    gR = None if gR is None else _f64(gR)
    nn, hh, bc = _i32(n), _f64(h), _i32(face_bc)
    lib().or_load_nodal(_p(nn), _p(hh), _p(f), _p(bc), _p(gR), _p(b))
    return b


def gauss3_unit():
    """3-point Gauss-Legendre rule on [0, 1]: nodes (1 - sqrt(3/5))/2, 1/2, (1 + sqrt(3/5))/2
    and weights 5/18, 8/18, 5/18 (exact for polynomials of degree <= 5)."""
    r = np.sqrt(0.6)
    return np.array([0.5 * (1.0 - r), 0.5, 0.5 * (1.0 + r)]), np.array([5.0, 8.0, 5.0]) / 18.0


def load_functional(n, lo, hi, f, q=6, faces=()):
    """Load functional of the weak form of Sec. 2 on the uniform grid of n = (nx, ny, nz)
    elements of the box [lo, hi]:  b_i = int_Omega f phi_i dx + sum over `faces` of
    int_F g phi_i dS,  written as the definition, element by element: on every element a q-point
    tensor Gauss-Legendre rule of f times each of the element's 8 trilinear hats, added into that
    hat's node; on every quad of a face likewise with q x q points and the quad's 4 bilinear
    hats. f(x, y, z) and g(x, y, z) take broadcastable coordinate arrays (points are interior to
    the elements and quads, so piecewise data may switch on element boundaries). faces: triples
    (axis, node index along that axis, g). Shape (nz+1, ny+1, nx+1)."""
    n = [int(v) for v in n]
    nx, ny, nz = n
    h = [(hi[a] - lo[a]) / n[a] for a in range(3)]
    t, w = np.polynomial.legendre.leggauss(int(q))
    t, w = 0.5 * (t + 1.0), 0.5 * w
    hat = {0: 1.0 - t, 1: t}  # the left and right hat of an interval at its points
    # the Gauss points of every element interval along each axis, shape (n_a, q)
    P = [lo[a] + (np.arange(n[a])[:, None] + t[None, :]) * h[a] for a in range(3)]
    b = np.zeros((nz + 1, ny + 1, nx + 1))
    vol = h[0] * h[1] * h[2]
    for ez in range(nz):
        X = P[0].reshape(1, nx, 1, 1, q)
        Y = P[1].reshape(ny, 1, 1, q, 1)
        Z = P[2][ez].reshape(1, 1, q, 1, 1)
        F = np.broadcast_to(f(X, Y, Z), (ny, nx, q, q, q))  # F[ey, ex, qz, qy, qx]
        for cz in (0, 1):
            for cy in (0, 1):
                for cx in (0, 1):
                    wphi = np.einsum("c,b,a->cba", w * hat[cz], w * hat[cy], w * hat[cx])
                    b[ez + cz, cy:cy + ny, cx:cx + nx] += vol * np.einsum("jicba,cba->ji", F, wphi)
    for axis, idx, g in faces:
        a1, a2 = [a for a in range(3) if a != axis]  # the face's two axes, a1 < a2
        c = lo[axis] + idx * h[axis]
        pts = [None, None, None]
        pts[axis] = np.full((1, 1, 1, 1), c)
        pts[a1] = P[a1].reshape(1, n[a1], 1, q)
        pts[a2] = P[a2].reshape(n[a2], 1, q, 1)
        G = np.broadcast_to(g(*pts), (n[a2], n[a1], q, q))  # G[e2, e1, q2, q1]
        area = h[a1] * h[a2]
        for c2 in (0, 1):
            for c1 in (0, 1):
                wphi = np.outer(w * hat[c2], w * hat[c1])
                v = area * np.einsum("jiba,ba->ji", G, wphi)
                if axis == 0:
                    b[c2:c2 + nz, c1:c1 + ny, idx] += v
                elif axis == 1:
                    b[c2:c2 + nz, idx, c1:c1 + nx] += v
                else:
                    b[idx, c2:c2 + ny, c1:c1 + nx] += v
    return b


def load_gauss(n, h, samples):
    """Load functional b_i = int f phi_i of Sec. 2 with f given at the 27 points of the 3-point
    Gauss-Legendre rule of every element (the ECMG_F_GAUSS layout: elements x fastest, then the
    points qx fastest, qy, qz). Written as the definition: on every element the rule's weights
    times f times each of the element's 8 trilinear hats at the points, added into the hat's
    node. Shape (nz+1, ny+1, nx+1)."""
    nx, ny, nz = (int(v) for v in n)
    F = np.asarray(samples, dtype=np.float64).reshape(nz, ny, nx, 3, 3, 3)  # [ez, ey, ex, qz, qy, qx]
    g, w = gauss3_unit()
    b = np.zeros((nz + 1, ny + 1, nx + 1))
    vol = h[0] * h[1] * h[2]
    for cz in (0, 1):
        for cy in (0, 1):
            for cx in (0, 1):
                phx = g if cx else 1.0 - g
                phy = g if cy else 1.0 - g
                phz = g if cz else 1.0 - g
                wphi = np.einsum("c,b,a->cba", w * phz, w * phy, w * phx)
                b[cz:cz + nz, cy:cy + ny, cx:cx + nx] += vol * np.einsum("kjicba,cba->kji", F, wphi)
    return b


def load_separable(n, h, terms, samples):
    """Load functional b_i = int f phi_i of Sec. 2 for f = sum_t fx_t(x) fy_t(y) fz_t(z), given by
    its factors at the 3-point Gauss nodes of every element interval (the ECMG_F_SEPARABLE
    layout: term-major, then x (3 per interval), y, z). Written as the definition: on every
    element, the 27-point tensor Gauss rule of f times each of the element's 8 trilinear hats,
    added into the hat's node. Exact when the factors have degree <= 4. Shape (nz+1, ny+1, nx+1)."""
    nx, ny, nz = (int(v) for v in n)
    s = np.asarray(samples, dtype=np.float64).reshape(int(terms), -1)
    fx = s[:, :3 * nx].reshape(-1, nx, 3)
    fy = s[:, 3 * nx:3 * (nx + ny)].reshape(-1, ny, 3)
    fz = s[:, 3 * (nx + ny):].reshape(-1, nz, 3)
    # f at the 27 points of every element: F[ez, ey, ex, qz, qy, qx]
    F = np.einsum("tkc,tjb,tia->kjicba", fz, fy, fx)
    g, w = gauss3_unit()
    b = np.zeros((nz + 1, ny + 1, nx + 1))
    vol = h[0] * h[1] * h[2]
    for cz in (0, 1):
        for cy in (0, 1):
            for cx in (0, 1):
                # the hat of corner (cx, cy, cz) at the 27 points, times the weights
                phx = g if cx else 1.0 - g
                phy = g if cy else 1.0 - g
                phz = g if cz else 1.0 - g
                wphi = np.einsum("c,b,a->cba", w * phz, w * phy, w * phx)
                b[cz:cz + nz, cy:cy + ny, cx:cx + nx] += vol * np.einsum("kjicba,cba->kji", F, wphi)
    return b


def nodal_separable(n, terms, factors):
    """g(x_i, y_j, z_k) = sum_t gx_t[i] gy_t[j] gz_t[k] from nodal factors (term-major, then x,
    y, z), shape (nz+1, ny+1, nx+1)."""
    nx, ny, nz = (int(v) for v in n)
    s = np.asarray(factors, dtype=np.float64).reshape(int(terms), -1)
    gx, gy, gz = s[:, :nx + 1], s[:, nx + 1:nx + ny + 2], s[:, nx + ny + 2:]
    return np.einsum("tk,tj,ti->kji", gz, gy, gx)


# ---- level transfer ---------------------------------------------------------------------
def coarsen_beta(nc, beta_fine):
    out = np.zeros(int(np.prod(nc)))
    bf, nn = _f64(beta_fine), _i32(nc)
    lib().or_coarsen_beta(_p(nn), _p(bf), _p(out))
    return out


def inject(nc, v_fine):
    out = np.zeros(num_nodes(nc))
    vf, nn = _f64(v_fine), _i32(nc)
    lib().or_inject(_p(nn), _p(vf), _p(out))
    return out


def restrict_load(nc, b_fine):
    out = np.zeros(num_nodes(nc))
    bf, nn = _f64(b_fine), _i32(nc)
    lib().or_restrict_load(_p(nn), _p(bf), _p(out))
    return out


# ---- solvers ----------------------------------------------------------------------------
def schedule_steps(L, l, mL, beta):
    """CG steps of level l in the fixed schedule of Alg. 3 (eq. (ee))."""
    return int(lib().or_schedule_steps(int(L), int(l), int(mL), float(beta)))


def apply_at(n, h, beta, face_bc, alpha, x, nodes):
    """(A x) at the given nodes [(i, j, k), ...] from the element matrices (or_apply_at)."""
    nn, hh, bc, al = _i32(n), _f64(h), _i32(face_bc), _f64(alpha)
    beta, x = _f64(beta), _f64(x)
    L = lib()
    return np.array([L.or_apply_at(_p(nn), _p(hh), _p(beta), _p(bc), _p(al), _p(x), int(i), int(j), int(k))
                     for i, j, k in nodes])


def exp_finite_at(n, U1, U0, nodes):
    """EXP_finite (Serendipity) of level n at the given nodes (or_exp_finite_at)."""
    nn, U1, U0 = _i32(n), _f64(U1), _f64(U0)
    L = lib()
    return np.array([L.or_exp_finite_at(_p(nn), _p(U1), _p(U0), int(i), int(j), int(k)) for i, j, k in nodes])


def exp_true_at(n, U1, U0, nodes):
    """EXP_true of level n at the given nodes (or_exp_true_at)."""
    nn, U1, U0 = _i32(n), _f64(U1), _f64(U0)
    L = lib()
    return np.array([L.or_exp_true_at(_p(nn), _p(U1), _p(U0), int(i), int(j), int(k)) for i, j, k in nodes])


def jcg(A: CSR, mask, b, gext, x0, rtol, max_iters=100000):
    x = _f64(x0).copy()
    it = C.c_int32()
    rr = C.c_double()
    fh = C.c_double()
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    b = _f64(b)
    g = _f64(gext)
    st = lib().or_jcg(A.N, _p(A.rowptr), _p(A.col), _p(A.val), _p(m), _p(b), _p(g), _p(x),
                      rtol, max_iters, C.byref(it), C.byref(rr), C.byref(fh))
    return x, dict(status=st, iters=it.value, rel_res=rr.value, rhs_norm=fh.value)


def pcg(A: CSR, mask, b, gext, x0, rtol, max_iters=100000, precond=1, fixed=0):
    """Textbook JCG / CG (or_pcg); fixed=1 runs exactly max_iters steps."""
    x = _f64(x0).copy()
    it, rr, fh = C.c_int32(), C.c_double(), C.c_double()
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    b, g = _f64(b), _f64(gext)
    st = lib().or_pcg(A.N, _p(A.rowptr), _p(A.col), _p(A.val), _p(m), _p(b), _p(g), _p(x), rtol, max_iters,
                      precond, fixed, C.byref(it), C.byref(rr), C.byref(fh))
    return x, dict(status=st, iters=it.value, rel_res=rr.value, rhs_norm=fh.value)


def pcg_single_pass(A: CSR, mask, b, gext, x0, rtol, max_iters=100000, precond=1):
    """The same iteration in the single-pass arrangement (or_pcg_single_pass)."""
    x = _f64(x0).copy()
    it, rr, fh = C.c_int32(), C.c_double(), C.c_double()
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    b, g = _f64(b), _f64(gext)
    st = lib().or_pcg_single_pass(A.N, _p(A.rowptr), _p(A.col), _p(A.val), _p(m), _p(b), _p(g), _p(x), rtol,
                                  max_iters, precond, C.byref(it), C.byref(rr), C.byref(fh))
    return x, dict(status=st, iters=it.value, rel_res=rr.value, rhs_norm=fh.value)


def dsolve(n, A: CSR, mask, b, x0):
    x = _f64(x0).copy()
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    b, nn = _f64(b), _i32(n)
    st = lib().or_dsolve_banded(_p(nn), A.N, _p(A.rowptr), _p(A.col), _p(A.val), _p(m),
                                _p(b), _p(x))
    return x, st


# ---- extrapolation ----------------------------------------------------------------------
def serendipity(xi, eta, zeta):
    N = np.zeros(20)
    lib().or_serendipity(xi, eta, zeta, _p(N))
    return N


def serendipity_nodes():
    a = np.zeros(60, dtype=np.int32)
    lib().or_serendipity_nodes(_p(a))
    return a.reshape(20, 3)


def exp_finite(n, U1, U0):
    W = np.zeros(num_nodes(n))
    U1 = _f64(U1)
    U0, nn = _f64(U0), _i32(n)
    lib().or_exp_finite(_p(nn), _p(U1), _p(U0), _p(W))
    return W


def exp_finite27(n, U1, U0):
    W = np.zeros(num_nodes(n))
    U1 = _f64(U1)
    U0, nn = _f64(U0), _i32(n)
    lib().or_exp_finite27(_p(nn), _p(U1), _p(U0), _p(W))
    return W


def exp_true(n, U1, U0):
    Ut = np.zeros(num_nodes(n))
    U1 = _f64(U1)
    U0, nn = _f64(U0), _i32(n)
    lib().or_exp_true(_p(nn), _p(U1), _p(U0), _p(Ut))
    return Ut


def norms(a, b=None):
    a = _f64(a)
    b = None if b is None else _f64(b)
    mx = C.c_double()
    rms = C.c_double()
    lib().or_norms(a.size, _p(a), _p(b), C.byref(mx), C.byref(rms))
    return mx.value, rms.value


# ---- the whole method -------------------------------------------------------------------
def ecmg(prob, rtol, max_iters=100000, exp_variant=EXP_SERENDIPITY20, precond=1, schedule=0, mL=0,
         sched_beta=0.0, threads=None):
    """Run Alg. 4 on a problem dict (see ``paper_1506_02983_gb300.inputs``). precond 1 = JCG
    (ECMG_jcg), 0 = plain CG (ECMG_cg); schedule 1 = the fixed step counts of Alg. 3 (eq. (ee),
    m_j = ceil(mL * sched_beta^(L-j))) instead of the tolerance. threads: None runs the one-thread
    build; a number runs the OpenMP build on that many threads (0: its default).

    Returns (levels, stats): levels[l] = dict(n=..., U=..., W=..., Ut=...) with nodal arrays
    shaped (nz+1, ny+1, nx+1); stats has per-level iters, rel_res, rhs_norm and status, the
    wall seconds of the set-up (seconds_assembly) and of the solves (seconds_solve), and the
    threads used.
    """
    L = int(prob["levels"])
    n0 = [int(v) for v in prob["n0"]]
    sizes = [num_nodes([v << l for v in n0]) for l in range(L)]
    tot = sum(sizes)
    U = np.zeros(tot)
    W = np.zeros(tot)
    Ut = np.zeros(tot)
    beta = _f64(prob["beta"]).ravel()
    f = _f64(prob["f"]).ravel()
    gD = None if prob.get("gD") is None else _f64(prob["gD"]).ravel()
    gR = None if prob.get("gR") is None else _f64(prob["gR"]).ravel()
    P = _Problem()
    P.n0[:] = n0
    P.levels = L
    P.lo[:] = list(prob["lo"])
    P.hi[:] = list(prob["hi"])
    P.face_bc[:] = list(prob["face_bc"])
    P.alpha[:] = list(prob["alpha"])
    P.beta, P.f, P.gD, P.gR = _p(beta), _p(f), _p(gD), _p(gR)
    P.f_mode = int(prob.get("f_mode", F_NODAL))
    S = _Stats()
    lb = lib() if threads is None else lib_omp()
    used = lb.or_set_threads(int(threads or 0))
    lb.or_ecmg_ex(C.byref(P), rtol, max_iters, int(exp_variant), int(precond), int(schedule), int(mL),
                  float(sched_beta), _p(U), _p(W), _p(Ut), C.byref(S))
    out = []
    off = 0
    for l in range(L):
        n = [v << l for v in n0]
        shp = (n[2] + 1, n[1] + 1, n[0] + 1)
        sl = slice(off, off + sizes[l])
        out.append(dict(n=n, U=U[sl].reshape(shp), W=W[sl].reshape(shp), Ut=Ut[sl].reshape(shp)))
        off += sizes[l]
    stats = dict(iters=list(S.iters[:L]), rel_res=list(S.rel_res[:L]),
                 rhs_norm=list(S.rhs_norm[:L]), status=S.status, seconds_assembly=S.seconds_assembly,
                 seconds_solve=S.seconds_solve, threads=used)
    return out, stats
