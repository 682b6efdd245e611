"""Seeded synthetic problem generators for eq. (bvp): -div(beta grad u) = f on a box.

This module holds none of the solver's arithmetic (no operator, no JCG, no extrapolation). It
evaluates problem data -- coefficient beta per element, nodal f, Dirichlet data g_D, Robin data
g_R, boundary types -- for manufactured solutions and for seeded random problems, and, for the
problems given in LOAD mode, the input functional b_i = int f phi_i (+ face terms) of the weak
form of Sec. 2 by Gauss quadrature (hat_integrals_1d / separable_load for separable f, the
per-element rule of jump_singular). That functional is an input of the library's LOAD mode; the
oracle's own per-element definition (oracle.load_functional) pins it. Both the CUDA path and
the CPU oracle receive exactly these arrays.

Every problem is a dict with keys
    n0 (3 ints, coarsest elements per axis), levels, lo, hi (box corners),
    face_bc (6 ints, faces x-,x+,y-,y+,z-,z+; 0 Dirichlet, 1 Robin), alpha (6 floats),
    beta  (finest elements, shape (nz, ny, nx), float64),
    f     (finest nodes, shape (nz+1, ny+1, nx+1)),
    gD, gR (finest nodes or None), f_mode (0 nodal f, 1 assembled load, 2 separable f),
    u_exact (finest nodes or None), rtol (relative-residual tolerance of the workload).
Arrays are C-ordered, so the flat index runs x fastest.

Compact problems (f_mode 2) carry instead: f = the Gauss samples of f_terms separable terms
(``separable_samples``), beta = None with beta_const, gD = the nodal factors of gD_terms
separable terms (``separable_nodal``).
"""
from __future__ import annotations

import numpy as np

DIRICHLET, ROBIN = 0, 1
PI = np.pi


def hat_integrals_1d(func, n, lo, hi, q=6):
    """I[i] = integral of func(t) * phi_i(t) over [lo, hi] for the piecewise-linear hat
    functions phi_i of a uniform n-interval grid, by q-point Gauss-Legendre per interval.
    With q = 6 the result is exact to rounding for the smooth data used here."""
    g, w = np.polynomial.legendre.leggauss(q)
    g = 0.5 * (g + 1.0)
    w = 0.5 * w
    h = (hi - lo) / n
    t = lo + (np.arange(n)[:, None] + g[None, :]) * h          # (n, q) points
    ft = func(t) * w[None, :] * h
    out = np.zeros(n + 1)
    out[:-1] += (ft * (1.0 - g)[None, :]).sum(axis=1)
    out[1:] += (ft * g[None, :]).sum(axis=1)
    return out


def separable_load(n, lo, hi, scale, fx, fy, fz):
    """Load functional f(phi_i) (Sec. 2) for a separable right-hand side
    f = scale * fx(x) fy(y) fz(z), shape (nz+1, ny+1, nx+1)."""
    ix = hat_integrals_1d(fx, n[0], lo[0], hi[0])
    iy = hat_integrals_1d(fy, n[1], lo[1], hi[1])
    iz = hat_integrals_1d(fz, n[2], lo[2], hi[2])
    return scale * iz[:, None, None] * iy[None, :, None] * ix[None, None, :]


def finest(n0, levels):
    return [int(v) << (levels - 1) for v in n0]


def _axes(n, lo, hi, centres=False):
    """Coordinates along x, y, z shaped for broadcasting to (z, y, x)."""
    out = []
    for a in range(3):
        if centres:
            t = lo[a] + (np.arange(n[a]) + 0.5) * (hi[a] - lo[a]) / n[a]
        else:
            t = lo[a] + np.arange(n[a] + 1) * (hi[a] - lo[a]) / n[a]
        shape = [1, 1, 1]
        shape[2 - a] = t.size
        out.append(t.reshape(shape))
    return out


def _base(n0, levels, lo, hi, face_bc, alpha, rtol):
    return dict(n0=[int(v) for v in n0], levels=int(levels), lo=[float(v) for v in lo],
                hi=[float(v) for v in hi], face_bc=[int(v) for v in face_bc],
                alpha=[float(v) for v in alpha], f_mode=0, rtol=float(rtol))


def exp_cube(levels=4, n0=(4, 4, 4), rtol=1e-10):
    """Unit cube, -Laplace u = f, all Dirichlet, u = exp(x+y+z) (the 32^3 parity workload
    with its default 4 levels 4^3 -> 32^3)."""
    p = _base(n0, levels, (0, 0, 0), (1, 1, 1), [DIRICHLET] * 6, [0.0] * 6, rtol)
    n = finest(n0, levels)
    x, y, z = _axes(n, p["lo"], p["hi"])
    u = np.exp(x) * np.exp(y) * np.exp(z)
    p.update(beta=np.ones((n[2], n[1], n[0])), f=-3.0 * u, gD=u, gR=None, u_exact=u)
    return p


def cos_cube(levels=7, n0=(8, 8, 8), rtol=1e-10, load="exact"):
    """Unit cube Poisson, u = cos(pi x) cos(pi y) cos(pi z), all Dirichlet, f = 3 pi^2 u.
    Default 8^3 -> 512^3 (7 levels): the mixed-vs-FP64 workload.
    load="exact": f is the load functional int f phi_i (f_mode 1); "nodal": nodal f."""
    p = _base(n0, levels, (0, 0, 0), (1, 1, 1), [DIRICHLET] * 6, [0.0] * 6, rtol)
    n = finest(n0, levels)
    x, y, z = _axes(n, p["lo"], p["hi"])
    c = [np.cos(PI * t) for t in (x, y, z)]
    u = c[0] * c[1] * c[2]
    if load == "exact":
        cp = lambda t: np.cos(PI * t)
        f = separable_load(n, p["lo"], p["hi"], 3.0 * PI * PI, cp, cp, cp)
        p["f_mode"] = 1
    else:
        f = (3.0 * PI * PI) * u
    p.update(beta=np.ones((n[2], n[1], n[0])), f=f, gD=u, gR=None, u_exact=u)
    return p


def paper_problem1(levels=7, n0=(8, 8, 8), rtol=1e-9, load="exact"):
    """Problem 1 of Sec. 5: Laplace u = -(3/4) pi^2 sin sin sin on [0,1]^3, u = 0 on x, y or
    z = 0, du/dn = 0 on x, y or z = 1; u = sin(pi x/2) sin(pi y/2) sin(pi z/2).
    load="exact": f is the load functional int f phi_i (f_mode 1); "nodal": nodal f."""
    bc = [DIRICHLET, ROBIN, DIRICHLET, ROBIN, DIRICHLET, ROBIN]
    p = _base(n0, levels, (0, 0, 0), (1, 1, 1), bc, [0.0] * 6, rtol)
    n = finest(n0, levels)
    x, y, z = _axes(n, p["lo"], p["hi"])
    u = np.sin(0.5 * PI * x) * np.sin(0.5 * PI * y) * np.sin(0.5 * PI * z)
    if load == "exact":
        sp_ = lambda t: np.sin(0.5 * PI * t)
        f = separable_load(n, p["lo"], p["hi"], 0.75 * PI * PI, sp_, sp_, sp_)
        p["f_mode"] = 1
    else:
        f = (0.75 * PI * PI) * u
    p.update(beta=np.ones((n[2], n[1], n[0])), f=f,
             gD=np.zeros_like(u), gR=np.zeros_like(u), u_exact=u)
    return p


def paper_problem2(levels=7, n0=(10, 4, 5), rtol=1e-12, load="exact"):
    """Problem 2 of Sec. 5: Laplace u = (1 - 2.5 pi^2) e^z sin(3 pi x/2) sin(pi y/2) on [0,1]^3,
    u = 0 on x = 0 and y = 0, u = sin(3 pi x/2) sin(pi y/2) on z = 0 and e times that on z = 1,
    du/dn = 0 on x = 1 and y = 1; u = e^z sin(3 pi x/2) sin(pi y/2). Anisotropic elements:
    coarsest 10 x 4 x 5 (the paper's choice), 7 levels to 640 x 256 x 320.
    load="exact": f is the load functional int f phi_i (f_mode 1); "nodal": nodal f."""
    bc = [DIRICHLET, ROBIN, DIRICHLET, ROBIN, DIRICHLET, DIRICHLET]
    p = _base(n0, levels, (0, 0, 0), (1, 1, 1), bc, [0.0] * 6, rtol)
    n = finest(n0, levels)
    x, y, z = _axes(n, p["lo"], p["hi"])
    u = np.exp(z) * np.sin(1.5 * PI * x) * np.sin(0.5 * PI * y)
    scale = 2.5 * PI * PI - 1.0
    if load == "exact":
        f = separable_load(n, p["lo"], p["hi"], scale, lambda t: np.sin(1.5 * PI * t),
                           lambda t: np.sin(0.5 * PI * t), np.exp)
        p["f_mode"] = 1
    else:
        f = scale * u
    p.update(beta=np.ones((n[2], n[1], n[0])), f=f, gD=u, gR=np.zeros_like(u), u_exact=u)
    return p


def variable_box(levels=7, n0=(8, 8, 16), rtol=1e-9):
    """Box (0,1)x(0,1)x(0,2) with beta = 1 + 0.5 sin(2 pi x) cos(2 pi y) sin(pi z) (at element
    centres), u = sin(pi x) sin(pi y) sin(pi z) + x y z, Dirichlet on five faces and Robin
    (alpha = 1) on z = 0. Default 8x8x16 -> 512x512x1024 (7 levels)."""
    bc = [DIRICHLET, DIRICHLET, DIRICHLET, DIRICHLET, ROBIN, DIRICHLET]
    alpha = [0.0, 0.0, 0.0, 0.0, 1.0, 0.0]
    p = _base(n0, levels, (0, 0, 0), (1, 1, 2), bc, alpha, rtol)
    n = finest(n0, levels)
    xc, yc, zc = _axes(n, p["lo"], p["hi"], centres=True)
    beta = 1.0 + 0.5 * np.sin(2 * PI * xc) * np.cos(2 * PI * yc) * np.sin(PI * zc)
    x, y, z = _axes(n, p["lo"], p["hi"])
    sx, sy, sz = np.sin(PI * x), np.sin(PI * y), np.sin(PI * z)
    cx, cy, cz = np.cos(PI * x), np.cos(PI * y), np.cos(PI * z)
    u = sx * sy * sz + x * y * z
    b = 1.0 + 0.5 * np.sin(2 * PI * x) * np.cos(2 * PI * y) * sz
    bx = PI * np.cos(2 * PI * x) * np.cos(2 * PI * y) * sz
    by = -PI * np.sin(2 * PI * x) * np.sin(2 * PI * y) * sz
    bz = 0.5 * PI * np.sin(2 * PI * x) * np.cos(2 * PI * y) * cz
    ux = PI * cx * sy * sz + y * z
    uy = PI * sx * cy * sz + x * z
    uz = PI * sx * sy * cz + x * y
    lap = -3.0 * PI * PI * sx * sy * sz
    f = -b * lap - (bx * ux + by * uy + bz * uz)
    # Robin on z = 0 (outward normal -z): g_R = alpha u + beta du/dn = u - beta u_z
    gR = u - b * uz
    p.update(beta=beta, f=f, gD=u, gR=gR, u_exact=u)
    return p


def random_problem(seed, n0=(2, 3, 2), levels=3, box=(1.0, 1.5, 0.75), face_bc=None,
                   alpha=None, rtol=1e-10, contrast=10.0):
    """Seeded random problem: lognormal beta (clipped to the given contrast), uniform f,
    g_D and g_R in [-1, 1], and (unless given) random boundary types and Robin alphas with at
    least one Dirichlet face."""
    rng = np.random.default_rng(seed)
    if face_bc is None:
        face_bc = list(rng.integers(0, 2, size=6))
        if all(b == ROBIN for b in face_bc):
            face_bc[int(rng.integers(0, 6))] = DIRICHLET
    if alpha is None:
        alpha = [float(rng.choice([0.0, 0.5, 2.0])) if b == ROBIN else 0.0 for b in face_bc]
    p = _base(n0, levels, (0, 0, 0), box, face_bc, alpha, rtol)
    n = finest(n0, levels)
    lnc = np.log(contrast)
    beta = np.exp(np.clip(rng.standard_normal((n[2], n[1], n[0])), -lnc / 2, lnc / 2))
    shp = (n[2] + 1, n[1] + 1, n[0] + 1)
    p.update(beta=beta, f=rng.uniform(-1, 1, shp), gD=rng.uniform(-1, 1, shp),
             gR=rng.uniform(-1, 1, shp), u_exact=None)
    return p


def random_vector(seed, shape):
    """Seeded uniform [-1, 1] nodal vector (for operator parity checks)."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, shape)


def coarsest_split(N, min_coarse=4):
    """Coarsest grid and level count for a finest grid of N = (Nx, Ny, Nz) elements: halve every
    axis while all are even and every half stays >= min_coarse."""
    n = [int(v) for v in N]
    levels = 1
    while all(v % 2 == 0 and v // 2 >= min_coarse for v in n):
        n = [v // 2 for v in n]
        levels += 1
    return n, levels


def batch_problems(count=64, seed=1506, sizes=(32, 48, 64, 96, 128), h=1.0 / 128, rtol=1e-8,
                   ln_contrast=np.log(10.0)):
    """Batched workload: `count` independent all-Dirichlet problems (g_D = 0) with cubic elements
    of side h. Per problem and axis the finest element count is drawn uniformly from `sizes`
    (box = N h); beta = exp(z) per element with z ~ N(0, 1) clipped to +-ln_contrast (a
    contrast of at most 1e2); f ~ U[-1, 1] per finest node (nodal data, injected to coarser
    levels). Levels from coarsest_split (at least 3 for these sizes)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        N = [int(v) for v in rng.choice(sizes, size=3)]
        n0, levels = coarsest_split(N)
        p = _base(n0, levels, (0.0, 0.0, 0.0), [v * h for v in N], [DIRICHLET] * 6, [0.0] * 6, rtol)
        beta = np.exp(np.clip(rng.standard_normal((N[2], N[1], N[0])), -ln_contrast, ln_contrast))
        f = rng.uniform(-1.0, 1.0, (N[2] + 1, N[1] + 1, N[0] + 1))
        p.update(beta=beta, f=f, gD=None, gR=None, u_exact=None)
        out.append(p)
    return out


def _gauss3():
    """3-point Gauss-Legendre nodes and weights on [0, 1]."""
    g, w = np.polynomial.legendre.leggauss(3)
    return 0.5 * (g + 1.0), 0.5 * w


def jump_singular(levels=7, n0=(16, 8, 8), rtol=1e-8, device=None):
    """Box (0,2)x(0,1)x(0,1), beta = 1 for x < 1 and 100 for x > 1 (element centres), singular
    manufactured solution u = r^1.5 (r = distance to the origin corner), Robin (alpha = 1) on
    x = 0 and Dirichlet (g_D = u) elsewhere. Default 16x8x8 -> 1024x512x512 (7 levels).

    u does not carry a continuous flux across x = 1, so the load functional (f_mode 1) is
        b_i = int f phi_i + int_{x=1} (beta- - beta+) du/dx phi_i dS + int_{x=0} g_R phi_i dS
    with f = -beta Laplace(u) = -3.75 beta r^-1/2, (beta- - beta+) du/dx = -99 * 1.5 r^-1/2 on
    x = 1, and g_R = beta du/dn + alpha u = r^1.5 on x = 0 (du/dx = 0 there); every integral by
    3-point Gauss per element or face quad (no evaluation at r = 0). device: None for numpy,
    or a torch device to evaluate the (large) arrays there."""
    if device is None:
        xp, mk = np, (lambda a: np.asarray(a, dtype=np.float64))
    else:
        import torch
        xp, mk = torch, (lambda a: torch.as_tensor(np.asarray(a, dtype=np.float64), device=device))
    bc = [ROBIN, DIRICHLET, DIRICHLET, DIRICHLET, DIRICHLET, DIRICHLET]
    alpha = [1.0, 0.0, 0.0, 0.0, 0.0, 0.0]
    p = _base(n0, levels, (0, 0, 0), (2, 1, 1), bc, alpha, rtol)
    p["f_mode"] = 1
    n = finest(n0, levels)
    h = [(p["hi"][a] - p["lo"][a]) / n[a] for a in range(3)]
    g, w = _gauss3()
    xs = mk(np.arange(n[0] + 1) * h[0])
    ys = mk(np.arange(n[1] + 1) * h[1])
    zs = mk(np.arange(n[2] + 1) * h[2])
    xc = mk((np.arange(n[0]) + 0.5) * h[0])
    beta_x = xp.where(xc < 1.0, mk(1.0), mk(100.0))                      # (nx,)
    beta = beta_x.reshape(1, 1, n[0]).expand(n[2], n[1], n[0]).contiguous() if device is not None else \
        np.broadcast_to(beta_x.reshape(1, 1, n[0]), (n[2], n[1], n[0])).copy()
    X, Y = xs.reshape(1, -1), ys.reshape(-1, 1)                          # (1, nx+1), (ny+1, 1)
    b = xp.zeros((n[2] + 1, n[1] + 1, n[0] + 1), dtype=xp.float64) if device is None else \
        xp.zeros((n[2] + 1, n[1] + 1, n[0] + 1), dtype=xp.float64, device=device)
    u = b.clone() if device is not None else b.copy()
    for k in range(n[2] + 1):
        u[k] = (X * X + Y * Y + zs[k] * zs[k]) ** 0.75
    # Gauss points of every element along each axis: (n, 3) coordinates and hat values
    def axis_pts(a):
        t = mk((np.arange(n[a])[:, None] + g[None, :]) * h[a])           # (n, 3)
        return t, mk(1.0 - g), mk(g)                                     # left / right hat at the points
    px, lx, rx = axis_pts(0)
    py, ly, ry = axis_pts(1)
    pz, lz, rz = axis_pts(2)
    wq = mk(w)
    jac = h[0] * h[1] * h[2]
    # volume term, one slab of elements at a time: contributions to the 8 corners
    for k in range(n[2]):
        # f at (ny, nx, 3z, 3y, 3x) points
        R2 = (px.reshape(1, n[0], 1, 1, 3) ** 2 + py.reshape(n[1], 1, 1, 3, 1) ** 2
              + pz[k].reshape(1, 1, 3, 1, 1) ** 2)
        fv = -3.75 * beta_x.reshape(1, n[0], 1, 1, 1) * R2 ** -0.25
        wz, wy, wx = wq.reshape(1, 1, 3, 1, 1), wq.reshape(1, 1, 1, 3, 1), wq.reshape(1, 1, 1, 1, 3)
        fw = fv * (wz * wy * wx) * jac
        for cz, hz in ((0, lz), (1, rz)):
            for cy, hy in ((0, ly), (1, ry)):
                for cx, hx in ((0, lx), (1, rx)):
                    phi = hz.reshape(1, 1, 3, 1, 1) * hy.reshape(1, 1, 1, 3, 1) * hx.reshape(1, 1, 1, 1, 3)
                    c = (fw * phi).sum(axis=(2, 3, 4)) if device is None else (fw * phi).sum(dim=(2, 3, 4))
                    b[k + cz, cy:cy + n[1], cx:cx + n[0]] += c
    # face terms: (values on the face's (nz, ny) quads at 3x3 points) -> 4 corners
    def face_add(i_node, xval, coef, power):
        R2 = xval * xval + py.reshape(1, n[1], 1, 3) ** 2 + pz.reshape(n[2], 1, 3, 1) ** 2
        fv = coef * R2 ** power * (wq.reshape(1, 1, 3, 1) * wq.reshape(1, 1, 1, 3)) * (h[1] * h[2])
        for cz, hz in ((0, lz), (1, rz)):
            for cy, hy in ((0, ly), (1, ry)):
                phi = hz.reshape(1, 1, 3, 1) * hy.reshape(1, 1, 1, 3)
                c = (fv * phi).sum(axis=(2, 3)) if device is None else (fv * phi).sum(dim=(2, 3))
                b[cz:cz + n[2], cy:cy + n[1], i_node] += c
    face_add(n[0] // 2, 1.0, -99.0 * 1.5, -0.25)    # interface x = 1: (beta- - beta+) du/dx
    face_add(0, 0.0, 1.0, 0.75)                     # Robin data on x = 0: g_R = r^1.5
    p.update(beta=beta, f=b, gD=u, gR=None, u_exact=u)
    return p


def gauss3_nodes():
    """The 3 Gauss-Legendre nodes on [0, 1] in the order the separable layout uses:
    (1 - sqrt(3/5))/2, 1/2, (1 + sqrt(3/5))/2."""
    r = np.sqrt(0.6)
    return np.array([0.5 * (1.0 - r), 0.5, 0.5 * (1.0 + r)])


def separable_samples(n, lo, hi, terms):
    """f = sum_t fx_t(x) fy_t(y) fz_t(z) (terms: list of (fx, fy, fz) callables) sampled at the
    3 Gauss nodes of every finest element interval: shape (T, 3 (nx + ny + nz)), per term x
    (interval-major, 3 per interval), then y, then z."""
    g = gauss3_nodes()
    rows = []
    for fac in terms:
        row = []
        for a in range(3):
            h = (hi[a] - lo[a]) / n[a]
            t = lo[a] + (np.arange(n[a])[:, None] + g[None, :]) * h
            row.append(np.broadcast_to(np.asarray(fac[a](t), dtype=np.float64), t.shape).ravel())
        rows.append(np.concatenate(row))
    return np.stack(rows)


def gauss_samples(n, lo, hi, f):
    """f(x, y, z) (broadcasting callable) at the 27 points of the 3-point Gauss-Legendre rule of
    every element of the uniform grid n on [lo, hi], in the ECMG_F_GAUSS layout: shape
    (nz, ny, nx, 3, 3, 3), elements x fastest, then the points qx fastest, qy, qz."""
    g = gauss3_nodes()
    pts = [lo[a] + (np.arange(n[a])[:, None] + g[None, :]) * (hi[a] - lo[a]) / n[a] for a in range(3)]
    X = pts[0].reshape(1, 1, n[0], 1, 1, 3)
    Y = pts[1].reshape(1, n[1], 1, 1, 3, 1)
    Z = pts[2].reshape(n[2], 1, 1, 3, 1, 1)
    return np.array(np.broadcast_to(f(X, Y, Z), (n[2], n[1], n[0], 3, 3, 3)), dtype=np.float64)


def exp_cube_gauss(levels=4, n0=(4, 4, 4), rtol=1e-10):
    """exp_cube with f = -Laplace(u) = -3 e^{x+y+z} given at the Gauss points of every finest
    element (f_mode 3)."""
    p = exp_cube(levels=levels, n0=n0, rtol=rtol)
    n = finest(n0, levels)
    p["f"] = gauss_samples(n, p["lo"], p["hi"], lambda x, y, z: -3.0 * np.exp(x + y + z))
    p["f_mode"] = 3
    return p


def random_gauss(seed, n0=(2, 3, 2), levels=3, face_bc=None):
    """A seeded random problem (lognormal beta, random boundary types, Robin alphas and data) with
    f a random trigonometric function given at the Gauss points of every finest element (f_mode 3)
    and nodal g_R on its Robin faces."""
    rng = np.random.default_rng(seed)
    p = random_problem(seed, n0=n0, levels=levels, face_bc=face_bc)
    n = finest(n0, levels)
    a, b, c, d = rng.uniform(0.5, 3.0, 4)
    p["f"] = gauss_samples(n, p["lo"], p["hi"],
                           lambda x, y, z: d * np.sin(a * x + 0.3) * np.cos(b * y - 0.2) + np.exp(-c * z))
    p["f_mode"] = 3
    return p


def separable_nodal(n, lo, hi, terms):
    """Nodal factors of g = sum_t gx_t(x) gy_t(y) gz_t(z): shape (T, (nx+1) + (ny+1) + (nz+1)),
    per term x, then y, then z."""
    rows = []
    for fac in terms:
        row = []
        for a in range(3):
            t = lo[a] + np.arange(n[a] + 1) * (hi[a] - lo[a]) / n[a]
            row.append(np.broadcast_to(np.asarray(fac[a](t), dtype=np.float64), t.shape).ravel())
        rows.append(np.concatenate(row))
    return np.stack(rows)


def cos_cube_compact(levels=7, n0=(8, 8, 8), rtol=1e-10, with_exact=True):
    """cos_cube in compact form: f = 3 pi^2 cos(pi x) cos(pi y) cos(pi z) as one separable term
    (Gauss samples), g_D = u as one separable term, beta_const = 1. O(n) input numbers instead
    of O(n^3). with_exact=False skips the dense u_exact (the 512^3 array is 1 GiB)."""
    p = _base(n0, levels, (0, 0, 0), (1, 1, 1), [DIRICHLET] * 6, [0.0] * 6, rtol)
    n = finest(n0, levels)
    c = lambda t: np.cos(PI * t)
    cs = lambda t: (3.0 * PI * PI) * np.cos(PI * t)
    p.update(f_mode=2, f_terms=1, f=separable_samples(n, p["lo"], p["hi"], [(cs, c, c)]),
             gD_terms=1, gD=separable_nodal(n, p["lo"], p["hi"], [(c, c, c)]),
             beta=None, beta_const=1.0, gR=None, u_exact=None)
    if with_exact:
        x, y, z = _axes(n, p["lo"], p["hi"])
        p["u_exact"] = c(x) * c(y) * c(z)
    return p


def random_separable(seed, n0=(3, 2, 2), levels=3, f_terms=3, gD_terms=2, face_bc=None, rtol=1e-10):
    """Seeded compact problem: a random box, f and g_D sums of products of random polynomials of
    degree <= 4 in each variable (the 3-point Gauss rule integrates them times a hat exactly),
    one random beta_const, Dirichlet faces unless face_bc says otherwise (Robin faces take
    random alpha and homogeneous data)."""
    rng = np.random.default_rng(seed)
    hi = tuple(float(v) for v in rng.uniform(0.5, 2.0, 3))
    lo = tuple(float(v) for v in rng.uniform(-0.5, 0.5, 3))
    hi = tuple(l + d for l, d in zip(lo, hi))
    bc = [DIRICHLET] * 6 if face_bc is None else list(face_bc)
    alpha = [0.0 if b == DIRICHLET else float(rng.uniform(0.5, 2.0)) for b in bc]
    p = _base(n0, levels, lo, hi, bc, alpha, rtol)
    n = finest(n0, levels)

    def poly():
        c = rng.standard_normal(int(rng.integers(1, 6)))
        return lambda t, c=c: np.polynomial.polynomial.polyval(t, c)

    fterms = [(poly(), poly(), poly()) for _ in range(f_terms)]
    gterms = [(poly(), poly(), poly()) for _ in range(gD_terms)]
    p.update(f_mode=2, f_terms=f_terms, f=separable_samples(n, lo, hi, fterms),
             gD_terms=gD_terms, gD=separable_nodal(n, lo, hi, gterms) if gD_terms else None,
             beta=None, beta_const=float(rng.uniform(0.5, 3.0)), gR=None, u_exact=None,
             f_factors=fterms, gD_factors=gterms)
    return p
