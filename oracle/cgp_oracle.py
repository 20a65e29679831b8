"""Plain FP64 CPU oracle for the coarse-grid projection (CGP) Poisson path.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this module:
only the tests, the smoke check and the benchmark's CPU-baseline leg do.  It
shares no code with the CUDA library; both sides receive the same inputs from
the seeded generators.

What it computes, step by step, in the paper's order (Sect. 2.2, Eqs. 12-20):

1. ``split4``     the nested fine mesh: each coarse triangle cut into four
                  (Sect. 2.3, Eq. 18 with k = 1).  Fine nodes are the coarse
                  nodes followed by the edge midpoints, edges ordered by
                  (min vertex, max vertex); child 4T+c of triangle (a, b, c)
                  is (a, m_ab, m_ca), (m_ab, b, m_bc), (m_ca, m_bc, c),
                  (m_ab, m_bc, m_ca).
2. ``assemble``   Galerkin P1 matrices (Sect. 2.3): stiffness
                  K_ij = int grad psi_i . grad psi_j and the divergence
                  operators Gx_ij = int psi_j d_x psi_i, Gy_ij likewise, by a
                  loop over triangles with scatter-add.
3. ``restrict``   injection, Eq. 19: q_c(beta) = q_f(alpha) where the nodes
                  coincide, found by matching coordinates.
4. ``rhs``        weak right-hand side of Delta x = div F with the natural
                  condition d_n x = F . n:  b_i = int F . grad psi_i, F the P1
                  interpolant.  Potential (Eqs. 5, 12): F = in-plane part of
                  u x B = (v B_z, -u B_z).  Pressure (Eq. 15):
                  F = (rho/dt)(u~, v~).
5. ``pcg``        Jacobi-preconditioned conjugate gradients (Saad, Iterative
                  Methods for Sparse Linear Systems, Alg. 9.1) on K x = b with
                  the Neumann null space removed by mean-zero projection of b,
                  x0 and the final x.
6. ``prolong``    Eq. 20: q_f(alpha) = sum_j q_c(beta_j) psi_j(x_alpha) with
                  psi_j the P1 shape functions of the coarse triangle that
                  contains the fine node (barycentric coordinates).
7. ``lorentz``    Ohm's law Eq. 4 / Eq. 7 and the Lorentz force of Eqs. 2, 8,
                  13-14 per fine triangle: g = grad phi_f (constant on P1),
                  u_bar the vertex mean, j = sigma(-g + u_bar x B), f = j x B.

``mixed_ir`` is the FP32-inner / FP64-outer iterative refinement variant and
``dense_solve`` the direct solve used to pin PCG on small meshes.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.csgraph  # noqa: F401  (connected components of the boundary curves)

# solver status codes of the oracle (its own numbering)
OK = 0
NOT_CONVERGED = 3
BREAKDOWN = 4
NONFINITE = 5

POTENTIAL = 0
PRESSURE = 1


# ----------------------------------------------------------------------------
# 1. nested 4-way split (Sect. 2.3, Eq. 18)
# ----------------------------------------------------------------------------
def split4(xy_c: np.ndarray, tri_c: np.ndarray):
    """Uniform 4-way split of a triangle mesh.

    Returns (xy_f, tri_f, edges, parent) where ``edges`` [E, 2] lists the
    coarse edges (a < b) in lexicographic order, fine node n_c + e is the
    midpoint of edge e, and ``parent[t]`` is the coarse triangle of fine
    triangle t.
    """
    xy_c = np.asarray(xy_c, dtype=np.float64)
    tri = np.asarray(tri_c, dtype=np.int64)
    n_c = xy_c.shape[0]
    t_c = tri.shape[0]
    # the three edges of each triangle: (a,b), (b,c), (c,a)
    ea = tri[:, [0, 1, 2]]
    eb = tri[:, [1, 2, 0]]
    lo = np.minimum(ea, eb)
    hi = np.maximum(ea, eb)
    key = lo * n_c + hi
    uniq, inv = np.unique(key.ravel(), return_inverse=True)
    edges = np.stack([uniq // n_c, uniq % n_c], axis=1)
    mid = n_c + inv.reshape(t_c, 3)          # m_ab, m_bc, m_ca
    xy_m = (xy_c[edges[:, 0]] + xy_c[edges[:, 1]]) * 0.5
    xy_f = np.concatenate([xy_c, xy_m], axis=0)
    a, b, c = tri[:, 0], tri[:, 1], tri[:, 2]
    m_ab, m_bc, m_ca = mid[:, 0], mid[:, 1], mid[:, 2]
    tri_f = np.empty((4 * t_c, 3), dtype=np.int64)
    tri_f[0::4] = np.stack([a, m_ab, m_ca], axis=1)
    tri_f[1::4] = np.stack([m_ab, b, m_bc], axis=1)
    tri_f[2::4] = np.stack([m_ca, m_bc, c], axis=1)
    tri_f[3::4] = np.stack([m_ab, m_bc, m_ca], axis=1)
    parent = np.repeat(np.arange(t_c), 4)
    return xy_f, tri_f.astype(np.int32), edges.astype(np.int32), parent


def split_levels(xy_c, tri_c, k: int):
    """k nested uniform 4-way splits (Eq. 18, P = 4^-k M): the list of levels
    [(xy_0, tri_0, None, None), (xy_1, tri_1, edges_0, parent_0), ...] where
    level l + 1 = split4(level l), edges_l are level l's edges and parent_l[t]
    the level-l triangle of level-(l+1) triangle t."""
    levels = [(np.asarray(xy_c, dtype=np.float64), np.asarray(tri_c, dtype=np.int32), None, None)]
    for _ in range(k):
        xy, tri = levels[-1][0], levels[-1][1]
        xy_n, tri_n, edges, parent = split4(xy, tri)
        levels.append((xy_n, tri_n, edges, parent))
    return levels


# ----------------------------------------------------------------------------
# 2. Galerkin P1 assembly (Sect. 2.3)
# ----------------------------------------------------------------------------
def p1_gradients(xy: np.ndarray, tri: np.ndarray):
    """Per triangle: twice the signed area and (b_i, c_i) with grad psi_i = (b_i, c_i) / (2A)."""
    x = xy[tri, 0]
    y = xy[tri, 1]
    i, j, k = [0, 1, 2], [1, 2, 0], [2, 0, 1]
    b = y[:, j] - y[:, k]
    c = x[:, k] - x[:, j]
    area2 = (x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0]) - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0])
    return area2, b, c


def assemble(xy: np.ndarray, tri: np.ndarray):
    """Assemble K, Gx, Gy (CSR, sorted columns, shared pattern) and diag(K).

    On triangle T with area A:  K_T[i, j] = A grad psi_i . grad psi_j
    = (b_i b_j + c_i c_j) / (4A);  Gx_T[i, j] = int_T psi_j d_x psi_i
    = (A/3)(b_i / 2A) = b_i / 6;  Gy_T[i, j] = c_i / 6.
    """
    xy = np.asarray(xy, dtype=np.float64)
    tri = np.asarray(tri, dtype=np.int64)
    n = xy.shape[0]
    area2, b, c = p1_gradients(xy, tri)
    if np.any(area2 <= 0):
        raise ValueError("triangles must be counter-clockwise and non-degenerate")
    A = 0.5 * area2
    kloc = (b[:, :, None] * b[:, None, :] + c[:, :, None] * c[:, None, :]) / (4.0 * A)[:, None, None]
    gxloc = np.repeat((b / 6.0)[:, :, None], 3, axis=2)
    gyloc = np.repeat((c / 6.0)[:, :, None], 3, axis=2)
    rows = np.repeat(tri[:, :, None], 3, axis=2)
    cols = np.repeat(tri[:, None, :], 3, axis=1)
    key = (rows * n + cols).ravel()
    uniq, inv = np.unique(key, return_inverse=True)
    col = (uniq % n).astype(np.int32)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(uniq // n, minlength=n), out=rowptr[1:])
    nnz = uniq.shape[0]
    kv = np.bincount(inv, weights=kloc.ravel(), minlength=nnz)
    gx = np.bincount(inv, weights=gxloc.ravel(), minlength=nnz)
    gy = np.bincount(inv, weights=gyloc.ravel(), minlength=nnz)
    K = sp.csr_matrix((kv, col, rowptr), shape=(n, n))
    Gx = sp.csr_matrix((gx, col, rowptr), shape=(n, n))
    Gy = sp.csr_matrix((gy, col, rowptr), shape=(n, n))
    d = K.diagonal().copy()
    return K, Gx, Gy, d


# ----------------------------------------------------------------------------
# 3. restriction by injection (Eq. 19)
# ----------------------------------------------------------------------------
def restrict(xy_c: np.ndarray, xy_f: np.ndarray, q_f: np.ndarray):
    """q_c(beta) = q_f(alpha) for the fine node alpha at the same position as beta."""
    rec = np.dtype([("x", np.float64), ("y", np.float64)])
    fk = np.ascontiguousarray(xy_f, dtype=np.float64).view(rec).ravel()
    ck = np.ascontiguousarray(xy_c, dtype=np.float64).view(rec).ravel()
    order = np.argsort(fk, kind="stable")
    pos = np.searchsorted(fk[order], ck)
    pos = np.minimum(pos, fk.shape[0] - 1)
    alpha = order[pos]
    if not np.all(fk[alpha] == ck):
        raise ValueError("a coarse node has no coincident fine node")
    return np.asarray(q_f)[alpha]


# ----------------------------------------------------------------------------
# 4. Poisson right-hand side (Eqs. 5, 12, 15)
# ----------------------------------------------------------------------------
def source_field(kind: int, u_c, v_c, B=(0.0, 0.0, 1.0), rho_over_dt: float = 1.0):
    """F with Delta x = div F: potential F = (u x B)_xy = (v B_z, -u B_z); pressure F = (rho/dt) u."""
    u_c = np.asarray(u_c, dtype=np.float64)
    v_c = np.asarray(v_c, dtype=np.float64)
    if kind == POTENTIAL:
        uvec = np.stack([u_c, v_c, np.zeros_like(u_c)], axis=1)
        uxb = np.cross(uvec, np.asarray(B, dtype=np.float64)[None, :])
        return uxb[:, 0], uxb[:, 1]
    if kind == PRESSURE:
        return rho_over_dt * u_c, rho_over_dt * v_c
    raise ValueError("kind")


def rhs(Gx, Gy, Fx, Fy):
    """b_i = int F . grad psi_i = sum_j Gx_ij Fx_j + Gy_ij Fy_j (no projection)."""
    return Gx @ Fx + Gy @ Fy


# ----------------------------------------------------------------------------
# 5. Jacobi PCG (Saad Alg. 9.1) with mean-zero projection
# ----------------------------------------------------------------------------
def project_mean(v):
    v = np.asarray(v, dtype=np.float64)
    return v - np.mean(v)


def pcg(K, d, b, x0=None, tol=1e-8, max_it=20000, project=True):
    """Solve K x = b with Jacobi-preconditioned CG.

    Stops when ||r||_2 <= tol ||b||_2 (recursive residual, b after projection),
    checked before every iteration.  Returns a dict with x (mean-zero when
    ``project``), iterations, recursive and true relative residuals, status.
    """
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    bp = project_mean(b) if project else b.copy()
    bnorm = math.sqrt(float(np.dot(bp, bp)))
    info = dict(iterations=0, rel_res_recursive=0.0, rel_res_true=0.0, status=OK)
    if not math.isfinite(bnorm):
        info.update(status=NONFINITE, x=np.zeros(n))
        return info
    if x0 is None:
        x = np.zeros(n)
    else:
        x = project_mean(x0) if project else np.asarray(x0, dtype=np.float64).copy()
    if bnorm == 0.0:
        info.update(x=np.zeros(n))
        return info
    r = bp - K @ x
    z = r / d
    p = z.copy()
    rz = float(np.dot(r, z))
    k = 0
    status = NOT_CONVERGED
    while True:
        rnorm = math.sqrt(float(np.dot(r, r)))
        if not math.isfinite(rnorm):
            status = NONFINITE
            break
        if rnorm <= tol * bnorm:
            status = OK
            break
        if k >= max_it:
            status = NOT_CONVERGED
            break
        if k > 0:
            rz_new = float(np.dot(r, z))
            beta = rz_new / rz
            rz = rz_new
            p = z + beta * p
        q = K @ p
        pq = float(np.dot(p, q))
        if not (pq > 0.0):
            status = BREAKDOWN if math.isfinite(pq) else NONFINITE
            break
        alpha = rz / pq
        x = x + alpha * p
        r = r - alpha * q
        z = r / d
        k += 1
    if project:
        x = project_mean(x)
    rt = bp - K @ x
    info.update(x=x, iterations=k, status=status,
                rel_res_recursive=math.sqrt(float(np.dot(r, r))) / bnorm,
                rel_res_true=math.sqrt(float(np.dot(rt, rt))) / bnorm)
    return info


def dense_solve(K, b):
    """Direct solve of (K + 1 1^T / n) x = b - mean(b): the mean-zero solution of K x = b."""
    Kd = K.toarray() if sp.issparse(K) else np.asarray(K)
    n = Kd.shape[0]
    return np.linalg.solve(Kd + np.ones((n, n)) / n, project_mean(b))


def outer_boundary(xy, tri):
    """Nodes on the outer boundary: boundary edges (sides of one triangle only), oriented as in
    their counter-clockwise triangle, grouped into connected boundary curves; a curve enclosing
    the domain has positive signed area, one around a hole negative."""
    xy = np.asarray(xy, dtype=np.float64)
    tri = np.asarray(tri, dtype=np.int64)
    n = xy.shape[0]
    sides = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]])
    key = np.minimum(sides[:, 0], sides[:, 1]) * n + np.maximum(sides[:, 0], sides[:, 1])
    uniq, cnt = np.unique(key, return_counts=True)
    bnd = sides[np.isin(key, uniq[cnt == 1])]
    G = sp.coo_matrix((np.ones(len(bnd)), (bnd[:, 0], bnd[:, 1])), shape=(n, n))
    _, label = sp.csgraph.connected_components(G, directed=False)
    a, b = bnd[:, 0], bnd[:, 1]
    area2 = np.bincount(label[a], weights=xy[a, 0] * xy[b, 1] - xy[b, 0] * xy[a, 1],
                        minlength=label.max() + 1)
    nodes = np.unique(bnd.ravel())
    return nodes[area2[label[nodes]] > 0]


def dirichlet_system(K, fixed):
    """K with the rows and columns of the fixed nodes replaced by the identity (their value is zero),
    and its diagonal: the far-field reading phi = 0 on the outer boundary."""
    n = K.shape[0]
    free = np.ones(n)
    free[fixed] = 0.0
    Df = sp.diags(free)
    Kd = (Df @ K @ Df + sp.diags(1.0 - free)).tocsr()
    Kd.sort_indices()
    return Kd, Kd.diagonal().copy()


# ----------------------------------------------------------------------------
# 6. prolongation by P1 shape functions (Eq. 20)
# ----------------------------------------------------------------------------
def prolong(xy_c, tri_c, xy_f, tri_f, parent, q_c):
    """q_f(alpha) = sum_j q_c(beta_j) psi_j(x_alpha) over the parent triangle containing alpha."""
    xy_c = np.asarray(xy_c, dtype=np.float64)
    n_f = xy_f.shape[0]
    q_c = np.asarray(q_c, dtype=np.float64)
    q_f = np.empty(n_f)
    # every fine node is a vertex of a child of some coarse triangle: interpolate there
    owner = np.full(n_f, -1, dtype=np.int64)
    owner[np.asarray(tri_f, dtype=np.int64).ravel()] = np.repeat(np.asarray(parent), 3)
    T = np.asarray(tri_c, dtype=np.int64)[owner]
    x = xy_c[T, 0]
    y = xy_c[T, 1]
    px = xy_f[:, 0]
    py = xy_f[:, 1]
    area2 = (x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0]) - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0])
    # barycentric coordinates: psi_i(p) = area(p, j, k) / area(i, j, k)
    l0 = ((x[:, 1] - px) * (y[:, 2] - py) - (x[:, 2] - px) * (y[:, 1] - py)) / area2
    l1 = ((x[:, 2] - px) * (y[:, 0] - py) - (x[:, 0] - px) * (y[:, 2] - py)) / area2
    l2 = ((x[:, 0] - px) * (y[:, 1] - py) - (x[:, 1] - px) * (y[:, 0] - py)) / area2
    q_f[:] = l0 * q_c[T[:, 0]] + l1 * q_c[T[:, 1]] + l2 * q_c[T[:, 2]]
    return q_f


# ----------------------------------------------------------------------------
# 7. gradient, current density and Lorentz force per fine triangle (Eqs. 4, 7)
# ----------------------------------------------------------------------------
def gradient(xy, tri, phi):
    """grad phi of the P1 field on each triangle: sum_i phi_i (b_i, c_i) / (2A)."""
    area2, b, c = p1_gradients(np.asarray(xy, dtype=np.float64), np.asarray(tri, dtype=np.int64))
    ph = np.asarray(phi, dtype=np.float64)[np.asarray(tri, dtype=np.int64)]
    gx = np.sum(ph * b, axis=1) / area2
    gy = np.sum(ph * c, axis=1) / area2
    return gx, gy


def lorentz(xy_f, tri_f, phi_f, u_f, v_f, B, sigma):
    """Per fine triangle: g = grad phi, j = sigma(-g + u_bar x B), f = j x B.

    Returns grad [T, 2] and force [T, 2] (the in-plane components).
    """
    gx, gy = gradient(xy_f, tri_f, phi_f)
    t = np.asarray(tri_f, dtype=np.int64)
    ub = np.asarray(u_f, dtype=np.float64)[t].mean(axis=1)
    vb = np.asarray(v_f, dtype=np.float64)[t].mean(axis=1)
    Bv = np.asarray(B, dtype=np.float64)[None, :]
    g3 = np.stack([gx, gy, np.zeros_like(gx)], axis=1)
    u3 = np.stack([ub, vb, np.zeros_like(ub)], axis=1)
    j = sigma * (-g3 + np.cross(u3, Bv))
    f = np.cross(j, Bv)
    return np.stack([gx, gy], axis=1), f[:, :2].copy()


# ----------------------------------------------------------------------------
# FP32-inner / FP64-outer iterative refinement
# ----------------------------------------------------------------------------
def pcg32(K32, d32, r32, tol, max_it, floor=0.0):
    """Jacobi PCG in float32 arithmetic from zero, stopping at ||r|| <= max(tol ||r0||, floor)."""
    n = r32.shape[0]
    x = np.zeros(n, dtype=np.float32)
    r = r32.astype(np.float32).copy()
    r0 = math.sqrt(float(np.dot(r, r)))
    if r0 == 0.0:
        return x, 0
    z = (r / d32).astype(np.float32)
    p = z.copy()
    rz = np.float32(np.dot(r, z))
    k = 0
    while k < max_it:
        if math.sqrt(float(np.dot(r, r))) <= max(tol * r0, floor):
            break
        if k > 0:
            rz_new = np.float32(np.dot(r, z))
            beta = np.float32(rz_new / rz)
            rz = rz_new
            p = (z + beta * p).astype(np.float32)
        q = (K32 @ p).astype(np.float32)
        pq = np.float32(np.dot(p, q))
        if not (pq > 0):
            break
        alpha = np.float32(rz / pq)
        x = (x + alpha * p).astype(np.float32)
        r = (r - alpha * q).astype(np.float32)
        z = (r / d32).astype(np.float32)
        k += 1
    return x, k


def mixed_ir(K, d, b, x0=None, tol=1e-8, inner_tol=1e-4, max_sweeps=50, inner_max_it=20000):
    """Iterative refinement: FP64 residual, correction sum and projection; FP32 inner PCG.

    The inner solve of K e = r stops at the relative reduction inner_tol, or
    as soon as its residual (the outer residual after the correction, up to
    FP32 rounding) is below half the outer target tol ||b||: solving further
    would only be thrown away by the next outer test.
    """
    bp = project_mean(b)
    n = bp.shape[0]
    bnorm = math.sqrt(float(np.dot(bp, bp)))
    x = np.zeros(n) if x0 is None else project_mean(x0)
    K32 = K.astype(np.float32)
    d32 = d.astype(np.float32)
    info = dict(iterations=0, outer_sweeps=0, status=NOT_CONVERGED)
    if bnorm == 0.0:
        info.update(x=np.zeros(n), status=OK, rel_res_true=0.0)
        return info
    total = 0
    sweeps = 0
    rel = float("inf")
    while True:
        r = project_mean(bp - K @ x)
        rel = math.sqrt(float(np.dot(r, r))) / bnorm
        if rel <= tol:
            info["status"] = OK
            break
        if sweeps >= max_sweeps:
            break
        dx, its = pcg32(K32, d32, r.astype(np.float32), inner_tol, inner_max_it, floor=0.5 * tol * bnorm)
        total += its
        x = project_mean(x + dx.astype(np.float64))
        sweeps += 1
    info.update(x=x, iterations=total, outer_sweeps=sweeps, rel_res_true=rel)
    return info


# ----------------------------------------------------------------------------
# 8. velocity correction (Eqs. 16-17), lumped P1 mass
# ----------------------------------------------------------------------------
def velocity_correct(xy_f, tri_f, p_f, u_t, v_t, dt_over_rho):
    """u = u~ - (dt/rho) (M_L^-1 int psi_i grad p), the Galerkin form of Eqs. 16-17 with the
    lumped mass M_L,ii = sum_{T ni i} |T| / 3 and int_T psi_i grad p = (|T| / 3) grad p|_T."""
    xy_f = np.asarray(xy_f, dtype=np.float64)
    tri = np.asarray(tri_f, dtype=np.int64)
    area2, _, _ = p1_gradients(xy_f, tri)
    gx, gy = gradient(xy_f, tri, p_f)
    w = np.repeat((0.5 * area2 / 3.0)[:, None], 3, axis=1).ravel()
    n = xy_f.shape[0]
    mass = np.bincount(tri.ravel(), weights=w, minlength=n)
    fx = np.bincount(tri.ravel(), weights=w * np.repeat(gx, 3), minlength=n)
    fy = np.bincount(tri.ravel(), weights=w * np.repeat(gy, 3), minlength=n)
    return np.asarray(u_t) - dt_over_rho * fx / mass, np.asarray(v_t) - dt_over_rho * fy / mass


# ----------------------------------------------------------------------------
# the whole CGP solve on one mesh pair
# ----------------------------------------------------------------------------
class OracleMesh:
    """Coarse mesh, its k nested 4-way splits (Eq. 18) and the assembled coarse operators."""

    def __init__(self, xy_c, tri_c, levels: int = 1):
        self.xy_c = np.asarray(xy_c, dtype=np.float64)
        self.tri_c = np.asarray(tri_c, dtype=np.int32)
        self.n_c = self.xy_c.shape[0]
        self.k = levels
        self.levels = split_levels(self.xy_c, self.tri_c, levels)
        self.xy_f, self.tri_f = self.levels[-1][0], self.levels[-1][1]
        self.edges = self.levels[1][2]              # the coarse edges
        self.parent = self.levels[1][3] if levels == 1 else None
        self.n_f = self.xy_f.shape[0]
        self.K, self.Gx, self.Gy, self.d = assemble(self.xy_c, self.tri_c)
        self._restrict_idx = None

    def restrict(self, q_f):
        if self._restrict_idx is None:
            self._restrict_idx = restrict(self.xy_c, self.xy_f, np.arange(self.n_f))
        return np.asarray(q_f)[self._restrict_idx]

    def prolong(self, q_c):
        """Eq. 20 one level at a time, k times (Sect. 2.3: prolongation only reaches the next nested space)."""
        q = np.asarray(q_c, dtype=np.float64)
        for l in range(self.k):
            xy, tri = self.levels[l][0], self.levels[l][1]
            xy_n, tri_n, _, parent = self.levels[l + 1]
            q = prolong(xy, tri, xy_n, tri_n, parent, q)
        return q

    def solve(self, u_f, v_f, kind=POTENTIAL, B=(0.0, 0.0, 1.0), sigma=1.0, rho_over_dt=20.0,
              tol=1e-8, x0=None, max_it=20000, mixed=False, inner_tol=1e-4, far_dirichlet=False):
        """One CGP solve: restrict, RHS, PCG (or mixed IR), prolong, gradient and force.
        far_dirichlet: phi = 0 on the outer boundary instead of the natural condition there."""
        u_c = self.restrict(u_f)
        v_c = self.restrict(v_f)
        Fx, Fy = source_field(kind, u_c, v_c, B, rho_over_dt)
        b = rhs(self.Gx, self.Gy, Fx, Fy)
        if far_dirichlet:
            fixed = outer_boundary(self.xy_c, self.tri_c)
            Kd, dd = dirichlet_system(self.K, fixed)
            bd = b.copy()
            bd[fixed] = 0.0
            info = pcg(Kd, dd, bd, x0, tol=tol, max_it=max_it, project=False)
        elif mixed:
            info = mixed_ir(self.K, self.d, b, x0, tol=tol, inner_tol=inner_tol)
        else:
            info = pcg(self.K, self.d, b, x0, tol=tol, max_it=max_it)
        phi_f = self.prolong(info["x"])
        grad, force = lorentz(self.xy_f, self.tri_f, phi_f, u_f, v_f, B, sigma)
        out = dict(info)
        out.update(b=b, phi_c=info["x"], phi_f=phi_f, grad=grad)
        if kind == POTENTIAL:
            out["force"] = force
        return out
