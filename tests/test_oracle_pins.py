"""Pins of the CPU oracle against facts fixed by the paper and by the mathematics.

None of these compares the oracle with itself: each checks a closed form, an
invariant, a worked example, a textbook identity or a brute-force answer.
The planted-mistake tests at the end mutate a copy of an oracle step and show
that the corresponding pin fails.
"""
import math
import os

import numpy as np
import pytest

from oracle import cgp_oracle as O
from paper_2003_00082_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def tiny_mesh():
    return inputs.ogrid(8, 4)


@pytest.fixture(scope="module")
def c1_mesh():
    xy, tri = inputs.ogrid(64, 32)
    return O.OracleMesh(xy, tri)


# ----------------------------------------------------------------------------
# mesh hierarchy (Sect. 2.3 Eq. 18, Sect. 3)
# ----------------------------------------------------------------------------
def test_paper_mesh_counts_follow_the_split_formula():
    rows = np.loadtxt(os.path.join(GOLDEN, "paper_mesh_counts.txt"), dtype=np.int64)
    by_k = {int(r[0]): (int(r[1]), int(r[2])) for r in rows}
    for k in (1, 2, 3):
        v_c, t_c = by_k[k]
        v_f, t_f = by_k[k - 1]
        assert t_f == 4 * t_c                    # Eq. 18, P = 4^-k M
        assert v_f == v_c + (v_c + t_c)          # one midpoint per edge, E = V + T (one hole)


@pytest.mark.parametrize("nt,nr", [(8, 4), (64, 32), (128, 64)])
def test_split_counts_match_closed_form(nt, nr):
    xy, tri = inputs.ogrid(nt, nr)
    xy_f, tri_f, edges, parent = O.split4(xy, tri)
    s = inputs.ogrid_sizes(nt, nr)
    assert xy.shape[0] == s["n_c"] and tri.shape[0] == s["t_c"]
    assert edges.shape[0] == s["e_c"]
    assert xy_f.shape[0] == s["n_f"] and tri_f.shape[0] == s["t_f"]
    if (nt, nr) == (64, 32):
        assert s["n_f"] == 8320
    # children are CCW, a quarter of the parent's area, and cover its vertices
    a2_c, _, _ = O.p1_gradients(xy, tri)
    a2_f, _, _ = O.p1_gradients(xy_f, tri_f)
    assert np.all(a2_f > 0)
    np.testing.assert_allclose(a2_f, np.repeat(a2_c, 4) / 4, rtol=1e-12)


def test_split_numbering_matches_hand_derived_example():
    path = os.path.join(GOLDEN, "split_two_triangles.txt")
    text = open(path).read().split("[tri_f]")
    xy_exp = np.loadtxt(text[0].split("[xy_f]")[1].splitlines())
    tri_exp = np.loadtxt(text[1].splitlines(), dtype=np.int64)
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    tri = np.array([[0, 1, 2], [0, 2, 3]])
    xy_f, tri_f, edges, parent = O.split4(xy, tri)
    np.testing.assert_array_equal(xy_f, xy_exp)
    np.testing.assert_array_equal(tri_f, tri_exp)
    np.testing.assert_array_equal(parent, [0, 0, 0, 0, 1, 1, 1, 1])


# ----------------------------------------------------------------------------
# assembly (P1 Galerkin, Sect. 2.3)
# ----------------------------------------------------------------------------
def cotangent_stiffness(xy, tri):
    """Textbook cotangent formula: K_ij = -1/2 sum over triangles of cot(angle opposite ij)."""
    n = xy.shape[0]
    K = np.zeros((n, n))
    for t in tri:
        for m in range(3):
            i, j, o = t[m], t[(m + 1) % 3], t[(m + 2) % 3]
            e1 = xy[i] - xy[o]
            e2 = xy[j] - xy[o]
            ang = math.acos(np.dot(e1, e2) / (np.linalg.norm(e1) * np.linalg.norm(e2)))
            w = 0.5 / math.tan(ang)
            K[i, j] -= w
            K[j, i] -= w
            K[i, i] += w
            K[j, j] += w
    return K


def check_stiffness(assemble_fn, xy, tri):
    K, Gx, Gy, d = assemble_fn(xy, tri)
    Kd = K.toarray()
    Kc = cotangent_stiffness(xy, tri)
    return np.max(np.abs(Kd - Kc)) <= 1e-10 * np.max(np.abs(Kc))


def test_stiffness_equals_cotangent_formula():
    xy, tri = tiny_mesh()
    assert check_stiffness(O.assemble, xy, tri)


def test_stiffness_invariants(c1_mesh):
    K = c1_mesh.K
    Kd = K.toarray()
    scale = np.max(np.abs(Kd))
    assert np.max(np.abs(Kd - Kd.T)) <= 1e-14 * scale              # symmetric
    assert np.max(np.abs(Kd.sum(axis=1))) <= 1e-13 * scale         # constants in the null space
    np.testing.assert_array_equal(c1_mesh.d, np.diag(Kd))
    # pattern: node adjacency plus the diagonal, nnz = n + 2E
    s = inputs.ogrid_sizes(64, 32)
    assert K.nnz == s["nnz"]


def test_stiffness_psd_with_one_dimensional_null_space():
    xy, tri = tiny_mesh()
    K, _, _, _ = O.assemble(xy, tri)
    w = np.linalg.eigvalsh(K.toarray())
    assert w[0] > -1e-12 * w[-1]
    assert abs(w[0]) < 1e-12 * w[-1]
    assert w[1] > 1e-6 * w[-1]                                     # rank n - 1


def interior_nodes(n_theta, n_r):
    return np.arange(n_theta, n_theta * n_r)                       # rings 1 .. n_r-1


def check_divergence_operators(assemble_fn, xy, tri, interior):
    """For interior i: int x d_x psi_i = -int psi_i = -|patch|/3, int y d_x psi_i = 0 (parts)."""
    K, Gx, Gy, d = assemble_fn(xy, tri)
    area2, _, _ = O.p1_gradients(xy, tri)
    patch = np.zeros(xy.shape[0])
    np.add.at(patch, tri.ravel(), np.repeat(area2 / 2.0, 3))
    x, y = xy[:, 0], xy[:, 1]
    want = -patch / 3.0
    tol = 1e-12 * np.max(np.abs(want))
    ok = np.max(np.abs((Gx @ x - want)[interior])) <= tol
    ok &= np.max(np.abs((Gy @ y - want)[interior])) <= tol
    ok &= np.max(np.abs((Gx @ y)[interior])) <= tol
    ok &= np.max(np.abs((Gy @ x)[interior])) <= tol
    # columns sum to zero: sum_i psi_i = 1 has zero gradient, so sum_i b_i = 0
    ok &= np.max(np.abs(np.asarray(Gx.sum(axis=0)))) <= 1e-13
    ok &= np.max(np.abs(np.asarray(Gy.sum(axis=0)))) <= 1e-13
    return bool(ok)


def test_divergence_operators_integration_by_parts():
    xy, tri = inputs.ogrid(16, 8)
    assert check_divergence_operators(O.assemble, xy, tri, interior_nodes(16, 8))


def test_patch_test_linear_potential_is_exact(c1_mesh):
    """F = grad(c0 + c1 x + c2 y) is reproduced exactly, boundary rows included (natural BC)."""
    xy = c1_mesh.xy_c
    phi = 0.3 + 1.7 * xy[:, 0] - 0.9 * xy[:, 1]
    b = O.rhs(c1_mesh.Gx, c1_mesh.Gy, np.full(c1_mesh.n_c, 1.7), np.full(c1_mesh.n_c, -0.9))
    np.testing.assert_allclose(c1_mesh.K @ phi, b, atol=1e-12 * np.max(np.abs(b)))
    out = O.pcg(c1_mesh.K, c1_mesh.d, b, tol=1e-14)
    ref = phi - phi.mean()
    assert np.linalg.norm(out["x"] - ref) <= 1e-10 * np.linalg.norm(ref)


def manufactured(nt):
    xy, tri = inputs.ogrid(nt, nt // 2)
    m = O.OracleMesh(xy, tri)
    x, y = m.xy_c[:, 0], m.xy_c[:, 1]
    e = np.exp(y / 15.0)
    phi = x * x - y * y + np.sin(x) * e                              # r^2 cos 2theta + sin(x) e^(y/15)
    Fx = 2 * x + np.cos(x) * e
    Fy = -2 * y + np.sin(x) * e / 15.0
    b = O.rhs(m.Gx, m.Gy, Fx, Fy)
    out = O.pcg(m.K, m.d, b, tol=1e-13)
    ref = phi - phi.mean()
    return np.sqrt(np.mean((out["x"] - ref) ** 2))


def test_manufactured_solution_converges_at_second_order():
    errs = [manufactured(nt) for nt in (16, 32, 64, 128)]
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    assert rates[-1] >= 1.8, rates
    assert rates[-2] >= 1.6, rates


def potential_flow_error(nt):
    xy, tri = inputs.ogrid(nt, nt // 2)
    m = O.OracleMesh(xy, tri)
    u, v = inputs.potential_flow(m.xy_f)
    out = m.solve(u, v, O.POTENTIAL, B=(0.0, 0.0, 1.0), sigma=1.0, tol=1e-13)
    x, y = m.xy_c[:, 0], m.xy_c[:, 1]
    exact = -y * (1.0 - 0.25 / (x * x + y * y))                     # phi = -B_z U y (1 - a^2/r^2)
    exact -= exact.mean()
    return np.sqrt(np.mean((out["phi_c"] - exact) ** 2)), out


def test_potential_flow_closed_form():
    errs = []
    for nt in (16, 32, 64):
        e, out = potential_flow_error(nt)
        errs.append(e)
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert rates[-1] >= 1.8, rates


def test_uniform_flow_gives_exact_potential_and_zero_current(c1_mesh):
    m = c1_mesh
    u = np.ones(m.n_f)
    v = np.zeros(m.n_f)
    out = m.solve(u, v, O.POTENTIAL, B=(0.0, 0.0, 1.0), sigma=2.0, tol=1e-14)
    y = m.xy_c[:, 1]
    ref = -(y - y.mean())                                           # phi = -B_z U y
    assert np.linalg.norm(out["phi_c"] - ref) <= 1e-10 * np.linalg.norm(ref)
    assert np.max(np.abs(out["force"])) <= 1e-8                     # j = 0


def test_dense_direct_matches_pcg():
    for nt in (8, 64):
        xy, tri = inputs.ogrid(nt, nt // 2)
        m = O.OracleMesh(xy, tri)
        u, v = inputs.velocity(m.xy_f, 3, 0, vortices=True, noise_std=1e-3)
        Fx, Fy = O.source_field(O.POTENTIAL, m.restrict(u), m.restrict(v), (0.0, 1.0, 1.0))
        b = O.rhs(m.Gx, m.Gy, Fx, Fy)
        xd = O.dense_solve(m.K, b)
        out = O.pcg(m.K, m.d, b, tol=1e-13)
        assert out["status"] == O.OK
        assert np.linalg.norm(out["x"] - xd) <= 1e-10 * np.linalg.norm(xd)
        assert abs(out["x"].mean()) <= 1e-13 * np.max(np.abs(xd))


def test_rhs_is_compatible(c1_mesh):
    m = c1_mesh
    u, v = inputs.velocity(m.xy_f, 5, 2, vortices=True, noise_std=1e-3)
    for kind in (O.POTENTIAL, O.PRESSURE):
        Fx, Fy = O.source_field(kind, m.restrict(u), m.restrict(v), (0.3, 0.1, 1.0), 20.0)
        b = O.rhs(m.Gx, m.Gy, Fx, Fy)
        assert abs(b.sum()) <= 1e-12 * np.sum(np.abs(b))


def test_pressure_rhs_of_a_uniform_field_is_boundary_flux_free(c1_mesh):
    """div of a constant field is zero: the solve returns phi = (rho/dt) U . x up to a constant."""
    m = c1_mesh
    u = np.full(m.n_f, 0.7)
    v = np.full(m.n_f, -0.2)
    out = m.solve(u, v, O.PRESSURE, rho_over_dt=20.0, tol=1e-14)
    x, y = m.xy_c[:, 0], m.xy_c[:, 1]
    ref = 20.0 * (0.7 * x - 0.2 * y)
    ref -= ref.mean()
    assert np.linalg.norm(out["phi_c"] - ref) <= 1e-10 * np.linalg.norm(ref)


# ----------------------------------------------------------------------------
# PCG special cases (Saad Alg. 9.1)
# ----------------------------------------------------------------------------
def test_pcg_zero_rhs_takes_no_iterations(c1_mesh):
    out = O.pcg(c1_mesh.K, c1_mesh.d, np.zeros(c1_mesh.n_c), tol=1e-8)
    assert out["iterations"] == 0 and out["status"] == O.OK
    assert np.all(out["x"] == 0)


def test_pcg_constant_rhs_projects_to_zero(c1_mesh):
    out = O.pcg(c1_mesh.K, c1_mesh.d, np.full(c1_mesh.n_c, 3.0), tol=1e-8)
    assert out["iterations"] == 0 and np.all(out["x"] == 0)


def test_pcg_max_it_and_nonfinite(c1_mesh):
    b = O.rhs(c1_mesh.Gx, c1_mesh.Gy, c1_mesh.xy_c[:, 1] ** 2, c1_mesh.xy_c[:, 0])
    out = O.pcg(c1_mesh.K, c1_mesh.d, b, tol=1e-12, max_it=5)
    assert out["status"] == O.NOT_CONVERGED and out["iterations"] == 5
    bn = b.copy()
    bn[7] = np.nan
    assert O.pcg(c1_mesh.K, c1_mesh.d, bn)["status"] == O.NONFINITE


def test_pcg_breakdown_on_indefinite_matrix():
    import scipy.sparse as sp
    A = sp.csr_matrix(np.diag([1.0, -1.0, 2.0]))
    out = O.pcg(A, np.array([1.0, 1.0, 1.0]), np.array([1.0, 1.0, 1.0]), project=False)
    assert out["status"] == O.BREAKDOWN


def test_pcg_terminates_in_n_steps_on_small_spd():
    """In exact arithmetic CG ends in at most n steps; FP64 on a well-conditioned 6x6 matches solve()."""
    import scipy.sparse as sp
    rng = np.random.default_rng(3)
    M = rng.standard_normal((6, 6))
    A = M @ M.T + 6 * np.eye(6)
    b = rng.standard_normal(6)
    out = O.pcg(sp.csr_matrix(A), np.diag(A).copy(), b, tol=1e-13, project=False)
    assert out["iterations"] <= 8
    np.testing.assert_allclose(out["x"], np.linalg.solve(A, b), rtol=1e-11)


# ----------------------------------------------------------------------------
# mapping operators (Eqs. 19, 20)
# ----------------------------------------------------------------------------
def test_injection_picks_coincident_nodes(c1_mesh):
    m = c1_mesh
    np.testing.assert_array_equal(m.restrict(m.xy_f[:, 0]), m.xy_c[:, 0])
    np.testing.assert_array_equal(m.restrict(m.xy_f[:, 1]), m.xy_c[:, 1])


def check_prolong_linear(prolong_fn, m):
    q = 0.25 - 1.5 * m.xy_c[:, 0] + 0.75 * m.xy_c[:, 1]
    qf = prolong_fn(m.xy_c, m.tri_c, m.xy_f, m.tri_f, m.parent, q)
    ref = 0.25 - 1.5 * m.xy_f[:, 0] + 0.75 * m.xy_f[:, 1]
    return np.max(np.abs(qf - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_prolongation_exact_on_linear_fields(c1_mesh):
    assert check_prolong_linear(O.prolong, c1_mesh)


def test_prolongation_at_midpoints_is_the_edge_average(c1_mesh):
    m = c1_mesh
    rng = np.random.default_rng(1)
    q = rng.standard_normal(m.n_c)
    qf = m.prolong(q)
    np.testing.assert_allclose(qf[: m.n_c], q, rtol=0, atol=1e-14 * np.max(np.abs(q)) * 10)
    avg = 0.5 * (q[m.edges[:, 0]] + q[m.edges[:, 1]])
    np.testing.assert_allclose(qf[m.n_c:], avg, atol=1e-14 * np.max(np.abs(q)) * 10)


def test_children_gradient_equals_parent_gradient(c1_mesh):
    m = c1_mesh
    rng = np.random.default_rng(2)
    q = rng.standard_normal(m.n_c)
    gx_c, gy_c = O.gradient(m.xy_c, m.tri_c, q)
    gx_f, gy_f = O.gradient(m.xy_f, m.tri_f, m.prolong(q))
    scale = np.max(np.abs(gx_c)) + np.max(np.abs(gy_c))
    assert np.max(np.abs(gx_f - np.repeat(gx_c, 4))) <= 1e-9 * scale
    assert np.max(np.abs(gy_f - np.repeat(gy_c, 4))) <= 1e-9 * scale


# ----------------------------------------------------------------------------
# Ohm's law and the Lorentz force (Eqs. 4, 7, 13-14)
# ----------------------------------------------------------------------------
def one_triangle_field(gx, gy, ux, uy):
    xy = np.array([[0.0, 0.0], [2.0, 0.0], [0.0, 1.0]])
    tri = np.array([[0, 1, 2]], dtype=np.int32)
    phi = gx * xy[:, 0] + gy * xy[:, 1] - 4.0
    return xy, tri, phi, np.full(3, ux), np.full(3, uy)


def check_lorentz_examples(lorentz_fn):
    rows = np.loadtxt(os.path.join(GOLDEN, "lorentz_worked_example.txt"))
    ok = True
    for s, ux, uy, gx, gy, bx, by, bz, fx, fy, jx, jy in rows:
        xy, tri, phi, u, v = one_triangle_field(gx, gy, ux, uy)
        g, f = lorentz_fn(xy, tri, phi, u, v, (bx, by, bz), s)
        ok &= np.allclose(g[0], [gx, gy], atol=1e-14)
        ok &= np.allclose(f[0], [fx, fy], atol=1e-13)
    return bool(ok)


def test_lorentz_worked_examples():
    assert check_lorentz_examples(O.lorentz)


def test_lorentz_with_axial_field_reduces_to_momentum_source():
    """B = B_o k: f = sigma B_o (-phi_y - B_o u, phi_x - B_o v), the RHS of Eqs. 13-14."""
    rng = np.random.default_rng(5)
    for _ in range(5):
        gx, gy, ux, uy, bo, s = rng.standard_normal(6)
        xy, tri, phi, u, v = one_triangle_field(gx, gy, ux, uy)
        _, f = O.lorentz(xy, tri, phi, u, v, (0.0, 0.0, bo), s)
        np.testing.assert_allclose(f[0], [s * bo * (-gy - bo * ux), s * bo * (gx - bo * uy)],
                                   rtol=1e-12, atol=1e-13)


def test_in_plane_field_is_the_degenerate_case(c1_mesh):
    """B in the x-y plane: div(u x B) = 0, so phi = 0 and f = sigma(-j_z B_y, j_z B_x), j_z = u B_y - v B_x."""
    m = c1_mesh
    u, v = inputs.velocity(m.xy_f, 0, 0, vortices=False, noise_std=1e-3)
    out = m.solve(u, v, O.POTENTIAL, B=(0.0, 1.0, 0.0), sigma=1.5, tol=1e-10)
    assert out["iterations"] == 0 and np.all(out["phi_c"] == 0)
    t = m.tri_f.astype(np.int64)
    ub, vb = u[t].mean(axis=1), v[t].mean(axis=1)
    jz = ub * 1.0 - vb * 0.0
    np.testing.assert_allclose(out["force"][:, 0], 1.5 * (-jz * 1.0), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(out["force"][:, 1], 0.0, atol=1e-15)


# ----------------------------------------------------------------------------
# mixed precision refinement
# ----------------------------------------------------------------------------
def test_mixed_precision_reaches_fp64_solution(c1_mesh):
    m = c1_mesh
    u, v = inputs.velocity(m.xy_f, 10, 0, vortices=True, noise_std=1e-3)
    Fx, Fy = O.source_field(O.POTENTIAL, m.restrict(u), m.restrict(v), (0.0, 0.0, 1.0))
    b = O.rhs(m.Gx, m.Gy, Fx, Fy)
    ref = O.dense_solve(m.K, b)
    out = O.mixed_ir(m.K, m.d, b, tol=1e-8, inner_tol=1e-4)
    assert out["status"] == O.OK
    assert out["outer_sweeps"] <= 4
    assert out["rel_res_true"] <= 1e-8
    fp64 = O.pcg(m.K, m.d, b, tol=1e-8)
    e_mixed = np.linalg.norm(out["x"] - ref) / np.linalg.norm(ref)
    e_fp64 = np.linalg.norm(fp64["x"] - ref) / np.linalg.norm(ref)
    # both are stopped at the same residual: their errors are of the same order
    assert e_mixed <= max(10 * e_fp64, 1e-7)


# ----------------------------------------------------------------------------
# planted mistakes: each pin above must catch a plausible error
# ----------------------------------------------------------------------------
def test_planted_mistakes_are_caught():
    xy, tri = inputs.ogrid(16, 8)

    def assemble_gy_sign(xy_, tri_):
        K, Gx, Gy, d = O.assemble(xy_, tri_)
        return K, Gx, -Gy, d

    def assemble_gx_transposed(xy_, tri_):
        K, Gx, Gy, d = O.assemble(xy_, tri_)
        return K, Gx.T.tocsr(), Gy, d

    def assemble_area_dropped(xy_, tri_):
        K, Gx, Gy, d = O.assemble(xy_, tri_)
        return K * 2.0, Gx, Gy, d

    interior = interior_nodes(16, 8)
    assert check_divergence_operators(O.assemble, xy, tri, interior)
    assert not check_divergence_operators(assemble_gy_sign, xy, tri, interior)
    assert not check_divergence_operators(assemble_gx_transposed, xy, tri, interior)
    xt, tt = tiny_mesh()
    assert not check_stiffness(assemble_area_dropped, xt, tt)

    def lorentz_no_uxb(xy_, tri_, phi, u, v, B, s):
        return O.lorentz(xy_, tri_, phi, 0 * u, 0 * v, B, s)

    def lorentz_wrong_sign(xy_, tri_, phi, u, v, B, s):
        g, f = O.lorentz(xy_, tri_, -phi, u, v, B, s)
        return -g, f

    assert not check_lorentz_examples(lorentz_no_uxb)
    assert not check_lorentz_examples(lorentz_wrong_sign)

    m = O.OracleMesh(xy, tri)

    def prolong_wrong_vertex(xy_c, tri_c, xy_f, tri_f, parent, q):
        qf = O.prolong(xy_c, tri_c, xy_f, tri_f, parent, q)
        n_c = xy_c.shape[0]
        e = m.edges
        qf[n_c:] = 0.5 * (q[e[:, 0]] + q[e[:, 0]])
        return qf

    assert not check_prolong_linear(prolong_wrong_vertex, m)


# ----------------------------------------------------------------------------
# nested coarsening levels k = 2, 3 (Sect. 2.3, Eq. 18; prolongation one level at a time)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("k", [2, 3])
def test_nested_levels_counts_prefix_and_areas(k):
    nt, nr = 12, 5
    xy, tri = inputs.ogrid(nt, nr)
    levels = O.split_levels(xy, tri, k)
    for l in range(k):
        xy_l, tri_l = levels[l][0], levels[l][1]
        xy_n, tri_n = levels[l + 1][0], levels[l + 1][1]
        # Eq. 18 per level, and the annulus count E = V + T the paper's four meshes obey (golden fixture)
        assert tri_n.shape[0] == 4 * tri_l.shape[0]
        assert xy_n.shape[0] == xy_l.shape[0] + (xy_l.shape[0] + tri_l.shape[0])
        np.testing.assert_array_equal(xy_n[: xy_l.shape[0]], xy_l)     # injection is a prefix at every level
    # level k of the n_theta x n_r O-grid has the node count of the 2^k n_theta x 2^k n_r O-grid
    assert levels[k][0].shape[0] == (2 ** k * nt) * (2 ** k * nr + 1)
    # the 4^k consecutive fine triangles from 4^k T tile coarse triangle T in equal, counter-clockwise parts
    a_c, _, _ = O.p1_gradients(levels[0][0], levels[0][1].astype(np.int64))
    a_f, _, _ = O.p1_gradients(levels[k][0], levels[k][1].astype(np.int64))
    assert np.all(a_f > 0)
    np.testing.assert_allclose(a_f.reshape(-1, 4 ** k), np.repeat(a_c[:, None], 4 ** k, axis=1) / 4 ** k,
                               rtol=1e-12)


@pytest.mark.parametrize("k", [2, 3])
def test_nested_prolongation_is_the_coarse_p1_interpolant(k):
    xy, tri = inputs.ogrid(10, 4)
    om = O.OracleMesh(xy, tri, levels=k)
    # exact on linear fields
    lin = lambda p: 0.3 + 1.7 * p[:, 0] - 0.4 * p[:, 1]  # noqa: E731
    np.testing.assert_allclose(om.prolong(lin(om.xy_c)), lin(om.xy_f), rtol=0, atol=1e-12)
    # k one-level prolongations equal Eq. 20 evaluated directly in the coarse triangle of each fine node
    rng = np.random.default_rng(5)
    q = rng.standard_normal(om.n_c)
    qf = om.prolong(q)
    parent_c = np.arange(om.tri_f.shape[0]) // 4 ** k
    direct = O.prolong(om.xy_c, om.tri_c, om.xy_f, om.tri_f, parent_c, q)
    np.testing.assert_allclose(qf, direct, rtol=0, atol=1e-12 * np.max(np.abs(q)))
    # so the fine gradients are the coarse triangle's gradient on all of its 4^k descendants
    gx_c, gy_c = O.gradient(om.xy_c, om.tri_c, q)
    gx_f, gy_f = O.gradient(om.xy_f, om.tri_f, qf)
    scale = np.max(np.abs(np.concatenate([gx_c, gy_c])))
    np.testing.assert_allclose(gx_f, np.repeat(gx_c, 4 ** k), rtol=0, atol=1e-10 * scale)
    np.testing.assert_allclose(gy_f, np.repeat(gy_c, 4 ** k), rtol=0, atol=1e-10 * scale)


# ----------------------------------------------------------------------------
# velocity correction (Eqs. 16-17) with the lumped P1 mass
# ----------------------------------------------------------------------------
def regular_grid(n):
    """Unit square, n x n cells, every cell cut by its rising diagonal (counter-clockwise)."""
    g = np.linspace(0.0, 1.0, n + 1)
    X, Y = np.meshgrid(g, g, indexing="xy")
    xy = np.stack([X.ravel(), Y.ravel()], axis=1)
    tri = []
    for j in range(n):
        for i in range(n):
            a, b, c, d = j * (n + 1) + i, j * (n + 1) + i + 1, (j + 1) * (n + 1) + i + 1, (j + 1) * (n + 1) + i
            tri += [[a, b, c], [a, c, d]]
    return xy, np.array(tri, dtype=np.int32)


def test_velocity_correction_is_exact_for_a_linear_pressure():
    xy, tri = inputs.ogrid(9, 4)
    xy_f, tri_f, _, _ = O.split4(xy, tri)
    rng = np.random.default_rng(8)
    ut, vt = rng.standard_normal(xy_f.shape[0]), rng.standard_normal(xy_f.shape[0])
    p = 2.0 - 0.7 * xy_f[:, 0] + 1.3 * xy_f[:, 1]
    u, v = O.velocity_correct(xy_f, tri_f, p, ut, vt, 0.05)
    np.testing.assert_allclose(u, ut - 0.05 * (-0.7), rtol=0, atol=1e-12)
    np.testing.assert_allclose(v, vt - 0.05 * 1.3, rtol=0, atol=1e-12)


def test_velocity_correction_recovers_quadratic_gradients_on_symmetric_patches():
    # the area-weighted mean of P1 gradients over a point-symmetric patch is exact for quadratics
    xy, tri = regular_grid(6)
    x, y = xy[:, 0], xy[:, 1]
    p = 0.5 * x * x - 1.2 * x * y + 0.8 * y * y
    u, v = O.velocity_correct(xy, tri, p, np.zeros_like(x), np.zeros_like(x), 1.0)
    interior = (x > 1e-9) & (x < 1 - 1e-9) & (y > 1e-9) & (y < 1 - 1e-9)
    np.testing.assert_allclose(-u[interior], (x - 1.2 * y)[interior], rtol=0, atol=1e-12)
    np.testing.assert_allclose(-v[interior], (-1.2 * x + 1.6 * y)[interior], rtol=0, atol=1e-12)
    # the check is not vacuous: on the one-sided boundary patches the recovery is not exact
    assert np.max(np.abs(-u[~interior] - (x - 1.2 * y)[~interior])) > 1e-3


def test_velocity_correction_integrates_to_the_boundary_integral():
    # sum_i M_L,ii (u~_i - u_i) / c = int grad p_h dx = closed integral of p_h n ds (Gauss), on an annulus
    xy, tri = inputs.ogrid(11, 5)
    xy_f, tri_f, _, _ = O.split4(xy, tri)
    rng = np.random.default_rng(4)
    p = rng.standard_normal(xy_f.shape[0])
    c = 0.05
    u, v = O.velocity_correct(xy_f, tri_f, p, np.zeros(xy_f.shape[0]), np.zeros(xy_f.shape[0]), c)
    area2, _, _ = O.p1_gradients(xy_f, tri_f.astype(np.int64))
    mass = np.bincount(tri_f.ravel(), weights=np.repeat(area2 / 6.0, 3), minlength=xy_f.shape[0])
    lhs = np.array([np.sum(mass * -u), np.sum(mass * -v)]) / c
    # boundary edges: sides used by one triangle only, oriented as in their (counter-clockwise) triangle
    sides = np.concatenate([tri_f[:, [0, 1]], tri_f[:, [1, 2]], tri_f[:, [2, 0]]])
    key = np.minimum(sides[:, 0], sides[:, 1]) * xy_f.shape[0] + np.maximum(sides[:, 0], sides[:, 1])
    uniq, cnt = np.unique(key, return_counts=True)
    bnd = sides[np.isin(key, uniq[cnt == 1])]
    a, b = bnd[:, 0], bnd[:, 1]
    pm = 0.5 * (p[a] + p[b])
    rhs = np.array([np.sum(pm * (xy_f[b, 1] - xy_f[a, 1])), np.sum(-pm * (xy_f[b, 0] - xy_f[a, 0]))])
    np.testing.assert_allclose(lhs, rhs, rtol=1e-10, atol=1e-10 * np.sum(np.abs(pm)))


# ----------------------------------------------------------------------------
# far-field Dirichlet variant: phi = 0 on the outer boundary (reading of "the electric field vanishes far away")
# ----------------------------------------------------------------------------
def test_outer_boundary_is_the_far_ring():
    nt, nr = 10, 4
    xy, tri = inputs.ogrid(nt, nr)
    np.testing.assert_array_equal(O.outer_boundary(xy, tri), np.arange(nr * nt, (nr + 1) * nt))
    # a mesh without a hole: its whole boundary
    sq = (np.array([[2.0, 1.0], [3.0, 1.0], [3.0, 2.0], [2.0, 2.0], [2.5, 1.5]]),
          np.array([[0, 1, 4], [1, 2, 4], [2, 3, 4], [3, 0, 4]]))
    np.testing.assert_array_equal(O.outer_boundary(*sq), [0, 1, 2, 3])


def test_far_field_dirichlet_potential_converges_to_its_closed_form():
    # potential flow, B = k: Laplace equation, d_r phi = -2 U sin(theta) on the cylinder (natural
    # condition j.n = 0), phi = 0 at r = R: phi = alpha (r - R^2 / r) sin(theta),
    # alpha = -2 U a^2 / (a^2 + R^2)
    a, R, U = inputs.R_IN, inputs.R_OUT, 1.0
    alpha = -2.0 * U * a * a / (a * a + R * R)
    errs = []
    for nt, nr in ((32, 16), (64, 32)):
        xy, tri = inputs.ogrid(nt, nr)
        om = O.OracleMesh(xy, tri)
        u, v = inputs.potential_flow(om.xy_f)
        out = om.solve(u, v, O.POTENTIAL, B=(0.0, 0.0, 1.0), tol=1e-13, far_dirichlet=True)
        r = np.hypot(xy[:, 0], xy[:, 1])
        exact = alpha * (r - R * R / r) * (xy[:, 1] / r)
        errs.append(np.linalg.norm(out["phi_c"] - exact) / np.linalg.norm(exact))
        assert np.all(out["phi_c"][nr * nt:] == 0.0)
    assert errs[1] < 0.05 and errs[0] / errs[1] > 3.0, errs     # second-order convergence
