"""Planted mistakes in the oracle (CPU): each test replaces one oracle function
by a copy with a plausible mistake and checks that the pins of that function
(the tests of tests/test_oracle_*.py, called directly) catch it.  A pin set
that still passes with the mistake in place would not pin the function."""
import numpy as np
import pytest

import synthgen as sg
from oracle import fem, gmg, indexing, learned, mesh, mlp, nedelec, quadrature, surrogate

import test_oracle_fem as pf
import test_oracle_gmg as pg
import test_oracle_indexing as pi
import test_oracle_learned as pl
import test_oracle_mesh as pm
import test_oracle_mlp as pn
import test_oracle_nedelec as pe
import test_oracle_surrogate as ps


def _caught(*pins):
    """True if at least one of the pins (callables without arguments) fails."""
    for pin in pins:
        try:
            pin()
        except AssertionError:
            return True
    return False


def test_pins_pass_on_the_oracle_as_written():
    assert not _caught(pf.test_p1_element_matrices_closed_forms,
                       lambda: pf.test_kuhn_cube_laplacian_is_h_times_7_point(1, 3),
                       pi.test_tw_worked_example_w3,
                       pg.test_chebyshev_error_polynomial_on_diagonal_matrix,
                       lambda: pl.test_one_hot_network_reads_the_neighbour_in_the_cells_frame(0),
                       lambda: pm.test_bey_equals_lattice_subgroups(2),
                       lambda: pf.test_p2_stiffness_and_mass_invariants(sg.kuhn_cube(1)),
                       pf.test_p2_stiffness_with_linear_k_matches_an_independent_rule,
                       pf.test_p1_divkgrad_is_the_exact_integral_for_linear_k,
                       pf.test_quadrature_exactness,
                       pg.test_chebyshev_order_one_is_weighted_jacobi,
                       pg.test_colour_gauss_seidel_is_the_sequential_sweep,
                       pn.test_gradient_matches_finite_differences,
                       pn.test_single_hidden_unit_closed_form,
                       lambda: pl.test_zero_network_is_weighted_jacobi(0),
                       pe.test_basis_curls_by_finite_differences,
                       lambda: ps.test_surrogate_is_exact_for_polynomial_coefficients(sg.kuhn_cube(1)),
                       pg.test_fmg_coarse_start_is_the_galerkin_projection,
                       pg.test_power_iteration_finds_the_largest_eigenvalue,
                       lambda: pe.test_prolongation_commutes_with_gradient_and_reproduces_rotations(
                           pe.PERM, 2),
                       pe.test_hiptmair_vcycle_is_level_independent_and_needs_the_potential_step,
                       pn.test_bf16_rounding_is_round_to_nearest_even,
                       pn.test_adam_first_step_is_lr_times_sign,
                       pl.test_samples_are_normalised_and_count_every_stride,
                       lambda: pi.test_subgroup_widths_count_every_micro_primitive(3),
                       lambda: pf.test_p1_laplace_symmetric_zero_rowsum_patch(sg.kuhn_cube(1), 2),
                       pe.test_mass_matrix_by_quadrature)


def test_a_missing_volume_factor_in_the_p1_stiffness_is_caught(monkeypatch):
    def wrong(X):
        G, vol = fem.bary_gradients(X)
        return np.einsum("tid,tjd->tij", G, G)              # |T| dropped
    monkeypatch.setattr(fem, "p1_stiffness", wrong)
    assert _caught(pf.test_p1_element_matrices_closed_forms,
                   lambda: pf.test_kuhn_cube_laplacian_is_h_times_7_point(1, 3))


def test_a_gradient_of_the_wrong_vertex_in_the_p1_stiffness_is_caught(monkeypatch):
    def wrong(X):
        G, vol = fem.bary_gradients(X)
        G = G[:, [1, 0, 2, 3]]                               # two vertices swapped
        return vol[:, None, None] * np.einsum("tid,tjd->tij", G, G)
    monkeypatch.setattr(fem, "p1_stiffness", wrong)
    assert _caught(pf.test_p1_element_matrices_closed_forms)


def test_a_wrong_term_in_the_index_function_is_caught(monkeypatch):
    def wrong(w, i, j, k):
        return (indexing.n_tet(w) - indexing.n_tet(w - k) + indexing.n_tri(w - k + 1)
                - indexing.n_tri(w - k - j + 1) + i)         # rows of length w - k - j + 1
    monkeypatch.setattr(indexing, "tw", wrong)
    assert _caught(pi.test_tw_worked_example_w3, lambda: pi.test_tw_closed_form_equals_loop_order_counting(4))


def test_a_wrong_chebyshev_recurrence_is_caught(monkeypatch):
    def wrong(A, D, x, b, lam_max, order=2, lo=0.1, hi=1.1):
        a, c = lo * lam_max, hi * lam_max
        theta, delta = 0.5 * (c + a), 0.5 * (c - a)
        sigma = theta / delta
        rho = 1.0 / sigma
        d = (b - A @ x) / (D * theta)
        x = x + d
        for _ in range(order - 1):
            rho_new = 1.0 / (2.0 * sigma - rho)
            d = rho_new * rho * d + (rho_new / delta) * ((b - A @ x) / D)   # factor 2 dropped
            x = x + d
            rho = rho_new
        return x
    monkeypatch.setattr(gmg, "chebyshev", wrong)
    assert _caught(pg.test_chebyshev_error_polynomial_on_diagonal_matrix)


def test_wrong_prolongation_weights_are_caught(monkeypatch):
    original = gmg.p1_prolongation

    def wrong(fine, coarse):
        P = original(fine, coarse).tocoo()
        v = np.where(P.data == 0.5, 0.25, P.data)            # midpoints from a quarter of each end
        return type(P)((v, (P.row, P.col)), shape=P.shape).tocsr()
    monkeypatch.setattr(gmg, "p1_prolongation", wrong)
    assert _caught(lambda: pg.test_prolongation_reproduces_linear_and_quadratic_functions(
        sg.kuhn_cube(1)))


def test_swapped_feature_directions_in_the_learned_step_are_caught(monkeypatch):
    dirs = learned.DIRS.copy()
    dirs[[7, 8]] = dirs[[8, 7]]                                # (-1,1,0) and (1,-1,0) swapped
    monkeypatch.setattr(learned, "DIRS", dirs)
    assert _caught(lambda: pl.test_one_hot_network_reads_the_neighbour_in_the_cells_frame(0))


def test_a_wrong_inner_diagonal_in_bey_refinement_is_caught(monkeypatch):
    def wrong(t):
        v0, v1, v2, v3 = t[:, 0], t[:, 1], t[:, 2], t[:, 3]
        m01, m02, m03 = (v0 + v1) // 2, (v0 + v2) // 2, (v0 + v3) // 2
        m12, m13, m23 = (v1 + v2) // 2, (v1 + v3) // 2, (v2 + v3) // 2
        # the octahedron split along v01-v23 instead of v02-v13
        kids = [(v0, m01, m02, m03), (m01, v1, m12, m13), (m02, m12, v2, m23),
                (m03, m13, m23, v3), (m01, m23, m02, m03), (m01, m23, m03, m13),
                (m01, m23, m13, m12), (m01, m23, m12, m02)]
        return np.stack([np.stack(k, axis=1) for k in kids], axis=1).reshape(-1, 4, 3)
    monkeypatch.setattr(mesh, "bey_children", wrong)
    assert _caught(lambda: pm.test_bey_equals_lattice_subgroups(1), pm.test_inner_edge_is_v02_v13)


def test_a_lumped_p1_mass_is_caught(monkeypatch):
    def wrong(X):
        _, vol = fem.bary_gradients(X)
        return vol[:, None, None] * (np.eye(4) / 4.0)[None]  # row sums kept, the matrix lumped
    monkeypatch.setattr(fem, "p1_mass", wrong)
    assert _caught(pf.test_p1_element_matrices_closed_forms)


def test_a_wrong_p2_edge_gradient_is_caught(monkeypatch):
    def wrong(lam, G):
        B = np.empty((G.shape[0], 10, 3))
        for i in range(4):
            B[:, i] = (4.0 * lam[i] - 1.0) * G[:, i]
        for e, (i, j) in enumerate(fem.P2_EDGES):
            B[:, 4 + e] = 2.0 * (lam[i] * G[:, j] + lam[j] * G[:, i])   # factor 4 halved
        return B
    monkeypatch.setattr(fem, "p2_basis_gradients", wrong)
    assert _caught(lambda: pf.test_p2_stiffness_and_mass_invariants(sg.kuhn_cube(1)),
                   pf.test_p2_stiffness_with_linear_k_matches_an_independent_rule)


def test_a_div_k_grad_coefficient_taken_at_one_vertex_is_caught(monkeypatch):
    def wrong(X, k_vertex):
        return k_vertex[:, 0][:, None, None] * fem.p1_stiffness(X)   # not the cell mean
    monkeypatch.setattr(fem, "p1_divkgrad", wrong)
    assert _caught(pf.test_p1_divkgrad_is_the_exact_integral_for_linear_k)


def test_jacobi_without_its_weight_is_caught(monkeypatch):
    monkeypatch.setattr(gmg, "jacobi", lambda A, D, x, b, omega: x + (b - A @ x) / D)
    assert _caught(pg.test_chebyshev_order_one_is_weighted_jacobi)


def test_gauss_seidel_with_one_residual_per_sweep_is_caught(monkeypatch):
    def wrong(A, D, x, b, colour):
        r = b - A @ x                                        # not refreshed between colours
        return x + r / D
    monkeypatch.setattr(gmg, "gauss_seidel_colours", wrong)
    assert _caught(pg.test_colour_gauss_seidel_is_the_sequential_sweep)


def test_a_missing_second_relu_in_the_network_is_caught(monkeypatch):
    def wrong(W1, W2, w3, X):
        z1 = X @ W1.T
        h1 = np.maximum(z1, 0.0)
        z2 = h1 @ W2.T
        h2 = z2                                              # second ReLU dropped
        return h2 @ w3, (X, z1, h1, z2, h2)
    monkeypatch.setattr(mlp, "forward", wrong)
    assert _caught(pn.test_gradient_matches_finite_differences,
                   pn.test_single_hidden_unit_closed_form)


def test_a_learned_step_without_the_jacobi_weight_is_caught(monkeypatch):
    original = learned.learned_step

    def wrong(macro, rm, x, r, D, W1, W2, w3, omega, forward=None):
        return original(macro, rm, x, r, D, W1, W2, w3, 1.0, forward)
    monkeypatch.setattr(learned, "learned_step", wrong)
    assert _caught(lambda: pl.test_zero_network_is_weighted_jacobi(0))


def test_a_whitney_function_of_the_opposite_orientation_is_caught(monkeypatch):
    def wrong(lam, G):
        out = np.empty(lam.shape[:-1] + (6, 3))
        for e, (a, b) in enumerate(nedelec.LOCAL_EDGES):
            out[..., e, :] = lam[..., b, None] * G[a] - lam[..., a, None] * G[b]
        return out
    monkeypatch.setattr(nedelec, "whitney", wrong)
    assert _caught(pe.test_basis_curls_by_finite_differences)


def test_a_surrogate_basis_missing_its_top_degree_is_caught(monkeypatch):
    import itertools

    def wrong(degree):
        return [e for e in itertools.product(range(degree + 1), repeat=3) if sum(e) < max(degree, 1)]
    monkeypatch.setattr(surrogate, "exponents", wrong)
    assert _caught(lambda: ps.test_surrogate_is_exact_for_polynomial_coefficients(sg.kuhn_cube(1)))


def test_a_perturbed_quadrature_weight_is_caught(monkeypatch):
    original = quadrature.sym14

    def wrong():
        bary, w = original()
        w = w.copy()
        w[0] += 1e-3
        w[-1] -= 1e-3                                        # total weight kept
        return bary, w
    monkeypatch.setattr(quadrature, "sym14", wrong)
    assert _caught(pf.test_quadrature_exactness)


def test_an_fmg_that_ignores_the_coarser_solution_is_caught(monkeypatch):
    def wrong(H, b, cycles=5, nu1=1, nu2=1, smoother=None, **kw):
        bs = {H.lmax: b}
        for l in range(H.lmax, H.lmin, -1):
            bs[l - 1] = H.P[l].T @ bs[l]
        x = None
        for l in range(H.lmin + 1, H.lmax + 1):
            x = np.zeros_like(bs[l])                          # no prolongated start
            for _ in range(cycles):
                x = gmg.vcycle(H, l, x, bs[l], nu1, nu2, smoother=smoother, **kw)
        return x
    monkeypatch.setattr(gmg, "fmg", wrong)
    assert _caught(pg.test_fmg_coarse_start_is_the_galerkin_projection)


def test_a_power_iteration_without_normalisation_is_caught(monkeypatch):
    def wrong(A, D, v0, iters=20):
        v = v0 / np.linalg.norm(v0)
        lam = 0.0
        for _ in range(iters):
            w = (A @ v) / D
            lam = np.linalg.norm(w)
            v = w                                             # not normalised
        return lam
    monkeypatch.setattr(gmg, "power_lambda_max", wrong)
    assert _caught(pg.test_power_iteration_finds_the_largest_eigenvalue)


def test_a_p2_prolongation_with_wrong_edge_functions_is_caught(monkeypatch):
    original = gmg.p2_prolongation

    def wrong(fine, coarse):
        P = original(fine, coarse).tocoo()
        v = np.where(np.isclose(P.data, 0.75), 0.5, P.data)   # 4 l_i l_j at (3/4, 1/4) off
        return type(P)((v, (P.row, P.col)), shape=P.shape).tocsr()
    monkeypatch.setattr(gmg, "p2_prolongation", wrong)
    assert _caught(lambda: pg.test_prolongation_reproduces_linear_and_quadratic_functions(
        sg.kuhn_cube(1)))


def test_a_nedelec_prolongation_without_the_coarse_orientation_is_caught(monkeypatch):
    import copy
    original = nedelec.nedelec_prolongation

    def wrong(fine, coarse):
        c = copy.copy(coarse)
        c.sign = np.ones_like(coarse.sign)                    # the cells' edge signs dropped
        return original(fine, c)
    monkeypatch.setattr(nedelec, "nedelec_prolongation", wrong)
    assert _caught(lambda: pe.test_prolongation_commutes_with_gradient_and_reproduces_rotations(
        pe.PERM, 2))


def test_a_hiptmair_step_without_its_potential_correction_is_caught(monkeypatch):
    def wrong(lev, x, b, edge_smoother, potential_smoother):
        return edge_smoother(lev.A, lev.D, x, b)              # potential space left out
    monkeypatch.setattr(nedelec, "hiptmair_step", wrong)
    assert _caught(pe.test_hiptmair_vcycle_is_level_independent_and_needs_the_potential_step)


def test_bf16_by_truncation_is_caught(monkeypatch):
    def wrong(a):
        f = np.asarray(a, dtype=np.float32)
        u = f.view(np.uint32)
        return ((u >> 16) << 16).astype(np.uint32).view(np.float32).astype(np.float64)
    monkeypatch.setattr(mlp, "bf16", wrong)
    assert _caught(pn.test_bf16_rounding_is_round_to_nearest_even)


def test_adam_without_bias_correction_is_caught(monkeypatch):
    def wrong(params, grads, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        for p, g, mi, vi in zip(params, grads, m, v):
            mi *= b1
            mi += (1 - b1) * g
            vi *= b2
            vi += (1 - b2) * g * g
            p -= lr * mi / (np.sqrt(vi) + eps)
    monkeypatch.setattr(mlp, "adam_step", wrong)
    assert _caught(pn.test_adam_first_step_is_lr_times_sign)


def test_training_targets_without_the_jacobi_part_are_caught(monkeypatch):
    original = learned.learned_samples

    def wrong(macro, rm, r, D, xstar, x, omega, stride, offset):
        return original(macro, rm, r, D, xstar, x, 0.0, stride, offset)   # target e, not e - omega s
    monkeypatch.setattr(learned, "learned_samples", wrong)
    assert _caught(pl.test_samples_are_normalised_and_count_every_stride)


def test_the_printed_xyz_down_face_width_is_caught(monkeypatch):
    original = indexing.subgroup_widths

    def wrong(level):
        wd = dict(original(level))
        wd[("face", "xyz-down")] = 2 ** level - 2            # Table 1 as printed
        return wd
    monkeypatch.setattr(indexing, "subgroup_widths", wrong)
    assert _caught(lambda: pi.test_subgroup_widths_count_every_micro_primitive(3))


def test_boundary_vertices_missing_from_the_dirichlet_set_are_caught(monkeypatch):
    def wrong(cell_ids, n_vertices):
        f = mesh.faces_of(cell_ids)
        uf, cnt = np.unique(f, axis=0, return_counts=True)
        mask = np.zeros(n_vertices, dtype=bool)
        mask[uf[cnt == 1][:, :2].ravel()] = True             # the third vertex of each face left out
        return mask
    monkeypatch.setattr(mesh, "dirichlet_vertices", wrong)
    assert _caught(lambda: pf.test_p1_laplace_symmetric_zero_rowsum_patch(sg.kuhn_cube(1), 2))


def test_a_nedelec_mass_with_a_dropped_term_is_caught(monkeypatch):
    def wrong(X):
        G, vol = fem.bary_gradients(X)
        GG = np.einsum("tid,tjd->tij", G, G)
        L = (np.ones((4, 4)) + np.eye(4)) / 20.0
        M = np.empty((X.shape[0], 6, 6))
        for e, (a, b) in enumerate(nedelec.LOCAL_EDGES):
            for f, (c, d) in enumerate(nedelec.LOCAL_EDGES):
                M[:, e, f] = (L[a, c] * GG[:, b, d] - L[a, d] * GG[:, b, c]
                              - L[b, c] * GG[:, a, d])             # + L[b, d] GG[a, c] dropped
        return vol[:, None, None] * M
    monkeypatch.setattr(nedelec, "mass_local", wrong)
    assert _caught(pe.test_mass_matrix_by_quadrature)
