"""Planted mistakes in the oracle, on the CPU.

Each mutant below changes one spot of ``oracle/vla_oracle.c`` the way a
plausible slip would: a dropped term or factor, a wrong sign, index or count,
a transposed operand.  The mutant is compiled into a scratch copy of the
oracle package, and the oracle's pin tests (values the paper prints, closed
forms, invariants, brute force, numpy) run against it in a child process;
every mutant must make at least one pin fail.  An unmutated copy run the same
way must pass them all, so that a failure means the planted slip was seen.
Every mutant keeps each array access in bounds.
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "vla_oracle.c")
PINS = [os.path.join(ROOT, "tests", f) for f in
        ("test_oracle_pins.py", "test_oracle_integrals.py", "test_oracle_pages_ext.py")]

pytestmark = pytest.mark.slow

# (name, text in the oracle, planted text)
MUTANTS = [
    # page primitives and the small dense helpers (Sections 2.3, 2.4)
    ("det3_cofactor_sign", "return A(0, 0) * c0 - A(0, 1) * c1 + A(0, 2) * c2;",
     "return A(0, 0) * c0 + A(0, 1) * c1 + A(0, 2) * c2;"),
    ("det2_index", "if (n == 2) return A(0, 0) * A(1, 1) - A(0, 1) * A(1, 0);",
     "if (n == 2) return A(0, 0) * A(1, 1) - A(0, 1) * A(0, 1);"),
    ("inv3_adjugate_not_transposed", "I(c, r) = cof / d;", "I(r, c) = cof / d;"),
    ("inv2_sign", "I(0, 1) = -A(0, 1) / d;", "I(0, 1) = A(0, 1) / d;"),
    ("amtam_first_operand_not_transposed", "s += a[r + i * p] * b[r + j * p];", "s += a[i + r * m] * b[r + j * p];"),
    ("astam_scalar_index", "C[k * m * n + e] = s[k] * A[k * m * n + e];", "C[k * m * n + e] = s[0] * A[k * m * n + e];"),
    ("avtam_page_transposed", "s += v[k * p + r] * A[k * p * n + r + j * p];", "s += v[k * p + r] * A[k * p * n + j + r * n];"),
    ("amt_not_transposed", "C[k * m * n + j + i * n] = A[k * m * n + i + j * m];",
     "C[k * m * n + i + j * m] = A[k * m * n + i + j * m];"),
    ("avtav_operand", "s += a[k * n + r] * b[k * n + r];", "s += a[k * n + r] * a[k * n + r];"),
    ("amsm_single_matrix_transposed", "s += A[k * m * p + i + r * m] * S[r + j * p];",
     "s += A[k * m * p + i + r * m] * S[j + r * n];"),
    ("amsv_page_transposed", "s += A[k * m * n + i + r * m] * sv[r];", "s += A[k * m * n + r + i * n] * sv[r];"),
    ("smamt_single_matrix_transposed", "s += S[i + r * m] * A[k * n * p + j + r * n];",
     "s += S[r + i * p] * A[k * n * p + j + r * n];"),
    ("svamt_page_transposed", "s += sv[r] * A[k * m * n + j + r * m];", "s += sv[r] * A[k * m * n + r + j * n];"),
    ("avtamav_page_transposed", "s += v[k * n + i] * A[k * n * n + i + j * n] * w[k * n + j];",
     "s += v[k * n + i] * A[k * n * n + j + i * n] * w[k * n + j];"),
    # geometry (Sections 3.1, 3.2)
    ("vectors_reversed", "V[d + j * dim] = xj[d] - xl[d];", "V[d + j * dim] = xl[d] - xj[d];"),
    ("volume_factorial", "det_signed[k] = d;\n        vol[k] = fabs(d) / factorial(dim);",
     "det_signed[k] = d;\n        vol[k] = fabs(d) / dim;"),
    ("normals_reference_sign", "(c == dim) ? 1.0 : (r == c ? -1.0 : 0.0);", "(c == dim) ? 1.0 : (r == c ? 1.0 : 0.0);"),
    ("normals_inverse_not_transposed", "s += Vi[q + r * dim] * ref[q + c * dim];", "s += Vi[r + q * dim] * ref[q + c * dim];"),
    # element matrices (Section 3.5)
    ("last_gradient_sign", "glam[r + dim * dim] = -s;", "glam[r + dim * dim] = s;"),
    ("gradients_not_transposed", "glam[r + j * dim] = Vi[j + r * dim];", "glam[r + j * dim] = Vi[r + j * dim];"),
    ("centroid_vertex_count", "xc[d] /= nv;", "xc[d] /= dim;"),
    ("exp_coefficient_argument", "if (kind == 1) return ca * exp(cb * sum);", "if (kind == 1) return ca * exp(cb * r2);"),
    ("p1_stiffness_dropped_coefficient", "Kp[p + q * nlb] = c * vol * s;", "Kp[p + q * nlb] = vol * s;"),
    ("p1_mass_diagonal", "(p == q ? 2.0 : 1.0) / ((dim + 1) * (dim + 2))", "(p == q ? 1.0 : 2.0) / ((dim + 1) * (dim + 2))"),
    ("p1_mass_denominator", "(p == q ? 2.0 : 1.0) / ((dim + 1) * (dim + 2))", "(p == q ? 2.0 : 1.0) / ((dim + 1) * (dim + 1))"),
    ("p2_edge_order_3d", "P2E3[6][2] = {{0, 1}, {1, 2}, {0, 2}, {0, 3}, {1, 3}, {2, 3}};",
     "P2E3[6][2] = {{0, 1}, {0, 2}, {1, 2}, {0, 3}, {1, 3}, {2, 3}};"),
    ("p2_edge_order_2d", "P2E2[3][2] = {{0, 1}, {1, 2}, {0, 2}};", "P2E2[3][2] = {{0, 1}, {0, 2}, {1, 2}};"),
    ("p2_vertex_basis_sign", "out->coef[1] = -1.0;", "out->coef[1] = 1.0;"),
    ("p2_derivative_dropped_exponent", "g->coef[i] = p->coef[t] * p->alpha[t][j];", "g->coef[i] = p->coef[t];"),
    ("monomial_integral_factorial", "return num * vol / factorial(s + dim);", "return num * vol / factorial(s + dim - 1);"),
    ("p2_mass_dropped_coefficient", "sm += P[p].coef[u] * P[q].coef[v] * bary_monomial_integral(dim, al, vol);",
     "sm += P[p].coef[u] * bary_monomial_integral(dim, al, vol);"),
    ("p2_stiffness_gradient_pair", "gg[G[p].j[u] + G[q].j[v] * 4]", "gg[G[p].j[u] + G[p].j[u] * 4]"),
    ("literal_point_coordinates", "x[r] += ip[i * (dim + 1) + j] * coords", "x[r] += ip[j] * coords"),
    ("literal_stiffness_weight", "cK += w[i] * cq[i];", "cK += cq[i];"),
    ("literal_mass_dropped_coefficient", "m += w[i] * cq[i] * ip[i * (dim + 1) + p] * ip[i * (dim + 1) + q];",
     "m += w[i] * ip[i * (dim + 1) + p] * ip[i * (dim + 1) + q];"),
    # sparse assembly (Section 3.5)
    ("csr_duplicates_kept", "if (q > 0 && keys[q] == keys[q - 1]) continue;", "if (q > 0 && keys[q] < keys[q - 1]) continue;"),
    ("scatter_column_index", "csr_find(row_ptr, col_idx, elems[k * nlb + j], elems[k * nlb + i]);",
     "csr_find(row_ptr, col_idx, elems[k * nlb + j], elems[k * nlb + j]);"),
    # boundary facets and facet enumeration (Section 3.2)
    ("boundary_inward", "double sgn = side > 0.0 ? -1.0 : 1.0;", "double sgn = side > 0.0 ? 1.0 : -1.0;"),
    ("boundary_area_half", "meas = 0.5 * sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);",
     "meas = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);"),
    ("boundary_2d_normal_sign", "n[1] = -(x2[0] - x1[0]);", "n[1] = (x2[0] - x1[0]);"),
    ("boundary_cross_product_sign", "n[1] = a[2] * b[0] - a[0] * b[2];", "n[1] = a[0] * b[2] - a[2] * b[0];"),
    ("facet_count_boundary", "if (r - q == 1) ++bnd;", "if (r - q <= 2) ++bnd;"),
    ("facet_list_pairing_two_vertices",
     "if (r[t].v[0] == r[t + 1].v[0] && r[t].v[1] == r[t + 1].v[1] && r[t].v[2] == r[t + 1].v[2]) {",
     "if (r[t].v[0] == r[t + 1].v[0] && r[t].v[1] == r[t + 1].v[1]) {"),
    ("facet_list_partner", "partner[r[t + 1].k * nv + r[t + 1].j] = r[t].k;",
     "partner[r[t + 1].k * nv + r[t + 1].j] = r[t + 1].k;"),
    ("facet_list_vertex_index", "if (i != j) faces[nf * dim + q++] = elems[k * nlb + i];",
     "if (i != j) faces[nf * dim + q++] = elems[k * nlb + j];"),
    # quadrature, GI, load vector, energies (Sections 3.4, 3.5)
    ("rule_segment_offset", "const double d = 0.5 / sqrt(3.0);", "const double d = 0.5 / sqrt(2.0);"),
    ("rule_triangle_degree2_points", "if (gqo == 2) big = 2.0 / 3.0, small = 1.0 / 6.0, wo = 1.0 / 3.0;",
     "if (gqo == 2) big = 0.5, small = 0.25, wo = 1.0 / 3.0;"),
    ("rule_triangle_degree3_weight", "wc = -27.0 / 48.0, wo = 25.0 / 48.0;", "wc = -25.0 / 48.0, wo = 25.0 / 48.0;"),
    ("rule_tet_degree2_root", "big = (5.0 + 3.0 * sqrt(5.0)) / 20.0, small = (5.0 - sqrt(5.0)) / 20.0",
     "big = (5.0 + 3.0 * sqrt(3.0)) / 20.0, small = (5.0 - sqrt(3.0)) / 20.0"),
    ("rule_tet_degree3_centroid_sign", "wc = -0.8, wo = 9.0 / 20.0;", "wc = 0.8, wo = 9.0 / 20.0;"),
    ("quad_points_vertex_index", "coords[(int64_t)cells[k * stride + j] * dim + d];", "coords[(int64_t)cells[k * stride] * dim + d];"),
    ("gi_weight_index", "avg[c] += w[q] * fip[(k * nip + q) * d + c];", "avg[c] += w[0] * fip[(k * nip + q) * d + c];"),
    ("gi_dropped_size", "for (int c = 0; c < d; ++c) out[c] += sizes[k] * avg[c];", "for (int c = 0; c < d; ++c) out[c] += avg[c];"),
    ("gi_flux_normal_index", "dot += avg[c] * normals[k * d + c];", "dot += avg[c] * normals[k * d];"),
    ("rhs_dropped_measure", "b2D[k * nlb + j] = vol[k] * s;", "b2D[k * nlb + j] = s;"),
    ("rhs_point_index", "basis_at(dim, order, j, ip + q * (dim + 1));", "basis_at(dim, order, j, ip);"),
    ("rhs_gather_index", "b[elems[k * nlb + j]] += b2D[k * nlb + j];", "b[elems[k * nlb]] += b2D[k * nlb + j];"),
    ("energy_half", "J[k * 3 + 0] = 0.5 * a;", "J[k * 3 + 0] = a;"),
    ("energy_load_sign", "J[k * 3 + 2] = -f;", "J[k * 3 + 2] = f;"),
    ("energy_mass_operand", "m += uk[i] * M3D[k * nlb * nlb + i + j * nlb] * uk[j];",
     "m += uk[i] * K3D[k * nlb * nlb + i + j * nlb] * uk[j];"),
    # second batch: operands, dropped factors and indices elsewhere in the same functions
    ("amsm_output_transposed", "C[k * m * n + i + j * m] = s;\n            }\n}\n\n/* y_k = A_k s",
     "C[k * m * n + j + i * n] = s;\n            }\n}\n\n/* y_k = A_k s"),
    ("aminv_singular_count", "if (d == 0.0) ++nsing;", "if (d != 0.0) ++nsing;"),
    ("vectors_from_first_vertex", "const double *xl = coords + (int64_t)e[dim] * dim;",
     "const double *xl = coords + (int64_t)e[0] * dim;"),
    ("poly_coefficient_uses_sum", "return ca + cb * r2;\n}", "return ca + cb * sum;\n}"),
    ("exp_coefficient_dropped_factor", "if (kind == 1) return ca * exp(cb * sum);", "if (kind == 1) return exp(cb * sum);"),
    ("centroid_vertex_index", "xc[d] += coords[(int64_t)elems[k * nlb + j] * dim + d];",
     "xc[d] += coords[(int64_t)elems[k * nlb] * dim + d];"),
    ("p2_stiffness_dropped_coefficient", "sk += G[p].coef[u] * G[q].coef[v] * gg[",
     "sk += G[p].coef[u] * gg["),
    ("p2_stiffness_exponent_operand", "al[j] = G[p].alpha[u][j] + G[q].alpha[v][j];",
     "al[j] = G[p].alpha[u][j] + G[p].alpha[u][j];"),
    ("literal_stiffness_dropped_coefficient", "Kp[p + q * nlb] = cK * vol * s;", "Kp[p + q * nlb] = vol * s;"),
    ("assemble_mass_from_stiffness_pages", "rc = orc_csr_scatter(ne, nlb, elems, M3D, row_ptr, col_idx, Mv);",
     "rc = orc_csr_scatter(ne, nlb, elems, K3D, row_ptr, col_idx, Mv);"),
    ("csr_column_from_row_bits", "col_idx[nnz] = (int32_t)(keys[q] & 0xffffffffu);", "col_idx[nnz] = (int32_t)(keys[q] >> 32);"),
    ("boundary_owner_test", "if (hits != dim) continue;", "if (hits < dim - 1) continue;"),
    ("rule_degree1_weight", "w[0] = 1.0;\n        return 1;", "w[0] = 0.5;\n        return 1;"),
    ("gi_flux_dropped_size", "out[0] += sizes[k] * dot;", "out[0] += dot;"),
    ("rhs_value_index", "s += w[q] * fip[k * nip + q] * basis_at", "s += w[q] * fip[k * nip] * basis_at"),
    ("energy_load_node_index", "f += b2D[k * nlb + j] * uk[j];", "f += b2D[k * nlb + j] * uk[0];"),
    ("facet_list_owner_facet", "owner[nf * 2 + 1] = j;", "owner[nf * 2 + 1] = 0;"),
    # third batch: more indices, factors and the literal variant's rule
    ("boundary_2d_length_sqrt", "meas = sqrt(n[0] * n[0] + n[1] * n[1]);", "meas = n[0] * n[0] + n[1] * n[1];"),
    ("boundary_2d_tangent_index", "n[0] = x2[1] - x1[1];", "n[0] = x2[0] - x1[0];"),
    ("energy_stiffness_right_node", "a += uk[i] * K3D[k * nlb * nlb + i + j * nlb] * uk[j];", "a += uk[i] * K3D[k * nlb * nlb + i + j * nlb] * uk[i];"),
    ("inv2_diagonal", "I(1, 1) = A(0, 0) / d;", "I(1, 1) = A(1, 1) / d;"),
    ("p2_vertex_basis_leading", "out->coef[0] = 2.0;", "out->coef[0] = 1.0;"),
    ("p2_derivative_exponent_kept", "g->alpha[i][j] -= 1;", "g->alpha[i][j] -= 0;"),
    ("monomial_integral_dropped_alpha_factorial", "num *= factorial(alpha[j]);", "num *= 1.0;"),
    ("centroid_radius_unsquared", "r2 += xc[d] * xc[d];", "r2 += xc[d];"),
    ("literal_rule_degree", "const int nip = orc_quad_rule(dim, 2, ip, w);", "const int nip = orc_quad_rule(dim, 3, ip, w);"),
    ("literal_point_coefficient_kind", "cq[i] = point_coeff(dim, ckind - 2, ca, cb, x);", "cq[i] = point_coeff(dim, 0, ca, cb, x);"),
    ("point_coeff_radius", "r2 += x[d] * x[d];\n        sum += x[d];\n    }\n    return kind == 1", "r2 += x[d];\n        sum += x[d];\n    }\n    return kind == 1"),
    ("quad_points_weight_index", "s += ip[q * nvert + j] * coords", "s += ip[j] * coords"),
    ("rhs_basis_order", "if (order == 1) return lam[j];", "if (order == 1) return lam[0];"),
    ("gi_component_index", "avg[c] += w[q] * fip[(k * nip + q) * d + c];", "avg[c] += w[q] * fip[(k * nip + q) * d];"),
    ("facet_count_drop_index", "if (j != drop) v[q++] = elems[k * nlb + j];", "if (j != drop) v[q++] = elems[k * nlb + drop];"),
    ("normals_last_reference_column", "(c == dim) ? 1.0 :", "(c == dim) ? -1.0 :"),
    ("volume_signed", "det_signed[k] = d;\n        vol[k] = fabs(d) / factorial(dim);", "det_signed[k] = d;\n        vol[k] = d / factorial(dim);"),
    ("p1_mass_dropped_coefficient", "Mp[p + q * nlb] = c * vol * (p == q", "Mp[p + q * nlb] = vol * (p == q"),
    # fourth batch: cofactor indices, outputs, P2 coefficients, search and facet outputs
    ("det3_minor_index", "double c1 = A(1, 0) * A(2, 2) - A(1, 2) * A(2, 0);", "double c1 = A(1, 0) * A(2, 2) - A(1, 2) * A(2, 1);"),
    ("det3_minor_sign", "double c2 = A(1, 0) * A(2, 1) - A(1, 1) * A(2, 0);", "double c2 = A(1, 1) * A(2, 0) - A(1, 0) * A(2, 1);"),
    ("inv3_row_cycle_swapped", "int r0 = (r + 1) % 3, r1 = (r + 2) % 3;", "int r0 = (r + 2) % 3, r1 = (r + 1) % 3;"),
    ("inv3_column_cycle", "int c0 = (c + 1) % 3, c1 = (c + 2) % 3;", "int c0 = (c + 1) % 3, c1 = (c + 1) % 3;"),
    ("smamt_output_transposed", "C[k * m * n + i + j * m] = s;\n            }\n}\n\n/* y_k = s^T", "C[k * m * n + j + i * n] = s;\n            }\n}\n\n/* y_k = s^T"),
    ("element_pages_volume_factorial", "if (vol) vol[k] = fabs(d) / factorial(dim);", "if (vol) vol[k] = fabs(d);"),
    ("p2_gradient_gram_operand", "s += glam[r + i * dim] * glam[r + j * dim];\n            gg", "s += glam[r + i * dim] * glam[r + i * dim];\n            gg"),
    ("rule_segment_weights", "w[0] = w[1] = 0.5;", "w[0] = w[1] = 1.0;"),
    ("rule_triangle_degree3_points", "else big = 0.6, small = 0.2,", "else big = 0.6, small = 0.25,"),
    ("csr_search_direction", "if (col_idx[mid] < c) lo = mid + 1;", "if (col_idx[mid] > c) lo = mid + 1;"),
    ("facet_list_neighbor_output", "if (neighbor) neighbor[nf] = (int32_t)p;", "if (neighbor) neighbor[nf] = (int32_t)k;"),
    ("rhs_p2_basis_index", "    p2_basis(dim, j, &p);\n    double v = 0.0;", "    p2_basis(dim, 0, &p);\n    double v = 0.0;"),
    ("energy_mass_uses_stiffness_sum", "J[k * 3 + 1] = 0.5 * m;", "J[k * 3 + 1] = 0.5 * a;"),
    ("literal_mass_coefficient_twice", "Mp[p + q * nlb] = vol * m;", "Mp[p + q * nlb] = cK * vol * m;"),
    ("p2_stiffness_dropped_coefficient_c", "Kp[p + q * nlb] = c * sk;", "Kp[p + q * nlb] = sk;"),
    ("p2_mass_dropped_coefficient_c", "Mp[p + q * nlb] = c * sm;", "Mp[p + q * nlb] = sm;"),
    ("avtamav_right_vector_index", "* w[k * n + j];\n        out[k] = s;", "* w[k * n + i];\n        out[k] = s;"),
    ("boundary_opposite_vertex", "if (!in) opp = v;", "if (in) opp = v;"),
    ("simplex_normals_inverse_operand", "        inv_small(dim, V, Vi);\n        double *out", "        inv_small(dim, V, Vi);\n        for (int q = 0; q < dim * dim; ++q) Vi[q] = V[q];\n        double *out"),
    # fifth batch: 2-D rules and facets, P2 basis, gradients and node values
    ("rule_segment_points_equal", "ip[2] = 0.5 - d, ip[3] = 0.5 + d;", "ip[2] = 0.5 + d, ip[3] = 0.5 - d;"),
    ("rule_centroid_not_barycentric", "for (int j = 0; j < nv; ++j) ip[j] = 1.0 / nv;", "for (int j = 0; j < nv; ++j) ip[j] = 1.0 / (nv + 1);"),
    ("p2_vertex_basis_exponent", "out->alpha[1][q] = 1;", "out->alpha[1][q] = 2;"),
    ("p2_edge_basis_node", "out->alpha[0][e[0]] += 1;", "out->alpha[0][e[1]] += 1;"),
    ("basis_value_power_index", "for (int e = 0; e < p.alpha[t][s]; ++e) m *= lam[s];", "for (int e = 0; e < p.alpha[t][s]; ++e) m *= lam[0];"),
    ("boundary_second_node", "*x2 = coords + (int64_t)fn[1] * dim;", "*x2 = coords + (int64_t)fn[2 % dim] * dim;"),
    ("quad_points_dropped_vertex", "for (int j = 0; j < nvert; ++j) s += ip", "for (int j = 0; j < nvert - 1; ++j) s += ip"),
    ("last_gradient_partial_sum", "for (int j = 0; j < dim; ++j) s += glam[r + j * dim];", "for (int j = 0; j < dim - 1; ++j) s += glam[r + j * dim];"),
    ("energy_node_values_index", "for (int j = 0; j < nlb; ++j) uk[j] = u[elems[k * nlb + j]];", "for (int j = 0; j < nlb; ++j) uk[j] = u[elems[k * nlb]];"),
    ("centroid_vertex_argument", "double c = centroid_coeff(dim, dim + 1, nlb,", "double c = centroid_coeff(dim, dim, nlb,"),
]


def _copy(base, name, old, new):
    """Scratch oracle package with one planted change, compiled here so that a
    compile error cannot pass for a caught mutant."""
    d = os.path.join(base, name)
    pkg = os.path.join(d, "oracle")
    os.makedirs(pkg)
    shutil.copy(os.path.join(ROOT, "oracle", "__init__.py"), pkg)
    src = open(SRC).read()
    if old is not None:
        assert src.count(old) == 1, f"{name}: the mutated text must occur exactly once in the oracle"
        src = src.replace(old, new)
    c = os.path.join(pkg, "vla_oracle.c")
    with open(c, "w") as f:
        f.write(src)
    subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", os.path.join(pkg, "liboracle.so"), c, "-lm"],
                   check=True, capture_output=True)
    return d


def _pins(d):
    """Runs the pin tests in a child whose first import path is the scratch
    copy (python -m puts the working directory first)."""
    env = dict(os.environ, PYTHONPATH=ROOT, PYTHONDONTWRITEBYTECODE="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu",
                        "-W", "ignore", *PINS], cwd=d, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-1500:]


def test_mutant_table_is_well_formed():
    names = [m[0] for m in MUTANTS]
    assert len(names) == len(set(names))
    src = open(SRC).read()
    for name, old, new in MUTANTS:
        assert old != new and src.count(old) == 1, name


def test_every_planted_mistake_fails_a_pin(tmp_path):
    base = str(tmp_path)
    control = _copy(base, "control", None, None)
    rc, out = _pins(control)
    assert rc == 0, "the unmutated scratch copy must pass every pin:\n" + out
    workers = max(1, min(8, os.cpu_count() or 1))
    with concurrent.futures.ThreadPoolExecutor(workers) as ex:
        runs = ex.map(lambda m: _pins(_copy(base, *m)), MUTANTS)
        res = dict(zip((m[0] for m in MUTANTS), runs))
    # pytest exit code 1: tests ran and at least one failed
    survivors = {n: out for n, (rc, out) in res.items() if rc != 1}
    assert not survivors, "mutants no pin caught: " + ", ".join(sorted(survivors))
