/*
 * vla_oracle.c -- plain, slow, obviously-correct FP64 reference of the
 * page-wise linear algebra and P1/P2 finite-element assembly of
 * "On a vectorized basic linear algebra package for prototyping codes in
 * MATLAB" (arXiv:2404.16039).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may link, load or
 * call this file: only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or constant
 * generator with the CUDA implementation.
 *
 * Style: explicit loops, element order ascending, one accumulation per
 * definition, FP64 throughout.  No blocking, fusion or reordering.
 *
 * Data layout (the paper's arrays, Section 2.4 and Section 3.1):
 *   page arrays   n x m x N, column-major per page: entry (r,c) of page k at
 *                 k*n*m + r + c*n.
 *   coords        dim x nn column-major: coordinate d of node i at i*dim + d.
 *   elems         nlb x ne column-major, 0-based: local node j of element k
 *                 at k*nlb + j.
 *   element pages nlb x nlb x ne, column-major per page.
 *   CSR           row_ptr[nn+1], col_idx[nnz] (ascending within a row),
 *                 values[nnz].
 *
 * Parity status: every function here is pinned by a test against values the
 * paper prints, closed forms, invariants or brute force (see the tests).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* small dense helpers (column-major)                                        */
/* ------------------------------------------------------------------------ */

/* determinant by cofactor expansion along the first row (page-wise
 * determinants, Section 2.3); n in {1,2,3}. */
static double det_small(int n, const double *a /* n x n col-major */) {
#define A(r, c) a[(r) + (c) * n]
    if (n == 1) return A(0, 0);
    if (n == 2) return A(0, 0) * A(1, 1) - A(0, 1) * A(1, 0);
    /* n == 3 */
    double c0 = A(1, 1) * A(2, 2) - A(1, 2) * A(2, 1);
    double c1 = A(1, 0) * A(2, 2) - A(1, 2) * A(2, 0);
    double c2 = A(1, 0) * A(2, 1) - A(1, 1) * A(2, 0);
    return A(0, 0) * c0 - A(0, 1) * c1 + A(0, 2) * c2;
#undef A
}

/* inverse = adjugate / det (page-wise inverses, Section 2.3).
 * Returns det.  A singular matrix yields IEEE inf/nan entries. */
static double inv_small(int n, const double *a, double *inv) {
#define A(r, c) a[(r) + (c) * n]
#define I(r, c) inv[(r) + (c) * n]
    double d = det_small(n, a);
    if (n == 1) {
        I(0, 0) = 1.0 / d;
    } else if (n == 2) {
        I(0, 0) = A(1, 1) / d;
        I(0, 1) = -A(0, 1) / d;
        I(1, 0) = -A(1, 0) / d;
        I(1, 1) = A(0, 0) / d;
    } else {
        /* cofactor C(r,c) = (-1)^(r+c) * minor(r,c); inverse = C^T / det */
        for (int r = 0; r < 3; ++r) {
            for (int c = 0; c < 3; ++c) {
                int r0 = (r + 1) % 3, r1 = (r + 2) % 3;
                int c0 = (c + 1) % 3, c1 = (c + 2) % 3;
                /* cyclic index choice already carries the cofactor sign */
                double cof = A(r0, c0) * A(r1, c1) - A(r0, c1) * A(r1, c0);
                I(c, r) = cof / d;
            }
        }
    }
    return d;
#undef A
#undef I
}

/* ------------------------------------------------------------------------ */
/* page primitives (Section 2.4: amtam, astam, avtam, amdet, aminv)          */
/* ------------------------------------------------------------------------ */

/* C_k = A_k^T B_k with A_k p x m, B_k p x n, C_k m x n.  Reading of the
 * amtam operand order: the transposed first operand times the second, as
 * the pagemtimes override in Section 2.4 and the call amtam(dphi,dphi) of the
 * P1 stiffness listing (Section 3.5) require. */
void orc_amtam(int64_t N, int p, int m, int n, const double *A, const double *B, double *C) {
    for (int64_t k = 0; k < N; ++k) {
        const double *a = A + k * p * m, *b = B + k * p * n;
        double *c = C + k * m * n;
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < n; ++j) {
                double s = 0.0;
                for (int r = 0; r < p; ++r) s += a[r + i * p] * b[r + j * p];
                c[i + j * m] = s;
            }
    }
}

/* C_k = s_k * A_k (page-wise scalar multiplication, Id (x) pi, Section 2.2). */
void orc_astam(int64_t N, int m, int n, const double *s, const double *A, double *C) {
    for (int64_t k = 0; k < N; ++k)
        for (int e = 0; e < m * n; ++e) C[k * m * n + e] = s[k] * A[k * m * n + e];
}

/* y_k = v_k^T A_k, v_k p-vector, A_k p x n, y_k 1 x n (Section 2.4, avtam). */
void orc_avtam(int64_t N, int p, int n, const double *v, const double *A, double *y) {
    for (int64_t k = 0; k < N; ++k)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int r = 0; r < p; ++r) s += v[k * p + r] * A[k * p * n + r + j * p];
            y[k * n + j] = s;
        }
}

/* C_k = A_k^T (page-wise transpose, pagemtranspose; Section 2.4).
 * A: m x n pages, C: n x m pages (column-major pages, page-major arrays). */
void orc_amt(int64_t N, int m, int n, const double *A, double *C) {
    for (int64_t k = 0; k < N; ++k)
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < n; ++j) C[k * m * n + j + i * n] = A[k * m * n + i + j * m];
}

/* out_k = a_k^T b_k (page-wise dot product of vector arrays; Section 2.4). */
void orc_avtav(int64_t N, int n, const double *a, const double *b, double *out) {
    for (int64_t k = 0; k < N; ++k) {
        double s = 0.0;
        for (int r = 0; r < n; ++r) s += a[k * n + r] * b[k * n + r];
        out[k] = s;
    }
}

/* C_k = A_k S: the single matrix S (p x n) copied to every page and
 * multiplied (amsm, Section 2.4).  A: m x p pages, C: m x n pages. */
void orc_amsm(int64_t N, int m, int p, int n, const double *A, const double *S, double *C) {
    for (int64_t k = 0; k < N; ++k)
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < n; ++j) {
                double s = 0.0;
                for (int r = 0; r < p; ++r) s += A[k * m * p + i + r * m] * S[r + j * p];
                C[k * m * n + i + j * m] = s;
            }
}

/* y_k = A_k s for the single vector s (amsv, Section 2.4).  A: m x n pages,
 * y: m values per page. */
void orc_amsv(int64_t N, int m, int n, const double *A, const double *sv, double *y) {
    for (int64_t k = 0; k < N; ++k)
        for (int i = 0; i < m; ++i) {
            double s = 0.0;
            for (int r = 0; r < n; ++r) s += A[k * m * n + i + r * m] * sv[r];
            y[k * m + i] = s;
        }
}

/* C_k = S A_k^T for the single matrix S (m x p) (smamt, Section 2.4).
 * A: n x p pages, C: m x n pages. */
void orc_smamt(int64_t N, int m, int p, int n, const double *S, const double *A, double *C) {
    for (int64_t k = 0; k < N; ++k)
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < n; ++j) {
                double s = 0.0;
                for (int r = 0; r < p; ++r) s += S[i + r * m] * A[k * n * p + j + r * n];
                C[k * m * n + i + j * m] = s;
            }
}

/* y_k = s^T A_k^T for the single vector s (svamt, Section 2.4): a 1 x m page.
 * A: m x n pages. */
void orc_svamt(int64_t N, int m, int n, const double *sv, const double *A, double *y) {
    for (int64_t k = 0; k < N; ++k)
        for (int j = 0; j < m; ++j) {
            double s = 0.0;
            for (int r = 0; r < n; ++r) s += sv[r] * A[k * m * n + j + r * m];
            y[k * m + j] = s;
        }
}

/* det_k = det(A_k), signed (Section 2.3 eq. of det_W; Section 3.2 example). */
void orc_amdet(int64_t N, int n, const double *A, double *det) {
    for (int64_t k = 0; k < N; ++k) det[k] = det_small(n, A + k * n * n);
}

/* Ainv_k = A_k^{-1}; det_k optional.  Returns the number of singular pages
 * (det == 0), whose inverse holds IEEE inf/nan (the paper defines the inverse
 * only where every determinant is non-zero, Section 2.3). */
int64_t orc_aminv(int64_t N, int n, const double *A, double *Ainv, double *det) {
    int64_t nsing = 0;
    for (int64_t k = 0; k < N; ++k) {
        double d = inv_small(n, A + k * n * n, Ainv + k * n * n);
        if (det) det[k] = d;
        if (d == 0.0) ++nsing;
    }
    return nsing;
}

/* ------------------------------------------------------------------------ */
/* geometry (Section 3.1 coords3D / vectors3D, Section 3.2)                  */
/* ------------------------------------------------------------------------ */

/* vectors3D page of element k: column j = x_{e_k[j]} - x_{e_k[dim]},
 * j = 0..dim-1 (vectors from the last vertex to the others). */
static void simplex_vectors(int dim, int nlb, const int32_t *elems, const double *coords, int64_t k,
                            double *V /* dim x dim */) {
    const int32_t *e = elems + k * nlb;
    const double *xl = coords + (int64_t)e[dim] * dim;
    for (int j = 0; j < dim; ++j) {
        const double *xj = coords + (int64_t)e[j] * dim;
        for (int d = 0; d < dim; ++d) V[d + j * dim] = xj[d] - xl[d];
    }
}

static double factorial(int n) {
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

void orc_vectors(int dim, int64_t ne, int nlb, const int32_t *elems, const double *coords, double *V) {
    for (int64_t k = 0; k < ne; ++k) simplex_vectors(dim, nlb, elems, coords, k, V + k * dim * dim);
}

/* signed det of vectors3D and volume |det| / dim! (Section 3.2 volume script). */
void orc_volumes(int dim, int64_t ne, int nlb, const int32_t *elems, const double *coords, double *vol,
                 double *det_signed) {
    double V[9];
    for (int64_t k = 0; k < ne; ++k) {
        simplex_vectors(dim, nlb, elems, coords, k, V);
        double d = det_small(dim, V);
        if (det_signed) det_signed[k] = d;
        vol[k] = fabs(d) / factorial(dim);
    }
}

/* Unnormalised outer normals of all simplex facets:
 * normals_k = (vectors3D_k)^{-T} * normalsRef  (Section 3.2, with the normal
 * transform X = A^{-T} of Section 2.3).  normalsRef columns are -e_1..-e_dim
 * and (1,..,1); column j is the normal of the facet opposite local vertex j. */
void orc_simplex_normals(int dim, int64_t ne, int nlb, const int32_t *elems, const double *coords,
                         double *normals /* dim x (dim+1) x ne */) {
    double V[9], Vi[9], ref[12];
    for (int r = 0; r < dim; ++r)
        for (int c = 0; c <= dim; ++c) ref[r + c * dim] = (c == dim) ? 1.0 : (r == c ? -1.0 : 0.0);
    for (int64_t k = 0; k < ne; ++k) {
        simplex_vectors(dim, nlb, elems, coords, k, V);
        inv_small(dim, V, Vi);
        double *out = normals + k * dim * (dim + 1);
        for (int r = 0; r < dim; ++r)
            for (int c = 0; c <= dim; ++c) {
                double s = 0.0;
                /* (Vi^T)(r, q) = Vi(q, r) */
                for (int q = 0; q < dim; ++q) s += Vi[q + r * dim] * ref[q + c * dim];
                out[r + c * dim] = s;
            }
    }
}

/* ------------------------------------------------------------------------ */
/* element matrices (Section 3.5)                                            */
/* ------------------------------------------------------------------------ */

/* Barycentric gradients of a simplex: with vectors3D V (last-vertex
 * convention), lambda_{0..dim-1}(x) = V^{-1}(x - x_last), so grad lambda_j is
 * row j of V^{-1} and grad lambda_dim = -sum of the others.
 * glam is dim x (dim+1) col-major: column j = grad lambda_j.  Returns det V. */
static double bary_gradients(int dim, const double *V, double *glam) {
    double Vi[9];
    double d = inv_small(dim, V, Vi);
    for (int j = 0; j < dim; ++j)
        for (int r = 0; r < dim; ++r) glam[r + j * dim] = Vi[j + r * dim];
    for (int r = 0; r < dim; ++r) {
        double s = 0.0;
        for (int j = 0; j < dim; ++j) s += glam[r + j * dim];
        glam[r + dim * dim] = -s;
    }
    return d;
}

/* Coefficient evaluated once per element at the vertex centroid x_c
 * (reading of the Section 3.5 remark on gqo = 1: the coefficient taken at a
 * single quadrature point):
 *   kind 0:  c = a + b |x_c|^2
 *   kind 1:  c = a * exp(b * sum_d x_c[d])   (the benchmark coefficient
 *            e^{x1+x2(+x3)} of Section 3.5.1 with a = b = 1). */
static double centroid_coeff(int dim, int nv, int nlb, const int32_t *elems, const double *coords, int64_t k,
                             int kind, double ca, double cb) {
    double xc[3] = {0, 0, 0};
    for (int j = 0; j < nv; ++j)
        for (int d = 0; d < dim; ++d) xc[d] += coords[(int64_t)elems[k * nlb + j] * dim + d];
    double r2 = 0.0, sum = 0.0;
    for (int d = 0; d < dim; ++d) {
        xc[d] /= nv;
        r2 += xc[d] * xc[d];
        sum += xc[d];
    }
    if (kind == 1) return ca * exp(cb * sum);
    return ca + cb * r2;
}

/* Integral over a simplex T of prod_j lambda_j^{alpha_j}:
 * alpha! * dim! * |T| / (|alpha| + dim)!  (standard barycentric formula). */
static double bary_monomial_integral(int dim, const int *alpha, double vol) {
    double num = factorial(dim);
    int s = 0;
    for (int j = 0; j <= dim; ++j) {
        num *= factorial(alpha[j]);
        s += alpha[j];
    }
    return num * vol / factorial(s + dim);
}

/* P2 basis in barycentric form.  Local order: the dim+1 vertices, then the
 * mid-edge nodes (2-D: (0,1),(1,2),(0,2); 3-D: (0,1),(1,2),(0,2),(0,3),(1,3),
 * (2,3)).  vertex j: lambda_j (2 lambda_j - 1); edge (a,b): 4 lambda_a lambda_b.
 * Each basis function is a sum of <= 2 monomials c * lambda^alpha. */
static const int P2E2[3][2] = {{0, 1}, {1, 2}, {0, 2}};
static const int P2E3[6][2] = {{0, 1}, {1, 2}, {0, 2}, {0, 3}, {1, 3}, {2, 3}};

typedef struct {
    int nterm;
    double coef[2];
    int alpha[2][4];
} poly_t;

static void p2_basis(int dim, int q, poly_t *out) {
    memset(out, 0, sizeof(*out));
    if (q <= dim) {
        out->nterm = 2;
        out->coef[0] = 2.0;
        out->alpha[0][q] = 2;
        out->coef[1] = -1.0;
        out->alpha[1][q] = 1;
    } else {
        const int *e = (dim == 2) ? P2E2[q - 3] : P2E3[q - 4];
        out->nterm = 1;
        out->coef[0] = 4.0;
        out->alpha[0][e[0]] += 1;
        out->alpha[0][e[1]] += 1;
    }
}

/* gradient of a P2 basis function: sum over terms and over the lambdas each
 * term contains: d(c lambda^alpha) = c alpha_j lambda^(alpha - e_j) grad lambda_j.
 * Represented as up to 4 pieces (coef, alpha', j). */
typedef struct {
    int n;
    double coef[4];
    int alpha[4][4];
    int j[4];
} gpoly_t;

static void p2_grad(int dim, const poly_t *p, gpoly_t *g) {
    memset(g, 0, sizeof(*g));
    for (int t = 0; t < p->nterm; ++t)
        for (int j = 0; j <= dim; ++j) {
            if (p->alpha[t][j] == 0) continue;
            int i = g->n++;
            g->coef[i] = p->coef[t] * p->alpha[t][j];
            memcpy(g->alpha[i], p->alpha[t], sizeof(g->alpha[i]));
            g->alpha[i][j] -= 1;
            g->j[i] = j;
        }
}

/* Element matrices of element k, P1 or P2, into Kp, Mp (nlb x nlb col-major):
 *   K_k(p,q) = c_k * int_T grad phi_p . grad phi_q,
 *   M_k(p,q) = c_k * int_T phi_p phi_q,
 * with c_k the centroid coefficient (kinds 0, 1); kinds 2, 3 (P1 only) take
 * the coefficient of kind 0, 1 at the points of the degree-2 rule instead.  P1: K_k = c_k vol G^T G,
 * M_k = c_k vol (1 + delta_pq) / ((dim+1)(dim+2)) (Section 3.5 stiffness and
 * mass listings; the integrals are evaluated exactly).  Returns signed det. */
int orc_quad_rule(int sdim, int gqo, double *ip, double *w);

/* coefficient at a point x: kind 0 a + b |x|^2, kind 1 a exp(b sum x) */
static double point_coeff(int dim, int kind, double ca, double cb, const double *x) {
    double r2 = 0.0, sum = 0.0;
    for (int d = 0; d < dim; ++d) {
        r2 += x[d] * x[d];
        sum += x[d];
    }
    return kind == 1 ? ca * exp(cb * sum) : ca + cb * r2;
}

static double element_matrices(int dim, int order, int nlb, const int32_t *elems, const double *coords, int64_t k,
                               int ckind, double ca, double cb, double *Kp, double *Mp, double *c_out) {
    double V[9], glam[12];
    simplex_vectors(dim, nlb, elems, coords, k, V);
    double d = bary_gradients(dim, V, glam);
    double vol = fabs(d) / factorial(dim);
    if (ckind >= 2 && order == 1) {
        /* the paper's literal P1 listing (stiffness_matrixP1, Section 3.5): the
         * degree-2 rule (gqo = 2) with the coefficient evaluated at every point;
         * the mass matrix the same way: M(p,q) = vol sum_i w_i c(x_i) lambda_p lambda_q */
        double ip[32], w[8], cq[8];
        const int nip = orc_quad_rule(dim, 2, ip, w);
        double cK = 0.0;
        for (int i = 0; i < nip; ++i) {
            double x[3] = {0, 0, 0};
            for (int j = 0; j <= dim; ++j)
                for (int r = 0; r < dim; ++r) x[r] += ip[i * (dim + 1) + j] * coords[(int64_t)elems[k * nlb + j] * dim + r];
            cq[i] = point_coeff(dim, ckind - 2, ca, cb, x);
            cK += w[i] * cq[i];
        }
        if (c_out) *c_out = cK;
        for (int p = 0; p < nlb; ++p)
            for (int q = 0; q < nlb; ++q) {
                double s = 0.0, m = 0.0;
                for (int r = 0; r < dim; ++r) s += glam[r + p * dim] * glam[r + q * dim];
                for (int i = 0; i < nip; ++i) m += w[i] * cq[i] * ip[i * (dim + 1) + p] * ip[i * (dim + 1) + q];
                Kp[p + q * nlb] = cK * vol * s;
                Mp[p + q * nlb] = vol * m;
            }
        return d;
    }
    double c = centroid_coeff(dim, dim + 1, nlb, elems, coords, k, ckind & 1, ca, cb);
    if (c_out) *c_out = c;
    if (order == 1) {
        for (int p = 0; p < nlb; ++p)
            for (int q = 0; q < nlb; ++q) {
                double s = 0.0;
                for (int r = 0; r < dim; ++r) s += glam[r + p * dim] * glam[r + q * dim];
                Kp[p + q * nlb] = c * vol * s;
                Mp[p + q * nlb] = c * vol * (p == q ? 2.0 : 1.0) / ((dim + 1) * (dim + 2));
            }
        return d;
    }
    /* P2: expand products into barycentric monomials and integrate exactly */
    double gg[16]; /* grad lambda_i . grad lambda_j */
    for (int i = 0; i <= dim; ++i)
        for (int j = 0; j <= dim; ++j) {
            double s = 0.0;
            for (int r = 0; r < dim; ++r) s += glam[r + i * dim] * glam[r + j * dim];
            gg[i + j * 4] = s;
        }
    poly_t P[10];
    gpoly_t G[10];
    for (int q = 0; q < nlb; ++q) {
        p2_basis(dim, q, &P[q]);
        p2_grad(dim, &P[q], &G[q]);
    }
    for (int p = 0; p < nlb; ++p)
        for (int q = 0; q < nlb; ++q) {
            double sk = 0.0, sm = 0.0;
            for (int u = 0; u < G[p].n; ++u)
                for (int v = 0; v < G[q].n; ++v) {
                    int al[4];
                    for (int j = 0; j < 4; ++j) al[j] = G[p].alpha[u][j] + G[q].alpha[v][j];
                    sk += G[p].coef[u] * G[q].coef[v] * gg[G[p].j[u] + G[q].j[v] * 4] *
                          bary_monomial_integral(dim, al, vol);
                }
            for (int u = 0; u < P[p].nterm; ++u)
                for (int v = 0; v < P[q].nterm; ++v) {
                    int al[4];
                    for (int j = 0; j < 4; ++j) al[j] = P[p].alpha[u][j] + P[q].alpha[v][j];
                    sm += P[p].coef[u] * P[q].coef[v] * bary_monomial_integral(dim, al, vol);
                }
            Kp[p + q * nlb] = c * sk;
            Mp[p + q * nlb] = c * sm;
        }
    return d;
}

/* All element pages (K3D, M3D of Section 3.5) plus volumes and coefficients. */
void orc_element_pages(int dim, int order, int64_t ne, int nlb, const int32_t *elems, const double *coords,
                       int ckind, double ca, double cb, double *K3D, double *M3D, double *vol, double *coef) {
    for (int64_t k = 0; k < ne; ++k) {
        double c;
        double d = element_matrices(dim, order, nlb, elems, coords, k, ckind, ca, cb, K3D + k * nlb * nlb,
                                    M3D + k * nlb * nlb, &c);
        if (vol) vol[k] = fabs(d) / factorial(dim);
        if (coef) coef[k] = c;
    }
}

/* ------------------------------------------------------------------------ */
/* sparse assembly with the semantics of MATLAB's sparse() on the row and    */
/* column index pages and the element pages (Section 3.5): all (row, col)   */
/* pairs of all elements, duplicates summed.                                */
/* Structural zeros are kept: the pattern depends on connectivity only.     */
/* ------------------------------------------------------------------------ */

static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

/* Pattern: returns nnz (or -1 on allocation failure).  If row_ptr/col_idx
 * are NULL only the count is returned. */
int64_t orc_csr_pattern(int64_t nn, int64_t ne, int nlb, const int32_t *elems, int32_t *row_ptr, int32_t *col_idx) {
    int64_t np = ne * nlb * nlb;
    uint64_t *keys = (uint64_t *)malloc((size_t)(np > 0 ? np : 1) * sizeof(uint64_t));
    if (!keys) return -1;
    int64_t t = 0;
    for (int64_t k = 0; k < ne; ++k)
        for (int i = 0; i < nlb; ++i)
            for (int j = 0; j < nlb; ++j) {
                /* X3D(i,j,k) = elems(k,j) is the row, Y3D(i,j,k) = elems(k,i) the column */
                uint64_t r = (uint32_t)elems[k * nlb + j], c = (uint32_t)elems[k * nlb + i];
                keys[t++] = (r << 32) | c;
            }
    qsort(keys, (size_t)np, sizeof(uint64_t), cmp_u64);
    int64_t nnz = 0;
    if (row_ptr)
        for (int64_t i = 0; i <= nn; ++i) row_ptr[i] = 0;
    for (int64_t q = 0; q < np; ++q) {
        if (q > 0 && keys[q] == keys[q - 1]) continue;
        if (col_idx) {
            col_idx[nnz] = (int32_t)(keys[q] & 0xffffffffu);
            row_ptr[(keys[q] >> 32) + 1] += 1;
        }
        ++nnz;
    }
    if (row_ptr)
        for (int64_t i = 0; i < nn; ++i) row_ptr[i + 1] += row_ptr[i];
    free(keys);
    return nnz;
}

/* position of column c in row r (binary search), -1 if absent */
static int64_t csr_find(const int32_t *row_ptr, const int32_t *col_idx, int32_t r, int32_t c) {
    int64_t lo = row_ptr[r], hi = row_ptr[r + 1] - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (col_idx[mid] == c) return mid;
        if (col_idx[mid] < c) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

/* Scatter element pages into CSR values, ascending k then (i, j):
 * vals(elems(k,j), elems(k,i)) += P_k(i,j).  Returns 0, or -1 if a pair is
 * missing from the pattern. */
int orc_csr_scatter(int64_t ne, int nlb, const int32_t *elems, const double *P3D, const int32_t *row_ptr,
                    const int32_t *col_idx, double *vals) {
    for (int64_t k = 0; k < ne; ++k)
        for (int j = 0; j < nlb; ++j)
            for (int i = 0; i < nlb; ++i) {
                int64_t pos = csr_find(row_ptr, col_idx, elems[k * nlb + j], elems[k * nlb + i]);
                if (pos < 0) return -1;
                vals[pos] += P3D[k * nlb * nlb + i + j * nlb];
            }
    return 0;
}

/* Whole assembly of K and M into an existing pattern (values zeroed first),
 * plus element volumes.  Page buffers are allocated internally if the
 * caller passes NULL for K3D/M3D. */
int orc_assemble(int dim, int order, int64_t nn, int64_t ne, int nlb, const int32_t *elems, const double *coords,
                 int ckind, double ca, double cb, const int32_t *row_ptr, const int32_t *col_idx, double *Kv, double *Mv,
                 double *vol, double *K3D, double *M3D) {
    int own = 0;
    if (!K3D || !M3D) {
        own = 1;
        K3D = (double *)malloc((size_t)(ne > 0 ? ne : 1) * nlb * nlb * sizeof(double));
        M3D = (double *)malloc((size_t)(ne > 0 ? ne : 1) * nlb * nlb * sizeof(double));
        if (!K3D || !M3D) {
            free(K3D);
            free(M3D);
            return -1;
        }
    }
    orc_element_pages(dim, order, ne, nlb, elems, coords, ckind, ca, cb, K3D, M3D, vol, NULL);
    int64_t nnz = row_ptr[nn];
    for (int64_t q = 0; q < nnz; ++q) Kv[q] = Mv[q] = 0.0;
    int rc = orc_csr_scatter(ne, nlb, elems, K3D, row_ptr, col_idx, Kv);
    if (rc == 0) rc = orc_csr_scatter(ne, nlb, elems, M3D, row_ptr, col_idx, Mv);
    if (own) {
        free(K3D);
        free(M3D);
    }
    return rc;
}

/* ------------------------------------------------------------------------ */
/* boundary facets: outward unit normals and measures                        */
/* ------------------------------------------------------------------------ */

/* For each boundary facet (dim nodes, vertex numbering), find the element
 * that owns it and its remaining vertex, then
 *   3-D: n = (x2 - x1) x (x3 - x1), area = |n| / 2,
 *   2-D: n = (t_y, -t_x) with t = x2 - x1, length = |t|,
 * oriented so that n points away from the remaining vertex, normalised.
 * Returns the number of facets without an owner (their outputs are NaN). */
int64_t orc_boundary(int dim, int64_t nn, int64_t ne, int nlb, const int32_t *elems, const double *coords,
                     int64_t nfb, const int32_t *faces, double *normals /* dim x nfb */, double *areas) {
    /* node -> element incidence lists (counting sort by node, ascending k) */
    int64_t *ptr = (int64_t *)calloc((size_t)nn + 1, sizeof(int64_t));
    int64_t *lst = (int64_t *)malloc((size_t)(ne > 0 ? ne : 1) * (dim + 1) * sizeof(int64_t));
    int64_t *cur = (int64_t *)malloc((size_t)(nn > 0 ? nn : 1) * sizeof(int64_t));
    int64_t missing = 0;
    for (int64_t k = 0; k < ne; ++k)
        for (int j = 0; j <= dim; ++j) ptr[elems[k * nlb + j] + 1] += 1;
    for (int64_t i = 0; i < nn; ++i) ptr[i + 1] += ptr[i];
    for (int64_t i = 0; i < nn; ++i) cur[i] = ptr[i];
    for (int64_t k = 0; k < ne; ++k)
        for (int j = 0; j <= dim; ++j) lst[cur[elems[k * nlb + j]]++] = k;
    for (int64_t f = 0; f < nfb; ++f) {
        const int32_t *fn = faces + f * dim;
        int32_t opp = -1;
        for (int64_t t = ptr[fn[0]]; t < ptr[fn[0] + 1] && opp < 0; ++t) {
            int64_t k = lst[t];
            int hits = 0;
            for (int j = 0; j <= dim; ++j)
                for (int q = 0; q < dim; ++q)
                    if (elems[k * nlb + j] == fn[q]) ++hits;
            if (hits != dim) continue;
            for (int j = 0; j <= dim; ++j) {
                int32_t v = elems[k * nlb + j];
                int in = 0;
                for (int q = 0; q < dim; ++q) in |= (v == fn[q]);
                if (!in) opp = v;
            }
        }
        double n[3] = {0, 0, 0}, meas;
        const double *x1 = coords + (int64_t)fn[0] * dim, *x2 = coords + (int64_t)fn[1] * dim;
        if (dim == 3) {
            const double *x3 = coords + (int64_t)fn[2] * dim;
            double a[3], b[3];
            for (int d = 0; d < 3; ++d) {
                a[d] = x2[d] - x1[d];
                b[d] = x3[d] - x1[d];
            }
            n[0] = a[1] * b[2] - a[2] * b[1];
            n[1] = a[2] * b[0] - a[0] * b[2];
            n[2] = a[0] * b[1] - a[1] * b[0];
            meas = 0.5 * sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        } else {
            n[0] = x2[1] - x1[1];
            n[1] = -(x2[0] - x1[0]);
            meas = sqrt(n[0] * n[0] + n[1] * n[1]);
        }
        double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (opp < 0) {
            ++missing;
            for (int d = 0; d < dim; ++d) normals[f * dim + d] = NAN;
            areas[f] = NAN;
            continue;
        }
        const double *xo = coords + (int64_t)opp * dim;
        double side = 0.0;
        for (int d = 0; d < dim; ++d) side += n[d] * (xo[d] - x1[d]);
        double sgn = side > 0.0 ? -1.0 : 1.0;
        for (int d = 0; d < dim; ++d) normals[f * dim + d] = sgn * n[d] / len;
        areas[f] = meas;
    }
    free(ptr);
    free(lst);
    free(cur);
    return missing;
}

/* ------------------------------------------------------------------------ */
/* facet enumeration (counts of the paper's normals table, Section 3.2)     */
/* ------------------------------------------------------------------------ */

static int cmp_face(const void *a, const void *b) {
    const int32_t *x = (const int32_t *)a, *y = (const int32_t *)b;
    for (int q = 0; q < 3; ++q) {
        if (x[q] != y[q]) return (x[q] > y[q]) - (x[q] < y[q]);
    }
    return 0;
}

/* Number of distinct facets of a simplicial mesh and number of facets that
 * belong to exactly one element (boundary facets).  Returns -1 on failure. */
int orc_count_facets(int dim, int64_t ne, int nlb, const int32_t *elems, int64_t *n_all, int64_t *n_boundary) {
    int64_t nf = ne * (dim + 1);
    int32_t *f = (int32_t *)malloc((size_t)(nf > 0 ? nf : 1) * 3 * sizeof(int32_t));
    if (!f) return -1;
    int64_t t = 0;
    for (int64_t k = 0; k < ne; ++k)
        for (int drop = 0; drop <= dim; ++drop) {
            int32_t v[3] = {-1, -1, -1};
            int q = 0;
            for (int j = 0; j <= dim; ++j)
                if (j != drop) v[q++] = elems[k * nlb + j];
            /* sort the facet's vertices (insertion sort) */
            for (int a = 1; a < dim; ++a)
                for (int b = a; b > 0 && v[b - 1] > v[b]; --b) {
                    int32_t tmp = v[b];
                    v[b] = v[b - 1];
                    v[b - 1] = tmp;
                }
            memcpy(f + 3 * t, v, sizeof(v));
            ++t;
        }
    qsort(f, (size_t)nf, 3 * sizeof(int32_t), cmp_face);
    int64_t all = 0, bnd = 0;
    for (int64_t q = 0; q < nf;) {
        int64_t r = q + 1;
        while (r < nf && cmp_face(f + 3 * q, f + 3 * r) == 0) ++r;
        ++all;
        if (r - q == 1) ++bnd;
        q = r;
    }
    *n_all = all;
    *n_boundary = bnd;
    free(f);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* quadrature on simplices (Section 3.4 Gauss_points, Section 3.5 intquad)  */
/* ------------------------------------------------------------------------ */

/* Symmetric rules in barycentric coordinates, weights summing to 1 (the
 * "averaged" normalisation of Gauss_points; intquad's weights are these
 * times 1/dim!).  gqo is the degree of exactness.  sdim is the simplex
 * dimension (1 segment, 2 triangle, 3 tetrahedron).  Published rules:
 *   segment   gqo 1: midpoint;  gqo 2-3: Gauss-Legendre, 1/2 +- 1/(2 sqrt 3).
 *   triangle  gqo 1: centroid;  gqo 2: (2/3,1/6,1/6) and permutations, 1/3 each;
 *             gqo 3: centroid -27/48, (3/5,1/5,1/5) and permutations 25/48.
 *   tet       gqo 1: centroid;  gqo 2: (a,b,b,b) and permutations, 1/4 each,
 *             a = (5 + 3 sqrt 5)/20, b = (5 - sqrt 5)/20;
 *             gqo 3: centroid -4/5, (1/2,1/6,1/6,1/6) and permutations 9/20.
 * ip: (sdim+1) x nip column-major (point q at q*(sdim+1)).  Returns nip, or
 * -1 for an unsupported (sdim, gqo). */
int orc_quad_rule(int sdim, int gqo, double *ip, double *w) {
    const int nv = sdim + 1;
    int nip = 0;
    if (gqo < 1 || gqo > 3 || sdim < 1 || sdim > 3) return -1;
    if (gqo == 1) {
        for (int j = 0; j < nv; ++j) ip[j] = 1.0 / nv;
        w[0] = 1.0;
        return 1;
    }
    if (sdim == 1) {
        const double d = 0.5 / sqrt(3.0);
        ip[0] = 0.5 + d, ip[1] = 0.5 - d;
        ip[2] = 0.5 - d, ip[3] = 0.5 + d;
        w[0] = w[1] = 0.5;
        return 2;
    }
    /* centroid (gqo 3) then one orbit of points with one distinguished coordinate */
    double big, small, wc = 0.0, wo;
    if (sdim == 2) {
        if (gqo == 2) big = 2.0 / 3.0, small = 1.0 / 6.0, wo = 1.0 / 3.0;
        else big = 0.6, small = 0.2, wc = -27.0 / 48.0, wo = 25.0 / 48.0;
    } else {
        if (gqo == 2) big = (5.0 + 3.0 * sqrt(5.0)) / 20.0, small = (5.0 - sqrt(5.0)) / 20.0, wo = 0.25;
        else big = 0.5, small = 1.0 / 6.0, wc = -0.8, wo = 9.0 / 20.0;
    }
    if (gqo == 3) {
        for (int j = 0; j < nv; ++j) ip[nip * nv + j] = 1.0 / nv;
        w[nip++] = wc;
    }
    for (int i = 0; i < nv; ++i) {
        for (int j = 0; j < nv; ++j) ip[nip * nv + j] = (i == j) ? big : small;
        w[nip++] = wo;
    }
    return nip;
}

/* Coordinates of the quadrature points of n simplices (elements or facets):
 * X(:,q,k) = sum_j ip(j,q) x_{cells(k,j)} -- the paper's X_ip =
 * amsm(coords3D, ip), dim x nip x n.  cells: stride entries per simplex, the
 * first nvert of which are its vertices. */
void orc_quad_points(int dim, int nvert, int64_t n, int stride, const int32_t *cells, const double *coords, int nip,
                     const double *ip, double *X) {
    for (int64_t k = 0; k < n; ++k)
        for (int q = 0; q < nip; ++q)
            for (int d = 0; d < dim; ++d) {
                double s = 0.0;
                for (int j = 0; j < nvert; ++j) s += ip[q * nvert + j] * coords[(int64_t)cells[k * stride + j] * dim + d];
                X[(k * nip + q) * dim + d] = s;
            }
}

/* The GI function of Section 3.4: value = sum_k sizes_k sum_q w_q f(:,q,k),
 * f of d components (fip: d x nip x n).  With normals (d x n) the components
 * are dotted with the simplex's normal first and out[0] is the scalar
 * integral; without, out[c] is the integral of component c. */
void orc_gi(int64_t n, int nip, int d, const double *fip, const double *w, const double *sizes, const double *normals,
            double *out) {
    for (int c = 0; c < d; ++c) out[c] = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        double avg[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        for (int c = 0; c < d; ++c)
            for (int q = 0; q < nip; ++q) avg[c] += w[q] * fip[(k * nip + q) * d + c];
        if (normals) {
            double dot = 0.0;
            for (int c = 0; c < d; ++c) dot += avg[c] * normals[k * d + c];
            out[0] += sizes[k] * dot;
        } else {
            for (int c = 0; c < d; ++c) out[c] += sizes[k] * avg[c];
        }
    }
}

/* local basis function j at barycentric point lam (P1: lambda_j; P2 as in
 * p2_basis) */
static double basis_at(int dim, int order, int j, const double *lam) {
    if (order == 1) return lam[j];
    poly_t p;
    p2_basis(dim, j, &p);
    double v = 0.0;
    for (int t = 0; t < p.nterm; ++t) {
        double m = p.coef[t];
        for (int s = 0; s <= dim; ++s)
            for (int e = 0; e < p.alpha[t][s]; ++e) m *= lam[s];
        v += m;
    }
    return v;
}

/* Right-hand side vector of Section 3.5 (rhs_vectorP1, and its P2 analogue):
 * b2D(j,k) = |T_k| sum_q w_q f(x_q) phi_j(ip_q) with f given at the rule's
 * points (fip: nip x ne), then b = accumarray(elems(:), b2D(:)). */
void orc_rhs(int dim, int order, int64_t nn, int64_t ne, int nlb, const int32_t *elems, const double *coords, int nip,
             const double *ip, const double *w, const double *fip, double *b, double *b2D) {
    double *vol = (double *)malloc((size_t)(ne > 0 ? ne : 1) * sizeof(double));
    orc_volumes(dim, ne, nlb, elems, coords, vol, NULL);
    for (int64_t i = 0; i < nn; ++i) b[i] = 0.0;
    for (int64_t k = 0; k < ne; ++k)
        for (int j = 0; j < nlb; ++j) {
            double s = 0.0;
            for (int q = 0; q < nip; ++q) s += w[q] * fip[k * nip + q] * basis_at(dim, order, j, ip + q * (dim + 1));
            b2D[k * nlb + j] = vol[k] * s;
        }
    for (int64_t k = 0; k < ne; ++k)
        for (int j = 0; j < nlb; ++j) b[elems[k * nlb + j]] += b2D[k * nlb + j];
    free(vol);
}

/* Local energies of Section 3.5 (eq. Jk_comps): with u_k the element's nodal
 * values, J(0,k) = u_k^T K_k u_k / 2, J(1,k) = u_k^T M_k u_k / 2,
 * J(2,k) = -b2D(:,k)^T u_k (b2D the element's own load contributions, so that
 * the J(.,k) sum to the global forms). */
void orc_energies(int64_t ne, int nlb, const int32_t *elems, const double *u, const double *K3D, const double *M3D,
                  const double *b2D, double *J) {
    for (int64_t k = 0; k < ne; ++k) {
        double uk[10];
        for (int j = 0; j < nlb; ++j) uk[j] = u[elems[k * nlb + j]];
        double a = 0.0, m = 0.0, f = 0.0;
        for (int i = 0; i < nlb; ++i)
            for (int j = 0; j < nlb; ++j) {
                a += uk[i] * K3D[k * nlb * nlb + i + j * nlb] * uk[j];
                m += uk[i] * M3D[k * nlb * nlb + i + j * nlb] * uk[j];
            }
        for (int j = 0; j < nlb; ++j) f += b2D[k * nlb + j] * uk[j];
        J[k * 3 + 0] = 0.5 * a;
        J[k * 3 + 1] = 0.5 * m;
        J[k * 3 + 2] = -f;
    }
}

/* out_k = v_k^T A_k w_k (Section 2.4, avtamav), v_k and w_k n-vectors,
 * A_k n x n column-major. */
void orc_avtamav(int64_t N, int n, const double *v, const double *A, const double *w, double *out) {
    for (int64_t k = 0; k < N; ++k) {
        double s = 0.0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) s += v[k * n + i] * A[k * n * n + i + j * n] * w[k * n + j];
        out[k] = s;
    }
}

/* ------------------------------------------------------------------------ */
/* facet list (Section 3.2: normals of all faces, boundary faces)            */
/* ------------------------------------------------------------------------ */

/* Every distinct facet once, in the order of its first element k ascending,
 * then its local facet j ascending (facet j is opposite local vertex j; its
 * vertices are the element's other vertices in local order).  A facet shared
 * by elements k < k' is listed with k.  faces: dim x nf; owner: 2 x nf
 * (k, j); neighbor: nf, the other element or -1 on the boundary.  Any output
 * may be NULL.  Returns nf (or -1 on allocation failure); *n_boundary the
 * number of facets without neighbour.  Brute force: all (sorted triple, k, j)
 * records sorted, equal triples paired. */
typedef struct {
    int32_t v[3];
    int64_t k;
    int32_t j;
} facet_rec;

static int cmp_facet_rec(const void *a, const void *b) {
    const facet_rec *x = (const facet_rec *)a, *y = (const facet_rec *)b;
    for (int q = 0; q < 3; ++q)
        if (x->v[q] != y->v[q]) return (x->v[q] > y->v[q]) - (x->v[q] < y->v[q]);
    if (x->k != y->k) return (x->k > y->k) - (x->k < y->k);
    return (x->j > y->j) - (x->j < y->j);
}

int64_t orc_facets(int dim, int64_t ne, int nlb, const int32_t *elems, int32_t *faces, int32_t *owner,
                   int32_t *neighbor, int64_t *n_boundary) {
    const int nv = dim + 1;
    const int64_t nr = ne * nv;
    facet_rec *r = (facet_rec *)malloc((size_t)(nr > 0 ? nr : 1) * sizeof(facet_rec));
    int64_t *partner = (int64_t *)malloc((size_t)(nr > 0 ? nr : 1) * sizeof(int64_t));
    if (!r || !partner) {
        free(r);
        free(partner);
        return -1;
    }
    for (int64_t k = 0; k < ne; ++k)
        for (int j = 0; j < nv; ++j) {
            facet_rec *f = r + k * nv + j;
            int q = 0;
            f->v[0] = f->v[1] = f->v[2] = -1;
            for (int i = 0; i < nv; ++i)
                if (i != j) f->v[q++] = elems[k * nlb + i];
            for (int a = 1; a < dim; ++a)
                for (int b = a; b > 0 && f->v[b - 1] > f->v[b]; --b) {
                    int32_t t = f->v[b];
                    f->v[b] = f->v[b - 1];
                    f->v[b - 1] = t;
                }
            f->k = k;
            f->j = j;
        }
    qsort(r, (size_t)nr, sizeof(facet_rec), cmp_facet_rec);
    /* partner element of record (k, j), indexed by k*nv + j */
    for (int64_t t = 0; t < nr; ++t) partner[r[t].k * nv + r[t].j] = -1;
    for (int64_t t = 0; t + 1 < nr; ++t)
        if (r[t].v[0] == r[t + 1].v[0] && r[t].v[1] == r[t + 1].v[1] && r[t].v[2] == r[t + 1].v[2]) {
            partner[r[t].k * nv + r[t].j] = r[t + 1].k;
            partner[r[t + 1].k * nv + r[t + 1].j] = r[t].k;
        }
    int64_t nf = 0, nb = 0;
    for (int64_t k = 0; k < ne; ++k)
        for (int j = 0; j < nv; ++j) {
            const int64_t p = partner[k * nv + j];
            if (p >= 0 && p < k) continue;   /* listed with the smaller element */
            if (faces) {
                int q = 0;
                for (int i = 0; i < nv; ++i)
                    if (i != j) faces[nf * dim + q++] = elems[k * nlb + i];
            }
            if (owner) owner[nf * 2] = (int32_t)k, owner[nf * 2 + 1] = j;
            if (neighbor) neighbor[nf] = (int32_t)p;
            if (p < 0) ++nb;
            ++nf;
        }
    if (n_boundary) *n_boundary = nb;
    free(r);
    free(partner);
    return nf;
}

/* ------------------------------------------------------------------------ */
/* Timing entry for the CPU baseline only (not pinned separately: it runs   */
/* the pinned functions above and gives their results bit for bit).  The    */
/* same assembly as orc_assemble on nthreads host threads: element pages    */
/* by orc_element_pages over contiguous element ranges, then each thread     */
/* scatters the entries whose row falls in its own block of rows, visiting  */
/* elements in ascending order, so every CSR value receives its terms in    */
/* the same order as the sequential scatter.                                */
/* ------------------------------------------------------------------------ */
#include <pthread.h>

typedef struct {
    int dim, order, nlb, ckind;
    int64_t ne, k0, k1;          /* element range of the page phase */
    int32_t r0, r1;              /* row block of the scatter phase */
    const int32_t *elems, *row_ptr, *col_idx;
    const double *coords;
    double ca, cb;
    double *K3D, *M3D, *vol, *Kv, *Mv;
    int phase, rc;
} orc_task;

static void *orc_task_run(void *p) {
    orc_task *t = (orc_task *)p;
    const int nlb = t->nlb;
    if (t->phase == 0) {
        orc_element_pages(t->dim, t->order, t->k1 - t->k0, nlb, t->elems + t->k0 * nlb, t->coords, t->ckind, t->ca,
                          t->cb, t->K3D + t->k0 * nlb * nlb, t->M3D + t->k0 * nlb * nlb, t->vol + t->k0, NULL);
        return NULL;
    }
    for (int64_t q = t->row_ptr[t->r0]; q < t->row_ptr[t->r1]; ++q) t->Kv[q] = t->Mv[q] = 0.0;
    for (int64_t k = 0; k < t->ne; ++k)
        for (int j = 0; j < nlb; ++j) {
            const int32_t r = t->elems[k * nlb + j];
            if (r < t->r0 || r >= t->r1) continue;
            for (int i = 0; i < nlb; ++i) {
                int64_t pos = csr_find(t->row_ptr, t->col_idx, r, t->elems[k * nlb + i]);
                if (pos < 0) {
                    t->rc = -1;
                    return NULL;
                }
                t->Kv[pos] += t->K3D[k * nlb * nlb + i + j * nlb];
                t->Mv[pos] += t->M3D[k * nlb * nlb + i + j * nlb];
            }
        }
    return NULL;
}

int orc_assemble_threads(int dim, int order, int64_t nn, int64_t ne, int nlb, const int32_t *elems,
                         const double *coords, int ckind, double ca, double cb, const int32_t *row_ptr,
                         const int32_t *col_idx, double *Kv, double *Mv, double *vol, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    double *K3D = (double *)malloc((size_t)(ne > 0 ? ne : 1) * nlb * nlb * sizeof(double));
    double *M3D = (double *)malloc((size_t)(ne > 0 ? ne : 1) * nlb * nlb * sizeof(double));
    orc_task *T = (orc_task *)calloc((size_t)nthreads, sizeof(orc_task));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    char *started = (char *)calloc((size_t)nthreads, 1);
    int rc = 0;
    if (!K3D || !M3D || !T || !th || !started) rc = -1;
    for (int phase = 0; phase < 2 && rc == 0; ++phase) {
        for (int t = 0; t < nthreads; ++t) {
            orc_task *x = &T[t];
            x->dim = dim;
            x->order = order;
            x->nlb = nlb;
            x->ckind = ckind;
            x->ne = ne;
            x->k0 = ne * t / nthreads;
            x->k1 = ne * (t + 1) / nthreads;
            x->r0 = (int32_t)(nn * t / nthreads);
            x->r1 = (int32_t)(nn * (t + 1) / nthreads);
            x->elems = elems;
            x->row_ptr = row_ptr;
            x->col_idx = col_idx;
            x->coords = coords;
            x->ca = ca;
            x->cb = cb;
            x->K3D = K3D;
            x->M3D = M3D;
            x->vol = vol;
            x->Kv = Kv;
            x->Mv = Mv;
            x->phase = phase;
            x->rc = 0;
        }
        for (int t = 1; t < nthreads; ++t) {
            started[t] = pthread_create(&th[t], NULL, orc_task_run, &T[t]) == 0;
            if (!started[t]) orc_task_run(&T[t]);   /* no thread to be had: run the task here */
        }
        orc_task_run(&T[0]);
        for (int t = 1; t < nthreads; ++t)
            if (started[t]) pthread_join(th[t], NULL);
        for (int t = 0; t < nthreads; ++t)
            if (T[t].rc) rc = T[t].rc;
    }
    free(K3D);
    free(M3D);
    free(T);
    free(th);
    free(started);
    return rc;
}
