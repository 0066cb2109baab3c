// vla_assemble.cu -- P1/P2 simplex stiffness and mass assembly into CSR
// (Section 3.5 stiffness/mass listings and their sparse() scatter), boundary
// facet normals and areas, and all-facet normals (Section 3.2).
//
// One CTA per row tile (built in vla_mesh.cu):
//   phase 0  the tile's vertex coordinates -> shared memory;
//   phase 1  every element touching the tile's rows: Jacobian, determinant,
//            cofactors, coefficient at the centroid, element matrix K_k and
//            mass scale -> shared memory (owned elements also write volume
//            and, on request, the K3D/M3D pages);
//   phase 2  every nonzero of the tile sums its contribution list (ascending
//            element id) from shared memory and writes its FP64 value once.
// No atomics, no global gathers in the hot loop; the order of every sum is
// fixed by the mesh, so results are bit-reproducible.
//
// Geometry (Sections 3.1-3.2): vectors3D V = [x_0 - x_d, ..., x_{d-1} - x_d];
// the cofactor vectors C_j (rows of adj V) give grad lambda_j = C_j / det V
// for j < d and C_d = -sum_j C_j.  P1: K_k(a,b) = c_k (C_a.C_b) / (d! |det V|),
// M_k = c_k |det V| / d! * (1 + delta_ab) / ((d+1)(d+2)).  P2: the same
// cofactor products weighted by reference tensors from the 4-point rule.
#include <cmath>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "vla_internal.cuh"

namespace vla {
namespace {

constexpr int kThreads = 256;

// ---------------------------------------------------------------------------
// P2 reference tables (built on the host once per device)
// ---------------------------------------------------------------------------
struct P2Tab {
    // stiffness: K_pq = sc * sum_t coef[u][t] * Cd[st[u][t]], u = packed (p<=q)
    unsigned char nterm[55];
    unsigned char st[55][4];
    float coef_f[55][4];
    double coef_d[55][4];
    float mhat_f[55];
    double mhat_d[55];
};
__constant__ P2Tab c_p2[2];   // [0] = 2-D (6 nodes), [1] = 3-D (10 nodes)

int packed_index(int p, int q, int n) {  // p <= q
    return p * n - p * (p - 1) / 2 + (q - p);
}

void p2_edges(int dim, int e, int &a, int &b) {
    static const int E2[3][2] = {{0, 1}, {1, 2}, {0, 2}};
    static const int E3[6][2] = {{0, 1}, {1, 2}, {0, 2}, {0, 3}, {1, 3}, {2, 3}};
    a = dim == 2 ? E2[e][0] : E3[e][0];
    b = dim == 2 ? E2[e][1] : E3[e][1];
}

// d(phi_p)/d(lambda_s) at barycentric point lam
double p2_dphi(int dim, int p, int s, const double *lam) {
    if (p <= dim) return (s == p) ? 4.0 * lam[p] - 1.0 : 0.0;
    int a, b;
    p2_edges(dim, p - dim - 1, a, b);
    if (s == a) return 4.0 * lam[b];
    if (s == b) return 4.0 * lam[a];
    return 0.0;
}

double p2_phi(int dim, int p, const double *lam) {
    if (p <= dim) return lam[p] * (2.0 * lam[p] - 1.0);
    int a, b;
    p2_edges(dim, p - dim - 1, a, b);
    return 4.0 * lam[a] * lam[b];
}

void build_p2_table(int dim, P2Tab &T) {
    const int n = dim == 2 ? 6 : 10, nv = dim + 1;
    // stiffness rule: 4 points, weights normalised to sum 1
    std::vector<std::vector<double>> pts;
    std::vector<double> wts;
    if (dim == 3) {
        const double a = 0.5854101966249685, b = 0.1381966011250105;
        for (int i = 0; i < 4; ++i) {
            std::vector<double> l(4, b);
            l[i] = a;
            pts.push_back(l);
            wts.push_back(0.25);
        }
    } else {
        pts.push_back({1.0 / 3, 1.0 / 3, 1.0 / 3});
        wts.push_back(-27.0 / 48.0);
        for (int i = 0; i < 3; ++i) {
            std::vector<double> l(3, 0.2);
            l[i] = 0.6;
            pts.push_back(l);
            wts.push_back(25.0 / 48.0);
        }
    }
    std::memset(&T, 0, sizeof(T));
    for (int p = 0; p < n; ++p)
        for (int q = p; q < n; ++q) {
            int u = packed_index(p, q, n);
            double acc[16] = {0};
            for (int s = 0; s < nv; ++s)
                for (int t = 0; t < nv; ++t)
                    for (size_t g = 0; g < pts.size(); ++g)
                        acc[std::min(s, t) * nv + std::max(s, t)] +=
                            wts[g] * p2_dphi(dim, p, s, pts[g].data()) * p2_dphi(dim, q, t, pts[g].data());
            int nt = 0;
            for (int s = 0; s < nv; ++s)
                for (int t = s; t < nv; ++t) {
                    double v = acc[s * nv + t];
                    if (std::fabs(v) < 1e-14) continue;
                    T.st[u][nt] = (unsigned char)packed_index(s, t, nv);
                    T.coef_d[u][nt] = v;
                    T.coef_f[u][nt] = (float)v;
                    ++nt;
                }
            T.nterm[u] = (unsigned char)nt;
        }
    // mass: collapsed Gauss-Legendre product rule (4 points per direction),
    // exact for the quartic integrand; normalised by the reference measure
    const double gx[4] = {-0.8611363115940526, -0.3399810435848563, 0.3399810435848563, 0.8611363115940526};
    const double gw[4] = {0.3478548451374538, 0.6521451548625461, 0.6521451548625461, 0.3478548451374538};
    double M[10][10] = {{0}};
    double refvol = dim == 2 ? 0.5 : 1.0 / 6.0;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j)
            for (int k = 0; k < (dim == 3 ? 4 : 1); ++k) {
                double a = 0.5 * (gx[i] + 1), b = 0.5 * (gx[j] + 1), c = 0.5 * (gx[k] + 1);
                double xi[3], w;
                if (dim == 2) {
                    xi[0] = a;
                    xi[1] = b * (1 - a);
                    w = 0.25 * gw[i] * gw[j] * (1 - a);
                } else {
                    xi[0] = a;
                    xi[1] = b * (1 - a);
                    xi[2] = c * (1 - a) * (1 - b);
                    w = 0.125 * gw[i] * gw[j] * gw[k] * (1 - a) * (1 - a) * (1 - b);
                }
                double lam[4];
                double sum = 0;
                for (int d = 0; d < dim; ++d) {
                    lam[d] = xi[d];
                    sum += xi[d];
                }
                lam[dim] = 1 - sum;
                for (int p = 0; p < n; ++p)
                    for (int q = 0; q < n; ++q) M[p][q] += w * p2_phi(dim, p, lam) * p2_phi(dim, q, lam);
            }
    for (int p = 0; p < n; ++p)
        for (int q = p; q < n; ++q) {
            int u = packed_index(p, q, n);
            T.mhat_d[u] = M[p][q] / refvol;
            T.mhat_f[u] = (float)T.mhat_d[u];
        }
}

std::mutex g_tab_mu;
bool g_tab_done[64] = {false};

vla_status ensure_p2_tables() {
    int dev = 0;
    VLA_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(VLA_ERR_INVALID_ARG, "device ordinal %d not supported", dev);
    std::lock_guard<std::mutex> lk(g_tab_mu);
    if (g_tab_done[dev]) return VLA_OK;
    P2Tab t[2];
    build_p2_table(2, t[0]);
    build_p2_table(3, t[1]);
    VLA_CUDA(cudaMemcpyToSymbol(c_p2, t, sizeof(t)));
    g_tab_done[dev] = true;
    return VLA_OK;
}

// ---------------------------------------------------------------------------
// element geometry
// ---------------------------------------------------------------------------
template <typename T>
struct Geo {
    T C[4][3];   // cofactor vectors (C_d = -sum)
    T det;       // signed det V (rounded)
    T xc[3];     // vertex centroid
};

// exact difference a - b = s + e (TwoSum with a negated operand)
__device__ __forceinline__ void two_diff(float a, float b, float &s, float &e) { two_sum(a, -b, s, e); }

// Mixed precision, 3-D.  V = Vh + Vl is the edge vector as a normalised
// float pair (Vh = fl(V), |Vl| <= ulp(Vh)/2), built error-free from the
// coordinate pairs; det V =
// det(Vh) (evaluated with an error-free cross product and a compensated dot
// product) + sum_j Vl_j . C_j (first-order correction; the remainder is
// O(|Vl|^2) ~ 2^-48 relative).
__device__ __forceinline__ void geo_mixed3(const float4 *__restrict__ sh, const float4 *__restrict__ sl, ushort4 v,
                                           Geo<float> &g) {
    const float4 h3 = sh[v.w], l3 = sl[v.w];
    float Vh[3][3], Vl[3][3];
    const unsigned short vi[3] = {v.x, v.y, v.z};
    float hs[3] = {h3.x, h3.y, h3.z};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float4 hj = sh[vi[j]], lj = sl[vi[j]];
        const float hjc[3] = {hj.x, hj.y, hj.z}, ljc[3] = {lj.x, lj.y, lj.z}, h3c[3] = {h3.x, h3.y, h3.z},
                    l3c[3] = {l3.x, l3.y, l3.z};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float s, e;
            two_diff(hjc[c], h3c[c], s, e);
            // renormalise so that |Vl| <= ulp(Vh)/2 even far from the origin,
            // where the lo parts are not small next to the edge length
            two_sum(s, __fadd_rn(e, __fsub_rn(ljc[c], l3c[c])), Vh[j][c], Vl[j][c]);
        }
        hs[0] += hj.x;
        hs[1] += hj.y;
        hs[2] += hj.z;
    }
    // C0 = Vh1 x Vh2 in float-float (exact products, one rounding in t)
    float s0[3], t0[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
        float p1, e1, p2, e2, s, es;
        two_prod(Vh[1][c1], Vh[2][c2], p1, e1);
        two_prod(Vh[1][c2], Vh[2][c1], p2, e2);
        two_sum(p1, -p2, s, es);
        s0[c] = s;
        t0[c] = __fadd_rn(es, __fsub_rn(e1, e2));
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
        g.C[0][c] = __fadd_rn(s0[c], t0[c]);
        g.C[1][c] = det2_kahan(Vh[2][c1], Vh[2][c2], Vh[0][c1], Vh[0][c2]);  // Vh2 x Vh0
        g.C[2][c] = det2_kahan(Vh[0][c1], Vh[0][c2], Vh[1][c1], Vh[1][c2]);  // Vh0 x Vh1
        g.C[3][c] = -((g.C[0][c] + g.C[1][c]) + g.C[2][c]);
    }
    // det(Vh) = Vh0 . (s0 + t0), compensated
    float P, E;
    two_prod(Vh[0][0], s0[0], P, E);
    float err = __fmaf_rn(Vh[0][0], t0[0], E);
#pragma unroll
    for (int c = 1; c < 3; ++c) {
        float p, e, q;
        two_prod(Vh[0][c], s0[c], p, e);
        two_sum(P, p, P, q);
        err = __fadd_rn(err, __fadd_rn(q, __fmaf_rn(Vh[0][c], t0[c], e)));
    }
    // first-order correction from Vl
    float corr = 0.f;
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int c = 0; c < 3; ++c) corr = __fmaf_rn(Vl[j][c], g.C[j][c], corr);
    g.det = __fadd_rn(P, __fadd_rn(err, corr));
    g.xc[0] = hs[0] * 0.25f;
    g.xc[1] = hs[1] * 0.25f;
    g.xc[2] = hs[2] * 0.25f;
}

// Mixed precision, 2-D.  C0 = (V1y, -V1x), C1 = (-V0y, V0x) (rows of adj V).
__device__ __forceinline__ void geo_mixed2(const float4 *__restrict__ sh, const float4 *__restrict__ sl, ushort4 v,
                                           Geo<float> &g) {
    const float4 h2 = sh[v.z], l2 = sl[v.z];
    float Vh[2][2], Vl[2][2];
    const unsigned short vi[2] = {v.x, v.y};
    float hs[2] = {h2.x, h2.y};
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const float4 hj = sh[vi[j]], lj = sl[vi[j]];
        float s, e;
        two_diff(hj.x, h2.x, s, e);
        two_sum(s, __fadd_rn(e, __fsub_rn(lj.x, l2.x)), Vh[j][0], Vl[j][0]);
        two_diff(hj.y, h2.y, s, e);
        two_sum(s, __fadd_rn(e, __fsub_rn(lj.y, l2.y)), Vh[j][1], Vl[j][1]);
        hs[0] += hj.x;
        hs[1] += hj.y;
    }
    g.C[0][0] = Vh[1][1];
    g.C[0][1] = -Vh[1][0];
    g.C[1][0] = -Vh[0][1];
    g.C[1][1] = Vh[0][0];
    g.C[2][0] = -(g.C[0][0] + g.C[1][0]);
    g.C[2][1] = -(g.C[0][1] + g.C[1][1]);
    g.C[0][2] = g.C[1][2] = g.C[2][2] = g.C[3][0] = g.C[3][1] = g.C[3][2] = 0.f;
    float p1, e1, p2, e2, s, es;
    two_prod(Vh[0][0], Vh[1][1], p1, e1);
    two_prod(Vh[0][1], Vh[1][0], p2, e2);
    two_sum(p1, -p2, s, es);
    float corr = 0.f;
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int c = 0; c < 2; ++c) corr = __fmaf_rn(Vl[j][c], g.C[j][c], corr);
    g.det = __fadd_rn(s, __fadd_rn(__fadd_rn(es, __fsub_rn(e1, e2)), corr));
    g.xc[0] = hs[0] * (1.0f / 3.0f);
    g.xc[1] = hs[1] * (1.0f / 3.0f);
    g.xc[2] = 0.f;
}

// FP64, 3-D and 2-D (coordinates as double4 in shared memory).
template <int DIM>
__device__ __forceinline__ void geo_f64(const double4 *__restrict__ sx, ushort4 v, Geo<double> &g) {
    const unsigned short vi[4] = {v.x, v.y, v.z, v.w};
    const double4 xl = sx[vi[DIM]];
    double V[3][3];
    double cs[3] = {xl.x, xl.y, xl.z};
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
        const double4 xj = sx[vi[j]];
        V[j][0] = xj.x - xl.x;
        V[j][1] = xj.y - xl.y;
        V[j][2] = xj.z - xl.z;
        cs[0] += xj.x;
        cs[1] += xj.y;
        cs[2] += xj.z;
    }
    if (DIM == 3) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
            g.C[0][c] = V[1][c1] * V[2][c2] - V[1][c2] * V[2][c1];
            g.C[1][c] = V[2][c1] * V[0][c2] - V[2][c2] * V[0][c1];
            g.C[2][c] = V[0][c1] * V[1][c2] - V[0][c2] * V[1][c1];
            g.C[3][c] = -((g.C[0][c] + g.C[1][c]) + g.C[2][c]);
        }
        g.det = V[0][0] * g.C[0][0] + V[0][1] * g.C[0][1] + V[0][2] * g.C[0][2];
        g.xc[0] = cs[0] * 0.25;
        g.xc[1] = cs[1] * 0.25;
        g.xc[2] = cs[2] * 0.25;
    } else {
        g.C[0][0] = V[1][1];
        g.C[0][1] = -V[1][0];
        g.C[1][0] = -V[0][1];
        g.C[1][1] = V[0][0];
        g.C[2][0] = -(g.C[0][0] + g.C[1][0]);
        g.C[2][1] = -(g.C[0][1] + g.C[1][1]);
        g.C[0][2] = g.C[1][2] = g.C[2][2] = g.C[3][0] = g.C[3][1] = g.C[3][2] = 0.0;
        g.det = V[0][0] * V[1][1] - V[0][1] * V[1][0];
        g.xc[0] = cs[0] / 3.0;
        g.xc[1] = cs[1] / 3.0;
        g.xc[2] = 0.0;
    }
}

template <typename T>
__device__ __forceinline__ T coeff(int kind, T ca, T cb, const T *xc, int dim) {
    if (kind == VLA_COEFF_EXP) {
        T s = xc[0] + xc[1] + (dim == 3 ? xc[2] : T(0));
        if constexpr (sizeof(T) == 4) return ca * expf(cb * s);
        else return ca * exp(cb * s);
    }
    T r2 = xc[0] * xc[0] + xc[1] * xc[1] + (dim == 3 ? xc[2] * xc[2] : T(0));
    return ca + cb * r2;
}

template <typename T>
__device__ __forceinline__ T dot3(const T *a, const T *b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// Mixed precision fast path: edge vectors rounded once to float, Kahan 2x2
// cofactors, plain dot for det.  The det error is below ~8u perm(|V|); if
// |det| < perm(|V|)/32 (a flat or sliver element) the exact float-pair path
// recomputes the geometry.
__device__ __forceinline__ void geo_mixed3_fast(const float4 *__restrict__ sh, const float4 *__restrict__ sl,
                                                ushort4 v, Geo<float> &g) {
    const float4 h3 = sh[v.w], l3 = sl[v.w];
    const unsigned short vi[3] = {v.x, v.y, v.z};
    float V[3][3];
    float sx = h3.x, sy = h3.y, sz = h3.z;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const float4 hj = sh[vi[j]], lj = sl[vi[j]];
        V[j][0] = __fadd_rn(__fsub_rn(hj.x, h3.x), __fsub_rn(lj.x, l3.x));
        V[j][1] = __fadd_rn(__fsub_rn(hj.y, h3.y), __fsub_rn(lj.y, l3.y));
        V[j][2] = __fadd_rn(__fsub_rn(hj.z, h3.z), __fsub_rn(lj.z, l3.z));
        sx += hj.x;
        sy += hj.y;
        sz += hj.z;
    }
    float perm = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
        // fast path: one FMA per cofactor; the exact path below takes over
        // whenever cancellation could matter (|det| small against perm(|V|))
        const float p12 = V[1][c2] * V[2][c1], p20 = V[2][c2] * V[0][c1], p01 = V[0][c2] * V[1][c1];
        g.C[0][c] = fmaf(V[1][c1], V[2][c2], -p12);
        g.C[1][c] = fmaf(V[2][c1], V[0][c2], -p20);
        g.C[2][c] = fmaf(V[0][c1], V[1][c2], -p01);
        g.C[3][c] = -((g.C[0][c] + g.C[1][c]) + g.C[2][c]);
        perm = fmaf(fabsf(V[0][c]), fabsf(V[1][c1] * V[2][c2]) + fabsf(p12), perm);
    }
    g.det = fmaf(V[0][0], g.C[0][0], fmaf(V[0][1], g.C[0][1], V[0][2] * g.C[0][2]));
    g.xc[0] = sx * 0.25f;
    g.xc[1] = sy * 0.25f;
    g.xc[2] = sz * 0.25f;
    if (fabsf(g.det) < 0.03125f * perm) geo_mixed3(sh, sl, v, g);
}

__device__ __forceinline__ void geo_mixed2_fast(const float4 *__restrict__ sh, const float4 *__restrict__ sl,
                                                ushort4 v, Geo<float> &g) {
    const float4 h2 = sh[v.z], l2 = sl[v.z];
    const float4 h0 = sh[v.x], l0 = sl[v.x], h1 = sh[v.y], l1 = sl[v.y];
    const float V00 = __fadd_rn(__fsub_rn(h0.x, h2.x), __fsub_rn(l0.x, l2.x));
    const float V01 = __fadd_rn(__fsub_rn(h0.y, h2.y), __fsub_rn(l0.y, l2.y));
    const float V10 = __fadd_rn(__fsub_rn(h1.x, h2.x), __fsub_rn(l1.x, l2.x));
    const float V11 = __fadd_rn(__fsub_rn(h1.y, h2.y), __fsub_rn(l1.y, l2.y));
    g.C[0][0] = V11;
    g.C[0][1] = -V10;
    g.C[1][0] = -V01;
    g.C[1][1] = V00;
    g.C[2][0] = -(V11 - V01);
    g.C[2][1] = -(V00 - V10);
    g.C[0][2] = g.C[1][2] = g.C[2][2] = g.C[3][0] = g.C[3][1] = g.C[3][2] = 0.f;
    g.det = det2_kahan(V00, V01, V10, V11);
    g.xc[0] = (h0.x + h1.x + h2.x) * (1.0f / 3.0f);
    g.xc[1] = (h0.y + h1.y + h2.y) * (1.0f / 3.0f);
    g.xc[2] = 0.f;
    if (fabsf(g.det) < 0.03125f * (fabsf(V00 * V11) + fabsf(V01 * V10))) geo_mixed2(sh, sl, v, g);
}

// ---------------------------------------------------------------------------
// compile-time configuration
// ---------------------------------------------------------------------------
template <int DIM, int ORDER, bool MIX>
struct Cfg {
    static constexpr int NV = DIM + 1;
    static constexpr int NLB = ORDER == 1 ? DIM + 1 : (DIM + 1) * (DIM + 2) / 2;
    static constexpr int NU = NLB * (NLB + 1) / 2;            // packed upper triangle
    static constexpr int RS = (NU + 1 + 3) / 4 * 4;            // record: NU entries, mass scale, padding
    static constexpr int UB = ORDER == 1 ? 4 : 8;              // code = element << UB | entry
    using T = typename std::conditional<MIX, float, double>::type;
    using CT = typename std::conditional<ORDER == 1, uint16_t, uint32_t>::type;
    static constexpr double DFACT = DIM == 3 ? 6.0 : 2.0;      // dim!
    static constexpr double MOFF = 1.0 / ((DIM + 1) * (DIM + 2));   // P1 off-diagonal mass / (c |T|)
};

struct AsmArgs {
    const vla::TileHdr *tiles;
    const int32_t *tile_nodes;
    const ushort4 *tile_elem;
    const int32_t *tile_own;
    const int2 *tile_nzpos;
    const int2 *tile_chunks;
    const void *codes;
    const float4 *xh, *xl;
    const double *coords;
    int n_tiles;
    int kind;
    double ca, cb;
    float caf, cbf;
    double *K, *M, *vol, *Kp, *Mp;
    unsigned long long *n_sing;
    int *err;
    int spin_limit;
    int stage_bytes;       // bytes of one input stage (segments + coordinates), 16-byte multiple
};

__host__ __device__ constexpr int padq(int x, int q) { return (x + q - 1) / q * q; }

// byte offsets of the staged segments of one tile inside a stage
struct StageMap {
    int ids, rec, gid, chk, nz, cod, xyz, end;
};
template <typename CT>
__device__ __forceinline__ StageMap stage_map(const vla::TileHdr &h) {
    StageMap m;
    m.ids = 0;
    m.rec = m.ids + 4 * padq(h.n_nodes, kTilePadNodes);
    m.gid = m.rec + 8 * padq(h.n_elems, kTilePadElems);
    m.chk = m.gid + 4 * padq(h.n_own, kTilePadOwn);
    m.nz = m.chk + 8 * padq(h.n_chunks, kTilePadChunks);
    m.cod = m.nz + 8 * padq(h.n_nz, kTilePadNz);
    m.xyz = m.cod + padq((int)sizeof(CT) * h.n_codes, 16);
    m.end = m.xyz + 32 * h.n_nodes;
    return m;
}

// packed f32x2 arithmetic (sm_100+): the K and M sums of a pair advance together
__device__ __forceinline__ unsigned long long pk(float a, float b) {
    unsigned long long d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(a), "f"(b));
    return d;
}
__device__ __forceinline__ void upk(unsigned long long d, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(d));
}
__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
// (hi, lo) += x, error-free on both lanes (TwoSum)
__device__ __forceinline__ void ff2_add(unsigned long long &hi, unsigned long long &lo, unsigned long long x) {
    const unsigned long long s = add2(hi, x);
    const unsigned long long bb = sub2(s, hi);
    const unsigned long long e = add2(sub2(hi, sub2(s, bb)), sub2(x, bb));
    hi = s;
    lo = add2(lo, e);
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Persistent CTA: tiles blockIdx.x, +gridDim.x, ...  Two input stages: while
// tile j is computed from stage j&1, the bulk copies of tile j+2 and the
// coordinate gathers (cp.async) of tile j+1 are in flight.
template <int DIM, int ORDER, bool MIX>
__global__ void __launch_bounds__(kThreads) k_assemble(AsmArgs A) {
    using C = Cfg<DIM, ORDER, MIX>;
    using T = typename C::T;
    using CT = typename C::CT;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int next_chunk[2];   // dynamic chunk counters, one per tile parity
    __shared__ vla::TileHdr s_hdr[2];   // header and segment map of the tile in each stage
    __shared__ StageMap s_map[2];
    if (threadIdx.x == 0) {
        next_chunk[0] = kThreads / 32;
        next_chunk[1] = kThreads / 32;
    }
    auto stage = [&](int st_) { return smem + (size_t)st_ * A.stage_bytes; };
    T *s_k = reinterpret_cast<T *>(smem + 2 * (size_t)A.stage_bytes);
    __shared__ T mhat[ORDER == 2 ? C::NU : 1];
    if constexpr (ORDER == 2) {
        for (int u = threadIdx.x; u < C::NU; u += kThreads)
            mhat[u] = MIX ? (T)c_p2[DIM - 2].mhat_f[u] : (T)c_p2[DIM - 2].mhat_d[u];
    }
    const int G = gridDim.x;
    int issued0 = 0, issued1 = 0;   // thread 0: loads issued per stage

    auto issue = [&](int t, int s) {   // thread 0 only
        const vla::TileHdr h = A.tiles[t];
        const StageMap mp = stage_map<CT>(h);
        s_hdr[s] = h;
        s_map[s] = mp;
        unsigned char *b = stage(s);
        mbar_expect_tx(&bar[s], (uint32_t)mp.xyz);
        if (mp.rec > mp.ids) bulk_g2s(b + mp.ids, A.tile_nodes + h.node_off, (uint32_t)(mp.rec - mp.ids), &bar[s]);
        if (mp.gid > mp.rec) bulk_g2s(b + mp.rec, A.tile_elem + h.elem_off, (uint32_t)(mp.gid - mp.rec), &bar[s]);
        if (mp.chk > mp.gid) bulk_g2s(b + mp.gid, A.tile_own + h.own_off, (uint32_t)(mp.chk - mp.gid), &bar[s]);
        if (mp.nz > mp.chk) bulk_g2s(b + mp.chk, A.tile_chunks + h.chunk_off, (uint32_t)(mp.nz - mp.chk), &bar[s]);
        if (mp.cod > mp.nz) bulk_g2s(b + mp.nz, A.tile_nzpos + h.nz_off, (uint32_t)(mp.cod - mp.nz), &bar[s]);
        if (mp.xyz > mp.cod)
            bulk_g2s(b + mp.cod, reinterpret_cast<const CT *>(A.codes) + h.code_off, (uint32_t)(mp.xyz - mp.cod), &bar[s]);
        if (s) ++issued1;
        else ++issued0;
    };
    // coordinate gathers of tile t into stage s (all threads, asynchronous)
    auto gather = [&](int t, int s) {
        const vla::TileHdr &h = s_hdr[s];
        const StageMap &mp = s_map[s];
        const int32_t *ids = reinterpret_cast<const int32_t *>(stage(s) + mp.ids);
        unsigned char *xyz = stage(s) + mp.xyz;
        for (int i = threadIdx.x; i < h.n_nodes; i += kThreads) {
            const int32_t g = ids[i];
            if constexpr (MIX) {
                cp_async16(xyz + 16 * i, A.xh + g);
                cp_async16(xyz + 16 * (h.n_nodes + i), A.xl + g);
            } else {
                double *dst = reinterpret_cast<double *>(xyz + 32 * i);
#pragma unroll
                for (int d = 0; d < DIM; ++d) cp_async8(dst + d, A.coords + (int64_t)g * DIM + d);
                if (DIM == 2) dst[2] = 0.0;
            }
        }
        cp_async_commit();
    };
    auto bail = [&]() {   // a bounded wait expired: record it, let copies in flight land, leave
        if (threadIdx.x == 0) {
            atomicOr(A.err, 1);
            if (issued0) mbar_wait_bounded(&bar[0], (uint32_t)((issued0 - 1) & 1), 1 << 24);
            if (issued1) mbar_wait_bounded(&bar[1], (uint32_t)((issued1 - 1) & 1), 1 << 24);
        }
        cp_async_wait_all();
    };

    const int t0 = blockIdx.x;
    if (t0 >= A.n_tiles) return;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_async_smem();
        issue(t0, 0);
        if (t0 + G < A.n_tiles) issue(t0 + G, 1);
    }
    __syncthreads();
    if (__syncthreads_or(!mbar_wait_bounded(&bar[0], 0, A.spin_limit))) {
        bail();
        return;
    }
    gather(t0, 0);

    const T ca = MIX ? (T)A.caf : (T)A.ca, cb = MIX ? (T)A.cbf : (T)A.cb;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr uint32_t UMASK = (1u << C::UB) - 1;
    unsigned long long sing = 0;

    for (int j = 0;; ++j) {
        const int t = t0 + j * G;
        if (t >= A.n_tiles) break;
        const int s = j & 1;
        const vla::TileHdr h = s_hdr[s];
        const StageMap mp = s_map[s];
        unsigned char *b = stage(s);
        const ushort4 *s_rec = reinterpret_cast<const ushort4 *>(b + mp.rec);
        const int32_t *s_gid = reinterpret_cast<const int32_t *>(b + mp.gid);
        const int2 *s_chk = reinterpret_cast<const int2 *>(b + mp.chk);
        const int2 *s_nz = reinterpret_cast<const int2 *>(b + mp.nz);
        const CT *s_cod = reinterpret_cast<const CT *>(b + mp.cod);
        const float4 *s_h = reinterpret_cast<const float4 *>(b + mp.xyz);
        const float4 *s_l = s_h + h.n_nodes;
        const double4 *s_x = reinterpret_cast<const double4 *>(b + mp.xyz);
        cp_async_wait_all();   // this thread's coordinate copies of tile t
        __syncthreads();       // everyone's

        // phase 1: element records (index n_elems is the zero record used by padding)
        for (int e = threadIdx.x; e <= h.n_elems; e += kThreads) {
            T *dst = s_k + (size_t)e * C::RS;
            if (e == h.n_elems) {
                for (int u = 0; u < C::RS; ++u) dst[u] = T(0);
                continue;
            }
            const ushort4 v = s_rec[e];
            Geo<T> g;
            if constexpr (MIX) {
                if constexpr (DIM == 3) geo_mixed3_fast(s_h, s_l, v, g);
                else geo_mixed2_fast(s_h, s_l, v, g);
            } else {
                geo_f64<DIM>(s_x, v, g);
            }
            const T c = coeff<T>(A.kind, ca, cb, g.xc, DIM);
            const T adet = g.det < T(0) ? -g.det : g.det;
            T sc;
            if constexpr (MIX) sc = c * __frcp_rn(T(C::DFACT) * adet);   // K(a,b) = sc * C_a . C_b
            else sc = c / (T(C::DFACT) * adet);
            T mscale;
            if constexpr (ORDER == 1) {
                T rec[C::RS];
#pragma unroll
                for (int u = 0; u < C::RS; ++u) rec[u] = T(0);
#pragma unroll
                for (int a = 0; a < C::NV; ++a)
#pragma unroll
                    for (int q = a; q < C::NV; ++q) rec[a * C::NLB - a * (a - 1) / 2 + (q - a)] = sc * dot3<T>(g.C[a], g.C[q]);
                mscale = c * adet * T(C::MOFF / C::DFACT);       // off-diagonal mass entry
                rec[C::NU] = mscale;
                if constexpr (MIX) {
#pragma unroll
                    for (int u = 0; u < C::RS; u += 4)
                        *reinterpret_cast<float4 *>(dst + u) = make_float4(rec[u], rec[u + 1], rec[u + 2], rec[u + 3]);
                } else {
#pragma unroll
                    for (int u = 0; u < C::RS; u += 2)
                        *reinterpret_cast<double2 *>(dst + u) = make_double2(rec[u], rec[u + 1]);
                }
            } else {
                T cd[10];
#pragma unroll
                for (int a = 0; a < C::NV; ++a)
#pragma unroll
                    for (int q = a; q < C::NV; ++q) cd[a * C::NV - a * (a - 1) / 2 + (q - a)] = dot3<T>(g.C[a], g.C[q]);
                const P2Tab &tb = c_p2[DIM - 2];
                for (int u = 0; u < C::NU; ++u) {
                    T acc = 0;
                    const int nt = tb.nterm[u];
                    for (int q = 0; q < nt; ++q) {
                        const T cf = MIX ? (T)tb.coef_f[u][q] : (T)tb.coef_d[u][q];
                        acc += cf * cd[tb.st[u][q]];
                    }
                    dst[u] = sc * acc;
                }
                mscale = c * adet * T(1.0 / C::DFACT);           // c |T|; entries scale the reference mass
                dst[C::NU] = mscale;
            }
            if (e < h.n_own) {
                const int64_t k = s_gid[e];
                if (g.det == T(0)) ++sing;
                if (A.vol) {
                    if constexpr (MIX) A.vol[k] = f32_to_f64(adet * (float)(1.0 / C::DFACT));
                    else A.vol[k] = adet / C::DFACT;
                }
                if (A.Kp || A.Mp) {
                    for (int a = 0; a < C::NLB; ++a)
                        for (int q = 0; q < C::NLB; ++q) {
                            const int p0 = a < q ? a : q, p1 = a < q ? q : a;
                            const int u = p0 * C::NLB - p0 * (p0 - 1) / 2 + (p1 - p0);
                            const int64_t pos = k * C::NLB * C::NLB + a + (int64_t)q * C::NLB;
                            const T kv = dst[u];
                            T mv;
                            if constexpr (ORDER == 1) mv = mscale * (a == q ? T(2) : T(1));
                            else mv = mscale * mhat[u];
                            if constexpr (MIX) {
                                if (A.Kp) A.Kp[pos] = f32_to_f64(kv);
                                if (A.Mp) A.Mp[pos] = f32_to_f64(mv);
                            } else {
                                if (A.Kp) A.Kp[pos] = kv;
                                if (A.Mp) A.Mp[pos] = mv;
                            }
                        }
                }
            }
        }
        // prefetch: coordinates of the next tile (its bulk copies were issued two tiles ago)
        const int tn = t + G;
        if (tn < A.n_tiles) {
            if (__syncthreads_or(!mbar_wait_bounded(&bar[s ^ 1], (uint32_t)(((j + 1) >> 1) & 1), A.spin_limit))) {
                bail();
                return;
            }
            gather(tn, s ^ 1);
        } else {
            __syncthreads();
        }

        // phase 2: pairs sorted by contribution count, 32 per warp-chunk,
        // contributions in ascending element order
        if (A.K || A.M) {
            // chunks are handed out dynamically: they are sorted by width, so a
            // static round-robin would give the first warps all the long ones
            for (int c = warp;;) {
                if (c >= h.n_chunks) break;
                const int q = c * 32 + lane;
                const int2 ch = s_chk[c];
                const CT *cp = s_cod + ch.x + lane;
                if constexpr (MIX) {
                    unsigned long long h0 = 0ull, l0 = 0ull, h1 = 0ull, l1 = 0ull;   // (K, M) pairs, 2 chains
                    int tt = 0;
                    for (; tt + 1 < ch.y; tt += 2) {
                        const uint32_t c0 = cp[tt * 32], c1 = cp[(tt + 1) * 32];
                        const float *r0 = s_k + (c0 >> C::UB) * C::RS, *r1 = s_k + (c1 >> C::UB) * C::RS;
                        float m0 = r0[C::NU], m1 = r1[C::NU];
                        if constexpr (ORDER == 2) {
                            m0 *= mhat[c0 & UMASK];
                            m1 *= mhat[c1 & UMASK];
                        }
                        ff2_add(h0, l0, pk(r0[c0 & UMASK], m0));
                        ff2_add(h1, l1, pk(r1[c1 & UMASK], m1));
                    }
                    if (tt < ch.y) {
                        const uint32_t c0 = cp[tt * 32];
                        const float *r0 = s_k + (c0 >> C::UB) * C::RS;
                        float m0 = r0[C::NU];
                        if constexpr (ORDER == 2) m0 *= mhat[c0 & UMASK];
                        ff2_add(h0, l0, pk(r0[c0 & UMASK], m0));
                    }
                    if (q < h.n_nz) {
                        ff2_add(h0, l0, h1);
                        ff2_add(h0, l0, l1);
                        // renormalise both sums at once: (hi, lo) <- TwoSum(hi, lo)
                        const unsigned long long s2 = add2(h0, l0);
                        const unsigned long long bb = sub2(s2, h0);
                        const unsigned long long e2 = add2(sub2(h0, sub2(s2, bb)), sub2(l0, bb));
                        float khi, mhi, klo, mlo;
                        upk(s2, khi, mhi);
                        upk(e2, klo, mlo);
                        const int2 pos = s_nz[q];
                        if (ORDER == 1 && pos.x == pos.y) {   // P1 diagonal mass: twice the off-diagonal scale
                            mhi *= 2.f;
                            mlo *= 2.f;
                        }
                        const double kd = ff_to_f64(khi, klo), md = ff_to_f64(mhi, mlo);
                        if (A.K) {
                            A.K[pos.x] = kd;
                            if (pos.y != pos.x) A.K[pos.y] = kd;
                        }
                        if (A.M) {
                            A.M[pos.x] = md;
                            if (pos.y != pos.x) A.M[pos.y] = md;
                        }
                    }
                } else {
                    double ks = 0.0, ms = 0.0;
                    for (int tt = 0; tt < ch.y; ++tt) {
                        const uint32_t c0 = cp[tt * 32];
                        const double *r0 = s_k + (c0 >> C::UB) * C::RS;
                        ks += r0[c0 & UMASK];
                        if constexpr (ORDER == 2) ms += r0[C::NU] * mhat[c0 & UMASK];
                        else ms += r0[C::NU];
                    }
                    if (q < h.n_nz) {
                        const int2 pos = s_nz[q];
                        if (ORDER == 1 && pos.x == pos.y) ms *= 2.0;
                        if (A.K) {
                            A.K[pos.x] = ks;
                            if (pos.y != pos.x) A.K[pos.y] = ks;
                        }
                        if (A.M) {
                            A.M[pos.x] = ms;
                            if (pos.y != pos.x) A.M[pos.y] = ms;
                        }
                    }
                }
                int nc = 0;
                if (lane == 0) nc = atomicAdd(&next_chunk[j & 1], 1);
                c = __shfl_sync(0xffffffffu, nc, 0);
            }
        }
        if (threadIdx.x == 0) next_chunk[(j + 1) & 1] = kThreads / 32;   // reset for the next tile
        __syncthreads();   // stage s and the element records are free
        if (threadIdx.x == 0 && t + 2 * G < A.n_tiles) issue(t + 2 * G, s);
    }
    if (A.n_sing && sing) atomicAdd(A.n_sing, sing);
}

template <int DIM, int ORDER, bool MIX>
size_t asm_smem(const vla_mesh *m, int &stage_bytes) {
    using C = Cfg<DIM, ORDER, MIX>;
    stage_bytes = (int)((m->tile_stage_bytes + 32 * (size_t)m->max_tile_nodes + 16 + 15) / 16 * 16);
    return 2 * (size_t)stage_bytes + ((size_t)m->max_tile_elems + 1) * C::RS * sizeof(typename C::T);
}

template <int DIM, int ORDER, bool MIX>
vla_status launch_assemble(const vla_mesh *m, AsmArgs a, cudaStream_t st) {
    int stage_bytes = 0;
    const size_t smem = asm_smem<DIM, ORDER, MIX>(m, stage_bytes);
    a.stage_bytes = stage_bytes;
    int dev = 0, maxsm = 0, nsm = 0;
    VLA_CUDA(cudaGetDevice(&dev));
    VLA_CUDA(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    VLA_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    if (smem + 1024 > (size_t)maxsm)
        return fail(VLA_ERR_UNSUPPORTED, "assembly tile needs %zu bytes of shared memory (limit %d)", smem, maxsm);
    auto kern = k_assemble<DIM, ORDER, MIX>;
    VLA_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    VLA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
    if (per_sm < 1) per_sm = 1;
    int grid = nsm * per_sm;
    if (grid > m->n_tiles) grid = m->n_tiles;
    kern<<<grid, kThreads, smem, st>>>(a);
    VLA_CUDA(cudaGetLastError());
    return VLA_OK;
}

// ---------------------------------------------------------------------------
// boundary facets
// ---------------------------------------------------------------------------
__global__ void k_boundary_f64(int64_t nfb, int dim, const double *__restrict__ x, const int32_t *__restrict__ faces,
                               const int32_t *__restrict__ opp, double *__restrict__ nrm, double *__restrict__ area) {
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < nfb; f += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = faces[f * dim], b = faces[f * dim + 1];
        const int32_t o = opp[f];
        double n[3] = {0, 0, 0}, meas;
        const double *x1 = x + (int64_t)a * dim, *x2 = x + (int64_t)b * dim, *xo = x + (int64_t)o * dim;
        if (dim == 3) {
            const double *x3 = x + (int64_t)faces[f * dim + 2] * dim;
            double u[3], w[3];
            for (int d = 0; d < 3; ++d) {
                u[d] = x2[d] - x1[d];
                w[d] = x3[d] - x1[d];
            }
            n[0] = u[1] * w[2] - u[2] * w[1];
            n[1] = u[2] * w[0] - u[0] * w[2];
            n[2] = u[0] * w[1] - u[1] * w[0];
        } else {
            n[0] = x2[1] - x1[1];
            n[1] = -(x2[0] - x1[0]);
        }
        const double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        meas = dim == 3 ? 0.5 * len : len;
        double side = 0;
        for (int d = 0; d < dim; ++d) side += n[d] * (xo[d] - x1[d]);
        const double sg = side > 0 ? -1.0 : 1.0;
        for (int d = 0; d < dim; ++d) nrm[f * dim + d] = sg * n[d] / len;
        area[f] = meas;
    }
}

__global__ void k_boundary_mixed(int64_t nfb, int dim, const float4 *__restrict__ xh, const float4 *__restrict__ xl,
                                 const int32_t *__restrict__ faces, const int32_t *__restrict__ opp,
                                 double *__restrict__ nrm, double *__restrict__ area) {
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < nfb; f += (int64_t)gridDim.x * blockDim.x) {
        const int32_t ia = faces[f * dim], ib = faces[f * dim + 1], io = opp[f];
        const float4 ha = xh[ia], la = xl[ia], hb = xh[ib], lb = xl[ib], ho = xh[io], lo = xl[io];
        auto dif = [](float h1, float l1, float h0, float l0) {
            return __fadd_rn(__fsub_rn(h1, h0), __fsub_rn(l1, l0));
        };
        float u[3] = {dif(hb.x, lb.x, ha.x, la.x), dif(hb.y, lb.y, ha.y, la.y), dif(hb.z, lb.z, ha.z, la.z)};
        float r[3] = {dif(ho.x, lo.x, ha.x, la.x), dif(ho.y, lo.y, ha.y, la.y), dif(ho.z, lo.z, ha.z, la.z)};
        float n[3];
        if (dim == 3) {
            const int32_t ic = faces[f * dim + 2];
            const float4 hc = xh[ic], lc = xl[ic];
            float w[3] = {dif(hc.x, lc.x, ha.x, la.x), dif(hc.y, lc.y, ha.y, la.y), dif(hc.z, lc.z, ha.z, la.z)};
            n[0] = det2_kahan(u[1], u[2], w[1], w[2]);
            n[1] = det2_kahan(u[2], u[0], w[2], w[0]);
            n[2] = det2_kahan(u[0], u[1], w[0], w[1]);
        } else {
            n[0] = u[1];
            n[1] = -u[0];
            n[2] = 0.f;
        }
        const float len = sqrtf(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        const float side = n[0] * r[0] + n[1] * r[1] + n[2] * r[2];
        const float inv = (side > 0.f ? -1.f : 1.f) / len;
        for (int d = 0; d < dim; ++d) nrm[f * dim + d] = f32_to_f64(n[d] * inv);
        area[f] = f32_to_f64(dim == 3 ? 0.5f * len : len);
    }
}

// all-facet normals V^{-T} normalsRef = -grad lambda_j = -C_j / det (FP64)
__global__ void k_simplex_normals(int64_t ne, int dim, int nlb, const double *__restrict__ x,
                                  const int32_t *__restrict__ elems, double *__restrict__ out) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < ne; k += (int64_t)gridDim.x * blockDim.x) {
        double V[3][3] = {{0}}, Cf[4][3] = {{0}}, det;
        const int32_t last = elems[k * nlb + dim];
        for (int j = 0; j < dim; ++j) {
            const int32_t vj = elems[k * nlb + j];
            for (int d = 0; d < dim; ++d) V[j][d] = x[(int64_t)vj * dim + d] - x[(int64_t)last * dim + d];
        }
        if (dim == 3) {
            for (int c = 0; c < 3; ++c) {
                const int c1 = (c + 1) % 3, c2 = (c + 2) % 3;
                Cf[0][c] = V[1][c1] * V[2][c2] - V[1][c2] * V[2][c1];
                Cf[1][c] = V[2][c1] * V[0][c2] - V[2][c2] * V[0][c1];
                Cf[2][c] = V[0][c1] * V[1][c2] - V[0][c2] * V[1][c1];
            }
            det = V[0][0] * Cf[0][0] + V[0][1] * Cf[0][1] + V[0][2] * Cf[0][2];
        } else {
            Cf[0][0] = V[1][1];
            Cf[0][1] = -V[1][0];
            Cf[1][0] = -V[0][1];
            Cf[1][1] = V[0][0];
            det = V[0][0] * V[1][1] - V[0][1] * V[1][0];
        }
        const double r = 1.0 / det;
        for (int d = 0; d < dim; ++d) {
            double s = 0;
            for (int j = 0; j < dim; ++j) {
                const double g = Cf[j][d] * r;       // grad lambda_j
                out[k * dim * (dim + 1) + d + j * dim] = -g;
                s += g;
            }
            out[k * dim * (dim + 1) + d + dim * dim] = s;  // -grad lambda_dim
        }
    }
}

}  // namespace
}  // namespace vla

using namespace vla;

extern "C" vla_status vla_assemble(const vla_mesh *m, int32_t kind, double ca, double cb, int32_t precision,
                                   double *K_vals, double *M_vals, double *vol, double *K_pages, double *M_pages,
                                   int64_t *n_singular, void *stream) {
    if (!m) return fail(VLA_ERR_INVALID_ARG, "null mesh");
    if (kind != VLA_COEFF_POLY && kind != VLA_COEFF_EXP) return fail(VLA_ERR_INVALID_ARG, "unknown coefficient kind");
    if (precision != VLA_PREC_FP64 && precision != VLA_PREC_MIXED)
        return fail(VLA_ERR_INVALID_ARG, "precision must be VLA_PREC_FP64 or VLA_PREC_MIXED");
    if (!std::isfinite(ca) || !std::isfinite(cb)) return fail(VLA_ERR_INVALID_ARG, "non-finite coefficient");
    cudaStream_t st = (cudaStream_t)stream;
    if (m->order == 2) {
        vla_status s = ensure_p2_tables();
        if (s) return s;
    }
    unsigned long long *ns = reinterpret_cast<unsigned long long *>(n_singular);
    if (ns) VLA_CUDA(cudaMemsetAsync(ns, 0, sizeof(unsigned long long), st));
    AsmArgs a;
    a.tiles = m->tiles;
    a.tile_nodes = m->tile_nodes;
    a.tile_elem = m->tile_elem;
    a.tile_own = m->tile_own;
    a.tile_nzpos = m->tile_nzpos;
    a.tile_chunks = m->tile_chunks;
    a.codes = m->tile_codes;
    a.xh = m->xh;
    a.xl = m->xl;
    a.coords = m->coords;
    a.kind = kind;
    a.ca = ca;
    a.cb = cb;
    a.K = K_vals;
    a.M = M_vals;
    a.vol = vol;
    a.Kp = K_pages;
    a.Mp = M_pages;
    a.n_sing = ns;
    a.err = m->d_err;
    a.spin_limit = m->spin_limit;
    a.n_tiles = m->n_tiles;
    a.caf = (float)ca;
    a.cbf = (float)cb;
    a.stage_bytes = 0;
    const bool mix = precision == VLA_PREC_MIXED;
    const int key = (m->dim == 3 ? 4 : 0) + (m->order == 2 ? 2 : 0) + (mix ? 1 : 0);
    switch (key) {
    case 0: return launch_assemble<2, 1, false>(m, a, st);
    case 1: return launch_assemble<2, 1, true>(m, a, st);
    case 2: return launch_assemble<2, 2, false>(m, a, st);
    case 3: return launch_assemble<2, 2, true>(m, a, st);
    case 4: return launch_assemble<3, 1, false>(m, a, st);
    case 5: return launch_assemble<3, 1, true>(m, a, st);
    case 6: return launch_assemble<3, 2, false>(m, a, st);
    default: return launch_assemble<3, 2, true>(m, a, st);
    }
}

extern "C" vla_status vla_boundary(const vla_mesh *m, int32_t precision, double *normals, double *areas,
                                   void *stream) {
    if (!m) return fail(VLA_ERR_INVALID_ARG, "null mesh");
    if (precision != VLA_PREC_FP64 && precision != VLA_PREC_MIXED)
        return fail(VLA_ERR_INVALID_ARG, "precision must be VLA_PREC_FP64 or VLA_PREC_MIXED");
    if (m->nfb == 0) return VLA_OK;
    if (!normals || !areas) return fail(VLA_ERR_INVALID_ARG, "null output");
    cudaStream_t st = (cudaStream_t)stream;
    const int g = grid_for(m->nfb, 256, 152 * 16);
    if (precision == VLA_PREC_FP64)
        k_boundary_f64<<<g, 256, 0, st>>>(m->nfb, m->dim, m->coords, m->faces, m->face_opp, normals, areas);
    else
        k_boundary_mixed<<<g, 256, 0, st>>>(m->nfb, m->dim, m->xh, m->xl, m->faces, m->face_opp, normals, areas);
    VLA_CUDA(cudaGetLastError());
    return VLA_OK;
}

extern "C" vla_status vla_simplex_normals(const vla_mesh *m, double *normals, void *stream) {
    if (!m) return fail(VLA_ERR_INVALID_ARG, "null mesh");
    if (!normals) return fail(VLA_ERR_INVALID_ARG, "null output");
    cudaStream_t st = (cudaStream_t)stream;
    k_simplex_normals<<<grid_for(m->ne, 256, 152 * 16), 256, 0, st>>>(m->ne, m->dim, m->nlb, m->coords, m->elems,
                                                                     normals);
    VLA_CUDA(cudaGetLastError());
    return VLA_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free element pages.
//
// Some callers cannot allocate device memory at the point where they need
// element matrices: code running while another framework owns the whole
// device heap, real-time loops that forbid allocator calls, or setups that
// must not create a persistent mesh handle.  vla_element_pages_static serves
// them: it takes the raw coordinate and connectivity arrays and writes the
// element pages and volumes, keeping its one scratch buffer (the float-pair
// split of the node coordinates used by the mixed-precision geometry) in a
// file-scope device array instead of allocating.  That array exists once per
// GPU that loads the library and lives until the process exits.
// ---------------------------------------------------------------------------
namespace vla {
namespace {

constexpr int64_t kStaticMaxNodes = int64_t(1) << 18;    // 262,144 nodes: 8 MiB of float pairs
static __device__ __align__(256) float4 g_static_xhl[2 * kStaticMaxNodes];

std::mutex g_static_mu;
void *g_static_ptr[64] = {nullptr};

// Device address of the scratch array for the current device (set up once
// per device with that device current; host code must not use the symbol's
// name as an address).
vla_status static_scratch(float4 **out) {
    int dev = 0;
    VLA_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(VLA_ERR_INVALID_ARG, "device ordinal %d not supported", dev);
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_xhl);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
        g_static_ptr[dev] = p;
    }
    *out = reinterpret_cast<float4 *>(g_static_ptr[dev]);
    return VLA_OK;
}

__global__ void k_static_split(int64_t nn, int dim, const double *__restrict__ x, float4 *__restrict__ xh,
                               float4 *__restrict__ xl) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x) {
        float h[3] = {0.f, 0.f, 0.f}, l[3] = {0.f, 0.f, 0.f};
        for (int d = 0; d < dim; ++d) {
            const double v = x[i * dim + d];
            h[d] = (float)v;
            l[d] = (float)(v - (double)h[d]);
        }
        xh[i] = make_float4(h[0], h[1], h[2], 0.f);
        xl[i] = make_float4(l[0], l[1], l[2], 0.f);
    }
}

// element pages and volumes straight from the mesh arrays, one thread per element
template <int DIM, int ORDER, bool MIX>
__global__ void __launch_bounds__(256) k_static_pages(int64_t ne, const int32_t *__restrict__ elems,
                                                      const float4 *__restrict__ xh, const float4 *__restrict__ xl,
                                                      const double *__restrict__ coords, int kind, double ca,
                                                      double cb, double *__restrict__ Kp, double *__restrict__ Mp,
                                                      double *__restrict__ vol, unsigned long long *__restrict__ n_sing) {
    using C = Cfg<DIM, ORDER, MIX>;
    using T = typename C::T;
    const T cat = (T)ca, cbt = (T)cb;
    unsigned long long sing = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < ne; k += (int64_t)gridDim.x * blockDim.x) {
        Geo<T> g;
        if constexpr (MIX) {
            float4 h[C::NV], l[C::NV];
#pragma unroll
            for (int j = 0; j < C::NV; ++j) {
                const int32_t v = elems[k * C::NLB + j];
                h[j] = xh[v];
                l[j] = xl[v];
            }
            // same geometry as the tiled assembly, from vertex arrays
            if constexpr (DIM == 3) {
                geo_mixed3_fast(h, l, make_ushort4(0, 1, 2, 3), g);
            } else {
                geo_mixed2_fast(h, l, make_ushort4(0, 1, 2, 0), g);
            }
        } else {
            double4 x[C::NV];
#pragma unroll
            for (int j = 0; j < C::NV; ++j) {
                const int32_t v = elems[k * C::NLB + j];
                x[j].x = coords[(int64_t)v * DIM];
                x[j].y = coords[(int64_t)v * DIM + 1];
                x[j].z = DIM == 3 ? coords[(int64_t)v * DIM + 2] : 0.0;
                x[j].w = 0.0;
            }
            geo_f64<DIM>(x, make_ushort4(0, 1, 2, DIM == 3 ? 3 : 0), g);
        }
        const T c = coeff<T>(kind, cat, cbt, g.xc, DIM);
        const T adet = g.det < T(0) ? -g.det : g.det;
        T sc;
        if constexpr (MIX) sc = c * __frcp_rn(T(C::DFACT) * adet);
        else sc = c / (T(C::DFACT) * adet);
        T cd[10];
#pragma unroll
        for (int a = 0; a < C::NV; ++a)
#pragma unroll
            for (int q = a; q < C::NV; ++q) cd[a * C::NV - a * (a - 1) / 2 + (q - a)] = dot3<T>(g.C[a], g.C[q]);
        const T mscale = ORDER == 1 ? c * adet * T(C::MOFF / C::DFACT) : c * adet * T(1.0 / C::DFACT);
        for (int a = 0; a < C::NLB; ++a)
            for (int q = 0; q < C::NLB; ++q) {
                const int p0 = a < q ? a : q, p1 = a < q ? q : a;
                T kv, mv;
                if constexpr (ORDER == 1) {
                    kv = sc * cd[p0 * C::NV - p0 * (p0 - 1) / 2 + (p1 - p0)];
                    mv = mscale * (a == q ? T(2) : T(1));
                } else {
                    const int u = p0 * C::NLB - p0 * (p0 - 1) / 2 + (p1 - p0);
                    const P2Tab &tb = c_p2[DIM - 2];
                    T acc = 0;
                    for (int t = 0; t < tb.nterm[u]; ++t) acc += (MIX ? (T)tb.coef_f[u][t] : (T)tb.coef_d[u][t]) * cd[tb.st[u][t]];
                    kv = sc * acc;
                    mv = mscale * (MIX ? (T)tb.mhat_f[u] : (T)tb.mhat_d[u]);
                }
                const int64_t pos = k * C::NLB * C::NLB + a + (int64_t)q * C::NLB;
                if constexpr (MIX) {
                    if (Kp) Kp[pos] = f32_to_f64(kv);
                    if (Mp) Mp[pos] = f32_to_f64(mv);
                } else {
                    if (Kp) Kp[pos] = kv;
                    if (Mp) Mp[pos] = mv;
                }
            }
        if (g.det == T(0)) ++sing;
        if (vol) {
            if constexpr (MIX) vol[k] = f32_to_f64(adet * (float)(1.0 / C::DFACT));
            else vol[k] = adet / C::DFACT;
        }
    }
    if (n_sing && sing) atomicAdd(n_sing, sing);
}

template <int DIM, int ORDER, bool MIX>
void launch_static_pages(int64_t ne, const int32_t *elems, const float4 *xh, const float4 *xl, const double *coords,
                         int kind, double ca, double cb, double *Kp, double *Mp, double *vol,
                         unsigned long long *ns, cudaStream_t st) {
    k_static_pages<DIM, ORDER, MIX><<<grid_for(ne, 256, 152 * 16), 256, 0, st>>>(ne, elems, xh, xl, coords, kind, ca,
                                                                                   cb, Kp, Mp, vol, ns);
}

}  // namespace
}  // namespace vla

extern "C" vla_status vla_element_pages_static(int32_t dim, int32_t order, int64_t nn, int64_t ne,
                                               const double *coords, const int32_t *elems, int32_t kind, double ca,
                                               double cb, int32_t precision, double *K_pages, double *M_pages,
                                               double *vol, int64_t *n_singular, void *stream) {
    if (dim != 2 && dim != 3) return fail(VLA_ERR_INVALID_ARG, "dim must be 2 or 3");
    if (order != VLA_P1 && order != VLA_P2) return fail(VLA_ERR_INVALID_ARG, "order must be VLA_P1 or VLA_P2");
    if (kind != VLA_COEFF_POLY && kind != VLA_COEFF_EXP) return fail(VLA_ERR_INVALID_ARG, "unknown coefficient kind");
    if (precision != VLA_PREC_FP64 && precision != VLA_PREC_MIXED)
        return fail(VLA_ERR_INVALID_ARG, "precision must be VLA_PREC_FP64 or VLA_PREC_MIXED");
    if (nn < 1 || ne < 0) return fail(VLA_ERR_INVALID_ARG, "need nn >= 1 and ne >= 0");
    if (nn > kStaticMaxNodes)
        return fail(VLA_ERR_BUDGET, "vla_element_pages_static: %lld nodes exceed its fixed scratch of %lld nodes; "
                                    "use vla_mesh_create + vla_assemble", (long long)nn, (long long)kStaticMaxNodes);
    if (ne >= ((int64_t)1 << 31) / 100) return fail(VLA_ERR_INVALID_ARG, "too many elements");
    if (ne > 0 && (!coords || !elems)) return fail(VLA_ERR_INVALID_ARG, "null mesh array");
    if (!std::isfinite(ca) || !std::isfinite(cb)) return fail(VLA_ERR_INVALID_ARG, "non-finite coefficient");
    cudaStream_t st = (cudaStream_t)stream;
    float4 *scratch = nullptr;
    vla_status s = static_scratch(&scratch);
    if (s) return s;
    if (order == 2) {
        s = ensure_p2_tables();
        if (s) return s;
    }
    unsigned long long *ns = reinterpret_cast<unsigned long long *>(n_singular);
    if (ns) VLA_CUDA(cudaMemsetAsync(ns, 0, sizeof(unsigned long long), st));
    if (ne == 0) return VLA_OK;
    const bool mix = precision == VLA_PREC_MIXED;
    float4 *xh = scratch, *xl = scratch + kStaticMaxNodes;
    if (mix) {
        k_static_split<<<grid_for(nn, 256, 152 * 16), 256, 0, st>>>(nn, dim, coords, xh, xl);
        VLA_CUDA(cudaGetLastError());
    }
    const int key = (dim == 3 ? 4 : 0) + (order == 2 ? 2 : 0) + (mix ? 1 : 0);
    switch (key) {
    case 0: launch_static_pages<2, 1, false>(ne, elems, xh, xl, coords, kind, ca, cb, K_pages, M_pages, vol, ns, st); break;
    case 1: launch_static_pages<2, 1, true>(ne, elems, xh, xl, coords, kind, ca, cb, K_pages, M_pages, vol, ns, st); break;
    case 2: launch_static_pages<2, 2, false>(ne, elems, xh, xl, coords, kind, ca, cb, K_pages, M_pages, vol, ns, st); break;
    case 3: launch_static_pages<2, 2, true>(ne, elems, xh, xl, coords, kind, ca, cb, K_pages, M_pages, vol, ns, st); break;
    case 4: launch_static_pages<3, 1, false>(ne, elems, xh, xl, coords, kind, ca, cb, K_pages, M_pages, vol, ns, st); break;
    case 5: launch_static_pages<3, 1, true>(ne, elems, xh, xl, coords, kind, ca, cb, K_pages, M_pages, vol, ns, st); break;
    case 6: launch_static_pages<3, 2, false>(ne, elems, xh, xl, coords, kind, ca, cb, K_pages, M_pages, vol, ns, st); break;
    default: launch_static_pages<3, 2, true>(ne, elems, xh, xl, coords, kind, ca, cb, K_pages, M_pages, vol, ns, st); break;
    }
    VLA_CUDA(cudaGetLastError());
    return VLA_OK;
}
