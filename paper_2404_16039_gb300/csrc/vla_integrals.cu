// vla_integrals.cu -- quadrature on simplices, the GI integrals of
// Section 3.4 (volume integrals and fluxes through boundary facets), the
// load vector and local energies of Section 3.5, and the avtamav page
// product of Section 2.4.
#include <cmath>
#include <cstring>

#include "vla_internal.cuh"

namespace vla {
namespace {

constexpr int kMaxIp = 8;   // points of the largest rule

// A symmetric simplex rule: barycentric points (sdim+1 coordinates) and
// weights summing to 1.
struct Rule {
    int sdim, nip;
    double ip[kMaxIp][4];
    double w[kMaxIp];
};

// Published rules of degree gqo = 1..3 on the segment (Gauss-Legendre), the
// triangle (centroid; three interior points; Strang-Fix 4-point with a
// negative centroid weight) and the tetrahedron (centroid; Hammer-Stroud
// 4-point; Keast 5-point with a negative centroid weight).  Each is the
// centroid with weight wc (if any) plus the orbit of (a, b, ..., b) under
// coordinate permutations with weight wo each.
bool make_rule(int sdim, int gqo, Rule &r) {
    std::memset(&r, 0, sizeof(r));
    r.sdim = sdim;
    if (sdim < 1 || sdim > 3 || gqo < 1 || gqo > 3) return false;
    const int nv = sdim + 1;
    double a = 0, b = 0, wo = 0, wc = 0;
    bool centroid = false, orbit = true;
    if (gqo == 1) {
        centroid = true, wc = 1.0, orbit = false;
    } else if (sdim == 1) {   // two Gauss points: lambda = (1 +- 1/sqrt3)/2
        a = 0.5 * (1.0 + 1.0 / std::sqrt(3.0)), b = 1.0 - a, wo = 0.5;
    } else if (sdim == 2) {
        if (gqo == 2) a = 2.0 / 3.0, b = 1.0 / 6.0, wo = 1.0 / 3.0;
        else centroid = true, wc = -27.0 / 48.0, a = 0.6, b = 0.2, wo = 25.0 / 48.0;
    } else {
        if (gqo == 2) {
            const double s5 = std::sqrt(5.0);
            a = (5.0 + 3.0 * s5) / 20.0, b = (5.0 - s5) / 20.0, wo = 0.25;
        } else {
            centroid = true, wc = -0.8, a = 0.5, b = 1.0 / 6.0, wo = 0.45;
        }
    }
    int q = 0;
    if (centroid) {
        for (int j = 0; j < nv; ++j) r.ip[q][j] = 1.0 / nv;
        r.w[q++] = wc;
    }
    if (orbit)
        for (int i = 0; i < nv; ++i) {
            for (int j = 0; j < nv; ++j) r.ip[q][j] = (j == i) ? a : b;
            r.w[q++] = wo;
        }
    r.nip = q;
    return true;
}

// basis function j of the element (P1 or P2) at barycentric point lam
double basis_value(int dim, int order, int j, const double *lam) {
    if (order == 1 || j <= dim) return order == 1 ? lam[j] : lam[j] * (2.0 * lam[j] - 1.0);
    static const int E2[3][2] = {{0, 1}, {1, 2}, {0, 2}};
    static const int E3[6][2] = {{0, 1}, {1, 2}, {0, 2}, {0, 3}, {1, 3}, {2, 3}};
    const int *e = dim == 2 ? E2[j - 3] : E3[j - 4];
    return 4.0 * lam[e[0]] * lam[e[1]];
}

struct QuadArgs {
    double ip[kMaxIp][4];
    int nip, nvert, stride, dim;
};

// X(:, q, k) = sum_j ip(j, q) x_{cells(k, j)}  (the paper's amsm(coords3D, ip));
// one point per thread, DIM coordinates and NV vertices compile-time
template <int DIM, int NV>
__global__ void __launch_bounds__(256, 8) k_quad_points(int64_t n, QuadArgs qa, const int32_t *__restrict__ cells,
                                                        const double *__restrict__ x, double *__restrict__ X) {
    const int64_t total = n * qa.nip;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / qa.nip;
        const int q = (int)(t - k * qa.nip);
        double s[DIM];
#pragma unroll
        for (int d = 0; d < DIM; ++d) s[d] = 0.0;
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            const int64_t node = cells[k * qa.stride + j];
            const double c = qa.ip[q][j];
#pragma unroll
            for (int d = 0; d < DIM; ++d) s[d] = fma(c, x[node * DIM + d], s[d]);
        }
#pragma unroll
        for (int d = 0; d < DIM; ++d) X[t * DIM + d] = s[d];
    }
}

// ---------------------------------------------------------------------------
// deterministic sums: a fixed grid of partial sums (each block a fixed
// strided subset in a fixed order, a fixed shuffle tree), then one block
// adding the partials in order -- the same bits on every run
// ---------------------------------------------------------------------------
constexpr int kRedThreads = 256;
constexpr int kRedMaxComp = 4;

__device__ __forceinline__ double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
    return s;   // valid in thread 0
}

struct GIArgs {
    double w[kMaxIp];
    int nip, d;
};

// partial[b][c] over simplices k = b*T + t, stride grid*T of
// sizes_k * sum_q w_q f(c, q, k)  (FLUX: the one sum of sizes_k *
// sum_c (sum_q w_q f(c, q, k)) n(c, k)); D components, compile-time, so the
// per-simplex averages stay in registers
template <int D, bool FLUX>
__global__ void k_gi_partial(int64_t n, GIArgs ga, const double *__restrict__ fip, const double *__restrict__ sizes,
                             const double *__restrict__ normals, double *__restrict__ partial) {
    __shared__ double sh[32];
    constexpr int NC = FLUX ? 1 : D;
    double acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const double *fk = fip + k * ga.nip * D;
        double avg[D];
#pragma unroll
        for (int c = 0; c < D; ++c) avg[c] = 0.0;
#pragma unroll
        for (int q = 0; q < kMaxIp; ++q) {
            if (q >= ga.nip) break;
#pragma unroll
            for (int c = 0; c < D; ++c) avg[c] = fma(ga.w[q], fk[q * D + c], avg[c]);
        }
        const double sk = sizes[k];
        if constexpr (FLUX) {
            double dot = 0.0;
#pragma unroll
            for (int c = 0; c < D; ++c) dot = fma(avg[c], normals[k * D + c], dot);
            acc[0] = fma(sk, dot, acc[0]);
        } else {
#pragma unroll
            for (int c = 0; c < D; ++c) acc[c] = fma(sk, avg[c], acc[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const double s = block_sum(acc[c], sh);
        if (threadIdx.x == 0) partial[(int64_t)blockIdx.x * kRedMaxComp + c] = s;
    }
}

__global__ void k_sum_partials(int nb, int ncomp, const double *__restrict__ partial, double *__restrict__ out) {
    __shared__ double sh[32];
    for (int c = 0; c < ncomp; ++c) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nb; b += blockDim.x) v += partial[(int64_t)b * kRedMaxComp + c];
        const double s = block_sum(v, sh);
        if (threadIdx.x == 0) out[c] = s;
    }
}

int red_blocks(int64_t n) {
    int64_t b = (n + kRedThreads - 1) / kRedThreads;
    if (b < 1) b = 1;
    if (b > 1024) b = 1024;
    return (int)b;
}

// ---------------------------------------------------------------------------
// load vector and energies
// ---------------------------------------------------------------------------
struct RhsArgs {
    double w[kMaxIp];
    double phi[kMaxIp][10];   // basis values at the rule's points
    int nip, dim, nlb;
};

// simplex measure |det V| / dim! from FP64 coordinates (vectors to the last vertex)
template <int DIM, int NLB>
__device__ __forceinline__ double simplex_measure(const int32_t *__restrict__ elems, int64_t k,
                                                  const double *__restrict__ x) {
    const int64_t last = elems[k * NLB + DIM];
    double V[DIM][DIM];
#pragma unroll
    for (int j = 0; j < DIM; ++j) {
        const int64_t vj = elems[k * NLB + j];
#pragma unroll
        for (int d = 0; d < DIM; ++d) V[j][d] = x[vj * DIM + d] - x[last * DIM + d];
    }
    double det;
    if constexpr (DIM == 3)
        det = V[0][0] * (V[1][1] * V[2][2] - V[1][2] * V[2][1]) - V[0][1] * (V[1][0] * V[2][2] - V[1][2] * V[2][0]) +
              V[0][2] * (V[1][0] * V[2][1] - V[1][1] * V[2][0]);
    else
        det = V[0][0] * V[1][1] - V[0][1] * V[1][0];
    return fabs(det) / (DIM == 3 ? 6.0 : 2.0);
}

// b2D(j, k) = |T_k| sum_q w_q f(q, k) phi_j(ip_q); DIM and NLB compile-time
template <int DIM, int NLB>
__global__ void __launch_bounds__(256, 8) k_rhs_local(int64_t ne, RhsArgs ra, const int32_t *__restrict__ elems,
                                                      const double *__restrict__ x, const double *__restrict__ fip,
                                                      double *__restrict__ b2D) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < ne; k += (int64_t)gridDim.x * blockDim.x) {
        const double vol = simplex_measure<DIM, NLB>(elems, k, x);
#pragma unroll
        for (int j = 0; j < NLB; ++j) {
            double s = 0.0;
            for (int q = 0; q < ra.nip; ++q) s = fma(ra.w[q] * fip[k * ra.nip + q], ra.phi[q][j], s);
            b2D[k * NLB + j] = vol * s;
        }
    }
}

// b_i = sum over node i's incidence list (ascending element, then local index)
__global__ void k_rhs_gather(int64_t nn, int nlb, const int32_t *__restrict__ n2e_ptr, const int32_t *__restrict__ n2e,
                             const double *__restrict__ b2D, double *__restrict__ b) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int32_t p = n2e_ptr[i]; p < n2e_ptr[i + 1]; ++p) {
            const int32_t c = n2e[p];
            s += b2D[(int64_t)(c >> 4) * nlb + (c & 15)];
        }
        b[i] = s;
    }
}

// J(0,k) = u_k^T K_k u_k / 2, J(1,k) = u_k^T M_k u_k / 2, J(2,k) = -b2D(:,k)^T u_k,
// plus block partials of the three sums; NLB nodes per element, compile-time
template <int NLB>
__global__ void k_energies(int64_t ne, const int32_t *__restrict__ elems, const double *__restrict__ u,
                           const double *__restrict__ Kp, const double *__restrict__ Mp, const double *__restrict__ b2D,
                           double *__restrict__ J, double *__restrict__ partial) {
    __shared__ double sh[32];
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < ne; k += (int64_t)gridDim.x * blockDim.x) {
        double uk[NLB];
#pragma unroll
        for (int j = 0; j < NLB; ++j) uk[j] = u[elems[k * NLB + j]];
        double e[3] = {0.0, 0.0, 0.0};
        const int64_t pg = k * NLB * NLB;
#pragma unroll
        for (int c = 0; c < NLB; ++c) {
            double kc = 0.0, mc = 0.0;   // (K_k u_k)_c and (M_k u_k)_c over rows r: A(r,c) at r + c NLB
#pragma unroll
            for (int r = 0; r < NLB; ++r) {
                if (Kp) kc = fma(Kp[pg + r + c * NLB], uk[r], kc);
                if (Mp) mc = fma(Mp[pg + r + c * NLB], uk[r], mc);
            }
            e[0] = fma(kc, uk[c], e[0]);
            e[1] = fma(mc, uk[c], e[1]);
            if (b2D) e[2] = fma(b2D[k * NLB + c], uk[c], e[2]);
        }
        e[0] *= 0.5;
        e[1] *= 0.5;
        e[2] = -e[2];
        if (J)
#pragma unroll
            for (int c = 0; c < 3; ++c) J[k * 3 + c] = e[c];
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[c] += e[c];
    }
    if (partial)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double s = block_sum(acc[c], sh);
            if (threadIdx.x == 0) partial[(int64_t)blockIdx.x * kRedMaxComp + c] = s;
        }
}

// out_k = v_k^T A_k w_k (page layout: v, w n x N; A n x n x N column-major;
// SoA: entry (r, c) of page k at (c n + r) N + k, vector entry r at r N + k)
template <typename T>
__global__ void k_avtamav(int64_t N, int n, int soa, const T *__restrict__ v, const T *__restrict__ A,
                          const T *__restrict__ w, T *__restrict__ out) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        T s = 0;
        for (int c = 0; c < n; ++c) {
            T col = 0;
            for (int r = 0; r < n; ++r) {
                const T a = soa ? A[((int64_t)c * n + r) * N + k] : A[k * n * n + r + (int64_t)c * n];
                const T vr = soa ? v[(int64_t)r * N + k] : v[k * n + r];
                col += vr * a;
            }
            s += col * (soa ? w[(int64_t)c * N + k] : w[k * n + c]);
        }
        out[k] = s;
    }
}

template <int D>
void launch_gi(int nb, cudaStream_t st, int64_t n, const GIArgs &ga, const double *fip, const double *sizes,
               const double *normals, double *partial) {
    if (normals) k_gi_partial<D, true><<<nb, kRedThreads, 0, st>>>(n, ga, fip, sizes, normals, partial);
    else k_gi_partial<D, false><<<nb, kRedThreads, 0, st>>>(n, ga, fip, sizes, normals, partial);
}

template <typename T>
vla_status scratch_alloc(T **p, size_t count, cudaStream_t st) {
    if (pool_malloc((void **)p, sizeof(T) * (count ? count : 1), st) != cudaSuccess) {
        cudaGetLastError();
        return fail(VLA_ERR_OOM, "scratch allocation of %zu bytes failed", sizeof(T) * count);
    }
    return VLA_OK;
}

}  // namespace
}  // namespace vla

using namespace vla;

extern "C" vla_status vla_quad_rule(int32_t sdim, int32_t gqo, int32_t *nip, double *ip, double *w) {
    Rule r;
    if (!make_rule(sdim, gqo, r)) return fail(VLA_ERR_UNSUPPORTED, "no rule for simplex dimension %d, degree %d", sdim, gqo);
    if (nip) *nip = r.nip;
    for (int q = 0; q < r.nip; ++q) {
        if (ip)
            for (int j = 0; j <= sdim; ++j) ip[q * (sdim + 1) + j] = r.ip[q][j];
        if (w) w[q] = r.w[q];
    }
    return VLA_OK;
}

extern "C" vla_status vla_quad_points(const vla_mesh *m, int32_t gqo, int32_t facets, double *X, void *stream) {
    if (!m || !X) return fail(VLA_ERR_INVALID_ARG, "null mesh or output");
    const int sdim = facets ? m->dim - 1 : m->dim;
    Rule r;
    if (!make_rule(sdim, gqo, r)) return fail(VLA_ERR_UNSUPPORTED, "no rule for simplex dimension %d, degree %d", sdim, gqo);
    if (facets && (m->nfb == 0 || !m->faces)) return fail(VLA_ERR_INVALID_ARG, "the mesh has no boundary facets");
    QuadArgs qa;
    std::memset(&qa, 0, sizeof(qa));
    std::memcpy(qa.ip, r.ip, sizeof(qa.ip));
    qa.nip = r.nip;
    qa.nvert = sdim + 1;
    qa.stride = facets ? m->dim : m->nlb;
    qa.dim = m->dim;
    const int64_t n = facets ? m->nfb : m->ne;
    if (n == 0) return VLA_OK;
    const int grid = grid_for(n * r.nip, 256);
    cudaStream_t st = (cudaStream_t)stream;
    const int32_t *cells = facets ? m->faces : m->elems;
    if (m->dim == 2) {
        if (qa.nvert == 2) k_quad_points<2, 2><<<grid, 256, 0, st>>>(n, qa, cells, m->coords, X);
        else k_quad_points<2, 3><<<grid, 256, 0, st>>>(n, qa, cells, m->coords, X);
    } else {
        if (qa.nvert == 3) k_quad_points<3, 3><<<grid, 256, 0, st>>>(n, qa, cells, m->coords, X);
        else k_quad_points<3, 4><<<grid, 256, 0, st>>>(n, qa, cells, m->coords, X);
    }
    VLA_CUDA(cudaGetLastError());
    return VLA_OK;
}

extern "C" vla_status vla_gi(int64_t n, int32_t nip, int32_t d, const double *fip, const double *w,
                             const double *sizes, const double *normals, double *out, void *stream) {
    if (n < 0 || nip < 1 || nip > kMaxIp || d < 1 || d > kRedMaxComp)
        return fail(VLA_ERR_INVALID_ARG, "need n >= 0, 1 <= nip <= %d, 1 <= d <= %d", kMaxIp, kRedMaxComp);
    if (!w || !out || (n > 0 && (!fip || !sizes))) return fail(VLA_ERR_INVALID_ARG, "null argument");
    cudaStream_t st = (cudaStream_t)stream;
    GIArgs ga;
    std::memset(&ga, 0, sizeof(ga));
    for (int q = 0; q < nip; ++q) ga.w[q] = w[q];
    ga.nip = nip;
    ga.d = d;
    const int nb = red_blocks(n);
    double *partial = nullptr;
    TRY(scratch_alloc(&partial, (size_t)nb * kRedMaxComp, st));
    switch (d) {
    case 1: launch_gi<1>(nb, st, n, ga, fip, sizes, normals, partial); break;
    case 2: launch_gi<2>(nb, st, n, ga, fip, sizes, normals, partial); break;
    case 3: launch_gi<3>(nb, st, n, ga, fip, sizes, normals, partial); break;
    default: launch_gi<4>(nb, st, n, ga, fip, sizes, normals, partial); break;
    }
    k_sum_partials<<<1, kRedThreads, 0, st>>>(nb, normals ? 1 : d, partial, out);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(partial, st);
    if (e != cudaSuccess) return cuda_fail(e, "vla_gi");
    return VLA_OK;
}

extern "C" vla_status vla_rhs(const vla_mesh *m, int32_t gqo, const double *fip, double *b, double *b2D, void *stream) {
    if (!m || !fip) return fail(VLA_ERR_INVALID_ARG, "null mesh or f values");
    Rule r;
    if (!make_rule(m->dim, gqo, r)) return fail(VLA_ERR_UNSUPPORTED, "no rule for dimension %d, degree %d", m->dim, gqo);
    cudaStream_t st = (cudaStream_t)stream;
    RhsArgs ra;
    std::memset(&ra, 0, sizeof(ra));
    ra.nip = r.nip;
    ra.dim = m->dim;
    ra.nlb = m->nlb;
    for (int q = 0; q < r.nip; ++q) {
        ra.w[q] = r.w[q];
        for (int j = 0; j < m->nlb; ++j) ra.phi[q][j] = basis_value(m->dim, m->order, j, r.ip[q]);
    }
    double *loc = b2D;
    if (!loc) TRY(scratch_alloc(&loc, (size_t)m->ne * m->nlb, st));
    const int grid = grid_for(m->ne, 256);
    switch (m->nlb) {
    case 3: k_rhs_local<2, 3><<<grid, 256, 0, st>>>(m->ne, ra, m->elems, m->coords, fip, loc); break;
    case 4: k_rhs_local<3, 4><<<grid, 256, 0, st>>>(m->ne, ra, m->elems, m->coords, fip, loc); break;
    case 6: k_rhs_local<2, 6><<<grid, 256, 0, st>>>(m->ne, ra, m->elems, m->coords, fip, loc); break;
    default: k_rhs_local<3, 10><<<grid, 256, 0, st>>>(m->ne, ra, m->elems, m->coords, fip, loc); break;
    }
    if (b) k_rhs_gather<<<grid_for(m->nn, 256), 256, 0, st>>>(m->nn, m->nlb, m->n2e_ptr, m->n2e, loc, b);
    cudaError_t e = cudaGetLastError();
    if (!b2D) cudaFreeAsync(loc, st);
    if (e != cudaSuccess) return cuda_fail(e, "vla_rhs");
    return VLA_OK;
}

extern "C" vla_status vla_energies(const vla_mesh *m, const double *u, const double *K_pages, const double *M_pages,
                                   const double *b2D, double *J_local, double *J_total, void *stream) {
    if (!m || !u) return fail(VLA_ERR_INVALID_ARG, "null mesh or u");
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = red_blocks(m->ne);
    double *partial = nullptr;
    if (J_total) TRY(scratch_alloc(&partial, (size_t)nb * kRedMaxComp, st));
#define VLA_ENERGIES(NLB) \
    k_energies<NLB><<<nb, kRedThreads, 0, st>>>(m->ne, m->elems, u, K_pages, M_pages, b2D, J_local, partial)
    switch (m->nlb) {
    case 3: VLA_ENERGIES(3); break;
    case 4: VLA_ENERGIES(4); break;
    case 6: VLA_ENERGIES(6); break;
    default: VLA_ENERGIES(10); break;
    }
#undef VLA_ENERGIES
    if (J_total) k_sum_partials<<<1, kRedThreads, 0, st>>>(nb, 3, partial, J_total);
    cudaError_t e = cudaGetLastError();
    if (partial) cudaFreeAsync(partial, st);
    if (e != cudaSuccess) return cuda_fail(e, "vla_energies");
    return VLA_OK;
}

extern "C" vla_status vla_avtamav(int32_t dtype, int32_t layout, int64_t N, int32_t n, const void *v, const void *A,
                                  const void *w, void *out, void *stream) {
    if (dtype != VLA_F32 && dtype != VLA_F64) return fail(VLA_ERR_INVALID_ARG, "dtype must be VLA_F32 or VLA_F64");
    if (layout != VLA_LAYOUT_PAGE && layout != VLA_LAYOUT_SOA) return fail(VLA_ERR_INVALID_ARG, "unknown layout");
    if (N < 0 || n < 1 || n > 16) return fail(VLA_ERR_INVALID_ARG, "need N >= 0 and 1 <= n <= 16");
    if (N == 0) return VLA_OK;
    if (!v || !A || !w || !out) return fail(VLA_ERR_INVALID_ARG, "null page array");
    cudaStream_t st = (cudaStream_t)stream;
    const int soa = layout == VLA_LAYOUT_SOA;
    if (dtype == VLA_F64)
        k_avtamav<double><<<grid_for(N, 256), 256, 0, st>>>(N, n, soa, (const double *)v, (const double *)A,
                                                            (const double *)w, (double *)out);
    else
        k_avtamav<float><<<grid_for(N, 256), 256, 0, st>>>(N, n, soa, (const float *)v, (const float *)A,
                                                           (const float *)w, (float *)out);
    VLA_CUDA(cudaGetLastError());
    return VLA_OK;
}
