// vla_pages.cu -- page-wise tiny-matrix primitives (Section 2.4 of the paper):
// amtam (A^T B), astam (s A), avtam (v^T A), amdet, aminv for 2x2 / 3x3 pages.
//
// These are HBM-streaming kernels with a handful of flops per page; no tensor
// cores (a 3x3 page is not a dense contraction).  Two data paths:
//  * page-major layout (each page contiguous, the MATLAB n x m x N layout):
//    a persistent kernel stages chunks of 128 pages through shared memory with
//    1-D TMA bulk copies (cp.async.bulk + mbarrier), double-buffered, computes
//    one page per thread from shared memory, and writes results back with bulk
//    stores.  Misaligned pointers and the tail chunk take a plain path.
//  * SoA layout (page index fastest): one page per thread, every load and
//    store coalesced across the warp.
#include <algorithm>
#include <mutex>

#include "vla_internal.cuh"

namespace vla {
namespace {

constexpr int kPagesPerChunk = 128;   // = threads per CTA of the staged kernel
constexpr int kSpinLimit = 1 << 22;   // bounded mbarrier wait

// ---------------------------------------------------------------------------
// page operations on register/shared arrays (column-major pages)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T det_n(const T *a, int n) {
    if (n == 2) return a[0] * a[3] - a[2] * a[1];
    // cofactor expansion along the first row
    T c0 = a[4] * a[8] - a[7] * a[5];
    T c1 = a[1] * a[8] - a[7] * a[2];
    T c2 = a[1] * a[5] - a[4] * a[2];
    return a[0] * c0 - a[3] * c1 + a[6] * c2;
}

template <typename T, int P, int M, int N>
struct OpAmtam {  // C (M x N) = A^T B, A: P x M, B: P x N
    static constexpr int I0 = P * M, I1 = P * N, O0 = M * N, O1 = 0;
    __device__ static bool apply(const T *a, const T *b, T *c, T *) {
#pragma unroll
        for (int j = 0; j < N; ++j)
#pragma unroll
            for (int i = 0; i < M; ++i) {
                T s = 0;
#pragma unroll
                for (int r = 0; r < P; ++r) s += a[r + i * P] * b[r + j * P];
                c[i + j * M] = s;
            }
        return false;
    }
};

template <typename T, int M, int N>
struct OpAstam {  // C = s A
    static constexpr int I0 = 1, I1 = M * N, O0 = M * N, O1 = 0;
    __device__ static bool apply(const T *s, const T *a, T *c, T *) {
        T v = s[0];
#pragma unroll
        for (int e = 0; e < M * N; ++e) c[e] = v * a[e];
        return false;
    }
};

template <typename T, int P, int N>
struct OpAvtam {  // y (1 x N) = v^T A, A: P x N
    static constexpr int I0 = P, I1 = P * N, O0 = N, O1 = 0;
    __device__ static bool apply(const T *v, const T *a, T *y, T *) {
#pragma unroll
        for (int j = 0; j < N; ++j) {
            T s = 0;
#pragma unroll
            for (int r = 0; r < P; ++r) s += v[r] * a[r + j * P];
            y[j] = s;
        }
        return false;
    }
};

template <typename T, int M, int N>
struct OpAmt {  // C (N x M) = A^T, A: M x N (pagemtranspose)
    static constexpr int I0 = M * N, I1 = 0, O0 = M * N, O1 = 0;
    __device__ static bool apply(const T *a, const T *, T *c, T *) {
#pragma unroll
        for (int j = 0; j < N; ++j)
#pragma unroll
            for (int i = 0; i < M; ++i) c[j + i * N] = a[i + j * M];
        return false;
    }
};

template <typename T, int N>
struct OpAvtav {  // s = a^T b, a and b: N-vectors
    static constexpr int I0 = N, I1 = N, O0 = 1, O1 = 0;
    __device__ static bool apply(const T *a, const T *b, T *c, T *) {
        T s = 0;
#pragma unroll
        for (int r = 0; r < N; ++r) s += a[r] * b[r];
        c[0] = s;
        return false;
    }
};

template <typename T, int N>
struct OpAmdet {
    static constexpr int I0 = N * N, I1 = 0, O0 = 1, O1 = 0;
    __device__ static bool apply(const T *a, const T *, T *d, T *) {
        d[0] = det_n<T>(a, N);
        return false;
    }
};

template <typename T, int N, bool WITH_DET>
struct OpAminv {  // Ainv = adj(A) / det(A); returns true for a singular page
    static constexpr int I0 = N * N, I1 = 0, O0 = N * N, O1 = WITH_DET ? 1 : 0;
    __device__ static bool apply(const T *a, const T *, T *inv, T *det) {
        T d = det_n<T>(a, N);
        T r = T(1) / d;
        if (N == 2) {
            inv[0] = a[3] * r;
            inv[1] = -a[1] * r;
            inv[2] = -a[2] * r;
            inv[3] = a[0] * r;
        } else {
#define A_(i, j) a[(i) + 3 * (j)]
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    int i0 = (i + 1) % 3, i1 = (i + 2) % 3, j0 = (j + 1) % 3, j1 = (j + 2) % 3;
                    // signed cofactor C(i,j); the inverse is C^T / det
                    inv[j + 3 * i] = (A_(i0, j0) * A_(i1, j1) - A_(i0, j1) * A_(i1, j0)) * r;
                }
#undef A_
        }
        if (WITH_DET) det[0] = d;
        return d == T(0);
    }
};

// ---------------------------------------------------------------------------
// staged page-major kernel: chunk c covers pages [c*128, c*128+128)
// ---------------------------------------------------------------------------
template <class OP, typename T>
__global__ void __launch_bounds__(kPagesPerChunk) k_page_staged(int64_t n_chunks, const T *__restrict__ in0,
                                                                 const T *__restrict__ in1, T *__restrict__ out0,
                                                                 T *__restrict__ out1,
                                                                 unsigned long long *__restrict__ n_sing,
                                                                 int *__restrict__ err) {
    constexpr int B = kPagesPerChunk;
    constexpr int I0 = OP::I0 * B, I1 = OP::I1 * B, O0 = OP::O0 * B, O1 = OP::O1 * B;
    constexpr uint32_t IN_BYTES = (uint32_t)((I0 + I1) * sizeof(T));
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *stage[2];
    stage[0] = reinterpret_cast<T *>(smem_raw);
    stage[1] = stage[0] + (I0 + I1);
    T *ob = stage[1] + (I0 + I1);
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int abort_flag;

    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        abort_flag = 0;
        fence_async_smem();
    }
    __syncthreads();

    int64_t c0 = blockIdx.x;
    auto issue = [&](int64_t c, int s) {
        mbar_expect_tx(&bar[s], IN_BYTES);
        bulk_g2s(stage[s], in0 + c * I0, (uint32_t)(I0 * sizeof(T)), &bar[s]);
        if (I1) bulk_g2s(stage[s] + I0, in1 + c * I1, (uint32_t)(I1 * sizeof(T)), &bar[s]);
    };
    int issued[2] = {0, 0};                  // loads issued per stage (thread 0's view)
    if (tid == 0 && c0 < n_chunks) {
        issue(c0, 0);
        issued[0] = 1;
    }

    unsigned long long local_sing = 0;
    int it = 0;
    for (int64_t c = c0; c < n_chunks; c += gridDim.x, ++it) {
        const int s = it & 1;
        const uint32_t parity = (uint32_t)((it >> 1) & 1);
        if (tid == 0) {
            int64_t cn = c + gridDim.x;
            if (cn < n_chunks) {               // stage s^1 was released by the barrier at the end of it-1
                issue(cn, s ^ 1);
                issued[s ^ 1] += 1;
            }
            bulk_wait_read0();                  // the previous bulk store finished reading ob
        }
        // wait for this chunk's inputs (bounded)
        bool ok = false;
        for (int spin = 0; spin < kSpinLimit; ++spin)
            if ((ok = mbar_try_wait(&bar[s], parity))) break;
        if (!ok) atomicExch(&abort_flag, 1);
        __syncthreads();
        if (abort_flag) break;

        const T *a = stage[s] + tid * OP::I0;
        const T *b = stage[s] + I0 + tid * OP::I1;
        T ra[OP::I0 > 0 ? OP::I0 : 1], rb[OP::I1 > 0 ? OP::I1 : 1], r0[OP::O0 > 0 ? OP::O0 : 1],
            r1[OP::O1 > 0 ? OP::O1 : 1];
#pragma unroll
        for (int e = 0; e < OP::I0; ++e) ra[e] = a[e];
#pragma unroll
        for (int e = 0; e < OP::I1; ++e) rb[e] = b[e];
        if (OP::apply(ra, rb, r0, r1)) ++local_sing;
#pragma unroll
        for (int e = 0; e < OP::O0; ++e) ob[tid * OP::O0 + e] = r0[e];
#pragma unroll
        for (int e = 0; e < OP::O1; ++e) ob[O0 + tid * OP::O1 + e] = r1[e];
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            bulk_s2g(out0 + c * O0, ob, (uint32_t)(O0 * sizeof(T)));
            if (O1) bulk_s2g(out1 + c * O1, ob + O0, (uint32_t)(O1 * sizeof(T)));
            bulk_commit();
        }
    }
    if (tid == 0) {
        bulk_wait0();
        if (abort_flag) {
            atomicOr(err, 1);
            // wait (bounded) for the last load issued into each stage before the CTA exits
            for (int s = 0; s < 2; ++s) {
                if (issued[s] == 0) continue;
                const uint32_t par = (uint32_t)((issued[s] - 1) & 1);
                for (int spin = 0; spin < kSpinLimit; ++spin)
                    if (mbar_try_wait(&bar[s], par)) break;
            }
        }
    }
    if (n_sing && local_sing) atomicAdd(n_sing, local_sing);
}

// ---------------------------------------------------------------------------
// plain page-major kernel (tail pages and misaligned pointers)
// ---------------------------------------------------------------------------
template <class OP, typename T>
__global__ void k_page_plain(int64_t begin, int64_t N, const T *__restrict__ in0, const T *__restrict__ in1,
                             T *__restrict__ out0, T *__restrict__ out1, unsigned long long *__restrict__ n_sing) {
    unsigned long long local_sing = 0;
    for (int64_t k = begin + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x) {
        T ra[OP::I0 > 0 ? OP::I0 : 1], rb[OP::I1 > 0 ? OP::I1 : 1], r0[OP::O0 > 0 ? OP::O0 : 1],
            r1[OP::O1 > 0 ? OP::O1 : 1];
#pragma unroll
        for (int e = 0; e < OP::I0; ++e) ra[e] = in0[k * OP::I0 + e];
#pragma unroll
        for (int e = 0; e < OP::I1; ++e) rb[e] = in1[k * OP::I1 + e];
        if (OP::apply(ra, rb, r0, r1)) ++local_sing;
#pragma unroll
        for (int e = 0; e < OP::O0; ++e) out0[k * OP::O0 + e] = r0[e];
#pragma unroll
        for (int e = 0; e < OP::O1; ++e) out1[k * OP::O1 + e] = r1[e];
    }
    if (n_sing && local_sing) atomicAdd(n_sing, local_sing);
}

// ---------------------------------------------------------------------------
// SoA kernel: entry e of page k at e*N + k
// ---------------------------------------------------------------------------
template <class OP, typename T>
__global__ void k_page_soa(int64_t N, const T *__restrict__ in0, const T *__restrict__ in1, T *__restrict__ out0,
                           T *__restrict__ out1, unsigned long long *__restrict__ n_sing) {
    unsigned long long local_sing = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        T ra[OP::I0 > 0 ? OP::I0 : 1], rb[OP::I1 > 0 ? OP::I1 : 1], r0[OP::O0 > 0 ? OP::O0 : 1],
            r1[OP::O1 > 0 ? OP::O1 : 1];
#pragma unroll
        for (int e = 0; e < OP::I0; ++e) ra[e] = in0[e * N + k];
#pragma unroll
        for (int e = 0; e < OP::I1; ++e) rb[e] = in1[e * N + k];
        if (OP::apply(ra, rb, r0, r1)) ++local_sing;
#pragma unroll
        for (int e = 0; e < OP::O0; ++e) out0[e * N + k] = r0[e];
#pragma unroll
        for (int e = 0; e < OP::O1; ++e) out1[e * N + k] = r1[e];
    }
    if (n_sing && local_sing) atomicAdd(n_sing, local_sing);
}

// ---------------------------------------------------------------------------
// products with one single matrix or vector (shapes chosen at run time, up to
// kBcastMax per side): one page per thread, the single object read through
// the read-only cache from device memory.  Page entry (i, j) of an r x c page
// k sits at k r c + i + j r (page layout) or (i + j r) N + k (SoA).
// ---------------------------------------------------------------------------
constexpr int kBcastMax = 16;
enum BcastOp { kAmsm, kAmsv, kSmamt, kSvamt };

template <typename T>
__global__ void k_page_bcast(int op, int64_t N, int soa, int m, int p, int n, const T *__restrict__ A,
                             const T *__restrict__ S, T *__restrict__ C) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        if (op == kAmsm) {   // A: m x p, S: p x n, C: m x n
            auto a = [&](int i, int r) { return soa ? A[(int64_t)(i + r * m) * N + k] : A[k * m * p + i + r * m]; };
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < m; ++i) {
                    T acc = 0;
                    for (int r = 0; r < p; ++r) acc += a(i, r) * __ldg(S + r + j * p);
                    const int64_t o = soa ? (int64_t)(i + j * m) * N + k : k * m * n + i + j * m;
                    C[o] = acc;
                }
        } else if (op == kSmamt) {   // S: m x p, A: n x p, C = S A^T: m x n
            auto a = [&](int j, int r) { return soa ? A[(int64_t)(j + r * n) * N + k] : A[k * n * p + j + r * n]; };
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < m; ++i) {
                    T acc = 0;
                    for (int r = 0; r < p; ++r) acc += __ldg(S + i + r * m) * a(j, r);
                    const int64_t o = soa ? (int64_t)(i + j * m) * N + k : k * m * n + i + j * m;
                    C[o] = acc;
                }
        } else {   // amsv / svamt: A: m x p, s: p, y_i = sum_r A(i, r) s_r (an m x 1 or 1 x m page)
            auto a = [&](int i, int r) { return soa ? A[(int64_t)(i + r * m) * N + k] : A[k * m * p + i + r * m]; };
            for (int i = 0; i < m; ++i) {
                T acc = 0;
                for (int r = 0; r < p; ++r) acc += a(i, r) * __ldg(S + r);
                C[soa ? (int64_t)i * N + k : k * m + i] = acc;
            }
        }
    }
}

// The same products for a page of compile-time shape R x CC held in
// registers; the single object's other dimension (`other`) stays a run-time
// loop.  amsm/amsv: page A (R x CC) times S (CC x other) -> R x other.
// smamt: S (other x CC) times the transposed page (R x CC) -> other x R.
template <typename T, int R, int CC>
__global__ void k_page_bcast_rc(int op, int64_t N, int soa, int other, const T *__restrict__ A,
                                const T *__restrict__ S, T *__restrict__ C) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        T a[R * CC];
#pragma unroll
        for (int e = 0; e < R * CC; ++e) a[e] = soa ? A[(int64_t)e * N + k] : A[k * (R * CC) + e];
        if (op == kSmamt) {
            for (int i = 0; i < other; ++i) {
                T srow[CC];
#pragma unroll
                for (int r = 0; r < CC; ++r) srow[r] = __ldg(S + i + r * other);
#pragma unroll
                for (int j = 0; j < R; ++j) {
                    T acc = 0;
#pragma unroll
                    for (int r = 0; r < CC; ++r) acc += srow[r] * a[j + r * R];
                    const int e = i + j * other;
                    C[soa ? (int64_t)e * N + k : k * (other * R) + e] = acc;
                }
            }
        } else {
            for (int j = 0; j < other; ++j) {
                T scol[CC];
#pragma unroll
                for (int r = 0; r < CC; ++r) scol[r] = __ldg(S + r + j * CC);
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    T acc = 0;
#pragma unroll
                    for (int r = 0; r < CC; ++r) acc += a[i + r * R] * scol[r];
                    const int e = i + j * R;
                    C[soa ? (int64_t)e * N + k : k * (R * other) + e] = acc;
                }
            }
        }
    }
}

int num_sms();

// Page-major pages of compile-time shape R x CC through shared memory.  A
// page-major page is R*CC contiguous words, so one page per thread reads and
// writes with a stride of a whole page per lane (one cache line per page per
// warp access, L1-wavefront bound).  Here the block reads its PB pages with
// consecutive threads on consecutive words, keeps them at an odd per-page
// stride (R*CC, or R*CC + 1 when that is even: the page reads of a warp fall
// on distinct banks), each thread forms its result page from there into a
// second area (odd stride likewise from OUT), and the block writes the result
// pages back with consecutive words.
// `div_in`/`div_out` are ceil(2^32 / size) for the page index of a word by one
// multiply-high (exact for words below 2^32 / size).
template <typename T, int R, int CC>
__global__ void __launch_bounds__(512 / sizeof(T)) k_page_bcast_staged(int op, int64_t N, int other,
                                                                      const T *__restrict__ A,
                                                                      const T *__restrict__ S, T *__restrict__ C,
                                                                      uint32_t div_out) {
    constexpr int PB = 512 / sizeof(T), IN = R * CC, INS = IN | 1;
    constexpr uint32_t DIV_IN = (uint32_t)((0x100000000ull + IN - 1) / IN);
    const int OUT = R * other, OUTS = OUT | 1;
    extern __shared__ __align__(16) unsigned char smraw[];
    T *sa = reinterpret_cast<T *>(smraw);
    T *sc = sa + PB * INS;
    // the single matrix, read once per block (its uses below are broadcast
    // shared-memory reads instead of a global load per entry and page)
    T *ss = sc + ((PB * OUTS + 15) & ~15);
    const int t = threadIdx.x;
    for (int i = t; i < CC * other; i += PB) ss[i] = S[i];   // visible after the loop's first barrier
    for (int64_t k0 = (int64_t)blockIdx.x * PB; k0 < N; k0 += (int64_t)gridDim.x * PB) {
        const int np = (int)(N - k0 < PB ? N - k0 : PB);
        const T *src = A + k0 * IN;
        {   // IN words per thread, all loads in flight before the first store
            T v[IN];
#pragma unroll
            for (int q = 0; q < IN; ++q) {
                const int f = t + q * PB;
                v[q] = f < np * IN ? src[f] : T(0);
            }
#pragma unroll
            for (int q = 0; q < IN; ++q) {
                const int f = t + q * PB;
                const int pg = (int)__umulhi((uint32_t)f, DIV_IN);
                if (f < np * IN) sa[pg * INS + (f - pg * IN)] = v[q];
            }
        }
        __syncthreads();
        if (t < np) {
            T a[IN];
#pragma unroll
            for (int e = 0; e < IN; ++e) a[e] = sa[t * INS + e];
            T *out = sc + t * OUTS;
            if (op == kSmamt) {   // S (other x CC) times the transposed page: other x R
                for (int i = 0; i < other; ++i) {
                    T srow[CC];
#pragma unroll
                    for (int r = 0; r < CC; ++r) srow[r] = ss[i + r * other];
#pragma unroll
                    for (int j = 0; j < R; ++j) {
                        T acc = 0;
#pragma unroll
                        for (int r = 0; r < CC; ++r) acc += srow[r] * a[j + r * R];
                        out[i + j * other] = acc;
                    }
                }
            } else {   // amsm / amsv: the page (R x CC) times S (CC x other): R x other
                for (int j = 0; j < other; ++j) {
                    T scol[CC];
#pragma unroll
                    for (int r = 0; r < CC; ++r) scol[r] = ss[r + j * CC];
#pragma unroll
                    for (int i = 0; i < R; ++i) {
                        T acc = 0;
#pragma unroll
                        for (int r = 0; r < CC; ++r) acc += a[i + r * R] * scol[r];
                        out[i + j * R] = acc;
                    }
                }
            }
        }
        __syncthreads();
        T *dst = C + k0 * OUT;
        for (int f = t; f < np * OUT; f += PB) {
            const int pg = (int)__umulhi((uint32_t)f, div_out);
            dst[f] = sc[pg * OUTS + (f - pg * OUT)];
        }
        __syncthreads();   // the next pages overwrite both areas
    }
}

// launches the register-page kernel when the page shape is one of the
// instantiated ones (rows 1-3; columns 2, 3, 4, 6, 10: vertices, P2 nodes and
// the quadrature points of the Section 3.4/3.5 uses); false otherwise
template <typename T>
bool launch_bcast_rc(int op, int64_t N, int soa, int R, int CC, int other, const T *A, const T *S, T *C, int g,
                     cudaStream_t st) {
    // page-major pages of the matrix products go through shared memory (see k_page_bcast_staged;
    // amsm 0.28 -> 0.40, smamt 0.37 -> 0.68 of HBM on 1e7 3x4 pages); SoA pages are coalesced as they are, and
    // the matrix-vector forms (other == 1: amsv, svamt) read a page's few outputs faster one page per thread
    // (0.79 against 0.62 staged)
    constexpr int PB = 512 / sizeof(T);
    const int OUT = R * other;
    const uint32_t div_out = (uint32_t)((0x100000000ull + OUT - 1) / OUT);
    // pages (odd stride R CC | 1), results (odd stride OUT | 1, area padded to 16 words), the single matrix
    const size_t smem = ((size_t)PB * (size_t)((R * CC) | 1) + (((size_t)PB * (size_t)(OUT | 1) + 15) & ~(size_t)15) +
                         (size_t)CC * other) * sizeof(T);
    const int gs = grid_for(N, PB, (int64_t)num_sms() * 16);
#define VLA_RC(r_, c_)                                                                               \
    if (R == r_ && CC == c_) {                                                                       \
        if (soa || other == 1)                                                                       \
            k_page_bcast_rc<T, r_, c_><<<g, 256, 0, st>>>(op, N, soa, other, A, S, C);               \
        else                                                                                         \
            k_page_bcast_staged<T, r_, c_><<<gs, PB, smem, st>>>(op, N, other, A, S, C, div_out);    \
        return true;                                                                                 \
    }
#define VLA_RC_ROW(r_) VLA_RC(r_, 2) VLA_RC(r_, 3) VLA_RC(r_, 4) VLA_RC(r_, 6) VLA_RC(r_, 10)
    VLA_RC_ROW(1) VLA_RC_ROW(2) VLA_RC_ROW(3)
#undef VLA_RC_ROW
#undef VLA_RC
    return false;
}

int g_num_sms = 0;
int *g_err_flag[64] = {nullptr};

int num_sms() {
    if (g_num_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 152;
    }
    return g_num_sms;
}

template <class OP, typename T>
vla_status launch_op(int32_t layout, int64_t N, const void *in0, const void *in1, void *out0, void *out1,
                     unsigned long long *n_sing, cudaStream_t st) {
    const T *a = (const T *)in0;
    const T *b = (const T *)in1;
    T *c = (T *)out0;
    T *d = (T *)out1;
    if (N == 0) return VLA_OK;
    if (layout == VLA_LAYOUT_SOA) {
        k_page_soa<OP, T><<<grid_for(N, 256, (int64_t)num_sms() * 16), 256, 0, st>>>(N, a, b, c, d, n_sing);
        VLA_CUDA(cudaGetLastError());
        return VLA_OK;
    }
    auto al16 = [](const void *p) { return p == nullptr || ((uintptr_t)p & 15u) == 0; };
    int64_t n_chunks = N / kPagesPerChunk;
    int64_t staged = 0;
    if (n_chunks > 0 && al16(a) && al16(b) && al16(c) && al16(d)) {
        const size_t smem = (size_t)(2 * (OP::I0 + OP::I1) + OP::O0 + OP::O1) * kPagesPerChunk * sizeof(T);
        int dev = 0;
        VLA_CUDA(cudaGetDevice(&dev));
        if (dev < 0 || dev >= 64) return fail(VLA_ERR_INVALID_ARG, "device ordinal %d not supported", dev);
        {   // the staged kernel's shared-memory size is fixed per operation: set once per device
            static std::mutex mu;
            static bool attr_done[64] = {};
            std::lock_guard<std::mutex> lk(mu);
            if (!attr_done[dev]) {
                VLA_CUDA(cudaFuncSetAttribute(k_page_staged<OP, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)smem));
                attr_done[dev] = true;
            }
        }
        if (!g_err_flag[dev]) {
            VLA_CUDA(cudaMalloc(&g_err_flag[dev], sizeof(int)));
            VLA_CUDA(cudaMemset(g_err_flag[dev], 0, sizeof(int)));
        }
        int per_sm = (int)((227 * 1024) / (smem + 1024));
        if (per_sm < 1) per_sm = 1;
        if (per_sm > 8) per_sm = 8;
        int64_t grid = (int64_t)num_sms() * per_sm;
        if (grid > n_chunks) grid = n_chunks;
        k_page_staged<OP, T><<<(int)grid, kPagesPerChunk, smem, st>>>(n_chunks, a, b, c, d, n_sing, g_err_flag[dev]);
        VLA_CUDA(cudaGetLastError());
        staged = n_chunks * kPagesPerChunk;
    }
    if (staged < N) {
        k_page_plain<OP, T><<<grid_for(N - staged, 256, (int64_t)num_sms() * 16), 256, 0, st>>>(staged, N, a, b, c,
                                                                                                   d, n_sing);
        VLA_CUDA(cudaGetLastError());
    }
    return VLA_OK;
}

vla_status check_common(int32_t dtype, int32_t layout, int64_t N) {
    if (dtype != VLA_F32 && dtype != VLA_F64) return fail(VLA_ERR_INVALID_ARG, "dtype must be VLA_F32 or VLA_F64");
    if (layout != VLA_LAYOUT_PAGE && layout != VLA_LAYOUT_SOA)
        return fail(VLA_ERR_INVALID_ARG, "layout must be VLA_LAYOUT_PAGE or VLA_LAYOUT_SOA");
    if (N < 0 || N > (int64_t)1 << 40) return fail(VLA_ERR_INVALID_ARG, "page count N=%lld out of range", (long long)N);
    return VLA_OK;
}

bool dim_ok(int x) { return x == 2 || x == 3; }

}  // namespace
}  // namespace vla

using namespace vla;

#define DISPATCH_T(dtype, ...)            \
    ((dtype) == VLA_F32 ? [&] {           \
        using T = float;                  \
        return __VA_ARGS__;               \
    }()                                   \
                        : [&] {           \
                              using T = double; \
                              return __VA_ARGS__; \
                          }())

extern "C" vla_status vla_amtam(int32_t dtype, int32_t layout, int64_t N, int32_t p, int32_t m, int32_t n,
                                const void *A, const void *B, void *C, void *stream) {
    vla_status st = check_common(dtype, layout, N);
    if (st) return st;
    if (!dim_ok(p) || !dim_ok(m) || !dim_ok(n)) return fail(VLA_ERR_INVALID_ARG, "amtam: p, m, n must be 2 or 3");
    if (N > 0 && (!A || !B || !C)) return fail(VLA_ERR_INVALID_ARG, "amtam: null array");
    cudaStream_t s = (cudaStream_t)stream;
    int code = (p - 2) * 4 + (m - 2) * 2 + (n - 2);
    return DISPATCH_T(dtype, ([&]() -> vla_status {
        switch (code) {
        case 0: return launch_op<OpAmtam<T, 2, 2, 2>, T>(layout, N, A, B, C, nullptr, nullptr, s);
        case 1: return launch_op<OpAmtam<T, 2, 2, 3>, T>(layout, N, A, B, C, nullptr, nullptr, s);
        case 2: return launch_op<OpAmtam<T, 2, 3, 2>, T>(layout, N, A, B, C, nullptr, nullptr, s);
        case 3: return launch_op<OpAmtam<T, 2, 3, 3>, T>(layout, N, A, B, C, nullptr, nullptr, s);
        case 4: return launch_op<OpAmtam<T, 3, 2, 2>, T>(layout, N, A, B, C, nullptr, nullptr, s);
        case 5: return launch_op<OpAmtam<T, 3, 2, 3>, T>(layout, N, A, B, C, nullptr, nullptr, s);
        case 6: return launch_op<OpAmtam<T, 3, 3, 2>, T>(layout, N, A, B, C, nullptr, nullptr, s);
        default: return launch_op<OpAmtam<T, 3, 3, 3>, T>(layout, N, A, B, C, nullptr, nullptr, s);
        }
    }()));
}

extern "C" vla_status vla_astam(int32_t dtype, int32_t layout, int64_t N, int32_t m, int32_t n, const void *sv,
                                const void *A, void *C, void *stream) {
    vla_status st = check_common(dtype, layout, N);
    if (st) return st;
    if (!dim_ok(m) || !dim_ok(n)) return fail(VLA_ERR_INVALID_ARG, "astam: m, n must be 2 or 3");
    if (N > 0 && (!sv || !A || !C)) return fail(VLA_ERR_INVALID_ARG, "astam: null array");
    cudaStream_t s = (cudaStream_t)stream;
    int code = (m - 2) * 2 + (n - 2);
    return DISPATCH_T(dtype, ([&]() -> vla_status {
        switch (code) {
        case 0: return launch_op<OpAstam<T, 2, 2>, T>(layout, N, sv, A, C, nullptr, nullptr, s);
        case 1: return launch_op<OpAstam<T, 2, 3>, T>(layout, N, sv, A, C, nullptr, nullptr, s);
        case 2: return launch_op<OpAstam<T, 3, 2>, T>(layout, N, sv, A, C, nullptr, nullptr, s);
        default: return launch_op<OpAstam<T, 3, 3>, T>(layout, N, sv, A, C, nullptr, nullptr, s);
        }
    }()));
}

extern "C" vla_status vla_avtam(int32_t dtype, int32_t layout, int64_t N, int32_t p, int32_t n, const void *v,
                                const void *A, void *y, void *stream) {
    vla_status st = check_common(dtype, layout, N);
    if (st) return st;
    if (!dim_ok(p) || !dim_ok(n)) return fail(VLA_ERR_INVALID_ARG, "avtam: p, n must be 2 or 3");
    if (N > 0 && (!v || !A || !y)) return fail(VLA_ERR_INVALID_ARG, "avtam: null array");
    cudaStream_t s = (cudaStream_t)stream;
    int code = (p - 2) * 2 + (n - 2);
    return DISPATCH_T(dtype, ([&]() -> vla_status {
        switch (code) {
        case 0: return launch_op<OpAvtam<T, 2, 2>, T>(layout, N, v, A, y, nullptr, nullptr, s);
        case 1: return launch_op<OpAvtam<T, 2, 3>, T>(layout, N, v, A, y, nullptr, nullptr, s);
        case 2: return launch_op<OpAvtam<T, 3, 2>, T>(layout, N, v, A, y, nullptr, nullptr, s);
        default: return launch_op<OpAvtam<T, 3, 3>, T>(layout, N, v, A, y, nullptr, nullptr, s);
        }
    }()));
}

extern "C" vla_status vla_amdet(int32_t dtype, int32_t layout, int64_t N, int32_t n, const void *A, void *det,
                                void *stream) {
    vla_status st = check_common(dtype, layout, N);
    if (st) return st;
    if (!dim_ok(n)) return fail(VLA_ERR_INVALID_ARG, "amdet: n must be 2 or 3");
    if (N > 0 && (!A || !det)) return fail(VLA_ERR_INVALID_ARG, "amdet: null array");
    cudaStream_t s = (cudaStream_t)stream;
    return DISPATCH_T(dtype, ([&]() -> vla_status {
        return n == 2 ? launch_op<OpAmdet<T, 2>, T>(layout, N, A, nullptr, det, nullptr, nullptr, s)
                      : launch_op<OpAmdet<T, 3>, T>(layout, N, A, nullptr, det, nullptr, nullptr, s);
    }()));
}

extern "C" vla_status vla_aminv(int32_t dtype, int32_t layout, int64_t N, int32_t n, const void *A, void *Ainv,
                                void *det, int64_t *n_singular, void *stream) {
    vla_status st = check_common(dtype, layout, N);
    if (st) return st;
    if (!dim_ok(n)) return fail(VLA_ERR_INVALID_ARG, "aminv: n must be 2 or 3");
    if (N > 0 && (!A || !Ainv)) return fail(VLA_ERR_INVALID_ARG, "aminv: null array");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *ns = reinterpret_cast<unsigned long long *>(n_singular);
    if (ns) VLA_CUDA(cudaMemsetAsync(ns, 0, sizeof(unsigned long long), s));
    return DISPATCH_T(dtype, ([&]() -> vla_status {
        if (det) {
            return n == 2 ? launch_op<OpAminv<T, 2, true>, T>(layout, N, A, nullptr, Ainv, det, ns, s)
                          : launch_op<OpAminv<T, 3, true>, T>(layout, N, A, nullptr, Ainv, det, ns, s);
        }
        return n == 2 ? launch_op<OpAminv<T, 2, false>, T>(layout, N, A, nullptr, Ainv, nullptr, ns, s)
                      : launch_op<OpAminv<T, 3, false>, T>(layout, N, A, nullptr, Ainv, nullptr, ns, s);
    }()));
}

extern "C" vla_status vla_amt(int32_t dtype, int32_t layout, int64_t N, int32_t m, int32_t n, const void *A, void *C,
                              void *stream) {
    vla_status st = check_common(dtype, layout, N);
    if (st) return st;
    if (!dim_ok(m) || !dim_ok(n)) return fail(VLA_ERR_INVALID_ARG, "amt: m, n must be 2 or 3");
    if (N > 0 && (!A || !C)) return fail(VLA_ERR_INVALID_ARG, "amt: null array");
    cudaStream_t s = (cudaStream_t)stream;
    int code = (m - 2) * 2 + (n - 2);
    return DISPATCH_T(dtype, ([&]() -> vla_status {
        switch (code) {
        case 0: return launch_op<OpAmt<T, 2, 2>, T>(layout, N, A, nullptr, C, nullptr, nullptr, s);
        case 1: return launch_op<OpAmt<T, 2, 3>, T>(layout, N, A, nullptr, C, nullptr, nullptr, s);
        case 2: return launch_op<OpAmt<T, 3, 2>, T>(layout, N, A, nullptr, C, nullptr, nullptr, s);
        default: return launch_op<OpAmt<T, 3, 3>, T>(layout, N, A, nullptr, C, nullptr, nullptr, s);
        }
    }()));
}

extern "C" vla_status vla_avtav(int32_t dtype, int32_t layout, int64_t N, int32_t n, const void *a, const void *b,
                                void *out, void *stream) {
    vla_status st = check_common(dtype, layout, N);
    if (st) return st;
    if (!dim_ok(n)) return fail(VLA_ERR_INVALID_ARG, "avtav: n must be 2 or 3");
    if (N > 0 && (!a || !b || !out)) return fail(VLA_ERR_INVALID_ARG, "avtav: null array");
    cudaStream_t s = (cudaStream_t)stream;
    return DISPATCH_T(dtype, ([&]() -> vla_status {
        return n == 2 ? launch_op<OpAvtav<T, 2>, T>(layout, N, a, b, out, nullptr, nullptr, s)
                      : launch_op<OpAvtav<T, 3>, T>(layout, N, a, b, out, nullptr, nullptr, s);
    }()));
}

namespace {
vla_status launch_bcast(const char *name, int op, int32_t dtype, int32_t layout, int64_t N, int m, int p, int n,
                        const void *A, const void *S, void *C, void *stream) {
    vla_status st = check_common(dtype, layout, N);
    if (st) return st;
    if (m < 1 || p < 1 || n < 1 || m > kBcastMax || p > kBcastMax || n > kBcastMax)
        return fail(VLA_ERR_INVALID_ARG, "%s: dimensions must be in [1, %d]", name, kBcastMax);
    if (N > 0 && (!A || !S || !C)) return fail(VLA_ERR_INVALID_ARG, "%s: null array", name);
    if (N == 0) return VLA_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int soa = layout == VLA_LAYOUT_SOA;
    const int g = grid_for(N, 256, (int64_t)num_sms() * 16);
    // page shape and the single object's other dimension
    const int R = op == kSmamt ? n : m, CC = p, other = op == kSmamt ? m : n;
    const bool fast = dtype == VLA_F32
                          ? launch_bcast_rc<float>(op, N, soa, R, CC, other, (const float *)A, (const float *)S,
                                                   (float *)C, g, s)
                          : launch_bcast_rc<double>(op, N, soa, R, CC, other, (const double *)A, (const double *)S,
                                                    (double *)C, g, s);
    if (fast) {
        VLA_CUDA(cudaGetLastError());
        return VLA_OK;
    }
    if (dtype == VLA_F32)
        k_page_bcast<float><<<g, 256, 0, s>>>(op, N, soa, m, p, n, (const float *)A, (const float *)S, (float *)C);
    else
        k_page_bcast<double><<<g, 256, 0, s>>>(op, N, soa, m, p, n, (const double *)A, (const double *)S, (double *)C);
    VLA_CUDA(cudaGetLastError());
    return VLA_OK;
}
}  // namespace

extern "C" vla_status vla_amsm(int32_t dtype, int32_t layout, int64_t N, int32_t m, int32_t p, int32_t n,
                               const void *A, const void *S, void *C, void *stream) {
    return launch_bcast("amsm", kAmsm, dtype, layout, N, m, p, n, A, S, C, stream);
}

extern "C" vla_status vla_amsv(int32_t dtype, int32_t layout, int64_t N, int32_t m, int32_t n, const void *A,
                               const void *sv, void *y, void *stream) {
    return launch_bcast("amsv", kAmsv, dtype, layout, N, m, n, 1, A, sv, y, stream);
}

extern "C" vla_status vla_smamt(int32_t dtype, int32_t layout, int64_t N, int32_t m, int32_t p, int32_t n,
                                const void *S, const void *A, void *C, void *stream) {
    return launch_bcast("smamt", kSmamt, dtype, layout, N, m, p, n, A, S, C, stream);
}

extern "C" vla_status vla_svamt(int32_t dtype, int32_t layout, int64_t N, int32_t m, int32_t n, const void *sv,
                                const void *A, void *y, void *stream) {
    return launch_bcast("svamt", kSvamt, dtype, layout, N, m, n, 1, A, sv, y, stream);
}
