// vla_internal.cuh -- shared internals of libvla (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>
#include <vector>

#include "vla.h"

namespace vla {

// ---------------------------------------------------------------------------
// error reporting (thread-local last message, see vla_last_error)
// ---------------------------------------------------------------------------
void set_error(const char *fmt, ...);
vla_status fail(vla_status st, const char *fmt, ...);
vla_status cuda_fail(cudaError_t e, const char *what);

// Launch parameters chosen by the autotuner (process-wide, all devices), per
// element type (dim - 2) * 2 + (order - 1): the incidence budget of a row
// tile used when a mesh is built, and the resident CTAs per SM of the
// assembly launch per precision.  0 means the library default.
int tuned_budget(int type);
int tile_budget(int dim, int order);   // the default per element type
// stream-ordered device allocation from the library's pool of this device,
// which keeps freed memory mapped for the next mesh build (up to a limit)
cudaError_t pool_malloc(void **p, size_t bytes, cudaStream_t st);
int tuned_ctas(int type, bool mix);
void set_tuned(int type, bool mix, int budget, int ctas);

// vla_mesh_create with an explicit tile budget (0: tuned or default)
vla_status mesh_create_budget(int32_t dim, int32_t order, int64_t nn, int64_t ne, const double *coords,
                              const int32_t *elems, int64_t nfb, const int32_t *faces, void *stream, int budget,
                              vla_mesh **out);

// returns the status of a library call that failed
#define TRY(...)                      \
    do {                              \
        vla_status s_ = (__VA_ARGS__); \
        if (s_ != VLA_OK) return s_;  \
    } while (0)

#define VLA_CUDA(call)                                              \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return ::vla::cuda_fail(e_, #call);  \
    } while (0)

inline int grid_for(int64_t n, int block, int64_t cap = 152 * 64) {
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

// ---------------------------------------------------------------------------
// float-float helpers (error-free transformations, round-to-nearest)
// ---------------------------------------------------------------------------

// s + e == a + b exactly (Knuth's TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// p + e == a * b exactly (FMA-based TwoProduct).
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// a*d - b*c with at most ~1.5 ulp error (Kahan's FMA algorithm).
__device__ __forceinline__ float det2_kahan(float a, float b, float c, float d) {
    float w = __fmul_rn(b, c);
    float e = __fmaf_rn(-b, c, w);
    float f = __fmaf_rn(a, d, -w);
    return __fadd_rn(f, e);
}

// compensated accumulator: value = hi + lo
struct ffacc {
    float hi, lo;
    __device__ __forceinline__ void zero() { hi = 0.f; lo = 0.f; }
    __device__ __forceinline__ void add(float x) {
        float s, e;
        two_sum(hi, x, s, e);
        hi = s;
        lo = __fadd_rn(lo, e);
    }
    // normalise so that |lo| <= ulp(hi)/2
    __device__ __forceinline__ void norm() {
        float s, e;
        two_sum(hi, lo, s, e);
        hi = s;
        lo = e;
    }
};

// ---------------------------------------------------------------------------
// FP32 -> FP64 conversions with integer instructions only.  The FP64 and
// conversion pipes of the GB300 SM run at a small fraction of the FP32 rate,
// so the mixed-precision kernels build the IEEE-754 binary64 bit patterns
// directly.
// ---------------------------------------------------------------------------

// exact conversion of any float (normal, subnormal, zero, inf, nan)
__device__ __forceinline__ unsigned long long f32_to_f64_bits(float x) {
    uint32_t u = __float_as_uint(x);
    unsigned long long s = (unsigned long long)(u >> 31) << 63;
    uint32_t e = (u >> 23) & 0xffu;
    uint32_t m = u & 0x7fffffu;
    if (e == 0xffu) return s | 0x7ff0000000000000ull | ((unsigned long long)m << 29);
    if (e == 0) {
        if (m == 0) return s;
        int p = 31 - __clz(m);                         // leading one of the subnormal mantissa, 0..22
        unsigned long long mant = ((unsigned long long)m << (52 - p)) & 0xfffffffffffffull;
        unsigned long long ex = (unsigned long long)(p - 149 + 1023);
        return s | (ex << 52) | mant;
    }
    return s | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)m << 29);
}

__device__ __forceinline__ double f32_to_f64(float x) { return __longlong_as_double((long long)f32_to_f64_bits(x)); }

// float -> double by integer widening of the bit pattern: exact for normal
// numbers and zeros; subnormal floats, inf and nan take the general path.
__device__ __forceinline__ double f32_to_f64_w(float x) {
    const uint32_t u = __float_as_uint(x);
    const uint32_t a = u & 0x7fffffffu;
    const uint32_t e = a >> 23;
    if (e == 0xffu || (e == 0u && a != 0u)) return f32_to_f64(x);
    const unsigned long long mag = a ? (((unsigned long long)a << 29) + (896ull << 52)) : 0ull;
    return __longlong_as_double((long long)(((unsigned long long)(u >> 31) << 63) | mag));
}

// hi + lo of a float pair as the correctly rounded double: both parts are
// widened exactly with integer instructions and added once in FP64 (one
// instruction on the otherwise idle FP64 pipe instead of a ~45-instruction
// integer significand construction).
__device__ __forceinline__ double ff_to_f64(float hi, float lo) { return f32_to_f64_w(hi) + f32_to_f64_w(lo); }

// hi + lo of a normalised float pair (|lo| <= ulp(hi)/2) as a double without
// the FP64 pipe: hi is widened exactly with integer instructions, and lo is
// counted in units of the double ulp of hi, d = trunc(lo * 2^(52 - E_hi)) (one
// exact power-of-two multiply carrying hi's sign, one float-to-int conversion;
// |d| <= 2^28, so adding d to the widened bit pattern never carries out of
// hi's significand).  When hi is a power of two and lo lowers it, the result
// lies one binade down, where the ulp halves and d counts twice.  Bits of lo
// below the double ulp of hi are dropped: the result is within one double ulp
// of hi + lo.  hi below 2^-75, zero, subnormal, inf or nan takes the FP64 path.
__device__ __forceinline__ double ff_to_f64_int(float hi, float lo) {
    const uint32_t uh = __float_as_uint(hi), eh = (uh >> 23) & 0xffu;
    if (eh < 52u || eh == 0xffu) return ff_to_f64(hi, lo);
    const float scale = __uint_as_float((uh & 0x80000000u) | ((306u - eh) << 23));   // +-2^(52 - E_hi)
    int d = __float2int_rz(__fmul_rn(lo, scale));
    if ((uh & 0x7fffffu) == 0u && d < 0) d *= 2;
    const unsigned long long bits = ((unsigned long long)(uh & 0x80000000u) << 32) |
                                    (((unsigned long long)(uh & 0x7fffffffu) << 29) + (896ull << 52));
    return __longlong_as_double((long long)(bits + (unsigned long long)(long long)d));
}

// ---------------------------------------------------------------------------
// PTX wrappers: mbarrier + 1-D bulk TMA (cp.async.bulk), sm_90+
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
        "r"(bytes)
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void bulk_s2g(void *dst, const void *src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// bounded wait on an mbarrier phase; false if the limit expired
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int limit) {
    for (int i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// ---------------------------------------------------------------------------
// mesh handle
// ---------------------------------------------------------------------------

// Per-tile header produced by the mesh build.  Every per-tile segment starts
// on a 16-byte boundary and its byte size is padded to a multiple of 16, so
// the assembly kernel can stage it into shared memory with one bulk copy.
struct TileHdr {
    int32_t node_off, n_nodes;    // tile_nodes: vertex node ids (int32)
    int32_t elem_off, n_elems;    // tile_elem: local vertex indices (ushort4); owned elements first
    int32_t own_off, n_own;       // tile_own: global ids of the owned elements (int32)
    int32_t nz_off, n_nz;         // tile_nzpos: (p_ij, p_ji) CSR positions (int2); upper pairs, then diagonals
    int32_t n_up;                 // number of off-diagonal pairs {i, j}
    int32_t chunk_off, n_chunks;  // tile_chunks: (code offset in the tile's segment, width) per 32 pairs
    int32_t code_off, n_codes;    // tile_codes segment (in codes; multiple of 32)
    int32_t rank_begin, n_rows;   // rows of the tile: ranks [rank_begin, rank_begin + n_rows) of the order
    int32_t pad;
};

constexpr int kTilePadNodes = 4, kTilePadElems = 2, kTilePadOwn = 4, kTilePadNz = 2, kTilePadChunks = 2;

}  // namespace vla

struct vla_mesh {
    int32_t dim, order, nlb;
    int64_t nn, ne, nfb, nnz;
    int32_t max_row_len;
    int32_t n_tiles;
    int32_t max_tile_nodes, max_tile_elems, max_tile_nz;
    int32_t tile_budget;
    int64_t n_codes;
    int64_t tile_elems_total;     // sum over tiles of their element counts (recompute factor * ne)
    size_t tile_stage_bytes;      // largest per-tile staged segment set (ids, records, owned, chunks, pairs, codes)
    size_t tile_smem;             // shared memory per CTA of the mixed-precision assembly launch
    int32_t spin_limit;           // bounded waits on bulk copies
    int32_t *d_err;               // device error word (bit 0: a bounded wait expired)
    int64_t device_bytes;
    int32_t row_begin = 0, row_end = -1;   // a row-block sub-mesh (vla_mesh_create_rows): its complete rows
    cudaStream_t stream;

    double *coords;        // nn x dim
    int32_t *elems;        // ne x nlb
    int32_t *faces;        // nfb x dim
    int32_t *face_opp;     // nfb: remaining vertex of the owning element
    float4 *xh, *xl;       // float pair split of coords (w = 0)
    int32_t *row_ptr, *col_idx;
    int32_t *n2e_ptr, *n2e;

    vla::TileHdr *tiles;
    int32_t *tile_nodes;   // global node ids per tile
    ushort4 *tile_elem;    // local vertex indices per tile element
    int32_t *tile_own;     // global ids of owned elements
    int32_t *tile_eid;     // global ids of every tile element (owned first), as tile_elem
    int2 *tile_nzpos;      // (p_ij, p_ji) CSR positions of each tile pair
    int2 *tile_chunks;     // (code offset within the tile segment, width) per 32-pair chunk
    void *tile_codes;      // uint16 (P1) or uint32 (P2) contribution codes, chunk-interleaved

    std::vector<void *> allocs;  // every device allocation owned by the handle
};
