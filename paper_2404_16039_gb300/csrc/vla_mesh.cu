// vla_mesh.cu -- mesh ingest on the device: validation, node->element
// incidence, the CSR pattern of the sparse assembly of Section 3.5,
// boundary-facet owners, the float-pair split of the coordinates, and the row
// tiles used by the assembly kernel.
//
// Row tiles.  Assembly is a gather problem: CSR entry (i,j) sums the
// (i,j) entries of every element containing nodes i and j.  The assembly
// kernel gives each CTA a set of rows that are close in space (nodes sorted
// by the Morton code of their cell), recomputes in shared memory the element
// matrices of every element touching those rows, and sums them per nonzero
// from shared memory.  The build below produces, per tile: its vertex nodes,
// its elements (local vertex indices), the elements it owns (writes volume and
// pages for), the global CSR position of each of its nonzeros, and for every
// nonzero the list of (local element, a, b) contribution codes in ascending
// element order, laid out 32 nonzeros at a time so that lane l of a warp reads
// code t of nonzero l from consecutive addresses.  The summation order of
// every CSR entry is therefore fixed by the mesh alone (ascending element id),
// which makes assembly bit-reproducible.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <set>

#include "vla_internal.cuh"

namespace vla {
namespace {

constexpr int kMaxRow = 255;   // CSR row length limit (slot fits a byte)
constexpr int kScanItems = 8;  // items per thread of the block scan
constexpr int kScanThreads = 256;

// ---------------------------------------------------------------------------
// device-wide exclusive scan of int32 or int64 values into int64
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long warp_incl_scan(long long v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        long long t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// block-wide exclusive scan of one value per thread; returns the block total in *total
__device__ long long block_excl_scan(long long v, long long *total) {
    __shared__ long long warp_sums[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    long long inc = warp_incl_scan(v);
    if (lane == 31) warp_sums[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        long long s = lane < nw ? warp_sums[lane] : 0;
        long long si = warp_incl_scan(s);
        if (lane < nw) warp_sums[lane] = si - s;
        if (lane == nw - 1) warp_sums[31] = si;
    }
    __syncthreads();
    long long res = inc - v + warp_sums[wid];
    long long tot = warp_sums[31];
    __syncthreads();
    if (total) *total = tot;
    return res;
}

template <typename TI>
__global__ void k_scan_blocks(int64_t n, const TI *__restrict__ in, long long *__restrict__ out,
                              long long *__restrict__ block_sums) {
    const int64_t base = (int64_t)blockIdx.x * kScanThreads * kScanItems + (int64_t)threadIdx.x * kScanItems;
    long long vals[kScanItems];
    long long s = 0;
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        int64_t i = base + q;
        vals[q] = (i < n) ? (long long)in[i] : 0;
        s += vals[q];
    }
    long long tot;
    long long pre = block_excl_scan(s, &tot);
#pragma unroll
    for (int q = 0; q < kScanItems; ++q) {
        int64_t i = base + q;
        if (i < n) out[i] = pre;
        pre += vals[q];
    }
    if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

__global__ void k_scan_add(int64_t n, long long *__restrict__ out, const long long *__restrict__ block_pre) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += block_pre[i / (kScanThreads * kScanItems)];
}

__global__ void k_i64_to_i32(int64_t n, const long long *__restrict__ in, int32_t *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (int32_t)in[i];
}

// Small pinned host buffer for the scalars a build reads back (one per host
// thread, allocated on first use): device-to-host copies into pageable memory
// would each wait for the whole stream.
// Pinned host buffers per host thread, freed when the thread ends (server
// ingest threads come and go with their servers)
struct PinnedBuf {
    void *p = nullptr;
    size_t cap = 0;
    ~PinnedBuf() {
        if (p) cudaFreeHost(p);
    }
    void *get(size_t bytes, size_t min_bytes) {
        if (bytes > cap) {
            if (p) cudaFreeHost(p);
            p = nullptr;
            cap = 0;
            const size_t want = bytes > min_bytes ? bytes + bytes / 4 : min_bytes;
            if (cudaMallocHost(&p, want) != cudaSuccess) {
                cudaGetLastError();
                return nullptr;
            }
            cap = want;
        }
        return p;
    }
};

// a growable buffer for the tile tables a build reads back and sends down
// (pageable copies of a few hundred KB go through a driver staging buffer);
// every build ends with a synchronisation before the thread's next build
// reuses it
void *pinned_tables(size_t bytes) {
    static thread_local PinnedBuf b;
    return b.get(bytes, (size_t)1 << 20);
}

// scalars read back through pinned memory (scan totals, error word, maxima)
long long *pinned_scalars() {
    static thread_local PinnedBuf b;
    return static_cast<long long *>(b.get(64 * sizeof(long long), 64 * sizeof(long long)));
}

// out[n] = out[n - 1] + in[n - 1] (the total), on the device
template <typename TI>
__global__ void k_scan_total(int64_t n, const TI *__restrict__ in, long long *__restrict__ out) {
    out[n] = n > 0 ? out[n - 1] + (long long)in[n - 1] : 0;
}

// out[0] = max(out[0], max_i in[i] + add) for non-negative values (out[0]
// zeroed beforehand); a max is independent of the order of the atomics
__global__ void k_max_i32(int64_t n, const int32_t *__restrict__ in, int add, long long *__restrict__ out) {
    int v = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v = max(v, in[i] + add);
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_down_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0 && v > 0) atomicMax(reinterpret_cast<unsigned long long *>(out), (unsigned long long)v);
}

// Device scratch of the mesh passes, per host thread and device, kept from
// one call to the next: a call's temporary buffers are carved in order from
// chunks of device memory the thread holds (a new chunk comes from the
// library pool only when the held ones are full) and given back in reverse
// order when the call's Scratch ends, instead of one pool allocation and one
// free per buffer.  The end of a thread's outermost Scratch is recorded as an
// event on its stream, and the thread's next call waits for it on its own
// stream (a call on the same stream is ordered anyway).  More than
// kScratchKeep bytes held are returned to the pool when the thread's
// outermost Scratch ends; the rest is freed when the thread ends.
constexpr size_t kScratchKeep = (size_t)512 << 20, kScratchChunk = (size_t)32 << 20, kScratchAlign = 256;
struct ScratchArena {
    struct Chunk {
        char *p;
        size_t cap, used;
    };
    std::vector<Chunk> chunks;
    size_t cur = 0, held = 0;
    int depth = 0, dev = -1;
    cudaEvent_t done = nullptr;   // recorded where the last outermost Scratch ended
    cudaStream_t done_st = nullptr;
    bool pending = false;
    void release(cudaStream_t st) {
        for (const Chunk &c : chunks) cudaFreeAsync(c.p, st);
        chunks.clear();
        cur = 0;
        held = 0;
    }
    ~ScratchArena() {
        if (chunks.empty() && !done) return;
        int old = 0;
        if (cudaGetDevice(&old) != cudaSuccess || cudaSetDevice(dev) != cudaSuccess) return;
        for (const Chunk &c : chunks) cudaFree(c.p);
        if (done) cudaEventDestroy(done);
        cudaSetDevice(old);
        cudaGetLastError();
    }
};
constexpr int kScratchDevices = 64;
ScratchArena *scratch_arena(int dev) {   // a fixed table: arenas never move while a Scratch points at one
    static thread_local ScratchArena a[kScratchDevices];
    if (dev < 0 || dev >= kScratchDevices) return nullptr;
    a[dev].dev = dev;
    return &a[dev];
}

struct Scratch {  // temporary device buffers of one call, given back when it ends
    cudaStream_t st = nullptr;
    ScratchArena *A = nullptr;
    size_t mark_cur = 0, mark_used = 0;
    template <typename T>
    vla_status get(T **p, size_t count) {
        void *q = nullptr;
        vla_status s = get_bytes(&q, sizeof(T) * (count > 0 ? count : 1));
        *p = static_cast<T *>(q);
        return s;
    }
    vla_status get_bytes(void **p, size_t bytes) {
        if (!A) {
            int dev = 0;
            VLA_CUDA(cudaGetDevice(&dev));
            A = scratch_arena(dev);
            if (!A) return fail(VLA_ERR_UNSUPPORTED, "device ordinal %d beyond the scratch table", dev);
            if (A->depth == 0 && A->pending && A->done_st != st) VLA_CUDA(cudaStreamWaitEvent(st, A->done, 0));
            A->depth += 1;
            mark_cur = A->cur;
            mark_used = A->chunks.empty() ? 0 : A->chunks[A->cur].used;
        }
        bytes = (bytes + kScratchAlign - 1) / kScratchAlign * kScratchAlign;
        while (!A->chunks.empty() && A->chunks[A->cur].cap - A->chunks[A->cur].used < bytes &&
               A->cur + 1 < A->chunks.size() && A->chunks[A->cur + 1].cap >= bytes)
            A->cur += 1;   // chunks past cur hold nothing
        if (A->chunks.empty() || A->chunks[A->cur].cap - A->chunks[A->cur].used < bytes) {
            const size_t last = A->chunks.empty() ? 0 : A->chunks.back().cap;
            const size_t cap = std::max(bytes, std::max(kScratchChunk, 2 * last));
            void *q = nullptr;
            cudaError_t e = pool_malloc(&q, cap, st);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(VLA_ERR_OOM, "device scratch allocation of %zu bytes failed", cap);
            }
            // the new chunk goes right after cur, so that chunks past cur stay empty
            A->chunks.insert(A->chunks.begin() + (A->chunks.empty() ? 0 : A->cur + 1),
                             ScratchArena::Chunk{static_cast<char *>(q), cap, 0});
            if (A->chunks.size() > 1) A->cur += 1;
            A->held += cap;
        }
        ScratchArena::Chunk &c = A->chunks[A->cur];
        *p = c.p + c.used;
        c.used += bytes;
        return VLA_OK;
    }
    ~Scratch() {
        if (!A) return;
        for (size_t i = mark_cur + 1; i < A->chunks.size(); ++i) A->chunks[i].used = 0;
        if (!A->chunks.empty()) A->chunks[mark_cur].used = mark_used;
        A->cur = mark_cur;
        A->depth -= 1;
        if (A->depth > 0) return;
        if (A->held > kScratchKeep) A->release(st);
        if (!A->done && cudaEventCreateWithFlags(&A->done, cudaEventDisableTiming) != cudaSuccess) {
            A->done = nullptr;
            cudaGetLastError();
            cudaStreamSynchronize(st);   // no event: leave nothing in flight on the memory
            A->pending = false;
            return;
        }
        cudaEventRecord(A->done, st);
        A->done_st = st;
        A->pending = true;
    }
};

// out[i] = sum_{j<i} in[j] for i in [0, n], all on the device; if total_host
// is given the total is read back (the only synchronisation).
template <typename TI>
vla_status excl_scan(const TI *in, int64_t n, long long *out, cudaStream_t st, long long *total_host) {
    const int64_t per = (int64_t)kScanThreads * kScanItems;
    int64_t nb = (n + per - 1) / per;
    if (nb < 1) nb = 1;
    Scratch S;   // the block sums
    S.st = st;
    long long *bs = nullptr, *bsp = nullptr;
    TRY(S.get(&bs, nb + 1));
    TRY(S.get(&bsp, nb + 1));
    k_scan_blocks<TI><<<(int)nb, kScanThreads, 0, st>>>(n, in, out, bs);
    VLA_CUDA(cudaGetLastError());
    if (nb > 1) {
        vla_status s = excl_scan<long long>(bs, nb, bsp, st, nullptr);
        if (s) return s;
        k_scan_add<<<grid_for(n, 256, 1 << 30), 256, 0, st>>>(n, out, bsp);
        VLA_CUDA(cudaGetLastError());
    }
    k_scan_total<TI><<<1, 1, 0, st>>>(n, in, out);
    VLA_CUDA(cudaGetLastError());
    if (total_host) {
        long long *hp = pinned_scalars();
        if (!hp) return fail(VLA_ERR_OOM, "pinned host scalars");
        VLA_CUDA(cudaMemcpyAsync(hp, out + n, sizeof(long long), cudaMemcpyDeviceToHost, st));
        VLA_CUDA(cudaStreamSynchronize(st));
        *total_host = hp[0];
    }
    return VLA_OK;
}

// ---------------------------------------------------------------------------
// validation and incidence
// ---------------------------------------------------------------------------
enum { ERR_OOB = 1, ERR_DUP = 2, ERR_ROWLEN = 4, ERR_FACE_OOB = 8, ERR_FACE_OWNER = 16, ERR_TILE_CAP = 32,
       ERR_NODE_CAP = 64 };

__global__ void k_validate_count(int64_t ne, int nlb, int64_t nn, const int32_t *__restrict__ elems,
                                 int32_t *__restrict__ cnt, int *__restrict__ err, long long *__restrict__ bad) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < ne; k += (int64_t)gridDim.x * blockDim.x) {
        int32_t v[10];
        bool ok = true;
        for (int j = 0; j < nlb; ++j) {
            v[j] = elems[k * nlb + j];
            if (v[j] < 0 || v[j] >= nn) ok = false;
        }
        if (!ok) {
            atomicOr(err, ERR_OOB);
            atomicMin(bad, (long long)k);
            continue;
        }
        for (int j = 0; j < nlb; ++j)
            for (int q = 0; q < j; ++q)
                if (v[q] == v[j]) ok = false;
        if (!ok) {
            atomicOr(err, ERR_DUP);
            atomicMin(bad, (long long)k);
            continue;
        }
        for (int j = 0; j < nlb; ++j) atomicAdd(&cnt[v[j]], 1);
    }
}

// does nothing when validation found a bad element (the build reads the error
// word at its next synchronisation and fails there)
__global__ void k_fill_n2e(int64_t ne, int nlb, const int32_t *__restrict__ elems, int32_t *__restrict__ cursor,
                           int32_t *__restrict__ n2e, const int *__restrict__ err) {
    if (*err & (ERR_OOB | ERR_DUP)) return;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < ne; k += (int64_t)gridDim.x * blockDim.x)
        for (int j = 0; j < nlb; ++j) {
            int32_t pos = atomicAdd(&cursor[elems[k * nlb + j]], 1);
            n2e[pos] = (int32_t)((k << 4) | j);
        }
}

// Sorts every segment [ptr[i], ptr[i+1]) of v ascending (the nodes'
// incidence lists by element id, the Morton buckets by node id), one warp per
// segment: up to 32 keys by a bitonic sort across the lanes (shuffles), longer
// ones by insertion on one lane
constexpr int kSegWarps = 8;
__global__ void __launch_bounds__(kSegWarps * 32) k_sort_segments(int64_t n, const int32_t *__restrict__ ptr,
                                                                  int32_t *__restrict__ v) {
    const int lane = threadIdx.x & 31;
    for (int64_t i = (int64_t)blockIdx.x * kSegWarps + (threadIdx.x >> 5); i < n;
         i += (int64_t)gridDim.x * kSegWarps) {
        const int32_t b = ptr[i], e = ptr[i + 1], len = e - b;
        if (len <= 1) continue;
        if (len <= 32) {
            int32_t x = lane < len ? v[b + lane] : 0x7fffffff;
            for (int k = 2; k <= 32; k <<= 1)
                for (int j = k >> 1; j > 0; j >>= 1) {
                    const int32_t y = __shfl_xor_sync(0xffffffffu, x, j);
                    const bool keep_min = ((lane & j) == 0) == ((lane & k) == 0);
                    x = keep_min ? min(x, y) : max(x, y);
                }
            if (lane < len) v[b + lane] = x;
        } else if (lane == 0) {
            for (int32_t p = b + 1; p < e; ++p) {
                const int32_t x = v[p];
                int32_t q = p - 1;
                while (q >= b && v[q] > x) {
                    v[q + 1] = v[q];
                    --q;
                }
                v[q + 1] = x;
            }
        }
        __syncwarp();
    }
}

// Sorts the 32 R keys x[h] of lane l (key index l + 32 h) ascending across
// the warp: a bitonic network, shuffles for the distances below 32 and
// register pairs of a lane for the others (all indices fixed at compile time).
template <int R>
__device__ __forceinline__ void warp_sort_regs(int32_t (&x)[R]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 32 * R; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
                const int hj = j >> 5;
#pragma unroll
                for (int h = 0; h < R; ++h)
                    if ((h & hj) == 0) {
                        const int h2 = h | hj;
                        const bool up = ((lane + 32 * h) & k) == 0;
                        const int32_t a = x[h], b = x[h2];
                        x[h] = up ? min(a, b) : max(a, b);
                        x[h2] = up ? max(a, b) : min(a, b);
                    }
            } else {
                const bool low = (lane & j) == 0;
#pragma unroll
                for (int h = 0; h < R; ++h) {
                    const int32_t y = __shfl_xor_sync(0xffffffffu, x[h], j);
                    const bool up = ((lane + 32 * h) & k) == 0;
                    x[h] = (low == up) ? min(x[h], y) : max(x[h], y);
                }
            }
        }
}

// the n keys ks[0..n) (n <= 32 R) sorted across the warp into u[0..n)
template <int R>
__device__ __forceinline__ void warp_sort_out(const int32_t *ks, int n, int32_t *u) {
    const int lane = threadIdx.x & 31;
    int32_t x[R];
#pragma unroll
    for (int h = 0; h < R; ++h) x[h] = lane + 32 * h < n ? ks[lane + 32 * h] : 0x7fffffff;
    warp_sort_regs<R>(x);
#pragma unroll
    for (int h = 0; h < R; ++h)
        if (lane + 32 * h < n) u[lane + 32 * h] = x[h];
}

// CSR row sets, one warp per row: the nodes of the row's incident elements
// (one candidate node per lane, four rounds of loads at a time) go into a
// hash set in shared memory of at least twice as many slots as candidates,
// up to 512 (a row longer than kMaxRow is an error, so a set of more than 256
// keys is never needed); the keys are sorted (up to 128 by a bitonic network
// over the lanes' registers, more by a bitonic sort in shared memory) and
// written to the row's scratch slot.
constexpr int kRowWarps = 8, kRowHash = 512;
template <int NLB>
__global__ void __launch_bounds__(kRowWarps * 32, 8) k_row_count(int64_t nn, const int32_t *__restrict__ elems,
                                                              const int32_t *__restrict__ n2e_ptr,
                                                              const int32_t *__restrict__ n2e,
                                                              int32_t *__restrict__ scratch,
                                                              int32_t *__restrict__ rowlen, int *__restrict__ err) {
    __shared__ int32_t hs[kRowWarps][kRowHash];
    __shared__ int32_t key[kRowWarps][kRowHash / 2];
    __shared__ int cnt[kRowWarps];
    if (*err & (ERR_OOB | ERR_DUP)) return;   // validation failed: the incidence lists were not filled
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t *tab = hs[w], *ks = key[w];
    for (int64_t i = (int64_t)blockIdx.x * kRowWarps + w; i < nn; i += (int64_t)gridDim.x * kRowWarps) {
        const int32_t b = n2e_ptr[i], e = n2e_ptr[i + 1];
        const int nq = e - b, ncand = nq * NLB;
        // a table of at least twice the candidates (at most kRowHash): the set never fills past half
        int H = 32;
        while (H < 2 * ncand && H < kRowHash) H <<= 1;
        for (int q = lane; q < H; q += 32) tab[q] = -1;
        if (lane == 0) cnt[w] = 0;
        __syncwarp();
        // candidate c = node c % NLB of incidence c / NLB, one per lane, four
        // rounds of loads in flight before their insertions
        for (int c0 = 0; c0 < ncand; c0 += 128) {
            int32_t xs[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int c = c0 + 32 * u + lane;
                xs[u] = c < ncand ? elems[(int64_t)(n2e[b + c / NLB] >> 4) * NLB + c % NLB] : -1;
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int32_t x = xs[u];
                if (x < 0) continue;
                uint32_t h = ((uint32_t)x * 2654435761u) & (uint32_t)(H - 1);
                for (int probe = 0; probe < H; ++probe) {
                    const int32_t prev = atomicCAS(&tab[h], -1, x);
                    if (prev == -1) {
                        atomicAdd(&cnt[w], 1);
                        break;
                    }
                    if (prev == x) break;
                    h = (h + 1) & (uint32_t)(H - 1);
                }
            }
        }
        __syncwarp();
        const int n = cnt[w];
        if (n > kMaxRow) {   // too long: report, skip the row
            if (lane == 0) {
                atomicOr(err, ERR_ROWLEN);
                rowlen[i] = 0;
            }
            __syncwarp();
            continue;
        }
        // compact
        int base = 0;
        for (int q0 = 0; q0 < H; q0 += 32) {
            const int32_t x = tab[q0 + lane];
            const unsigned m = __ballot_sync(0xffffffffu, x >= 0);
            if (x >= 0) ks[base + __popc(m & ((1u << lane) - 1u))] = x;
            base += __popc(m);
        }
        __syncwarp();
        int32_t *u = scratch + (int64_t)NLB * b;
        if (n <= 32) {   // up to 128 keys: a bitonic network over the lanes' registers
            warp_sort_out<1>(ks, n, u);
        } else if (n <= 64) {
            warp_sort_out<2>(ks, n, u);
        } else if (n <= 128) {
            warp_sort_out<4>(ks, n, u);
        } else {   // pad to a power of two, bitonic sort in shared memory
            int P = 1;
            while (P < n) P <<= 1;
            for (int q = n + lane; q < P; q += 32) ks[q] = 0x7fffffff;
            __syncwarp();
            for (int kk = 2; kk <= P; kk <<= 1)
                for (int j = kk >> 1; j > 0; j >>= 1) {
                    for (int q = lane; q < P; q += 32) {
                        const int l = q ^ j;
                        if (l > q) {
                            const bool up = (q & kk) == 0;
                            const int32_t x = ks[q], y = ks[l];
                            if ((x > y) == up) {
                                ks[q] = y;
                                ks[l] = x;
                            }
                        }
                    }
                    __syncwarp();
                }
            for (int q = lane; q < n; q += 32) u[q] = ks[q];
        }
        if (lane == 0) rowlen[i] = n;
        __syncwarp();
    }
}

__global__ void k_row_fill(int64_t nn, int nlb, const int32_t *__restrict__ n2e_ptr,
                           const int32_t *__restrict__ scratch, const int32_t *__restrict__ row_ptr,
                           int32_t *__restrict__ col_idx) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t *u = scratch + (int64_t)nlb * n2e_ptr[i];
        int32_t b = row_ptr[i], e = row_ptr[i + 1];
        for (int32_t p = b; p < e; ++p) col_idx[p] = u[p - b];
    }
}

// owner element and remaining vertex of each boundary facet
__global__ void k_face_owner(int64_t nfb, int dim, int nlb, int64_t nn, const int32_t *__restrict__ faces,
                             const int32_t *__restrict__ elems, const int32_t *__restrict__ n2e_ptr,
                             const int32_t *__restrict__ n2e, int32_t *__restrict__ opp, int *__restrict__ err) {
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < nfb; f += (int64_t)gridDim.x * blockDim.x) {
        int32_t fn[3] = {0, 0, 0};
        bool ok = true;
        for (int q = 0; q < dim; ++q) {
            fn[q] = faces[f * dim + q];
            if (fn[q] < 0 || fn[q] >= nn) ok = false;
        }
        if (!ok) {
            atomicOr(err, ERR_FACE_OOB);
            opp[f] = -1;
            continue;
        }
        int32_t found = -1;
        for (int32_t t = n2e_ptr[fn[0]]; t < n2e_ptr[fn[0] + 1] && found < 0; ++t) {
            int64_t k = (int64_t)(n2e[t] >> 4);
            int hits = 0;
            int32_t rest = -1;
            for (int j = 0; j <= dim; ++j) {
                int32_t v = elems[k * nlb + j];
                bool in = false;
                for (int q = 0; q < dim; ++q) in |= (v == fn[q]);
                if (in) ++hits;
                else rest = v;
            }
            if (hits == dim) found = rest;
        }
        opp[f] = found;
        if (found < 0) atomicOr(err, ERR_FACE_OWNER);
    }
}

// float pair split: x = hi + lo with hi = fl32(x), lo = fl32(x - hi)
__global__ void k_split_coords(int64_t nn, int dim, const double *__restrict__ x, float4 *__restrict__ xh,
                               float4 *__restrict__ xl) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x) {
        float h[3] = {0.f, 0.f, 0.f}, l[3] = {0.f, 0.f, 0.f};
        for (int d = 0; d < dim; ++d) {
            double v = x[i * dim + d];
            h[d] = (float)v;
            l[d] = (float)(v - (double)h[d]);
        }
        xh[i] = make_float4(h[0], h[1], h[2], 0.f);
        xl[i] = make_float4(l[0], l[1], l[2], 0.f);
    }
}

// ---------------------------------------------------------------------------
// spatial ordering of the rows
// ---------------------------------------------------------------------------
// bounding box from the per-block partials (lo[3], hi[3] each): warp c
// reduces component c
__global__ void k_bbox_final(int nb, const double *__restrict__ part, double *__restrict__ bb) {
    const int c = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (c >= 6) return;
    double v = c < 3 ? 1e300 : -1e300;
    for (int b = lane; b < nb; b += 32) v = c < 3 ? fmin(v, part[b * 6 + c]) : fmax(v, part[b * 6 + c]);
    for (int o = 16; o > 0; o >>= 1) {
        const double y = __shfl_down_sync(0xffffffffu, v, o);
        v = c < 3 ? fmin(v, y) : fmax(v, y);
    }
    if (lane == 0) bb[c] = v;
}

__global__ void k_bbox_partial(int64_t nn, int dim, const double *__restrict__ x, double *__restrict__ part) {
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x)
        for (int d = 0; d < dim; ++d) {
            double v = x[i * dim + d];
            lo[d] = fmin(lo[d], v);
            hi[d] = fmax(hi[d], v);
        }
    __shared__ double s[6][256];
    for (int d = 0; d < 3; ++d) {
        s[d][threadIdx.x] = lo[d];
        s[3 + d][threadIdx.x] = hi[d];
    }
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
            for (int d = 0; d < 3; ++d) {
                s[d][threadIdx.x] = fmin(s[d][threadIdx.x], s[d][threadIdx.x + o]);
                s[3 + d][threadIdx.x] = fmax(s[3 + d][threadIdx.x], s[3 + d][threadIdx.x + o]);
            }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int d = 0; d < 6; ++d) part[blockIdx.x * 6 + d] = s[d][0];
}

__device__ __forceinline__ uint32_t spread3(uint32_t v) {  // 10 bits -> every third bit
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}
__device__ __forceinline__ uint32_t spread2(uint32_t v) {  // 16 bits -> every second bit
    v &= 0xffffu;
    v = (v | (v << 8)) & 0x00ff00ffu;
    v = (v | (v << 4)) & 0x0f0f0f0fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

__global__ void k_cell_keys(int64_t nn, int dim, int bits, const double *__restrict__ x,
                            const double *__restrict__ bb, int32_t *__restrict__ key) {
    const uint32_t G = 1u << bits;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t q[3] = {0, 0, 0};
        for (int d = 0; d < dim; ++d) {
            double ext = bb[3 + d] - bb[d];
            double t = ext > 0 ? (x[i * dim + d] - bb[d]) / ext : 0.0;
            int64_t c = (int64_t)(t * G);
            if (c < 0) c = 0;
            if (c >= (int64_t)G) c = G - 1;
            q[d] = (uint32_t)c;
        }
        key[i] = (int32_t)(dim == 3 ? (spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2))
                                    : (spread2(q[0]) | (spread2(q[1]) << 1)));
    }
}

__global__ void k_hist(int64_t n, const int32_t *__restrict__ key, int32_t *__restrict__ h) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&h[key[i]], 1);
}

__global__ void k_bucket_scatter(int64_t n, const int32_t *__restrict__ key, int32_t *__restrict__ cursor,
                                 int32_t *__restrict__ perm) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        perm[atomicAdd(&cursor[key[i]], 1)] = (int32_t)i;
}

// tile = consecutive ranks whose incidence-weight prefix falls in [t*B, (t+1)*B)
__global__ void k_rank_weights(int64_t nn, const int32_t *__restrict__ perm, const int32_t *__restrict__ cnt,
                               int32_t *__restrict__ w) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nn; r += (int64_t)gridDim.x * blockDim.x)
        w[r] = cnt[perm[r]] + 1;
}

__global__ void k_tile_flags(int64_t nn, int64_t B, const long long *__restrict__ pre, int32_t *__restrict__ flag) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nn; r += (int64_t)gridDim.x * blockDim.x)
        flag[r] = (r == 0 || pre[r - 1] / B != pre[r] / B) ? 1 : 0;
}

__global__ void k_tile_assign(int64_t nn, const int32_t *__restrict__ flag, const long long *__restrict__ fpre,
                              const int32_t *__restrict__ perm, int32_t *__restrict__ tile_begin,
                              int32_t *__restrict__ node_tile) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nn; r += (int64_t)gridDim.x * blockDim.x) {
        int32_t t = (int32_t)(fpre[r] + flag[r] - 1);
        if (flag[r]) tile_begin[t] = (int32_t)r;
        node_tile[perm[r]] = t;
    }
}

// ---------------------------------------------------------------------------
// per-tile sets (one CTA per tile)
// ---------------------------------------------------------------------------
// Sorts n distinct keys (n <= capacity of a, which is a multiple of 64)
// ascending from a into out.  Each warp sorts runs of 64 keys in registers (a
// bitonic network over its lanes, two keys per lane, shuffles for the
// distances below 32), the runs go back to a, padded with INT_MAX; then every
// key's place is its index in its run plus the number of smaller keys in each
// other run (a binary search per run).  The keys are distinct, so the places
// are a permutation.  Ends with a block barrier.
__device__ void sort_distinct(int32_t *a, int n, int32_t *out) {
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int nruns = (n + 63) >> 6;
    for (int r = threadIdx.x >> 5; r < nruns; r += nw) {
        int32_t *run = a + r * 64;
        int32_t x0 = r * 64 + lane < n ? run[lane] : 0x7fffffff;
        int32_t x1 = r * 64 + 32 + lane < n ? run[32 + lane] : 0x7fffffff;
        // key q = lane + 32 h sits in register h; stage (k, j) pairs q with q ^ j
        // and keeps the smaller key at the lower index where (q & k) == 0
#pragma unroll
        for (int k = 2; k <= 64; k <<= 1)
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
                if (j == 32) {   // only with k == 64: the two registers of a lane, ascending
                    const int32_t lo = min(x0, x1), hi = max(x0, x1);
                    x0 = lo;
                    x1 = hi;
                } else {
                    const int32_t y0 = __shfl_xor_sync(0xffffffffu, x0, j);
                    const int32_t y1 = __shfl_xor_sync(0xffffffffu, x1, j);
                    const bool low = (lane & j) == 0;
                    const bool up0 = (lane & k) == 0, up1 = ((lane + 32) & k) == 0;
                    x0 = (low == up0) ? min(x0, y0) : max(x0, y0);
                    x1 = (low == up1) ? min(x1, y1) : max(x1, y1);
                }
            }
        run[lane] = x0;
        run[32 + lane] = x1;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int32_t x = a[i];
        const int r = i >> 6;
        int pos = i & 63;
        for (int s2 = 0; s2 < nruns; ++s2) {
            if (s2 == r) continue;
            const int32_t *run = a + s2 * 64;
            int lo = 0;   // keys of run s2 below x
#pragma unroll
            for (int step = 64; step > 0; step >>= 1)
                if (lo + step <= 64 && run[lo + step - 1] < x) lo += step;
            pos += lo;
        }
        out[pos] = x;
    }
    __syncthreads();
}

struct TileCounts {
    int32_t n_nodes, n_elems, n_own, n_up, n_diag, n_rows, rank_begin, pad;
};

__device__ __forceinline__ int lower_bound_i32(const int32_t *a, int n, int32_t x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// insert a non-negative key into an open-addressing set in shared memory
// (H a power of two, empty slots -1); the probe sequence visits every slot, so
// it ends once the set holds fewer than H keys.  Returns false when the key
// found no slot (the set was full)
__device__ __forceinline__ bool hset_insert(int32_t *tab, int H, int32_t x) {
    uint32_t h = ((uint32_t)x * 2654435761u) & (uint32_t)(H - 1);
    for (int probe = 0; probe < H; ++probe) {
        const int32_t prev = atomicCAS(&tab[h], -1, x);
        if (prev == -1 || prev == x) return true;
        h = (h + 1) & (uint32_t)(H - 1);
    }
    return false;
}

// the set's keys, in no particular order, into out[0..count); returns count
// (warp-aggregated slot claims: one shared atomic per warp and pass)
__device__ int hset_compact(const int32_t *tab, int H, int32_t *out) {
    __shared__ int s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (int c0 = 0; c0 < H; c0 += blockDim.x) {
        const int i = c0 + threadIdx.x;
        const int32_t x = i < H ? tab[i] : -1;
        const unsigned m = __ballot_sync(0xffffffffu, x >= 0);
        int base = 0;
        if (lane == 0 && m) base = atomicAdd(&s_cnt, __popc(m));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (x >= 0) out[base + __popc(m & ((1u << lane) - 1u))] = x;
    }
    __syncthreads();
    const int n = s_cnt;
    __syncthreads();
    return n;
}

// number of entries of the ascending array a[0..n) that are <= x
__device__ __forceinline__ int upper_bound_i32(const int32_t *a, int n, int32_t x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (a[mid] <= x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Pass A of the tile build: the tile's elements (every element incident to
// one of its rows: deduplicated in a shared-memory hash set, then sorted;
// owned elements -- those whose first vertex's row is in the tile -- first),
// the vertex nodes of those elements (likewise), and the counts of its pairs.
// The global loads of each step are issued in batches ahead of the set
// insertions, so a CTA waits for one memory round trip per batch.
__global__ void k_tile_sets(int n_tiles, int64_t nn, int dim, int nlb, int cap_e, int cap_n,
                            const int32_t *__restrict__ tile_begin, const int32_t *__restrict__ perm,
                            const int32_t *__restrict__ n2e_ptr, const int32_t *__restrict__ n2e,
                            const int32_t *__restrict__ elems, const int32_t *__restrict__ row_ptr,
                            const int32_t *__restrict__ col_idx, const int32_t *__restrict__ node_tile,
                            int32_t *__restrict__ sc_elems, int32_t *__restrict__ sc_nodes,
                            TileCounts *__restrict__ counts, int *__restrict__ err) {
    extern __shared__ int32_t sm[];
    const int t = blockIdx.x;
    if (t >= n_tiles) return;
    // cap_e >= B + wmax >= the tile's weight >= its rows and its candidates;
    // cap_n bounds the tile's distinct vertex nodes (a tile with more reports
    // ERR_NODE_CAP, and the host runs the pass again with a larger cap_n)
    const int hs_len = 3 * cap_e > 2 * cap_n ? 3 * cap_e : 2 * cap_n;
    int32_t *ce = sm;                 // cap_e: the tile's elements
    int32_t *hs = sm + cap_e;         // hs_len: hash sets, then scratch of the partition
    int32_t *cn = hs + hs_len;        // max(cap_e, cap_n) + 64: the rows' prefix, then the tile's vertex nodes
    int32_t *tmp = hs;
    const int rb = tile_begin[t];
    const int re = (t + 1 < n_tiles) ? tile_begin[t + 1] : (int)nn;
    const int nr = re - rb;
    const int He = 2 * cap_e;
    // the rows' incidence-list starts (past the element table) and the prefix
    // of their lengths (in the node list's space, unused until the node phase)
    int32_t *r_start = hs + He, *r_pre = cn;
    for (int i = threadIdx.x; i < He; i += blockDim.x) hs[i] = -1;
    // one scan carries both the incidence counts (low word) and the CSR row
    // lengths (high word); the row lengths bound the tile's vertex nodes, all
    // of which are columns of the tile's rows
    long long ncand_l = 0, cols_l = 0;
    for (int c0 = 0; c0 < nr; c0 += blockDim.x) {
        const int rr = c0 + threadIdx.x;
        long long len = 0;
        int32_t st = 0;
        if (rr < nr) {
            const int32_t i = perm[rb + rr];
            st = n2e_ptr[i];
            len = (long long)(n2e_ptr[i + 1] - st) | ((long long)(row_ptr[i + 1] - row_ptr[i]) << 32);
        }
        long long tot;
        const long long pre = block_excl_scan(len, &tot);
        if (rr < nr) {
            r_pre[rr] = (int32_t)(ncand_l + (pre & 0xffffffffll));
            r_start[rr] = st;
        }
        ncand_l += tot & 0xffffffffll;
        cols_l += tot >> 32;
    }
    if (ncand_l > cap_e) {   // more candidates than the tile was sized for
        if (threadIdx.x == 0) atomicOr(err, ERR_TILE_CAP);
        return;
    }
    const int ncand = (int)ncand_l;
    if (threadIdx.x == 0) r_pre[nr] = ncand;
    __syncthreads();
    // the rows' incidences as one flat list, four per thread per batch
    for (int x0 = threadIdx.x; x0 < ncand; x0 += 4 * blockDim.x) {
        int32_t kk[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int x = x0 + u * blockDim.x;
            kk[u] = -1;
            if (x < ncand) {
                const int rr = upper_bound_i32(r_pre, nr + 1, x) - 1;   // the row whose range holds x
                kk[u] = n2e[r_start[rr] + (x - r_pre[rr])] >> 4;
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (kk[u] >= 0) hset_insert(hs, He, kk[u]);
    }
    __syncthreads();
    // the set's keys past the table, sorted into ce
    const int n_el = hset_compact(hs, He, hs + He);
    sort_distinct(hs + He, n_el, ce);
    // owner flags (past the partition's output in the scratch region)
    int32_t *oflag = hs + cap_e;
    long long own = 0;
    for (int i0 = threadIdx.x; i0 < n_el; i0 += 4 * blockDim.x) {
        int32_t f[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * blockDim.x;
            f[u] = i < n_el ? elems[(int64_t)ce[i] * nlb] : 0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * blockDim.x;
            if (i < n_el) {
                const int o = node_tile[f[u]] == t;
                oflag[i] = o;
                own += o;
            }
        }
    }
    long long n_own = 0;
    block_excl_scan(own, &n_own);   // synchronises: the flags are visible below
    // owned elements first (stable partition)
    long long obase = 0, hbase = 0;
    for (int c0 = 0; c0 < n_el; c0 += blockDim.x) {
        const int i = c0 + threadIdx.x;
        int o = 0, halo = 0;
        if (i < n_el) {
            o = oflag[i];
            halo = !o;
        }
        long long tot_o, tot_h;
        long long po = block_excl_scan(o, &tot_o);
        long long ph = block_excl_scan(halo, &tot_h);
        if (o) tmp[obase + po] = ce[i];
        if (halo) tmp[n_own + hbase + ph] = ce[i];
        obase += tot_o;
        hbase += tot_h;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n_el; i += blockDim.x) sc_elems[(int64_t)t * cap_e + i] = tmp[i];
    __syncthreads();
    // vertex nodes of those elements
    const int nv = dim + 1;
    const int nnc = n_el * nv;
    // a table of at least twice the distinct nodes the tile can have (the
    // candidates, or the columns of its rows if fewer), at most cap_n slots, so
    // that the keys it holds fit the node list
    const int nnb = nnc < cols_l ? nnc : (int)cols_l;   // at most this many distinct nodes
    int Hu = cap_n < 64 ? cap_n : 64;
    while (Hu < 2 * nnb && Hu < cap_n) Hu <<= 1;
    for (int i = threadIdx.x; i < Hu; i += blockDim.x) hs[i] = -1;
    __syncthreads();
    bool fits = true;
    for (int x0 = threadIdx.x; x0 < nnc; x0 += 8 * blockDim.x) {
        int32_t vv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int x = x0 + u * blockDim.x;
            vv[u] = x < nnc ? elems[(int64_t)ce[x / nv] * nlb + (x % nv)] : -1;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (vv[u] >= 0) fits &= hset_insert(hs, Hu, vv[u]);
    }
    if (__syncthreads_or(!fits)) {   // more distinct nodes than cap_n: the host sizes the pass again
        if (threadIdx.x == 0) atomicOr(err, ERR_NODE_CAP);
        return;
    }
    const int n_nd = hset_compact(hs, Hu, cn);
    sort_distinct(cn, n_nd, hs);   // the table is dead after the compaction
    for (int i = threadIdx.x; i < n_nd; i += blockDim.x) sc_nodes[(int64_t)t * cap_n + i] = hs[i];
    // upper pairs {i, j > i} and diagonals of the tile's rows
    long long up = 0, dg = 0;
    for (int r = rb + threadIdx.x; r < re; r += blockDim.x) {
        const int32_t i = perm[r];
        const int32_t b = row_ptr[i], len = row_ptr[i + 1] - b;
        if (len == 0) continue;
        const int ds = lower_bound_i32(col_idx + b, len, i);
        up += len - ds - 1;
        dg += 1;
    }
    long long tot_up, tot_dg;
    block_excl_scan(up, &tot_up);
    block_excl_scan(dg, &tot_dg);
    if (threadIdx.x == 0) {
        TileCounts c;
        c.n_nodes = n_nd;
        c.n_elems = n_el;
        c.n_own = (int32_t)n_own;
        c.n_up = (int32_t)tot_up;
        c.n_diag = (int32_t)tot_dg;
        c.n_rows = re - rb;
        c.rank_begin = rb;
        c.pad = 0;
        counts[t] = c;
    }
}

// local index of global element k in a tile's element list (owned block then halo block)
__device__ __forceinline__ int tile_local_elem(const int32_t *te, int n_own, int n_el, int32_t k) {
    int p = lower_bound_i32(te, n_own, k);
    if (p < n_own && te[p] == k) return p;
    return n_own + lower_bound_i32(te + n_own, n_el - n_own, k);
}

// What the warp passes need of a tile row, written once by the row pass of
// k_tile_fill: its node, CSR start and length, the diagonal's offset, its
// incidence list, and the indices of its first upper pair and its diagonal
// among the tile's pairs (one 32-byte load instead of a chain of dependent ones)
struct __align__(16) RowInfo {
    int32_t qu, qd, i, b, len, ds, q0, nq;
};

// The rows of a tile are visited by warps, one row at a time.  A row's pairs
// are its upper pairs {i, c > i} in column order, then the diagonal {i, i};
// its incidences come in ascending element order.  The count pass holds the
// pairs one per lane and the incidences one per lane, 32 at a time: for each
// pair, the ballot of the incidences whose element holds the pair's other
// node counts its contributions.  The code pass (below) walks the incidences
// as (incidence, local node) items instead and ranks the items that hit the
// same pair by lane; both see the contributions in the order a single thread
// walking the row would (element order).

// Pass B: node lists, element records, owned ids, pair positions and the
// contribution count of every pair.  Dynamic shared memory: the tile's node
// list (n_nodes ints), searched for the elements' local vertex indices.
template <int NLB>
__global__ void __launch_bounds__(256) k_tile_fill(int n_tiles, int dim, int cap_e, int cap_n,
                                                   const TileHdr *__restrict__ hdr, const int32_t *__restrict__ perm,
                                                   const int32_t *__restrict__ n2e_ptr, const int32_t *__restrict__ n2e,
                                                   const int32_t *__restrict__ elems, const int32_t *__restrict__ row_ptr,
                                                   const int32_t *__restrict__ col_idx,
                                                   const int32_t *__restrict__ sc_elems,
                                                   const int32_t *__restrict__ sc_nodes, int32_t *__restrict__ tile_nodes,
                                                   ushort4 *__restrict__ tile_elem, int32_t *__restrict__ tile_own,
                                                   int32_t *__restrict__ tile_eid,
                                                   int2 *__restrict__ tile_nzpos, int32_t *__restrict__ nz_count,
                                                   RowInfo *__restrict__ row_info) {
    extern __shared__ int32_t s_tn[];
    const int t = blockIdx.x;
    if (t >= n_tiles) return;
    const TileHdr h = hdr[t];
    const int32_t *te = sc_elems + (int64_t)t * cap_e;
    const int32_t *tn = sc_nodes + (int64_t)t * cap_n;
    for (int i = threadIdx.x; i < h.n_nodes; i += blockDim.x) {
        const int32_t v = tn[i];
        s_tn[i] = v;
        tile_nodes[h.node_off + i] = v;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < h.n_elems; e += blockDim.x) {
        const int64_t k = te[e];
        unsigned short v[4] = {0, 0, 0, 0};
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (j <= dim) v[j] = (unsigned short)lower_bound_i32(s_tn, h.n_nodes, elems[k * NLB + j]);
        tile_elem[h.elem_off + e] = make_ushort4(v[0], v[1], v[2], v[3]);
        if (e < h.n_own) tile_own[h.own_off + e] = (int32_t)k;
        tile_eid[h.elem_off + e] = (int32_t)k;
    }
    // per-row base of its upper pairs and index of its diagonal (rank order)
    long long ubase = 0, dbase = 0;
    for (int c0 = 0; c0 < h.n_rows; c0 += blockDim.x) {
        const int rr = c0 + threadIdx.x;
        long long up = 0, hasd = 0;
        int32_t i = -1, b = 0, len = 0, ds = 0;
        if (rr < h.n_rows) {
            i = perm[h.rank_begin + rr];
            b = row_ptr[i];
            len = row_ptr[i + 1] - b;
            if (len > 0) {
                ds = lower_bound_i32(col_idx + b, len, i);
                up = len - ds - 1;
                hasd = 1;
            }
        }
        long long tot_u, tot_d;
        const long long pu = block_excl_scan(up, &tot_u);
        const long long pd = block_excl_scan(hasd, &tot_d);
        if (rr < h.n_rows) {
            const int32_t qu = (int32_t)(ubase + pu);
            const int32_t qd = hasd ? h.n_up + (int32_t)(dbase + pd) : -1;
            if (hasd) tile_nzpos[h.nz_off + qd] = make_int2(b + ds, b + ds);
            const int32_t q0 = n2e_ptr[i];
            row_info[h.rank_begin + rr] = RowInfo{qu, qd, i, b, len, ds, q0, n2e_ptr[i + 1] - q0};
        }
        ubase += tot_u;
        dbase += tot_d;
    }
    __syncthreads();
    // CSR positions (p_ij, p_ji) of the upper pairs and contribution counts of
    // every pair (each written once)
    const int lane = threadIdx.x & 31;
    for (int rr = threadIdx.x >> 5; rr < h.n_rows; rr += blockDim.x >> 5) {
        const RowInfo ri = row_info[h.rank_begin + rr];
        const int32_t i = ri.i, b = ri.b, len = ri.len, ds = ri.ds, q0 = ri.q0, nq = ri.nq;
        if (len == 0) continue;
        const int np = len - ds;
        for (int p0 = 0; p0 < np; p0 += 32) {
            const int pp = p0 + lane, npq = min(32, np - p0);
            const int32_t c_pp = pp < np - 1 ? col_idx[b + ds + 1 + pp] : i;
            if (pp < np - 1) {   // upper pair {i, c}: its place in row c by a search of that row
                const int32_t bj = row_ptr[c_pp], lj = row_ptr[c_pp + 1] - bj;
                tile_nzpos[h.nz_off + ri.qu + pp] = make_int2(b + ds + 1 + pp, bj + lower_bound_i32(col_idx + bj, lj, i));
            }
            int cnt = 0;
            for (int j0 = 0; j0 < nq; j0 += 32) {
                const bool valid = j0 + lane < nq;
                const int64_t k = valid ? (int64_t)(n2e[q0 + j0 + lane] >> 4) : 0;
                int32_t v[NLB];
#pragma unroll
                for (int bb = 0; bb < NLB; ++bb) v[bb] = valid ? elems[k * NLB + bb] : -1;
                for (int q = 0; q < npq; ++q) {
                    const int32_t c = __shfl_sync(0xffffffffu, c_pp, q);
                    bool hit = false;
#pragma unroll
                    for (int bb = 0; bb < NLB; ++bb) hit |= v[bb] == c;
                    const int n = __popc(__ballot_sync(0xffffffffu, hit));
                    if (lane == q) cnt += n;
                }
            }
            if (pp < np) nz_count[h.nz_off + (pp == np - 1 ? ri.qd : ri.qu + pp)] = cnt;
        }
    }
}

// Orders every tile's pairs by contribution count (descending, stable), so
// that the 32 pairs of a chunk need nearly the same number of iterations, then
// writes the chunk table (tile-relative code offset, width) and the permuted
// pair positions.  order[nz_off + q] = new index of row-major pair q.  Each
// warp places a contiguous range of the row-major pairs (whole 32-pair
// windows): per-warp count histograms give every (count, warp) its first slot
// (counts descending, then warps in range order, which keeps the order
// stable), and within a window a pair's slot is its bucket's next slot plus
// the number of earlier lanes with the same count.
constexpr int kChunkWarps = 8, kMaxCount = 512;
__global__ void __launch_bounds__(kChunkWarps * 32) k_chunk_table(int n_tiles, const TileHdr *__restrict__ hdr,
                                                                  const int32_t *__restrict__ nz_count,
                                                                  const int2 *__restrict__ nzpos_rowmajor,
                                                                  int2 *__restrict__ nzpos, int32_t *__restrict__ order,
                                                                  int2 *__restrict__ chunks,
                                                                  int32_t *__restrict__ tile_codes_n) {
    const int t = blockIdx.x;
    if (t >= n_tiles) return;
    const TileHdr h = hdr[t];
    __shared__ int32_t hist[kChunkWarps][kMaxCount + 1];
    __shared__ int32_t w[1024];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kChunkWarps * (kMaxCount + 1); i += blockDim.x) (&hist[0][0])[i] = 0;
    for (int i = threadIdx.x; i < 1024; i += blockDim.x) w[i] = 0;
    __syncthreads();
    const int nwin = (h.n_nz + 31) >> 5, per = (nwin + kChunkWarps - 1) / kChunkWarps;
    const int q_begin = min(wid * per, nwin) * 32, q_end = min(min((wid + 1) * per, nwin) * 32, h.n_nz);
    for (int q = q_begin + lane; q < q_end; q += 32) atomicAdd(&hist[wid][min(nz_count[h.nz_off + q], kMaxCount)], 1);
    __syncthreads();
    // first slot of every (count, warp): a block scan over the counts in
    // descending order of the per-count totals, then the warps in order
    long long base = 0;
    for (int r0 = 0; r0 <= kMaxCount; r0 += blockDim.x) {
        const int r = r0 + threadIdx.x, c = kMaxCount - r;
        int tot = 0;
        if (r <= kMaxCount)
            for (int ww = 0; ww < kChunkWarps; ++ww) tot += hist[ww][c];
        long long all;
        const long long pre = block_excl_scan(tot, &all);
        if (r <= kMaxCount) {
            int run = (int)(base + pre);
            for (int ww = 0; ww < kChunkWarps; ++ww) {
                const int n = hist[ww][c];
                hist[ww][c] = run;
                run += n;
            }
        }
        base += all;
    }
    __syncthreads();
    for (int q0 = q_begin; q0 < q_end; q0 += 32) {
        const int q = q0 + lane;
        const bool valid = q < q_end;
        const int n = valid ? nz_count[h.nz_off + q] : 0;
        const int c = valid ? min(n, kMaxCount) : -1 - lane;   // invalid lanes match nobody
        const unsigned peers = __match_any_sync(0xffffffffu, c);
        const int rank = __popc(peers & ((1u << lane) - 1u));
        const int bs = valid ? hist[wid][c] : 0;
        __syncwarp();
        if (valid) {
            const int32_t nq = bs + rank;
            order[h.nz_off + q] = nq;
            nzpos[h.nz_off + nq] = nzpos_rowmajor[h.nz_off + q];
            if ((nq >> 5) < 1024) atomicMax(&w[nq >> 5], n);   // chunk width: its largest count
            if (rank == 0) hist[wid][c] = bs + __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
    // chunk table: code offsets by a block scan of 32 x width
    const int nch = min(h.n_chunks, 1024);
    long long off = 0;
    for (int c0 = 0; c0 < nch; c0 += blockDim.x) {
        const int c = c0 + threadIdx.x;
        const long long v = c < nch ? 32LL * w[c] : 0;
        long long all;
        const long long pre = block_excl_scan(v, &all);
        if (c < nch) chunks[h.chunk_off + c] = make_int2((int)(off + pre), w[c]);
        off += all;
    }
    if (threadIdx.x == 0) tile_codes_n[t] = (int32_t)off;
}

// Pass C: contribution codes, element * rsc + packed (a,b) entry (the entry's
// word offset in a record of stride rsc), ascending element order per pair;
// padding slots point at the tile's zero element.  A warp takes a row and
// walks its incidence list as (incidence, local node) items, 32 at a time:
// an item whose node c is at or above the row's node is a contribution to
// pair (i, c), found by a binary search of the row's upper columns staged in
// shared memory; the items of a batch that hit the same pair are ranked by
// lane (match), which keeps the ascending element order, and the pair's
// running count sits in shared memory.  Dynamic shared memory: per warp the
// row's upper columns, pair slot bases and counts (kMaxRow + 1 each), then the
// tile's element list (n_elems ints), searched for local element indices.
constexpr int kCodeWarps = 8;
template <int NLB, typename CT>
__global__ void __launch_bounds__(kCodeWarps * 32, NLB == 4 ? 8 : 4) k_tile_codes(int n_tiles, int cap_e, int rsc,
                                                                const TileHdr *__restrict__ hdr,
                                                                const int32_t *__restrict__ n2e,
                                                                const int32_t *__restrict__ elems,
                                                                const int32_t *__restrict__ col_idx,
                                                                const int32_t *__restrict__ sc_elems,
                                                                const RowInfo *__restrict__ row_info,
                                                                const int32_t *__restrict__ order,
                                                                const int2 *__restrict__ chunks,
                                                                CT *__restrict__ codes) {
    extern __shared__ int32_t s_dyn[];
    constexpr int W = kMaxRow + 1;
    const int t = blockIdx.x;
    if (t >= n_tiles) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int32_t *s_col = s_dyn + warp * 3 * W, *s_base = s_col + W, *s_cnt = s_base + W;
    int32_t *s_te = s_dyn + kCodeWarps * 3 * W;
    const TileHdr h = hdr[t];
    const int32_t *te = sc_elems + (int64_t)t * cap_e;
    for (int i = threadIdx.x; i < h.n_elems; i += blockDim.x) s_te[i] = te[i];
    const CT dummy = (CT)((uint32_t)h.n_elems * (uint32_t)rsc);
    for (int i = threadIdx.x; i < h.n_codes; i += blockDim.x) codes[(int64_t)h.code_off + i] = dummy;
    __syncthreads();
    const unsigned below = (1u << lane) - 1u;
    CT *out = codes + h.code_off;
    for (int rr = warp; rr < h.n_rows; rr += kCodeWarps) {
        const RowInfo ri = row_info[h.rank_begin + rr];
        const int32_t i = ri.i, len = ri.len, q0 = ri.q0, nq = ri.nq;
        if (len == 0) continue;
        const int np = len - ri.ds, nu = np - 1;   // pairs: the nu upper columns, then the diagonal
        for (int pp = lane; pp < np; pp += 32) {
            if (pp < nu) s_col[pp] = col_idx[ri.b + ri.ds + 1 + pp];
            const int nqo = order[h.nz_off + (pp == nu ? ri.qd : ri.qu + pp)];
            s_base[pp] = chunks[h.chunk_off + (nqo >> 5)].x + (nqo & 31);
            s_cnt[pp] = 0;
        }
        __syncwarp();
        const int top = nu > 0 ? 1 << (31 - __clz(nu)) : 0;
        for (int j0 = 0; j0 < nq; j0 += 32) {
            const int nj = min(32, nq - j0);
            int32_t kl = 0, ea = 0;   // this lane's incidence: element, (local element << 4 | local node)
            if (lane < nj) {
                const int32_t word = n2e[q0 + j0 + lane];
                kl = word >> 4;
                ea = (tile_local_elem(s_te, h.n_own, h.n_elems, kl) << 4) | (word & 15);
            }
            const int nit = nj * NLB;
            for (int it0 = 0; it0 < nit; it0 += 32) {
                const int it = it0 + lane, jj = it / NLB, bb = it - jj * NLB;
                const int32_t k = __shfl_sync(0xffffffffu, kl, jj & 31);
                const int32_t e = __shfl_sync(0xffffffffu, ea, jj & 31);
                int pp = -1;
                if (it < nit) {
                    const int32_t c = elems[(int64_t)k * NLB + bb];
                    if (c == i) {
                        pp = nu;
                    } else if (c > i) {
                        int pos = 0;   // upper columns below c
                        for (int s = top; s > 0; s >>= 1)
                            if (pos + s <= nu && s_col[pos + s - 1] < c) pos += s;
                        pp = pos;
                    }
                }
                const unsigned grp = __match_any_sync(0xffffffffu, pp);
                const int rank = __popc(grp & below), gsz = __popc(grp);
                const int cnt = pp >= 0 ? s_cnt[pp] : 0;
                __syncwarp();
                if (pp >= 0) {
                    const int a = e & 15, p = a < bb ? a : bb, r = a < bb ? bb : a;
                    const uint32_t u = (uint32_t)(p * NLB - p * (p - 1) / 2 + (r - p));
                    out[s_base[pp] + (cnt + rank) * 32] = (CT)((uint32_t)(e >> 4) * (uint32_t)rsc + u);
                    if (rank == gsz - 1) s_cnt[pp] = cnt + gsz;
                }
                __syncwarp();
            }
        }
    }
}

int next_pow2(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

template <typename T>
vla_status dalloc(vla_mesh *m, T **p, size_t count, cudaStream_t st) {
    size_t bytes = sizeof(T) * (count > 0 ? count : 1);
    cudaError_t e = pool_malloc((void **)p, bytes, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(VLA_ERR_OOM, "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    m->allocs.push_back((void *)*p);
    m->device_bytes += (int64_t)bytes;
    return VLA_OK;
}



// the tile kernels take dynamic shared-memory sizes that depend on the mesh;
// a kernel's limit is raised to the device maximum once per device (meshes
// built concurrently on several host threads must not change it under each
// other)
vla_status allow_max_smem(const void *fn) {
    static std::mutex mu;
    static std::set<std::pair<int, const void *>> done;
    int dev = 0, maxsm = 0;
    VLA_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(mu);
    if (done.count({dev, fn})) return VLA_OK;
    VLA_CUDA(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cudaFuncAttributes fa;
    VLA_CUDA(cudaFuncGetAttributes(&fa, fn));
    VLA_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm - (int)fa.sharedSizeBytes));
    done.insert({dev, fn});
    return VLA_OK;
}

// largest shared-memory footprint of a tile's assembly launch that still lets
// two CTAs share an SM (VLA_TILE_SMEM_CAP overrides, for experiments)
size_t tile_smem_cap() {
    if (const char *c = getenv("VLA_TILE_SMEM_CAP")) return (size_t)std::max(16384ll, atoll(c));
    int dev = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 233472;
    }
    return (size_t)per_sm / 2 - 4096;
}

// incidence budget of a tile (sum over its rows of 1 + incident elements)
vla_status build(vla_mesh *m, const double *coords, const int32_t *elems, const int32_t *faces) {
    cudaStream_t st = m->stream;
    const int dim = m->dim, nlb = m->nlb;
    const int64_t nn = m->nn, ne = m->ne, nfb = m->nfb;
    Scratch S;
    S.st = st;
    const int TB = 256;

    TRY(dalloc(m, &m->coords, nn * dim, st));
    TRY(dalloc(m, &m->elems, ne * nlb, st));
    VLA_CUDA(cudaMemcpyAsync(m->coords, coords, sizeof(double) * nn * dim, cudaMemcpyDeviceToDevice, st));
    VLA_CUDA(cudaMemcpyAsync(m->elems, elems, sizeof(int32_t) * ne * nlb, cudaMemcpyDeviceToDevice, st));
    if (nfb > 0) {
        TRY(dalloc(m, &m->faces, nfb * dim, st));
        TRY(dalloc(m, &m->face_opp, nfb, st));
        VLA_CUDA(cudaMemcpyAsync(m->faces, faces, sizeof(int32_t) * nfb * dim, cudaMemcpyDeviceToDevice, st));
    }

    // ---- validation + incidence counts
    int *d_err;
    long long *d_bad;
    int32_t *cnt;
    TRY(S.get(&d_err, 1));
    TRY(S.get(&d_bad, 1));
    TRY(S.get(&cnt, nn));
    VLA_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), st));
    const long long big = 0x7fffffffffffffffll;
    VLA_CUDA(cudaMemcpyAsync(d_bad, &big, sizeof(long long), cudaMemcpyHostToDevice, st));
    VLA_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t) * nn, st));
    k_validate_count<<<grid_for(ne, TB), TB, 0, st>>>(ne, nlb, nn, m->elems, cnt, d_err, d_bad);
    VLA_CUDA(cudaGetLastError());
    // scalars read back through pinned memory: [0] scan totals, [1] error word,
    // [2] bad element, [3] max incidence + 1, [4] max row length
    long long *hp = pinned_scalars();
    if (!hp) return fail(VLA_ERR_OOM, "pinned host scalars");
    long long *dsc;
    TRY(S.get(&dsc, 8));
    // the validation result is read at the next synchronisation (after the CSR row
    // counts); until then the kernels that follow index through the elements only
    // when the error word is clear
    int h_err = 0;

    // ---- node -> element incidence (sorted by element)
    long long *pre;
    TRY(S.get(&pre, nn + 1));
    // every element of a validated mesh puts each of its nlb nodes in one incidence list: no count to read back
    const long long n2e_total = (long long)ne * nlb;
    TRY(excl_scan<int32_t>(cnt, nn, pre, st, nullptr));
    TRY(dalloc(m, &m->n2e_ptr, nn + 1, st));
    TRY(dalloc(m, &m->n2e, n2e_total, st));
    k_i64_to_i32<<<grid_for(nn + 1, TB, 1 << 30), TB, 0, st>>>(nn + 1, pre, m->n2e_ptr);
    int32_t *cursor;
    TRY(S.get(&cursor, nn + 1));
    VLA_CUDA(cudaMemcpyAsync(cursor, m->n2e_ptr, sizeof(int32_t) * (nn + 1), cudaMemcpyDeviceToDevice, st));
    k_fill_n2e<<<grid_for(ne, TB), TB, 0, st>>>(ne, nlb, m->elems, cursor, m->n2e, d_err);
    k_sort_segments<<<grid_for((nn + kSegWarps - 1) / kSegWarps, 1), kSegWarps * 32, 0, st>>>(nn, m->n2e_ptr, m->n2e);
    VLA_CUDA(cudaGetLastError());

    // ---- CSR pattern
    int32_t *scratch, *rowlen;
    TRY(S.get(&scratch, (size_t)n2e_total * nlb));
    TRY(S.get(&rowlen, nn));
    {
        auto kr = nlb == 3 ? k_row_count<3> : nlb == 4 ? k_row_count<4> : nlb == 6 ? k_row_count<6> : k_row_count<10>;
        kr<<<grid_for((nn + kRowWarps - 1) / kRowWarps, 1), kRowWarps * 32, 0, st>>>(nn, m->elems, m->n2e_ptr, m->n2e,
                                                                                     scratch, rowlen, d_err);
    }
    VLA_CUDA(cudaGetLastError());
    long long nnz = 0;
    VLA_CUDA(cudaMemsetAsync(dsc + 1, 0, sizeof(long long), st));
    k_max_i32<<<grid_for(nn, 256), 256, 0, st>>>(nn, rowlen, 0, dsc + 1);
    hp[1] = 0;
    VLA_CUDA(cudaMemcpyAsync(&hp[1], d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    VLA_CUDA(cudaMemcpyAsync(&hp[2], d_bad, sizeof(long long), cudaMemcpyDeviceToHost, st));
    VLA_CUDA(cudaMemcpyAsync(&hp[4], dsc + 1, sizeof(long long), cudaMemcpyDeviceToHost, st));
    TRY(excl_scan<int32_t>(rowlen, nn, pre, st, &nnz));   // synchronises: the copies above have landed
    h_err = (int)hp[1];
    const long long h_bad = hp[2];
    if (h_err & ERR_OOB) return fail(VLA_ERR_INDEX_OOB, "element %lld references a node outside [0, %lld)", h_bad, (long long)nn);
    if (h_err & ERR_DUP) return fail(VLA_ERR_DEGENERATE, "element %lld repeats a node", h_bad);
    m->max_row_len = (int32_t)hp[4];
    if (h_err & ERR_ROWLEN) return fail(VLA_ERR_UNSUPPORTED, "a CSR row has more than %d entries", kMaxRow);
    if (nnz > 0x7fffffffll) return fail(VLA_ERR_UNSUPPORTED, "nnz %lld exceeds int32", nnz);
    m->nnz = nnz;
    TRY(dalloc(m, &m->row_ptr, nn + 1, st));
    TRY(dalloc(m, &m->col_idx, nnz, st));
    k_i64_to_i32<<<grid_for(nn + 1, TB, 1 << 30), TB, 0, st>>>(nn + 1, pre, m->row_ptr);
    k_row_fill<<<grid_for(nn, TB), TB, 0, st>>>(nn, nlb, m->n2e_ptr, scratch, m->row_ptr, m->col_idx);
    VLA_CUDA(cudaGetLastError());

    // ---- boundary facet owners
    if (nfb > 0) {
        k_face_owner<<<grid_for(nfb, TB), TB, 0, st>>>(nfb, dim, nlb, nn, m->faces, m->elems, m->n2e_ptr, m->n2e,
                                                        m->face_opp, d_err);
        VLA_CUDA(cudaGetLastError());
        // its error bits are read with the tile counts below (nothing before reads the facets)
    }

    // ---- float pair coordinates
    TRY(dalloc(m, &m->xh, nn, st));
    TRY(dalloc(m, &m->xl, nn, st));
    k_split_coords<<<grid_for(nn, TB), TB, 0, st>>>(nn, dim, m->coords, m->xh, m->xl);
    VLA_CUDA(cudaGetLastError());

    // ---- spatial order of the rows (Morton code of the cell, then node id)
    const int nbb = 256;
    double *bbp, *bbf;
    TRY(S.get(&bbp, nbb * 6));
    TRY(S.get(&bbf, 6));
    k_bbox_partial<<<nbb, 256, 0, st>>>(nn, dim, m->coords, bbp);
    k_bbox_final<<<1, 192, 0, st>>>(nbb, bbp, bbf);
    VLA_CUDA(cudaGetLastError());
    int bits = 1;
    {
        double cells = (double)nn / 8.0;
        while (bits < (dim == 3 ? 7 : 10) && std::pow(2.0, (double)(bits * dim)) < cells) ++bits;
    }
    const int64_t nkeys = (int64_t)1 << (bits * dim);
    int32_t *key, *hist, *perm;
    long long *hpre;
    TRY(S.get(&key, nn));
    TRY(S.get(&hist, nkeys));
    TRY(S.get(&hpre, nkeys + 1));
    TRY(S.get(&perm, nn));
    k_cell_keys<<<grid_for(nn, TB), TB, 0, st>>>(nn, dim, bits, m->coords, bbf, key);
    VLA_CUDA(cudaMemsetAsync(hist, 0, sizeof(int32_t) * nkeys, st));
    k_hist<<<grid_for(nn, TB), TB, 0, st>>>(nn, key, hist);
    VLA_CUDA(cudaGetLastError());
    TRY(excl_scan<int32_t>(hist, nkeys, hpre, st, nullptr));
    int32_t *bptr;
    TRY(S.get(&bptr, nkeys + 1));
    k_i64_to_i32<<<grid_for(nkeys + 1, TB, 1 << 30), TB, 0, st>>>(nkeys + 1, hpre, bptr);
    int32_t *bcur;
    TRY(S.get(&bcur, nkeys + 1));
    VLA_CUDA(cudaMemcpyAsync(bcur, bptr, sizeof(int32_t) * (nkeys + 1), cudaMemcpyDeviceToDevice, st));
    k_bucket_scatter<<<grid_for(nn, TB), TB, 0, st>>>(nn, key, bcur, perm);
    k_sort_segments<<<grid_for((nkeys + kSegWarps - 1) / kSegWarps, 1), kSegWarps * 32, 0, st>>>(nkeys, bptr, perm);
    VLA_CUDA(cudaGetLastError());

    // ---- tiles: consecutive ranks, incidence-weight budget B
    // budget: the caller's (autotuner candidates), else the tuned one, else the default;
    // VLA_TILE_BUDGET overrides all three (experiments)
    int B = m->tile_budget > 0 ? m->tile_budget : tuned_budget((dim - 2) * 2 + (m->order - 1));
    const int B_default = tile_budget(dim, m->order);
    bool adaptive = false;
    if (B <= 0) {
        B = B_default;
        adaptive = true;
    }
    if (const char *tb = getenv("VLA_TILE_BUDGET")) {
        B = std::max(64, atoi(tb));
        adaptive = false;
    }
    if (adaptive) {
        // under the default budget a small mesh is cut into about two tiles per
        // SM, where tiles of at least 128 incidences allow it: its per-tile
        // build passes and its assembly then spread over the GPU instead of
        // running on a few CTAs (the results do not depend on the tiling)
        int dev_ = 0, nsm = 0;
        VLA_CUDA(cudaGetDevice(&dev_));
        VLA_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev_));
        const int64_t total_w = nn + n2e_total, per = (total_w + 2 * (int64_t)nsm - 1) / (2 * (int64_t)std::max(nsm, 1));
        B = (int)std::min<int64_t>(B, std::max<int64_t>(128, per));
    }
    const size_t mark_allocs = m->allocs.size();
    const int64_t mark_bytes = m->device_bytes;
    const size_t cap = tile_smem_cap();
    for (int attempt = 0;; ++attempt) {
        m->tile_budget = B;
        int32_t *w, *flag, *tile_begin, *node_tile;
        long long *fpre;
        TRY(S.get(&w, nn));
        TRY(S.get(&flag, nn));
        TRY(S.get(&fpre, nn + 1));
        TRY(S.get(&node_tile, nn));
        k_rank_weights<<<grid_for(nn, TB), TB, 0, st>>>(nn, perm, cnt, w);
        TRY(excl_scan<int32_t>(w, nn, pre, st, nullptr));
        k_tile_flags<<<grid_for(nn, TB), TB, 0, st>>>(nn, B, pre, flag);
        long long n_tiles = 0;
        VLA_CUDA(cudaMemsetAsync(dsc + 2, 0, sizeof(long long), st));
        k_max_i32<<<grid_for(nn, 256), 256, 0, st>>>(nn, cnt, 1, dsc + 2);   // max incidence + 1
        VLA_CUDA(cudaMemcpyAsync(&hp[3], dsc + 2, sizeof(long long), cudaMemcpyDeviceToHost, st));
        TRY(excl_scan<int32_t>(flag, nn, fpre, st, &n_tiles));   // synchronises
        TRY(S.get(&tile_begin, n_tiles + 1));
        k_tile_assign<<<grid_for(nn, TB), TB, 0, st>>>(nn, flag, fpre, perm, tile_begin, node_tile);
        VLA_CUDA(cudaGetLastError());
        m->n_tiles = (int32_t)n_tiles;

        // max incidence of a single node bounds the tile's candidate count: B + max weight
        const int wmax = (int)hp[3];
        if (wmax > B && adaptive && B < B_default) {   // a small-mesh budget below a node's weight: cut again
            B = std::min(B_default, std::max(wmax, 2 * B));
            continue;
        }
        if (wmax > B) return fail(VLA_ERR_UNSUPPORTED, "a node belongs to %d elements (tile budget %d)", wmax - 1, B);
        // cap_n bounds a tile's distinct vertex nodes: first the element bound
        // cap_e (a few times what Kuhn-like meshes need), and only if some tile
        // has more, the bound no tile can exceed, (dim + 1) (B + wmax).
        // VLA_TILE_NODE_CAP sets the first bound instead (experiments, tests)
        const int cap_e = next_pow2(B + wmax);
        const int cap_n_max = next_pow2((dim + 1) * (B + wmax));
        int cap_n = cap_e;
        if (const char *nc = getenv("VLA_TILE_NODE_CAP")) cap_n = std::min(cap_n_max, next_pow2(std::max(64, atoi(nc))));
        int32_t *sc_elems, *sc_nodes;
        TileCounts *tcnt;
        TRY(S.get(&sc_elems, (size_t)n_tiles * cap_e));
        TRY(S.get(&tcnt, n_tiles));
        auto launch_sets = [&]() -> vla_status {
            TRY(S.get(&sc_nodes, (size_t)n_tiles * cap_n));
            const size_t hs_len = std::max(3 * (size_t)cap_e, 2 * (size_t)cap_n);
            const size_t smemA = sizeof(int32_t) * ((size_t)cap_e + hs_len + (size_t)std::max(cap_e, cap_n) + 64);
            int dev_ = 0, maxsm_ = 0;
            VLA_CUDA(cudaGetDevice(&dev_));
            VLA_CUDA(cudaDeviceGetAttribute(&maxsm_, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev_));
            if (smemA + 1024 > (size_t)maxsm_)
                return fail(VLA_ERR_UNSUPPORTED, "tile budget %d too large for the tile builder", B);
            TRY(allow_max_smem((const void *)k_tile_sets));
            k_tile_sets<<<(int)n_tiles, 256, smemA, st>>>((int)n_tiles, nn, dim, nlb, cap_e, cap_n, tile_begin,
                                                           perm, m->n2e_ptr, m->n2e, m->elems, m->row_ptr,
                                                           m->col_idx, node_tile, sc_elems, sc_nodes, tcnt, d_err);
            VLA_CUDA(cudaGetLastError());
            return VLA_OK;
        };
        TRY(launch_sets());
        // pinned tables: the tile counts (read back), the headers (sent down), the code counts (read back)
        unsigned char *tb = static_cast<unsigned char *>(
            pinned_tables((sizeof(TileCounts) + sizeof(TileHdr) + sizeof(int32_t)) * (size_t)n_tiles));
        if (!tb) return fail(VLA_ERR_OOM, "pinned host tile tables");
        TileCounts *hc = reinterpret_cast<TileCounts *>(tb);
        TileHdr *hh = reinterpret_cast<TileHdr *>(tb + sizeof(TileCounts) * (size_t)n_tiles);
        int32_t *hnc = reinterpret_cast<int32_t *>(tb + (sizeof(TileCounts) + sizeof(TileHdr)) * (size_t)n_tiles);
        VLA_CUDA(cudaMemcpyAsync(hc, tcnt, sizeof(TileCounts) * n_tiles, cudaMemcpyDeviceToHost, st));
        hp[1] = 0;
        VLA_CUDA(cudaMemcpyAsync(&hp[1], d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
        VLA_CUDA(cudaStreamSynchronize(st));
        h_err = (int)hp[1];
        if (h_err == ERR_NODE_CAP && cap_n < cap_n_max) {   // a tile with more vertex nodes than cap_n: size up once
            cap_n = cap_n_max;
            VLA_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int32_t), st));
            TRY(launch_sets());
            VLA_CUDA(cudaMemcpyAsync(hc, tcnt, sizeof(TileCounts) * n_tiles, cudaMemcpyDeviceToHost, st));
            hp[1] = 0;
            VLA_CUDA(cudaMemcpyAsync(&hp[1], d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
            VLA_CUDA(cudaStreamSynchronize(st));
            h_err = (int)hp[1];
        }
        if (h_err & ERR_FACE_OOB)
            return fail(VLA_ERR_INDEX_OOB, "a boundary facet references a node outside [0, %lld)", (long long)nn);
        if (h_err & ERR_FACE_OWNER) return fail(VLA_ERR_DEGENERATE, "a boundary facet is not a facet of any element");
        if (h_err & (ERR_TILE_CAP | ERR_NODE_CAP)) return fail(VLA_ERR_UNSUPPORTED, "tile candidate capacity exceeded");

        // tile offsets (host scan over a few thousand tiles); every segment padded for bulk copies
        auto pad = [](int64_t x, int64_t q) { return (x + q - 1) / q * q; };
        int64_t o_node = 0, o_elem = 0, o_own = 0, o_nz = 0, o_chunk = 0, n_own_total = 0, nz_total = 0;
        m->max_tile_nodes = m->max_tile_elems = m->max_tile_nz = 0;
        m->tile_elems_total = 0;
        for (int64_t t = 0; t < n_tiles; ++t) {
            TileHdr &h = hh[t];
            std::memset(&h, 0, sizeof(h));
            const TileCounts &c = hc[t];
            h.node_off = (int32_t)o_node;
            h.n_nodes = c.n_nodes;
            h.elem_off = (int32_t)o_elem;
            h.n_elems = c.n_elems;
            h.own_off = (int32_t)o_own;
            h.n_own = c.n_own;
            h.nz_off = (int32_t)o_nz;
            h.n_nz = c.n_up + c.n_diag;
            h.n_up = c.n_up;
            h.chunk_off = (int32_t)o_chunk;
            h.n_chunks = (c.n_up + c.n_diag + 31) / 32;
            h.rank_begin = c.rank_begin;
            h.n_rows = c.n_rows;
            o_node += pad(c.n_nodes, kTilePadNodes);
            o_elem += pad(c.n_elems, kTilePadElems);
            o_own += pad(c.n_own, kTilePadOwn);
            o_nz += pad(h.n_nz, kTilePadNz);
            o_chunk += pad(h.n_chunks, kTilePadChunks);
            n_own_total += c.n_own;
            nz_total += 2LL * c.n_up + c.n_diag;
            m->tile_elems_total += c.n_elems;
            m->max_tile_nodes = std::max(m->max_tile_nodes, c.n_nodes);
            m->max_tile_elems = std::max(m->max_tile_elems, c.n_elems);
            m->max_tile_nz = std::max(m->max_tile_nz, h.n_nz);
            if (h.n_chunks > 1024) return fail(VLA_ERR_UNSUPPORTED, "tile has more than 1024 chunks");
        }
        if (n_own_total != ne) return fail(VLA_ERR_CUDA, "internal: tiles own %lld of %lld elements", (long long)n_own_total, (long long)ne);
        if (nz_total != nnz) return fail(VLA_ERR_CUDA, "internal: tiles cover %lld of %lld nonzeros", (long long)nz_total, nnz);
        if (m->max_tile_elems >= 0xffff || m->max_tile_nodes > 0xffff)
            return fail(VLA_ERR_UNSUPPORTED, "tile exceeds 65534 elements or 65535 nodes");
        if (m->order == 1 && m->max_tile_elems >= 4095)
            return fail(VLA_ERR_UNSUPPORTED, "P1 tile has %d elements (limit 4094)", m->max_tile_elems);
        TRY(dalloc(m, &m->tiles, n_tiles, st));
        VLA_CUDA(cudaMemcpyAsync(m->tiles, hh, sizeof(TileHdr) * n_tiles, cudaMemcpyHostToDevice, st));
        // +16 bytes of slack: bulk copies round sizes up to 16 bytes
        TRY(dalloc(m, &m->tile_nodes, o_node + 4, st));
        TRY(dalloc(m, &m->tile_elem, o_elem + 2, st));
        TRY(dalloc(m, &m->tile_own, o_own + 4, st));
        TRY(dalloc(m, &m->tile_eid, o_elem + 4, st));
        TRY(dalloc(m, &m->tile_nzpos, o_nz + 2, st));
        TRY(dalloc(m, &m->tile_chunks, o_chunk + 2, st));
        VLA_CUDA(cudaMemsetAsync(m->tile_nodes, 0, sizeof(int32_t) * (o_node + 4), st));
        VLA_CUDA(cudaMemsetAsync(m->tile_elem, 0, sizeof(ushort4) * (o_elem + 2), st));
        VLA_CUDA(cudaMemsetAsync(m->tile_own, 0, sizeof(int32_t) * (o_own + 4), st));
        VLA_CUDA(cudaMemsetAsync(m->tile_eid, 0, sizeof(int32_t) * (o_elem + 4), st));
        VLA_CUDA(cudaMemsetAsync(m->tile_nzpos, 0, sizeof(int2) * (o_nz + 2), st));
        VLA_CUDA(cudaMemsetAsync(m->tile_chunks, 0, sizeof(int2) * (o_chunk + 2), st));
        int32_t *nz_count, *tile_ncodes, *nz_order;
        RowInfo *row_info;
        int2 *nzpos_rm;
        TRY(S.get(&nz_count, o_nz + 2));
        TRY(S.get(&nz_order, o_nz + 2));
        TRY(S.get(&nzpos_rm, o_nz + 2));
        TRY(S.get(&row_info, nn));
        TRY(S.get(&tile_ncodes, n_tiles));
        {
            auto kf = nlb == 3 ? k_tile_fill<3> : nlb == 4 ? k_tile_fill<4> : nlb == 6 ? k_tile_fill<6> : k_tile_fill<10>;
            TRY(allow_max_smem((const void *)kf));
            kf<<<(int)n_tiles, 256, sizeof(int32_t) * (size_t)std::max(1, m->max_tile_nodes), st>>>(
                (int)n_tiles, dim, cap_e, cap_n, m->tiles, perm, m->n2e_ptr, m->n2e, m->elems, m->row_ptr, m->col_idx,
                sc_elems, sc_nodes, m->tile_nodes, m->tile_elem, m->tile_own, m->tile_eid, nzpos_rm, nz_count,
                row_info);
            VLA_CUDA(cudaGetLastError());
        }
        k_chunk_table<<<(int)n_tiles, kChunkWarps * 32, 0, st>>>((int)n_tiles, m->tiles, nz_count, nzpos_rm, m->tile_nzpos, nz_order,
                                                    m->tile_chunks, tile_ncodes);
        VLA_CUDA(cudaGetLastError());
        VLA_CUDA(cudaMemcpyAsync(hnc, tile_ncodes, sizeof(int32_t) * n_tiles, cudaMemcpyDeviceToHost, st));
        VLA_CUDA(cudaStreamSynchronize(st));
        int64_t o_code = 0;
        const size_t code_bytes = (m->order == 1) ? 2 : 4;
        size_t stage_max = 0;
        for (int64_t t = 0; t < n_tiles; ++t) {
            hh[t].code_off = (int32_t)o_code;
            hh[t].n_codes = hnc[t];
            o_code += hnc[t];
            if (o_code > 0x7fffffffll) return fail(VLA_ERR_UNSUPPORTED, "too many contribution codes");
            const TileHdr &h = hh[t];
            size_t stage = 4 * pad(h.n_nodes, kTilePadNodes) + 8 * pad(h.n_elems, kTilePadElems) +
                           4 * pad(h.n_own, kTilePadOwn) + 8 * pad(h.n_chunks, kTilePadChunks) +
                           8 * pad(h.n_nz, kTilePadNz) + code_bytes * h.n_codes;
            stage_max = std::max(stage_max, stage);
        }
        m->tile_stage_bytes = stage_max;
        {
            // shared-memory footprint of the mixed-precision assembly launch: two input
            // stages and the element records.  Each part is capped on its own (stage
            // 30%, records 40% of the two-CTAs-per-SM limit), so a batched launch over
            // meshes of any types, which sizes each part for its largest tile, keeps
            // two CTAs per SM too; above a cap the tiles are cut with a smaller budget
            const int nu = nlb * (nlb + 1) / 2, rs = (nu + 1) | 1;
            const size_t stg = (stage_max + 32 * (size_t)m->max_tile_nodes + 16 + 15) / 16 * 16;
            const size_t rec = ((size_t)m->max_tile_elems + 1) * rs * 4;
            m->tile_smem = 2 * stg + rec;
            const double over = std::max((double)stg / (0.3 * (double)cap), (double)rec / (0.4 * (double)cap));
            if (over > 1.0 && attempt < 4 && B > wmax) {
                for (size_t a = mark_allocs; a < m->allocs.size(); ++a) cudaFreeAsync(m->allocs[a], st);
                m->allocs.resize(mark_allocs);
                m->device_bytes = mark_bytes;
                B = std::max(wmax, (int)((double)B / over * 0.95));
                continue;
            }
        }
        m->n_codes = o_code;
        VLA_CUDA(cudaMemcpyAsync(m->tiles, hh, sizeof(TileHdr) * n_tiles, cudaMemcpyHostToDevice, st));
        const int rsc = (nlb * (nlb + 1) / 2 + 1) | 1;   // code stride: the mixed-precision record stride
        const size_t smem_codes = sizeof(int32_t) * ((size_t)kCodeWarps * 3 * (kMaxRow + 1) + std::max(1, m->max_tile_elems));
        if (m->order == 1) {
            uint16_t *codes;
            TRY(dalloc(m, &codes, o_code + 64, st));
            auto kc = nlb == 3 ? k_tile_codes<3, uint16_t> : k_tile_codes<4, uint16_t>;
            TRY(allow_max_smem((const void *)kc));
            kc<<<(int)n_tiles, kCodeWarps * 32, smem_codes, st>>>((int)n_tiles, cap_e, rsc, m->tiles, m->n2e, m->elems,
                                                                  m->col_idx, sc_elems, row_info, nz_order,
                                                                  m->tile_chunks, codes);
            m->tile_codes = codes;
        } else {
            uint32_t *codes;
            TRY(dalloc(m, &codes, o_code + 64, st));
            auto kc = nlb == 6 ? k_tile_codes<6, uint32_t> : k_tile_codes<10, uint32_t>;
            TRY(allow_max_smem((const void *)kc));
            kc<<<(int)n_tiles, kCodeWarps * 32, smem_codes, st>>>((int)n_tiles, cap_e, rsc, m->tiles, m->n2e, m->elems,
                                                                  m->col_idx, sc_elems, row_info, nz_order,
                                                                  m->tile_chunks, codes);
            m->tile_codes = codes;
        }
        VLA_CUDA(cudaGetLastError());
        break;
    }
    TRY(dalloc(m, &m->d_err, 1, st));
    VLA_CUDA(cudaMemsetAsync(m->d_err, 0, sizeof(int32_t), st));
    m->spin_limit = 1 << 22;
    if (const char *sl = getenv("VLA_DEBUG_SPIN_LIMIT")) m->spin_limit = atoi(sl);
    return VLA_OK;
}

// ---------------------------------------------------------------------------
// facet list: facet j of element k (opposite local vertex j) and the other
// element holding it, found in the incidence list of the facet's first vertex
// ---------------------------------------------------------------------------
template <int DIM>
__global__ void k_facet_neighbors(int64_t ne, int nlb, const int32_t *__restrict__ elems,
                                  const int32_t *__restrict__ n2e_ptr, const int32_t *__restrict__ n2e,
                                  int32_t *__restrict__ nbr, int32_t *__restrict__ flag) {
    constexpr int NV = DIM + 1;
    // vertex ids of element e: one 16-byte load for P1 tetrahedra
    auto verts = [&](int64_t e, int32_t (&v)[NV]) {
        if (DIM == 3 && nlb == 4) {
            const int4 q = __ldg(reinterpret_cast<const int4 *>(elems) + e);
            v[0] = q.x, v[1] = q.y, v[2] = q.z, v[NV - 1] = q.w;
        } else {
#pragma unroll
            for (int i = 0; i < NV; ++i) v[i] = __ldg(elems + e * nlb + i);
        }
    };
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ne * NV; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / NV;
        const int j = (int)(t - k * NV);
        int32_t kv[NV], fv[DIM];
        verts(k, kv);
        int q = 0;
#pragma unroll
        for (int i = 0; i < NV; ++i)
            if (i != j) fv[q++] = kv[i];
        int32_t found = -1;
        for (int32_t p = n2e_ptr[fv[0]]; p < n2e_ptr[fv[0] + 1] && found < 0; ++p) {
            const int32_t e = n2e[p] >> 4;
            if (e == k) continue;
            int32_t ev[NV];
            verts(e, ev);
            int hits = 1;   // fv[0] is in e by construction
#pragma unroll
            for (int a = 1; a < DIM; ++a)
#pragma unroll
                for (int i = 0; i < NV; ++i) hits += ev[i] == fv[a];
            if (hits == DIM) found = e;
        }
        nbr[t] = found;
        flag[t] = (found < 0 || found > k) ? 1 : 0;   // listed with the smaller element
    }
}

__global__ void k_facet_write(int64_t ne, int dim, int nlb, const int32_t *__restrict__ elems,
                              const int32_t *__restrict__ nbr, const int32_t *__restrict__ flag,
                              const long long *__restrict__ pos, int32_t *__restrict__ faces,
                              int32_t *__restrict__ owner, int32_t *__restrict__ neighbor) {
    const int nv = dim + 1;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ne * nv; t += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[t]) continue;
        const int64_t k = t / nv, f = pos[t];
        const int j = (int)(t - k * nv);
        if (faces) {
            int q = 0;
            for (int i = 0; i < nv; ++i)
                if (i != j) faces[f * dim + q++] = elems[k * nlb + i];
        }
        if (owner) {
            owner[2 * f] = (int32_t)k;
            owner[2 * f + 1] = j;
        }
        if (neighbor) neighbor[f] = nbr[t];
    }
}

__global__ void k_count_boundary(int64_t n, const int32_t *__restrict__ nbr, const int32_t *__restrict__ flag,
                                 int32_t *__restrict__ bflag) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
        bflag[t] = flag[t] && nbr[t] < 0;
}

}  // namespace

vla_status mesh_build(vla_mesh *m, const double *coords, const int32_t *elems, const int32_t *faces) {
    return build(m, coords, elems, faces);
}

}  // namespace vla

using namespace vla;

namespace vla {
vla_status mesh_create_budget(int32_t dim, int32_t order, int64_t nn, int64_t ne, const double *coords,
                              const int32_t *elems, int64_t nfb, const int32_t *faces, void *stream, int budget,
                              vla_mesh **out) {
    if (!out) return fail(VLA_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (dim != 2 && dim != 3) return fail(VLA_ERR_INVALID_ARG, "dim must be 2 or 3");
    if (order != VLA_P1 && order != VLA_P2) return fail(VLA_ERR_INVALID_ARG, "order must be VLA_P1 or VLA_P2");
    if (nn < 1 || ne < 1 || nfb < 0) return fail(VLA_ERR_INVALID_ARG, "need nn >= 1, ne >= 1, nfb >= 0");
    if (nn > 0x7fffffffll || nfb > 0x7fffffffll) return fail(VLA_ERR_INVALID_ARG, "counts must fit int32");
    if (ne >= ((int64_t)1 << 27)) return fail(VLA_ERR_UNSUPPORTED, "ne must be below 2^27");
    if (!coords || !elems || (nfb > 0 && !faces)) return fail(VLA_ERR_INVALID_ARG, "null mesh array");
    vla_mesh *m = new (std::nothrow) vla_mesh();
    if (!m) return fail(VLA_ERR_OOM, "host allocation failed");
    m->dim = dim;
    m->order = order;
    m->nlb = order == VLA_P1 ? dim + 1 : (dim + 1) * (dim + 2) / 2;
    m->nn = nn;
    m->ne = ne;
    m->nfb = nfb;
    m->stream = (cudaStream_t)stream;
    m->tile_budget = budget;
    vla_status s = mesh_build(m, coords, elems, faces);
    if (s != VLA_OK) {
        char keep[512];
        vla_last_error(keep, sizeof(keep));
        cudaStreamSynchronize(m->stream);   // no copy from this thread's pinned tables left in flight
        cudaGetLastError();
        vla_mesh_destroy(m);
        set_error("%s", keep);
        return s;
    }
    cudaError_t e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) {
        vla_mesh_destroy(m);
        return cuda_fail(e, "mesh build");
    }
    *out = m;
    return VLA_OK;
}
}  // namespace vla

extern "C" vla_status vla_mesh_create(int32_t dim, int32_t order, int64_t nn, int64_t ne, const double *coords,
                                      const int32_t *elems, int64_t nfb, const int32_t *faces, void *stream,
                                      vla_mesh **out) {
    return vla::mesh_create_budget(dim, order, nn, ne, coords, elems, nfb, faces, stream, 0, out);
}

extern "C" vla_status vla_mesh_destroy(vla_mesh *m) {
    if (!m) return VLA_OK;
    cudaStreamSynchronize(m->stream);
    for (void *p : m->allocs) cudaFreeAsync(p, m->stream);
    cudaStreamSynchronize(m->stream);
    delete m;
    return VLA_OK;
}

extern "C" vla_status vla_mesh_check(vla_mesh *m, void *stream) {
    if (!m) return fail(VLA_ERR_INVALID_ARG, "null mesh");
    cudaStream_t st = (cudaStream_t)stream;
    int h = 0;
    VLA_CUDA(cudaMemcpyAsync(&h, m->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    VLA_CUDA(cudaStreamSynchronize(st));
    if (h) {
        VLA_CUDA(cudaMemsetAsync(m->d_err, 0, sizeof(int), st));
        VLA_CUDA(cudaStreamSynchronize(st));
        return fail(VLA_ERR_TIMEOUT, "a bounded wait of a kernel on this mesh expired (error word %d)", h);
    }
    return VLA_OK;
}

extern "C" vla_status vla_mesh_info(const vla_mesh *m, vla_mesh_info_t *info) {
    if (!m || !info) return fail(VLA_ERR_INVALID_ARG, "null argument");
    info->dim = m->dim;
    info->order = m->order;
    info->nlb = m->nlb;
    info->nn = m->nn;
    info->ne = m->ne;
    info->nfb = m->nfb;
    info->nnz = m->nnz;
    info->max_row_len = m->max_row_len;
    info->n_tiles = m->n_tiles;
    info->device_bytes = m->device_bytes;
    info->tile_elems = m->tile_elems_total;
    info->n_codes = m->n_codes;
    info->tile_budget = m->tile_budget;
    info->reserved = 0;
    info->smem_bytes = (int64_t)m->tile_smem;
    return VLA_OK;
}

extern "C" vla_status vla_mesh_csr_view(const vla_mesh *m, const int32_t **row_ptr, const int32_t **col_idx) {
    if (!m || !row_ptr || !col_idx) return fail(VLA_ERR_INVALID_ARG, "vla_mesh_csr_view: NULL argument");
    *row_ptr = m->row_ptr;
    *col_idx = m->col_idx;
    return VLA_OK;
}

extern "C" vla_status vla_mesh_csr(const vla_mesh *m, int32_t *row_ptr, int32_t *col_idx, void *stream) {
    if (!m) return fail(VLA_ERR_INVALID_ARG, "null mesh");
    cudaStream_t st = (cudaStream_t)stream;
    if (row_ptr)
        VLA_CUDA(cudaMemcpyAsync(row_ptr, m->row_ptr, sizeof(int32_t) * (m->nn + 1), cudaMemcpyDeviceToDevice, st));
    if (col_idx && m->nnz > 0)
        VLA_CUDA(cudaMemcpyAsync(col_idx, m->col_idx, sizeof(int32_t) * m->nnz, cudaMemcpyDeviceToDevice, st));
    return VLA_OK;
}

extern "C" vla_status vla_mesh_facets(const vla_mesh *m, int32_t *faces, int32_t *owner, int32_t *neighbor,
                                      int64_t *n_faces, int64_t *n_boundary, void *stream) {
    if (!m) return fail(VLA_ERR_INVALID_ARG, "null mesh");
    cudaStream_t st = (cudaStream_t)stream;
    const int nv = m->dim + 1;
    const int64_t nt = m->ne * nv;
    Scratch S;
    S.st = st;
    int32_t *nbr, *flag, *bflag;
    long long *pos;
    TRY(S.get(&nbr, nt));
    TRY(S.get(&flag, nt));
    TRY(S.get(&bflag, nt));
    TRY(S.get(&pos, nt + 1));
    if (m->dim == 3)
        k_facet_neighbors<3><<<grid_for(nt, 256), 256, 0, st>>>(m->ne, m->nlb, m->elems, m->n2e_ptr, m->n2e, nbr, flag);
    else
        k_facet_neighbors<2><<<grid_for(nt, 256), 256, 0, st>>>(m->ne, m->nlb, m->elems, m->n2e_ptr, m->n2e, nbr, flag);
    VLA_CUDA(cudaGetLastError());
    long long total = 0, nb = 0;
    TRY(excl_scan<int32_t>(flag, nt, pos, st, &total));
    if (faces || owner || neighbor)
        k_facet_write<<<grid_for(nt, 256), 256, 0, st>>>(m->ne, m->dim, m->nlb, m->elems, nbr, flag, pos, faces,
                                                          owner, neighbor);
    k_count_boundary<<<grid_for(nt, 256), 256, 0, st>>>(nt, nbr, flag, bflag);
    VLA_CUDA(cudaGetLastError());
    TRY(excl_scan<int32_t>(bflag, nt, pos, st, &nb));
    VLA_CUDA(cudaStreamSynchronize(st));
    if (n_faces) *n_faces = total;
    if (n_boundary) *n_boundary = nb;
    return VLA_OK;
}

// ---------------------------------------------------------------------------
// Row-block partition (assembly on several GPUs by blocks of rows).  Every
// element and every page is independent; the one exchange step is the CSR
// sum.  A GPU that owns the contiguous rows [r0, r1) takes every element with
// a node in that range -- the elements it shares with its neighbours (the
// halo) are duplicated -- and so holds every contribution to its rows: it
// assembles complete rows and no reduction across GPUs is needed.  Node
// numbering stays global, so the rows [r0, r1) of the sub-mesh's CSR are the
// rows [r0, r1) of the whole mesh's CSR, with the same summation order
// (ascending element id) and therefore the same bits.
// ---------------------------------------------------------------------------
namespace vla {
namespace {

// flag[k] = 1 if element k has a node (vertex or P2 mid-edge node) in [r0, r1)
__global__ void k_block_elem_flags(int64_t ne, int nlb, const int32_t *__restrict__ elems, int32_t r0, int32_t r1,
                                   int32_t *__restrict__ flag) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < ne; k += (int64_t)gridDim.x * blockDim.x) {
        int32_t f = 0;
        for (int j = 0; j < nlb; ++j) {
            const int32_t v = elems[k * nlb + j];
            f |= (v >= r0 && v < r1) ? 1 : 0;
        }
        flag[k] = f;
    }
}

// flag[f] = 1 if the smallest node of facet f lies in [r0, r1): the facets are split among the blocks
__global__ void k_block_facet_flags(int64_t nf, int dim, const int32_t *__restrict__ faces, int32_t r0, int32_t r1,
                                    int32_t *__restrict__ flag) {
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += (int64_t)gridDim.x * blockDim.x) {
        int32_t v = faces[f * dim];
        for (int j = 1; j < dim; ++j) v = min(v, faces[f * dim + j]);
        flag[f] = (v >= r0 && v < r1) ? 1 : 0;
    }
}

__global__ void k_compact_flags(int64_t n, const int32_t *__restrict__ flag, const long long *__restrict__ pre,
                                int32_t *__restrict__ ids) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        if (flag[k]) ids[pre[k]] = (int32_t)k;
}

// dst row i = src row ids[i] (rows of w int32)
__global__ void k_gather_rows(int64_t n, int w, const int32_t *__restrict__ ids, const int32_t *__restrict__ src,
                              int32_t *__restrict__ dst) {
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n * w; q += (int64_t)gridDim.x * blockDim.x)
        dst[q] = src[(int64_t)ids[q / w] * w + q % w];
}

// ascending ids of the flagged items into a stream-ordered allocation; synchronises for the count
vla_status select_flagged(int64_t n, const int32_t *flag, int32_t **ids, int64_t *count, cudaStream_t st) {
    *ids = nullptr;
    *count = 0;
    long long *pre = nullptr;
    VLA_CUDA(pool_malloc((void **)&pre, sizeof(long long) * (n + 1), st));
    long long total = 0;
    vla_status s = excl_scan<int32_t>(flag, n, pre, st, &total);
    if (s == VLA_OK && total > 0) {
        cudaError_t e = pool_malloc((void **)ids, sizeof(int32_t) * total, st);
        if (e != cudaSuccess) s = cuda_fail(e, "partition ids");
        else k_compact_flags<<<grid_for(n, 256), 256, 0, st>>>(n, flag, pre, *ids);
    }
    cudaFreeAsync(pre, st);
    if (s == VLA_OK) {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) s = cuda_fail(e, "partition compaction");
    }
    *count = total;
    return s;
}

vla_status check_block(int64_t nn, int32_t row_begin, int32_t row_end) {
    if (row_begin < 0 || row_end <= row_begin || (int64_t)row_end > nn)
        return fail(VLA_ERR_INVALID_ARG, "row block [%d, %d) must be a non-empty range inside [0, %lld)", row_begin,
                    row_end, (long long)nn);
    return VLA_OK;
}

}  // namespace
}  // namespace vla

extern "C" vla_status vla_partition_rows(int32_t nlb, int64_t ne, const int32_t *elems, int32_t row_begin,
                                         int32_t row_end, int32_t *elem_ids, int64_t *n_elems, void *stream) {
    if (!n_elems) return fail(VLA_ERR_INVALID_ARG, "n_elems is NULL");
    *n_elems = 0;
    if (nlb < 3 || nlb > 10) return fail(VLA_ERR_INVALID_ARG, "nlb must be in [3, 10]");
    if (ne < 0 || ne > 0x7fffffffll) return fail(VLA_ERR_INVALID_ARG, "ne must be in [0, 2^31-1]");
    if (row_begin < 0 || row_end < row_begin) return fail(VLA_ERR_INVALID_ARG, "need 0 <= row_begin <= row_end");
    if (ne == 0 || row_end == row_begin) return VLA_OK;
    if (!elems) return fail(VLA_ERR_INVALID_ARG, "elems is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *flag = nullptr, *ids = nullptr;
    VLA_CUDA(pool_malloc((void **)&flag, sizeof(int32_t) * ne, st));
    k_block_elem_flags<<<grid_for(ne, 256), 256, 0, st>>>(ne, nlb, elems, row_begin, row_end, flag);
    int64_t cnt = 0;
    vla_status s = select_flagged(ne, flag, &ids, &cnt, st);
    if (s == VLA_OK && elem_ids && cnt > 0) {
        cudaError_t e = cudaMemcpyAsync(elem_ids, ids, sizeof(int32_t) * cnt, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) s = cuda_fail(e, "partition copy");
    }
    cudaFreeAsync(flag, st);
    if (ids) cudaFreeAsync(ids, st);
    if (s == VLA_OK) *n_elems = cnt;
    return s;
}

extern "C" vla_status vla_mesh_create_rows(int32_t dim, int32_t order, int64_t nn, int64_t ne, const double *coords,
                                           const int32_t *elems, int64_t nfb, const int32_t *faces, int32_t row_begin,
                                           int32_t row_end, void *stream, vla_mesh **out) {
    if (!out) return fail(VLA_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (dim != 2 && dim != 3) return fail(VLA_ERR_INVALID_ARG, "dim must be 2 or 3");
    if (order != VLA_P1 && order != VLA_P2) return fail(VLA_ERR_INVALID_ARG, "order must be VLA_P1 or VLA_P2");
    if (nn < 1 || nn > 0x7fffffffll || ne < 1 || ne > 0x7fffffffll || nfb < 0 || nfb > 0x7fffffffll)
        return fail(VLA_ERR_INVALID_ARG, "need 1 <= nn, ne < 2^31 and 0 <= nfb < 2^31");
    TRY(check_block(nn, row_begin, row_end));
    if (!coords || !elems || (nfb > 0 && !faces)) return fail(VLA_ERR_INVALID_ARG, "null mesh array");
    const int nlb = order == VLA_P1 ? dim + 1 : (dim + 1) * (dim + 2) / 2;
    cudaStream_t st = (cudaStream_t)stream;
    int32_t *flag = nullptr, *ids = nullptr, *sub = nullptr, *fflag = nullptr, *fids = nullptr, *fsub = nullptr;
    int64_t nes = 0, nfs = 0;
    vla_status s = VLA_OK;
    auto ck = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess && s == VLA_OK) s = cuda_fail(e, what);
    };
    ck(pool_malloc((void **)&flag, sizeof(int32_t) * ne, st), "partition flags");
    if (s == VLA_OK) {
        k_block_elem_flags<<<grid_for(ne, 256), 256, 0, st>>>(ne, nlb, elems, row_begin, row_end, flag);
        s = select_flagged(ne, flag, &ids, &nes, st);
    }
    if (s == VLA_OK && nes == 0)
        s = fail(VLA_ERR_INVALID_ARG, "no element has a node in rows [%d, %d)", row_begin, row_end);
    if (s == VLA_OK) {
        ck(pool_malloc((void **)&sub, sizeof(int32_t) * nes * nlb, st), "sub-mesh elements");
        if (s == VLA_OK) k_gather_rows<<<grid_for(nes * nlb, 256), 256, 0, st>>>(nes, nlb, ids, elems, sub);
    }
    if (s == VLA_OK && nfb > 0) {
        ck(pool_malloc((void **)&fflag, sizeof(int32_t) * nfb, st), "partition facet flags");
        if (s == VLA_OK) {
            k_block_facet_flags<<<grid_for(nfb, 256), 256, 0, st>>>(nfb, dim, faces, row_begin, row_end, fflag);
            s = select_flagged(nfb, fflag, &fids, &nfs, st);
        }
        if (s == VLA_OK && nfs > 0) {
            ck(pool_malloc((void **)&fsub, sizeof(int32_t) * nfs * dim, st), "sub-mesh facets");
            if (s == VLA_OK) k_gather_rows<<<grid_for(nfs * dim, 256), 256, 0, st>>>(nfs, dim, fids, faces, fsub);
        }
    }
    if (s == VLA_OK) ck(cudaGetLastError(), "partition gather");
    if (s == VLA_OK) s = mesh_create_budget(dim, order, nn, nes, coords, sub, nfs, fsub, stream, 0, out);
    for (int32_t *p : {flag, ids, sub, fflag, fids, fsub})
        if (p) cudaFreeAsync(p, st);
    if (s == VLA_OK) {
        (*out)->row_begin = row_begin;
        (*out)->row_end = row_end;
    }
    return s;
}
