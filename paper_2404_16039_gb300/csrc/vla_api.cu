// vla_api.cu -- library-wide entry points: version, error reporting, and the
// device error word polled after bounded waits.
#include <algorithm>
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "vla_internal.cuh"

namespace vla {

static thread_local std::string t_last_error;

void set_error(const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_last_error = buf;
}

vla_status fail(vla_status st, const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_last_error = buf;
    return st;
}

vla_status cuda_fail(cudaError_t e, const char *what) {
    return fail(VLA_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
}

static std::mutex g_tune_mu;
static int g_budget[4] = {0, 0, 0, 0};
static int g_ctas[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};

// default incidence budget of a row tile per element type.  Smaller tiles
// assemble a little faster in 2-D (the autotuner picks half these budgets
// there), and P2 tetrahedra assemble faster in batches at 480, but both cost
// mesh-build time (more tiles; P2 tiles at 480 often exceed the shared-memory
// caps and are cut again), which dominates ingest-bound serving.
int tile_budget(int dim, int order) {
    if (order == 1) return dim == 3 ? 800 : 2048;
    return dim == 3 ? 384 : 1024;
}

int tuned_budget(int type) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return (type >= 0 && type < 4) ? g_budget[type] : 0;
}

int tuned_ctas(int type, bool mix) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return (type >= 0 && type < 4) ? g_ctas[type][mix ? 1 : 0] : 0;
}

void set_tuned(int type, bool mix, int budget, int ctas) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (type < 0 || type >= 4) return;
    g_budget[type] = budget;
    g_ctas[type][mix ? 1 : 0] = ctas;
}

// Device memory of mesh builds, batches, servers and integral scratch comes
// from one memory pool per device that keeps up to min(8 GiB, 1/16 of the
// device) of freed memory mapped between calls.  The device's default pool
// keeps none: every synchronisation returns what was freed to the driver, and
// the next build maps it again (a few hundred MB of scratch per million
// elements).  VLA_POOL_KEEP (bytes) sets the amount kept; 0 keeps none.  If
// the pool cannot be made, the device's default pool serves the allocations.
cudaError_t pool_malloc(void **p, size_t bytes, cudaStream_t st) {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    static bool tried[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaMallocAsync(p, bytes, st);
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!tried[dev]) {   // one attempt per device; without a pool the device's default one serves
            tried[dev] = true;
            cudaMemPoolProps pp;
            std::memset(&pp, 0, sizeof(pp));
            pp.allocType = cudaMemAllocationTypePinned;
            pp.handleTypes = cudaMemHandleTypeNone;
            pp.location.type = cudaMemLocationTypeDevice;
            pp.location.id = dev;
            cudaMemPool_t np;
            size_t fr = 0, total = 0;
            if (cudaMemPoolCreate(&np, &pp) == cudaSuccess) {
                unsigned long long keep = 0;
                if (cudaMemGetInfo(&fr, &total) == cudaSuccess) keep = std::min<unsigned long long>(8ull << 30, total / 16);
                if (const char *k = getenv("VLA_POOL_KEEP")) keep = strtoull(k, nullptr, 10);
                if (cudaMemPoolSetAttribute(np, cudaMemPoolAttrReleaseThreshold, &keep) == cudaSuccess) pools[dev] = np;
                else cudaMemPoolDestroy(np);
            }
            cudaGetLastError();   // a failed attempt leaves no sticky error behind
        }
        pool = pools[dev];
    }
    return pool ? cudaMallocFromPoolAsync(p, bytes, pool, st) : cudaMallocAsync(p, bytes, st);
}

}  // namespace vla

extern "C" int32_t vla_version(void) { return 100; }

extern "C" size_t vla_last_error(char *buf, size_t len) {
    const std::string &s = vla::t_last_error;
    if (buf && len > 0) {
        size_t n = s.size() < len - 1 ? s.size() : len - 1;
        std::memcpy(buf, s.data(), n);
        buf[n] = '\0';
    }
    return s.size();
}
