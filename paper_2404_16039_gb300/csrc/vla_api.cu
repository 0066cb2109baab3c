// vla_api.cu -- library-wide entry points: version, error reporting, and the
// device error word polled after bounded waits.
#include <cstdarg>
#include <cstring>

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
