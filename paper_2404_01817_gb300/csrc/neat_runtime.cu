// Host-side runtime pieces of libneat.so: error reporting, argument checks
// and kernel shared-memory limits.
#include <map>
#include <mutex>
#include <string>
#include <utility>

#include "neat_internal.h"

namespace neat {

namespace {
thread_local std::string t_last_error;
}

void set_error(const std::string &msg) { t_last_error = msg; }
void clear_error() { t_last_error.clear(); }

int cuda_fail(cudaError_t e, const char *what)
{
    t_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return NEAT_ECUDA;
}

int invalid(const char *what)
{
    t_last_error = what;
    return NEAT_EINVAL;
}

bool dims_ok(const neat_dims &d)
{
    return d.num_inputs >= 0 && d.num_outputs >= 1 && d.max_nodes >= 1 && d.max_nodes <= NEAT_MAX_NODES &&
           d.max_conns >= 0 && d.max_conns <= NEAT_MAX_CONNS &&
           (int64_t)d.num_inputs + d.num_outputs <= d.max_nodes;
}

namespace {
std::mutex g_smem_mu;
std::map<std::pair<int, const void *>, size_t> g_smem_allowed;   // (device, kernel) -> dynamic bytes allowed
}

int allow_dynamic_smem(const void *kernel, size_t dynamic_bytes, const char *what)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, what);
    std::lock_guard<std::mutex> lk(g_smem_mu);
    size_t &allowed = g_smem_allowed[{dev, kernel}];
    if (allowed >= dynamic_bytes) return NEAT_OK;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return cuda_fail(e, what);
    if (fa.sharedSizeBytes + dynamic_bytes > kMaxSmemPerBlock) return invalid(what);
    if (fa.sharedSizeBytes + dynamic_bytes > 48u * 1024u) {
        // never lowered: launches of the same kernel with larger needs may be in flight
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dynamic_bytes);
        if (e != cudaSuccess) return cuda_fail(e, what);
    }
    allowed = dynamic_bytes;
    return NEAT_OK;
}

}  // namespace neat

extern "C" const char *neat_last_error(void) { return neat::t_last_error.c_str(); }

extern "C" const char *neat_version(void) { return "neat-gb300 0.1 (sm_103a)"; }
