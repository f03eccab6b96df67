// Host-side runtime pieces of libneat.so: error reporting and argument checks.
#include <string>

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

}  // namespace neat

extern "C" const char *neat_last_error(void) { return neat::t_last_error.c_str(); }

extern "C" const char *neat_version(void) { return "neat-gb300 0.1 (sm_103a)"; }
