// Diagnostics shared by every entry point.
#include <atomic>

#include "common.cuh"

namespace tw {
static std::atomic<int> g_last_cuda_error{0};
static std::atomic<unsigned long long> g_launches{0};
void set_cuda_error(cudaError_t e) { g_last_cuda_error.store((int)e); }
static thread_local int g_count_paused = 0;
void count_launches(unsigned long long n) {
    if (!g_count_paused) g_launches.fetch_add(n);
}
void pause_launch_count(bool on) { g_count_paused += on ? 1 : -1; }
}  // namespace tw

extern "C" const char *tw_status_string(int status) {
    switch (status) {
        case TW_OK: return "ok";
        case TW_NOT_CONVERGED: return "not converged: sweep cap reached before the residual tolerance";
        case TW_NO_PATH: return "no path: the descent stalled or exceeded max_len";
        case TW_EINVAL: return "invalid argument";
        case TW_EGOAL_BLOCKED: return "goal cell is occupied, on the border or out of range";
        case TW_ESTART_BLOCKED: return "start cell is occupied";
        case TW_ECUDA: return "CUDA error (see tw_last_cuda_error)";
        case TW_EWORKSPACE: return "workspace missing, misaligned or too small";
        default: return "unknown status";
    }
}

extern "C" int tw_last_cuda_error(void) { return tw::g_last_cuda_error.load(); }

extern "C" unsigned long long tw_launch_count(void) { return tw::g_launches.load(); }

extern "C" const char *tw_version(void) { return "twgrid 0.1 (sm_103a)"; }
