// Mixed-precision defect correction (placeholder until the correction sweeps land).
#include "common.cuh"
#include "hp_internal.cuh"

namespace tw {

size_t carve_mixed(Carver &cv, int nx, int ny, int storage, RelaxLayout *R) {
    (void)storage;
    carve_rb(cv, nx, ny, R ? &R->rb : nullptr, true);
    return cv.need;
}

int relax_mixed(const uint8_t *, int, int, int, int, float *, int, const hp_params *, hp_stats *,
                RelaxLayout &, cudaStream_t) {
    return TW_EINVAL;
}

}  // namespace tw
