// semistoch.cu -- deterministic projection inside the space D (Sec. III).
#include "fq_internal.h"

struct fciqmc_handle;

namespace fq {
void launch_semistoch(const DevInst *, int, int, cudaStream_t) {}
}  // namespace fq

int build_semistochastic(fciqmc_handle *) { return FCIQMC_ERR_UNSUPPORTED; }

extern "C" int fciqmc_step_batch(fciqmc_handle **, int32_t, int64_t) { return FCIQMC_ERR_UNSUPPORTED; }
