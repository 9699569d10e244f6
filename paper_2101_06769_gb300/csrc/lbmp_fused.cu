// lbmp_fused.cu -- fused single-pass step kernel (placeholder until written)
#include "lbmp_internal.h"

namespace lbmp {

bool fused_supported(const lbmp_handle*) { return false; }
cudaError_t launch_step_fused(lbmp_handle* h) { return launch_step_simple(h); }

}  // namespace lbmp
