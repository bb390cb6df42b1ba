// Persistent fused forward + L1 + backward over (view, tile) work items (batched path).
#include "tgs_internal.cuh"

namespace tgs {}  // namespace tgs
