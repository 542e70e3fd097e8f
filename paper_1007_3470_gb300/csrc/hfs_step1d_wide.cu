// hfs_step1d_wide.cu -- the generic wide FP32 fused 1D step kernel (every
// plan, including the alternative radix orders and four values per thread;
// perturbation kind and box symmetry read per instance).
#include "hfs_step1d.cuh"

namespace hfs {
HFS_STEP1D_VARIANT(, float, -1, true)
}  // namespace hfs
