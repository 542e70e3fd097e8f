// hfs_step1d_wide_vinone.cu -- the wide FP32 fused 1D step kernel (every plan,
// including the alternative radix orders and four values per thread) for
// batches whose instances all have perturbation kind HFS_VI_NONE and symmetric
// boxes (one translation unit per variant, compiled in parallel).
#include "hfs_step1d.cuh"

namespace hfs {
HFS_STEP1D_VARIANT(, float, HFS_VI_NONE, true)
}  // namespace hfs
