// hfs_step1d_vicos.cu -- the FP32 fused 1D step kernel specialised for
// batches whose instances all have perturbation kind HFS_VI_COS and boxes
// symmetric about 0 (one translation unit per variant, compiled in parallel).
#include "hfs_step1d.cuh"

namespace hfs {
HFS_STEP1D_VARIANT(, float, HFS_VI_COS, false)
}  // namespace hfs
