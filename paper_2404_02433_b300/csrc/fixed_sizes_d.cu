// Block-floating-point transform launchers for n = 384 and 1024 (one
// translation unit per group of lengths, so that the library compiles in
// parallel).
#include "fixed_kernels.cuh"

namespace etc {
ETC_FX_INSTANTIATE(384)
ETC_FX_INSTANTIATE(1024)
ETC_FX_Y3_INSTANTIATE(1024)
}  // namespace etc
