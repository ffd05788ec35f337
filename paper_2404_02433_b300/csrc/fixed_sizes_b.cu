// Block-floating-point transform launchers for n = 160, 192, 256 (one
// translation unit per group of lengths, so that the library compiles in
// parallel).
#include "fixed_kernels.cuh"

namespace etc {
ETC_FX_INSTANTIATE(160)
ETC_FX_INSTANTIATE(192)
ETC_FX_INSTANTIATE(256)
ETC_FX_Y3_INSTANTIATE(256)
}  // namespace etc
