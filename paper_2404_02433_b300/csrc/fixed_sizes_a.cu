// Block-floating-point transform launchers for n = 32, 64, 96, 128 (one
// translation unit per group of lengths, so that the library compiles in
// parallel).
#include "fixed_kernels.cuh"

namespace etc {
ETC_FX_INSTANTIATE(32)
ETC_FX_INSTANTIATE(64)
ETC_FX_INSTANTIATE(96)
ETC_FX_INSTANTIATE(128)
}  // namespace etc
