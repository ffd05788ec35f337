// Register-resident transform launchers for n = 32, 64, 96, 128 (one translation unit
// per group of lengths, so that the library compiles in parallel).
#include "fast_kernels.cuh"

namespace etc {
ETC_FAST_INSTANTIATE(32)
ETC_FAST_INSTANTIATE(64)
ETC_FAST_INSTANTIATE(96)
ETC_FAST_INSTANTIATE(128)
}  // namespace etc
