// Register-resident transform launchers for n = 160, 192, 256 (one translation unit
// per group of lengths, so that the library compiles in parallel).
#include "fast_kernels.cuh"

namespace etc {
ETC_FAST_INSTANTIATE(160)
ETC_FAST_INSTANTIATE(192)
ETC_FAST_INSTANTIATE(256)
}  // namespace etc
