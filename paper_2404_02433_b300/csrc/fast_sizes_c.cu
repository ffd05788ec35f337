// Register-resident transform launchers for n = 384, 512 (one translation unit
// per group of lengths, so that the library compiles in parallel).
#include "fast_kernels.cuh"

namespace etc {
ETC_FAST_INSTANTIATE(384)
ETC_FAST_INSTANTIATE(512)
}  // namespace etc
