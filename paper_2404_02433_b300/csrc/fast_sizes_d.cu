// Register-resident transform launchers for n = 1024 (one translation unit
// per group of lengths, so that the library compiles in parallel).
#include "fast_kernels.cuh"

namespace etc {
ETC_FAST_INSTANTIATE(1024)
}  // namespace etc
