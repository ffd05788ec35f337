// Block-floating-point transform launchers for n = 512 (one translation unit
// per group of lengths, so that the library compiles in parallel).
#include "fixed_kernels.cuh"

namespace etc {
ETC_FX_INSTANTIATE(512)
ETC_FX_Y3_INSTANTIATE(512)
}  // namespace etc
