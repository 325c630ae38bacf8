// Detector instantiations for up to 8 users (own translation unit: parallel compile).
#include "detect_kernel.cuh"

namespace rapro {
RAPRO_DETECT_DEFINE_KT(8)
}  // namespace rapro
