// Detector instantiations for up to 4 users (own translation unit: parallel compile).
#include "detect_kernel.cuh"

namespace rapro {
RAPRO_DETECT_DEFINE_KT(4)
}  // namespace rapro
