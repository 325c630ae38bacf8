// Detector instantiations for up to 12 users (own translation unit: parallel compile).
#include "detect_kernel.cuh"

namespace rapro {
RAPRO_DETECT_DEFINE_KT(12)
}  // namespace rapro
