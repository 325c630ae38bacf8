// Detector instantiations for up to 16 users (own translation unit: parallel compile).
#include "detect_kernel.cuh"

namespace rapro {
RAPRO_DETECT_DEFINE_KT(16)
}  // namespace rapro
