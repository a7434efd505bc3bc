// Complex128 instantiations (FP64 path and FP32-bulk variant).
#include "tho_launch.cuh"

namespace tho {
const Launcher kLaunchC128 = make_launcher<z64, z64>();
const Launcher kLaunchC128Bulk32 = make_launcher<z64, z32>();
const Launcher kLaunchC128Emu = make_launcher<z64, z64, true>();
}  // namespace tho
