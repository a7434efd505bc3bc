// Real FP64 instantiations (FP64 path and FP32-bulk variant).
#include "tho_launch.cuh"

namespace tho {
const Launcher kLaunchF64 = make_launcher<double, double>();
const Launcher kLaunchF64Bulk32 = make_launcher<double, float>();
const Launcher kLaunchF64Emu = make_launcher<double, double, true>();
}  // namespace tho
