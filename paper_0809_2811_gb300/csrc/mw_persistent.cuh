// mw_persistent.cuh -- persistent cooperative engine (device side).
#pragma once
#include "mw_device.cuh"

namespace mw {
constexpr int kPersThreads = 128;
}  // namespace mw
