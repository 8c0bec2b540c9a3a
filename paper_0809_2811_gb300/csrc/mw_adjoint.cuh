// mw_adjoint.cuh -- adjoint of the forces (device side).
#pragma once
#include "mw_device.cuh"
