// mhd_thermal_launch.h -- host entry of the thermal-source kernels.
#pragma once
#include <cuda_runtime.h>

namespace mhd {
struct PatchDev;
struct ThermalDev;
int issue_thermal(const PatchDev& P, const ThermalDev& th, cudaStream_t s, long long* launches);
int issue_thermal_cells(long long n, const double* T0, const double* nh, const double* ce, const double* dt,
                        const ThermalDev& th, double* T_out, int* status, cudaStream_t s);
}  // namespace mhd
