// mhd_mlp_launch.h -- host entries of the surrogate kernels (mhd_mlp.cu).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace mhd {
struct PatchDev;
struct ThermalDev;
struct MlpDev;
int mlp_forward(long long n, const float* xs, const MlpDev& M, float* y, cudaStream_t s);
int mlp_grad(const MlpDev& M, const float* data, long long nrows, unsigned long long seed, long long step, int batch,
             float* grad, float* loss_sum, cudaStream_t s);
int mlp_grad_tc_setup();  // opt-in to the kernel's shared memory (call before a stream capture)
int mlp_grad_tc(const MlpDev& M, const float* data, long long nrows, unsigned long long seed, long long step,
                const long long* step_dev, long long loss_from, int batch, float* grad, float* loss_sum, int* err,
                cudaStream_t s);
int mlp_adam_sched(float* p, float* grad, float* m, float* v, double lr0, long long total, long long* step_dev,
                   __nv_bfloat16* W2h, cudaStream_t s);
int mlp_refresh(const float* p, __nv_bfloat16* W2h, cudaStream_t s);
int mlp_forward_tc(long long n, const float* xs, const float* p, const __nv_bfloat16* W2h, float* y, int* err,
                   int sms, cudaStream_t s);
// Wst != nullptr (mixed path): the kernels also store W of the updated cells there and the
// CFL limit into the patch's slot, which the caller resets; the caller then fills W's ghost
// shell.
int issue_surrogate_tc(const PatchDev& P, const ThermalDev& th, const MlpDev& M, int* fb_list,
                       unsigned long long* fb_count, float* Wst, int sms, cudaStream_t s, long long* launches);
int issue_surrogate(const PatchDev& P, const ThermalDev& th, const MlpDev& M, int* fb_list,
                    unsigned long long* fb_count, float* Wst, int sms, cudaStream_t s, long long* launches);
}  // namespace mhd
