// bs_step.cu -- the position updates of a Heun (RK2) step of the Lagrangian
// vortex method (the nodes move with the velocity, Section 1):
//   x* = x0 + dt v(x0);   x1 = x0 + dt/2 (v(x0) + v(x*)).
#include "bs_internal.cuh"

namespace bs {
namespace {

__global__ void euler_kernel(const double *__restrict__ x0, const double *__restrict__ v0, double dt, int64_t n,
                             double *__restrict__ x)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) x[i] = x0[i] + dt * v0[i];
}

__global__ void heun_kernel(const double *__restrict__ x0, const double *__restrict__ v0,
                            const double *__restrict__ v1, double dt, int64_t n, double *__restrict__ x)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) x[i] = x0[i] + 0.5 * dt * (v0[i] + v1[i]);
}

}  // namespace

cudaError_t launch_euler(const double *x0, const double *v0, double dt, int64_t n_values, double *x, cudaStream_t st)
{
    euler_kernel<<<(unsigned)((n_values + 255) / 256), 256, 0, st>>>(x0, v0, dt, n_values, x);
    return cudaGetLastError();
}

cudaError_t launch_heun(const double *x0, const double *v0, const double *v1, double dt, int64_t n_values, double *x,
                        cudaStream_t st)
{
    heun_kernel<<<(unsigned)((n_values + 255) / 256), 256, 0, st>>>(x0, v0, v1, dt, n_values, x);
    return cudaGetLastError();
}

}  // namespace bs
