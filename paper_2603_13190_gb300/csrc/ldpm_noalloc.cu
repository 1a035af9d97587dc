// ldpm_noalloc.cu -- kinetic energy of caller-provided device arrays with no allocation at all.
//
// This is the energy reduction of ldpm_energy (per-block partial sums, then one block adding the
// partials in a fixed order) restricted to W_kin = sum 1/2 m v^2, with its scratch (the per-block
// partials) in a file-scope device array instead of memory allocated by a handle.  It exists for
// callers that may not allocate device memory; see ldpm_kinetic_energy_noalloc in include/ldpm.h.
#include <cstdint>
#include <cstdio>
#include <mutex>

#include <cuda_runtime.h>

#include "../../include/ldpm.h"
#include "ldpm_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 4;
constexpr int kMaxBlocks = 4096;
constexpr int64_t kMaxDof = (int64_t)kMaxBlocks * kThreads * kPerThread;  // 4,194,304 DOFs
constexpr int kMaxDevices = 64;

// Per-block partial sums (32 KiB on every device that loads the library, held until exit).
static __device__ __align__(256) double g_ke_scratch[kMaxBlocks];

std::mutex g_mu;
double *g_scratch_addr[kMaxDevices] = {};

__global__ void __launch_bounds__(kThreads) ke_partial_kernel(const double *__restrict__ v,
                                                              const double *__restrict__ mass, int64_t n,
                                                              double *__restrict__ partial)
{
    __shared__ double red[kThreads];
    const int tid = threadIdx.x;
    const int64_t base = (int64_t)blockIdx.x * kThreads * kPerThread + tid;
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
        const int64_t i = base + (int64_t)k * kThreads;
        if (i < n) acc += 0.5 * mass[i] * v[i] * v[i];
    }
    red[tid] = acc;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (tid < w) red[tid] += red[tid + w];
        __syncthreads();
    }
    if (tid == 0) partial[blockIdx.x] = red[0];
}

__global__ void __launch_bounds__(kThreads) ke_final_kernel(const double *__restrict__ partial, int nb,
                                                            double *__restrict__ out)
{
    __shared__ double red[kThreads];
    const int tid = threadIdx.x;
    double acc = 0.0;
    for (int b = tid; b < nb; b += kThreads) acc += partial[b];
    red[tid] = acc;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (tid < w) red[tid] += red[tid + w];
        __syncthreads();
    }
    if (tid == 0) out[0] = red[0];
}

int reject(int code, const char *msg, const char *detail)
{
    char buf[256];
    snprintf(buf, sizeof buf, "ldpm_kinetic_energy_noalloc: %s%s", msg, detail ? detail : "");
    ldpm::set_last_error(buf);
    return code;
}

}  // namespace

extern "C" int ldpm_kinetic_energy_noalloc(const double *v, const double *mass, int64_t n_dof, double *out,
                                           void *stream)
{
    ldpm::set_last_error("");
    if (!v || !mass || !out || n_dof < 0) return reject(LDPM_E_INVALID_ARG, "NULL pointer or negative n_dof", nullptr);
    if (n_dof > kMaxDof) {
        char d[96];
        snprintf(d, sizeof d, "%lld > %lld", (long long)n_dof, (long long)kMaxDof);
        return reject(LDPM_E_INVALID_ARG, "n_dof exceeds the static scratch limit: ", d);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return reject(LDPM_E_CUDA, "cudaGetDevice: ", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return reject(LDPM_E_INVALID_ARG, "device ordinal out of range", nullptr);
    double *scratch = nullptr;
    {
        // Set-up, once per device, with that device current: the device address of the array.
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_scratch_addr[dev]) {
            e = cudaGetSymbolAddress((void **)&g_scratch_addr[dev], g_ke_scratch);
            if (e != cudaSuccess) {
                g_scratch_addr[dev] = nullptr;
                return reject(LDPM_E_CUDA, "cudaGetSymbolAddress: ", cudaGetErrorString(e));
            }
        }
        scratch = g_scratch_addr[dev];
    }
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nb = (int)((n_dof + kThreads * kPerThread - 1) / (kThreads * kPerThread));
    if (nb > 0) ke_partial_kernel<<<nb, kThreads, 0, s>>>(v, mass, n_dof, scratch);
    ke_final_kernel<<<1, kThreads, 0, s>>>(scratch, nb, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return reject(LDPM_E_CUDA, "launch: ", cudaGetErrorString(e));
    return LDPM_OK;
}
