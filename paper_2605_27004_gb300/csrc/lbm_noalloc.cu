// lbm_totals_noalloc: FP64 mass and momentum totals of a caller-owned population array, with
// no device allocation at all. It is a variant of the block-partial reduction behind
// lbm_totals for callers that cannot call cudaMalloc (or any allocating routine) at the point
// where they need the totals: code running under an external memory manager that owns every
// device byte, code inside a region where allocation would synchronise the device or break a
// strict memory budget, or plug-ins that only receive pointers to existing buffers.
//
// The per-block partial sums live in one file-scope __device__ array of fixed size, which every
// GPU that loads this library holds until the process exits. Host code never passes the
// array's name to a kernel (in host code that name is only a stand-in, not a device address);
// it looks the device address up once per device with cudaGetSymbolAddress.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/lbm.h"
#include "lbm_lattice.cuh"

namespace {

constexpr int kBlocks = 1216;  // 152 SMs x 8 resident blocks: the reduction grid never exceeds it
constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

// 1216 records x 4 doubles = 38,912 bytes per device.
static __device__ __align__(256) double g_noalloc_partials[kBlocks * 4];

std::mutex g_mu;
double* g_scratch[kMaxDevices] = {nullptr};

template <int Q, typename T>
__global__ void __launch_bounds__(kThreads) k_totals_noalloc(const T* __restrict__ f, long long N,
                                                             double* __restrict__ partials) {
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += stride) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const double fi = (double)f[(long long)i * N + n];
            const lbm::Vec3 c = lbm::vel<Q>(i);
            v[0] += fi;
            v[1] += c.x * fi;
            v[2] += c.y * fi;
            v[3] += c.z * fi;
        }
    }
    __shared__ double sh[kThreads / 32][4];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        double s = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) sh[warp][k] = s;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) s += sh[w][threadIdx.x];
        partials[blockIdx.x * 4 + threadIdx.x] = s;  // every launched block writes its record
    }
}

// One block adds the nb records in a fixed order.
__global__ void __launch_bounds__(kThreads) k_totals_noalloc_finish(const double* __restrict__ partials, int nb,
                                                                    double* __restrict__ out) {
    __shared__ double sh[kThreads];
    for (int k = 0; k < 4; ++k) {
        double s = 0.0;
        for (int b = threadIdx.x; b < nb; b += kThreads) s += partials[b * 4 + k];
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int o = kThreads / 2; o > 0; o >>= 1) {
            if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) out[k] = sh[0];
        __syncthreads();
    }
}

// Device address of the scratch array on the current device, looked up once per device. The
// cached address belongs to the device's primary context as it was at the first call: after a
// cudaDeviceReset (or anything else that destroys that context) the module is loaded anew and
// the cached address is stale, so this entry point must not be used across a reset.
int scratch_for_current_device(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        (void)cudaGetLastError();
        return LBM_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) {
            (void)cudaGetLastError();
            return LBM_ERR_CUDA;
        }
        g_scratch[dev] = static_cast<double*>(p);
    }
    *out = g_scratch[dev];
    return LBM_OK;
}

// Both launches go through cudaLaunchKernel, whose return value is the status of that launch
// alone: an earlier, unrelated error left in the runtime's last-error slot is neither reported
// as this call's failure nor cleared.
template <int Q, typename T>
int launch(const void* f, long long N, double* totals, cudaStream_t s, double* scratch) {
    long long nb = (N + kThreads - 1) / kThreads;
    if (nb > kBlocks) nb = kBlocks;
    if (nb < 1) nb = 1;
    const T* fp = static_cast<const T*>(f);
    void* a1[] = {(void*)&fp, (void*)&N, (void*)&scratch};
    if (cudaLaunchKernel((const void*)&k_totals_noalloc<Q, T>, dim3((unsigned)nb), dim3(kThreads), a1, 0, s) !=
        cudaSuccess)
        return LBM_ERR_CUDA;
    int nbi = (int)nb;
    void* a2[] = {(void*)&scratch, (void*)&nbi, (void*)&totals};
    if (cudaLaunchKernel((const void*)&k_totals_noalloc_finish, dim3(1), dim3(kThreads), a2, 0, s) != cudaSuccess)
        return LBM_ERR_CUDA;
    return LBM_OK;
}

}  // namespace

extern "C" int lbm_totals_noalloc(int lattice, int nx, int ny, int nz, int fp64, const void* f, double* totals,
                                  void* stream) {
    if (lattice != 9 && lattice != 19 && lattice != 27) return LBM_ERR_INVALID_ARG;
    if (nx < 1 || ny < 1 || nz < 1 || (lattice == 9 && nz != 1) || !f || !totals) return LBM_ERR_INVALID_ARG;
    // nx * ny < 2^62 cannot overflow; the product with nz is checked by division first
    const long long nxy = (long long)nx * ny;
    if (nxy > 2147483647LL / nz) return LBM_ERR_INVALID_ARG;  // beyond the supported 2^31 - 1 cells
    const long long N = nxy * nz;
    double* scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc != LBM_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    switch (lattice) {
        case 9: return fp64 ? launch<9, double>(f, N, totals, s, scratch) : launch<9, float>(f, N, totals, s, scratch);
        case 19:
            return fp64 ? launch<19, double>(f, N, totals, s, scratch) : launch<19, float>(f, N, totals, s, scratch);
        default:
            return fp64 ? launch<27, double>(f, N, totals, s, scratch) : launch<27, float>(f, N, totals, s, scratch);
    }
}
