// noalloc.cu -- smg_apply_A_dot_static: out = A u and (u, A u) with no device allocation.
//
// Some callers cannot allocate device memory at the point where they need this product: a
// host framework that owns every device allocation and hands the library only its input and
// output buffers, or a timing-critical section where cudaMalloc / cudaFree are not acceptable
// because they can synchronise the device.  smg_setup allocates (the hierarchy and the work
// vectors), so such callers cannot use a handle.  This entry point needs none: the block
// partial sums of the inner product live in a file-scope device array that every GPU which
// loads the library holds until the process exits.
//
// It is a variant of the Krylov SpMV kernel (q = A p with the fused inner product (p, q)); the
// 7-point operator is the model problem of the paper, which has no counterpart of this
// allocation-free form.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/smg.h"
#include "smg_internal.h"

namespace {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocChunk = 8192;     // points per CTA
constexpr int kNoAllocBlocks = 4096;    // CTAs at most, hence points at most:
constexpr long long kNoAllocMaxPoints = static_cast<long long>(kNoAllocChunk) * kNoAllocBlocks;  // 33,554,432
constexpr int kMaxDevices = 64;

// The shared scratch: one partial sum per CTA and the finished-CTA counter.  In host code these
// names are host-side stand-ins, not device addresses; their device addresses come from
// cudaGetSymbolAddress, per device.
static __device__ __align__(256) double g_noalloc_partials[kNoAllocBlocks];
static __device__ __align__(256) unsigned int g_noalloc_counter;

struct DevScratch {
    bool ready = false;
    double *partials = nullptr;
    unsigned int *counter = nullptr;
};
DevScratch g_scratch[kMaxDevices];
std::mutex g_scratch_mutex;

__global__ void __launch_bounds__(kNoAllocThreads) apply_A_dot_static_kernel(int nx, int ny, int nz,
                                                                            const double *__restrict__ u,
                                                                            double *__restrict__ out,
                                                                            double *__restrict__ dot,
                                                                            double *partials, unsigned int *counter) {
    const int npi = nx * ny, n = npi * nz;
    const long long np = npi;
    const int i0 = blockIdx.x * kNoAllocChunk;
    const int i1 = min(n, i0 + kNoAllocChunk);
    double acc = 0.0;
    for (int i = i0 + threadIdx.x; i < i1; i += kNoAllocThreads) {
        const int z = i / npi, ip = i - z * npi, y = ip / nx, x = ip - y * nx;
        double nb = 0.0;
        if (x > 0) nb += u[i - 1];
        if (x < nx - 1) nb += u[i + 1];
        if (y > 0) nb += u[i - nx];
        if (y < ny - 1) nb += u[i + nx];
        if (z > 0) nb += u[i - np];
        if (z < nz - 1) nb += u[i + np];
        const double q = 6.0 * u[i] - nb;
        out[i] = q;
        acc = fma(u[i], q, acc);
    }
    // block sum (pairwise), then the last CTA adds the partials in CTA order
    __shared__ double sh[kNoAllocThreads / 32];
    __shared__ bool last;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < kNoAllocThreads / 32; ++w) b += sh[w];
        partials[blockIdx.x] = b;
        __threadfence();
        last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (last && threadIdx.x < 32) {
        // the last CTA's first warp: each lane sums every 32nd partial with TwoSum (error-free
        // addition, errors carried in c), then the lanes' (s, c) pairs are combined the same way
        __threadfence();
        const int lane = threadIdx.x;
        double s = 0.0, c = 0.0;
        for (unsigned b = lane; b < gridDim.x; b += 32) {
            const double v = *reinterpret_cast<volatile double *>(&partials[b]);
            const double t = s + v;
            const double bp = t - s;
            c += (s - (t - bp)) + (v - bp);
            s = t;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double vs = __shfl_down_sync(0xffffffffu, s, o), vc = __shfl_down_sync(0xffffffffu, c, o);
            const double t = s + vs;
            const double bp = t - s;
            c += ((s - (t - bp)) + (vs - bp)) + vc;
            s = t;
        }
        if (lane == 0) *dot = s + c;
    }
}

// Device addresses of the scratch on the current device, looked up once per device.
int scratch_for_current_device(DevScratch &out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        smg::set_last_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return SMG_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        smg::set_last_error("device ordinal beyond the 64 this entry point supports");
        return SMG_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    DevScratch &s = g_scratch[dev];
    if (!s.ready) {
        void *p = nullptr, *q = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e == cudaSuccess) e = cudaGetSymbolAddress(&q, g_noalloc_counter);
        if (e != cudaSuccess) {
            smg::set_last_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return SMG_ERR_CUDA;
        }
        s.partials = static_cast<double *>(p);
        s.counter = static_cast<unsigned int *>(q);
        s.ready = true;
    }
    out = s;
    return SMG_OK;
}

}  // namespace

extern "C" int smg_apply_A_dot_static(int nx, int ny, int nz, const double *u, double *out, double *dot,
                                      void *stream) {
    if (nx < 1 || ny < 1 || nz < 1) {
        smg::set_last_error("grid sizes must be >= 1");
        return SMG_ERR_ARG;
    }
    if (static_cast<long long>(nx) * ny * nz > kNoAllocMaxPoints) {
        smg::set_last_error("nx*ny*nz exceeds the 33,554,432 points the static scratch covers");
        return SMG_ERR_ARG;
    }
    if (u == nullptr || out == nullptr || dot == nullptr) {
        smg::set_last_error("null pointer");
        return SMG_ERR_ARG;
    }
    DevScratch s;
    int rc = scratch_for_current_device(s);
    if (rc != SMG_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the counter must start at zero: the scratch keeps whatever the previous call left
    cudaError_t e = cudaMemsetAsync(s.counter, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) {
        smg::set_last_error(std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
        return SMG_ERR_CUDA;
    }
    const int n = nx * ny * nz;
    const int blocks = (n + kNoAllocChunk - 1) / kNoAllocChunk;
    apply_A_dot_static_kernel<<<blocks, kNoAllocThreads, 0, st>>>(nx, ny, nz, u, out, dot, s.partials, s.counter);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        smg::set_last_error(std::string("kernel launch: ") + cudaGetErrorString(e));
        return SMG_ERR_CUDA;
    }
    return SMG_OK;
}
