// batched_inst.cu -- instantiates the persistent multi-system V-cycle kernel for one x-line chunk
// size K = SMG_K (1..4, i.e. nx <= 128), FP32 storage (FP32 cycle, FP64 coarsest plane).
// The persistent kernel holds the FP32 and the FP64 plane cycles in one body; the FP64 factors
// (K > 2) go out of line so that their registers do not weigh on the whole kernel.
#define SMG_FAC_REG_BYTES 16
#include "batched.cuh"

#ifndef SMG_K
#error "compile with -DSMG_K=<rows per lane>"
#endif

namespace smg {

#define SMG_CAT2(a, b) a##b
#define SMG_CAT(a, b) SMG_CAT2(a, b)

template <class S>
static cudaError_t launch_one(int blocks, int threads, size_t smem, const PersistArgs &p, cudaStream_t st,
                              bool cooperative) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = cooperative ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, persistent_vcycle_kernel<S, SMG_K>, p);
}

cudaError_t SMG_CAT(launch_persistent_vcycle_k, SMG_K)(Prec storage, int blocks, int threads, size_t smem,
                                                       const PersistArgs &p, cudaStream_t st, bool cooperative) {
    switch (storage) {
    case Prec::F64: return cudaErrorInvalidValue;
    case Prec::F32: return launch_one<float>(blocks, threads, smem, p, st, cooperative);
    case Prec::BF16: return cudaErrorInvalidValue;
    }
    return cudaErrorInvalidValue;
}

int SMG_CAT(set_persistent_smem_k, SMG_K)(Prec storage, size_t smem) {
    cudaError_t e = cudaErrorInvalidValue;
    switch (storage) {
    case Prec::F32:
        e = raise_smem_attr(reinterpret_cast<const void *>(&persistent_vcycle_kernel<float, SMG_K>), smem);
        break;
    default: break;
    }
    return static_cast<int>(e);
}

int SMG_CAT(persistent_blocks_per_sm_k, SMG_K)(Prec storage, int threads, size_t smem) {
    int n = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (storage) {
    case Prec::F32:
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, persistent_vcycle_kernel<float, SMG_K>, threads, smem);
        break;
    default: break;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

}  // namespace smg
