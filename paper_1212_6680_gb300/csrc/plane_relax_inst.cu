// plane_relax_inst.cu -- instantiates the plane-relaxation kernel for one x-line chunk size
// K = SMG_K (rows per lane; nx <= 32 K) and one storage precision SMG_PREC (0 FP64, 1 FP32,
// 2 BF16).  The build compiles this unit once per (K, precision) so the instantiations
// compile in parallel.
#include "plane_lean.cuh"
#include "plane_relax.cuh"

#if !defined(SMG_K) || !defined(SMG_PREC)
#error "compile with -DSMG_K=<rows per lane> -DSMG_PREC=<0|1|2>"
#endif

namespace smg {

#define SMG_CAT4(a, b, c, d) a##b##c##d
#define SMG_NAME(base, k, p) SMG_CAT4(base, k, _p, p)

#if SMG_PREC == 0
using StorageT = double;
#elif SMG_PREC == 1
using StorageT = float;
#else
using StorageT = __nv_bfloat16;
#endif

// a.R > 1: one thread-block cluster of a.R CTAs per plane.
cudaError_t SMG_NAME(launch_plane_relax_k, SMG_K, SMG_PREC)(bool f64, int nplanes, int nb, int threads,
                                                            const PlaneRelaxArgs &a, size_t smem, cudaStream_t st) {
    const bool cl = a.R > 1;
    if (f64 || SMG_PREC == 0)
        return cl ? launch_pr<StorageT, double, SMG_K, true>(nplanes, nb, threads, a, smem, st)
                  : launch_pr<StorageT, double, SMG_K, false>(nplanes, nb, threads, a, smem, st);
#if SMG_PREC != 0
    return cl ? launch_pr<StorageT, float, SMG_K, true>(nplanes, nb, threads, a, smem, st)
              : launch_pr<StorageT, float, SMG_K, false>(nplanes, nb, threads, a, smem, st);
#else
    return cudaErrorInvalidValue;
#endif
}

int SMG_NAME(set_plane_relax_smem_k, SMG_K, SMG_PREC)(bool f64, bool cl, size_t smem) {
    if (f64 || SMG_PREC == 0)
        return cl ? set_smem_attr<StorageT, double, SMG_K, true>(smem) : set_smem_attr<StorageT, double, SMG_K, false>(smem);
#if SMG_PREC != 0
    return cl ? set_smem_attr<StorageT, float, SMG_K, true>(smem) : set_smem_attr<StorageT, float, SMG_K, false>(smem);
#else
    return static_cast<int>(cudaErrorInvalidValue);
#endif
}

bool SMG_NAME(cluster_resident_k, SMG_K, SMG_PREC)(bool f64, int R, int threads, size_t smem) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(R, 1, 1);
    cfg.blockDim = dim3(threads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = R;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    cudaError_t e;
#if SMG_PREC != 0
    if (!f64)
        e = cudaOccupancyMaxActiveClusters(&n, plane_relax_kernel<StorageT, float, SMG_K, true>, &cfg);
    else
#endif
        e = cudaOccupancyMaxActiveClusters(&n, plane_relax_kernel<StorageT, double, SMG_K, true>, &cfg);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return n > 0;
}

#if SMG_K <= 8
// The shortened-step plane cycle (plane_lean.cuh): FP32 or FP64 compute, on one CTA or a cluster
// (a.R > 1) per plane.
cudaError_t SMG_NAME(launch_plane_lean_k, SMG_K, SMG_PREC)(bool f64, int nplanes, int nb, int threads,
                                                           const PlaneRelaxArgs &a, size_t smem, cudaStream_t st) {
    const bool cl = a.R > 1;
    if (f64 || SMG_PREC == 0)
        return cl ? launch_lean<StorageT, double, SMG_K, true>(nplanes, nb, threads, a, smem, st)
                  : launch_lean<StorageT, double, SMG_K, false>(nplanes, nb, threads, a, smem, st);
#if SMG_PREC != 0
    return cl ? launch_lean<StorageT, float, SMG_K, true>(nplanes, nb, threads, a, smem, st)
              : launch_lean<StorageT, float, SMG_K, false>(nplanes, nb, threads, a, smem, st);
#else
    return cudaErrorInvalidValue;
#endif
}
int SMG_NAME(set_plane_lean_smem_k, SMG_K, SMG_PREC)(bool f64, bool cl, size_t smem) {
    if (f64 || SMG_PREC == 0)
        return cl ? set_lean_smem_attr<StorageT, double, SMG_K, true>(smem)
                  : set_lean_smem_attr<StorageT, double, SMG_K, false>(smem);
#if SMG_PREC != 0
    return cl ? set_lean_smem_attr<StorageT, float, SMG_K, true>(smem)
              : set_lean_smem_attr<StorageT, float, SMG_K, false>(smem);
#else
    return static_cast<int>(cudaErrorInvalidValue);
#endif
}
bool SMG_NAME(lean_cluster_resident_k, SMG_K, SMG_PREC)(bool f64, int R, int threads, size_t smem) {
#if SMG_PREC != 0
    if (!f64) return lean_cluster_resident<StorageT, float, SMG_K>(R, threads, smem);
#endif
    return lean_cluster_resident<StorageT, double, SMG_K>(R, threads, smem);
}
#endif

}  // namespace smg
