// plane_relax_inst.cu -- instantiates the plane-relaxation kernel for one x-line chunk size
// K = SMG_K (rows per lane; nx <= 32 K).  The build compiles this unit once per K so the
// instantiations compile in parallel.
#include "plane_relax.cuh"

#ifndef SMG_K
#error "compile with -DSMG_K=<rows per lane>"
#endif

namespace smg {

#define SMG_CAT2(a, b) a##b
#define SMG_CAT(a, b) SMG_CAT2(a, b)

cudaError_t SMG_CAT(launch_plane_relax_k, SMG_K)(Prec storage, bool f64, int nplanes, int nb, int threads,
                                                 const PlaneRelaxArgs &a, size_t smem, cudaStream_t st) {
    switch (storage) {
    case Prec::F64: return launch_pr<double, double, SMG_K>(nplanes, nb, threads, a, smem, st);
    case Prec::F32:
        return f64 ? launch_pr<float, double, SMG_K>(nplanes, nb, threads, a, smem, st)
                   : launch_pr<float, float, SMG_K>(nplanes, nb, threads, a, smem, st);
    case Prec::BF16:
        return f64 ? launch_pr<__nv_bfloat16, double, SMG_K>(nplanes, nb, threads, a, smem, st)
                   : launch_pr<__nv_bfloat16, float, SMG_K>(nplanes, nb, threads, a, smem, st);
    }
    return cudaErrorInvalidValue;
}

int SMG_CAT(set_plane_relax_smem_k, SMG_K)(Prec storage, bool f64, size_t smem) {
    switch (storage) {
    case Prec::F64: return set_smem_attr<double, double, SMG_K>(smem);
    case Prec::F32: return f64 ? set_smem_attr<float, double, SMG_K>(smem) : set_smem_attr<float, float, SMG_K>(smem);
    case Prec::BF16:
        return f64 ? set_smem_attr<__nv_bfloat16, double, SMG_K>(smem) : set_smem_attr<__nv_bfloat16, float, SMG_K>(smem);
    }
    return static_cast<int>(cudaErrorInvalidValue);
}

}  // namespace smg
