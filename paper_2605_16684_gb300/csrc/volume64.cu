// volume64.cu -- FP64 instantiations of the flux-differencing volume kernel.
#include "volume_impl.cuh"

cudaError_t esdg_launch_volume_f64(const EsdgGrid& g, const EsdgLGL& L, const EsdgPhys& P, int mode,
                                   const EsdgVolArgs& a, cudaStream_t s) {
  return esdg_vol::launch_volume_t<false>(g, L, P, mode, a, s);
}
