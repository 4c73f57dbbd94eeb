// volume32.cu -- mixed-precision instantiations (FP32 pairs, FP64 state and
// pressure recovery) of the flux-differencing volume kernel.
#include "volume_impl.cuh"

cudaError_t esdg_launch_volume_mixed(const EsdgGrid& g, const EsdgLGL& L, const EsdgPhys& P,
                                     int mode, const EsdgVolArgs& a, cudaStream_t s) {
  return esdg_vol::launch_volume_t<true>(g, L, P, mode, a, s);
}
