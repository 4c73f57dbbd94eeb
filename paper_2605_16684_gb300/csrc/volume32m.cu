// volume32m.cu -- the mixed-precision volume kernel relative to a moving
// background (a flow carried by the background, e.g. the channel's balanced
// jet): FP32 pairs formed as differences against the background's fluxes
// (pair32bgm), per-tile kernel for every order.
#include "volume_tile.cuh"

cudaError_t esdg_launch_volume_mixed_moving(const EsdgGrid& g, const EsdgLGL& L, const EsdgPhys& P,
                                            int mode, const EsdgVolArgs& a, cudaStream_t s) {
  using namespace esdg_vol;
#define ESDG_MV(NN)                                                                   \
  case NN:                                                                            \
    return mode ? launch_one<NN, true, 1, 2>(g, P, L, a, s) : launch_one<NN, true, 0, 2>(g, P, L, a, s);
  switch (g.N) {
    ESDG_MV(1)
    ESDG_MV(2)
    ESDG_MV(3)
    ESDG_MV(4)
    ESDG_MV(5)
    ESDG_MV(6)
    ESDG_MV(7)
    default:
      return cudaErrorInvalidValue;
  }
#undef ESDG_MV
}
