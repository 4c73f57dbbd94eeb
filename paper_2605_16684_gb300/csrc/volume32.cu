// volume32.cu -- mixed-precision instantiations (FP32 pairs, FP64 state and
// pressure recovery) of the flux-differencing volume kernel: single-mesh
// launches and the persistent batched kernel with a background (two tile shapes).
#include "volume_impl.cuh"

int esdg_volume_mixed_take_timeout() {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, esdg_vol::g_esdg_vol_timeout, sizeof(int)) != cudaSuccess) return -1;
  if (v) {
    const int z = 0;
    if (cudaMemcpyToSymbol(esdg_vol::g_esdg_vol_timeout, &z, sizeof(int)) != cudaSuccess) return -1;
  }
  return v ? 1 : 0;
}

cudaError_t esdg_launch_volume_mixed(const EsdgGrid& g, const EsdgLGL& L, const EsdgPhys& P,
                                     int mode, const EsdgVolArgs& a, cudaStream_t s) {
  return esdg_vol::launch_volume_t<true>(g, L, P, mode, a, s);
}

namespace {
template <int N> struct Alt32 { static constexpr int EPB = 0; };
template <> struct Alt32<1> { static constexpr int EPB = 8; };
template <> struct Alt32<2> { static constexpr int EPB = 8; };
template <> struct Alt32<3> { static constexpr int EPB = 4; };
template <> struct Alt32<4> { static constexpr int EPB = 3; };
template <> struct Alt32<5> { static constexpr int EPB = 2; };
template <> struct Alt32<6> { static constexpr int EPB = 1; };
template <> struct Alt32<7> { static constexpr int EPB = 1; };
}  // namespace

int esdg_volume_batch_variants_mixed(int N) { return (N >= 1 && N <= 7) ? 2 : 1; }

#define ESDG_V32(NN)                                                                          \
  case NN:                                                                                    \
    if (variant == 1 && Alt32<NN>::EPB > 0) {                                                 \
      if (what == 0) return esdg_vol::launch_batch_one<NN, true, true, Alt32<NN>::EPB>(      \
                                members, tiles, ntiles, grid, L, A, B, s) == cudaSuccess ? 0 : -1; \
      if (what == 1) return esdg_vol::Shape<NN, true, true, Alt32<NN>::EPB>::EPB;             \
      return esdg_vol::batch_occupancy<NN, true, true, Alt32<NN>::EPB>();                     \
    }                                                                                         \
    if (what == 0) return esdg_vol::launch_batch_one<NN, true, true, 0>(                     \
                              members, tiles, ntiles, grid, L, A, B, s) == cudaSuccess ? 0 : -1; \
    if (what == 1) return esdg_vol::Shape<NN, true, true, 0>::EPB;                            \
    return esdg_vol::batch_occupancy<NN, true, true, 0>();

// mixed members of a batch always carry a background (set by their initial state)
int esdg_volume_batch_mixed(int what, int N, int variant, const EsdgMember* members,
                            const int2* tiles, const int* ntiles, int grid, const EsdgLGL& L,
                            double A, double B, cudaStream_t s) {
  switch (N) {
    ESDG_V32(1) ESDG_V32(2) ESDG_V32(3) ESDG_V32(4) ESDG_V32(5) ESDG_V32(6) ESDG_V32(7)
    default: return -1;
  }
}
#undef ESDG_V32
