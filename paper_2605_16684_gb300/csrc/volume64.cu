// volume64.cu -- FP64 instantiations of the flux-differencing volume kernel:
// single-mesh launches and the persistent batched kernel (two tile shapes).
#include "volume_impl.cuh"

int esdg_volume_f64_take_timeout() {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, esdg_vol::g_esdg_vol_timeout, sizeof(int)) != cudaSuccess) return -1;
  if (v) {
    const int z = 0;
    if (cudaMemcpyToSymbol(esdg_vol::g_esdg_vol_timeout, &z, sizeof(int)) != cudaSuccess) return -1;
  }
  return v ? 1 : 0;
}

cudaError_t esdg_launch_volume_f64(const EsdgGrid& g, const EsdgLGL& L, const EsdgPhys& P, int mode,
                                   const EsdgVolArgs& a, cudaStream_t s) {
  return esdg_vol::launch_volume_t<false>(g, L, P, mode, a, s);
}

namespace {
// alternative tile shapes (elements per CTA) offered to the batch autotuner
template <int N> struct Alt64 { static constexpr int EPB = 0; };
template <> struct Alt64<1> { static constexpr int EPB = 4; };
template <> struct Alt64<2> { static constexpr int EPB = 8; };
template <> struct Alt64<3> { static constexpr int EPB = 4; };
template <> struct Alt64<4> { static constexpr int EPB = 3; };
}  // namespace

int esdg_volume_batch_variants_f64(int N) { return (N >= 1 && N <= 4) ? 2 : 1; }

#define ESDG_V64(NN)                                                                          \
  case NN:                                                                                    \
    if (variant == 1 && Alt64<NN>::EPB > 0) {                                                 \
      if (what == 0) return esdg_vol::launch_batch_one<NN, false, false, Alt64<NN>::EPB>(    \
                                members, tiles, ntiles, grid, L, A, B, s) == cudaSuccess ? 0 : -1; \
      if (what == 1) return esdg_vol::Shape<NN, false, false, Alt64<NN>::EPB>::EPB;           \
      return esdg_vol::batch_occupancy<NN, false, false, Alt64<NN>::EPB>();                   \
    }                                                                                         \
    if (what == 0) return esdg_vol::launch_batch_one<NN, false, false, 0>(                   \
                              members, tiles, ntiles, grid, L, A, B, s) == cudaSuccess ? 0 : -1; \
    if (what == 1) return esdg_vol::Shape<NN, false, false, 0>::EPB;                          \
    return esdg_vol::batch_occupancy<NN, false, false, 0>();

// what: 0 launch (returns 0 / -1), 1 elements per tile, 2 CTAs per SM
int esdg_volume_batch_f64(int what, int N, int variant, const EsdgMember* members, const int2* tiles,
                          const int* ntiles, int grid, const EsdgLGL& L, double A, double B,
                          cudaStream_t s) {
  switch (N) {
    ESDG_V64(1) ESDG_V64(2) ESDG_V64(3) ESDG_V64(4) ESDG_V64(5) ESDG_V64(6) ESDG_V64(7)
    default: return -1;
  }
}
#undef ESDG_V64
