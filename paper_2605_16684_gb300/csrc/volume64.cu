// volume64.cu -- FP64 instantiations of the flux-differencing volume kernel:
// single-mesh launches and the batched variants (pipelined persistent kernel,
// per-tile kernel at two tile shapes).
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

namespace {
// Batched volume variants offered to the autotuner, in order: the pipelined
// persistent kernel (when its tile fits in shared memory), the per-tile kernel
// at the default tile shape, and at the alternative shape (when there is one).
template <int NN>
int batch_variant(int what, int variant, const EsdgMember* members, const int2* tiles,
                  const int* ntiles, int grid, const EsdgLGL& L, double A, double B, cudaStream_t s) {
  constexpr bool pipe_ok = esdg_vol::Pipe64<NN, 1>::SMEM <= ESDG_PIPE_SMEM_MAX;
  constexpr bool alt_ok = Alt64<NN>::EPB > 0;
  int kinds[3], nk = 0;
  if (pipe_ok) kinds[nk++] = 0;
  kinds[nk++] = 1;
  if (alt_ok) kinds[nk++] = 2;
  if (what == 3) return nk;
  if (variant < 0 || variant >= nk) return -1;
  switch (kinds[variant]) {
    case 0:
      if constexpr (pipe_ok) return esdg_vol::pipe_batch<NN, false>(what, members, tiles, ntiles, grid, L, A, B, s);
      return -1;
    case 1:
      if (what == 0) return esdg_vol::launch_batch_one<NN, false, false, 0>(members, tiles, ntiles, grid, L, A, B, s) == cudaSuccess ? 0 : -1;
      if (what == 1) return esdg_vol::Shape<NN, false, false, 0>::EPB;
      return esdg_vol::batch_occupancy<NN, false, false, 0>();
    default:
      if constexpr (alt_ok) {
        if (what == 0) return esdg_vol::launch_batch_one<NN, false, false, Alt64<NN>::EPB>(members, tiles, ntiles, grid, L, A, B, s) == cudaSuccess ? 0 : -1;
        if (what == 1) return esdg_vol::Shape<NN, false, false, Alt64<NN>::EPB>::EPB;
        return esdg_vol::batch_occupancy<NN, false, false, Alt64<NN>::EPB>();
      }
      return -1;
  }
}

int batch_dispatch(int what, int N, int variant, const EsdgMember* members, const int2* tiles,
                   const int* ntiles, int grid, const EsdgLGL& L, double A, double B, cudaStream_t s) {
  switch (N) {
    case 1: return batch_variant<1>(what, variant, members, tiles, ntiles, grid, L, A, B, s);
    case 2: return batch_variant<2>(what, variant, members, tiles, ntiles, grid, L, A, B, s);
    case 3: return batch_variant<3>(what, variant, members, tiles, ntiles, grid, L, A, B, s);
    case 4: return batch_variant<4>(what, variant, members, tiles, ntiles, grid, L, A, B, s);
    case 5: return batch_variant<5>(what, variant, members, tiles, ntiles, grid, L, A, B, s);
    case 6: return batch_variant<6>(what, variant, members, tiles, ntiles, grid, L, A, B, s);
    case 7: return batch_variant<7>(what, variant, members, tiles, ntiles, grid, L, A, B, s);
    default: return -1;
  }
}
}  // namespace

int esdg_volume_batch_variants_f64(int N) {
  const int n = batch_dispatch(3, N, 0, nullptr, nullptr, nullptr, 0, EsdgLGL{}, 0, 0, 0);
  return n > 0 ? n : 1;
}

// what: 0 launch (returns 0 / -1), 1 elements per tile, 2 CTAs per SM
int esdg_volume_batch_f64(int what, int N, int variant, const EsdgMember* members,
                          const int2* tiles, const int* ntiles, int grid, const EsdgLGL& L,
                          double A, double B, cudaStream_t s) {
  return batch_dispatch(what, N, variant, members, tiles, ntiles, grid, L, A, B, s);
}
