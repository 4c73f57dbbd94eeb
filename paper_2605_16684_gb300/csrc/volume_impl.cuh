// volume_impl.cuh -- flux-differencing volume kernel (Section 3, the volume term
// of Eq. (nm:semi), with the optimisations of Section 4.1).
// The arithmetic lives in volume_pairs.cuh, the per-tile kernels in
// volume_tile.cuh, the pipelined persistent kernels in volume_pipe.cuh; this
// file dispatches the single-mesh launches.
//
//   rhs_i = -(1/J_i) [ sum_d sum_l Dt^{(d)}_{il} H^d(q_i, q_l) + face lifts ] + h_i
//
// H^d is the two-point entropy-conservative flux with the metric average
// n = {{Ja^d}}_{il} plus the non-symmetric gravity term 1/2 rho_hat [[phi]] n.
//
// Layout on the GPU (one CTA = EPB elements):
//   prologue   one thread per node: primitives once per node (u = rho u/rho, p,
//              b = rho/(2p), 1/b), staged in shared memory with 1/2 Ja;
//   pair pass  one thread per pencil (element, direction d, transverse node):
//              every unordered pair (i < l) of the pencil is evaluated once and
//              added to both nodes in registers -- node i gets Dt_il H(i,l),
//              node l gets Dt_li H(l,i), where H(l,i) shares the symmetric flux
//              and takes the gravity part -G(i,l) b_i/b_l (Section 4.1).  The
//              pencil's two end nodes also receive the interface fluxes of the
//              two faces the pencil pierces;
//   epilogue   one thread per node: sum the three directions, scale by -1/J,
//              add the Coriolis source, then write rhs or apply the LSRK stage.
//
// The pencil-per-thread pair pass evaluates exactly N_q (N_q - 1)/2 pairs per
// pencil for every N (no antipodal double counting at odd N, no load
// imbalance, no shuffles or atomics); the pencil's accumulators live in
// registers and are exchanged once through shared memory.
//
// FP64: log means use the artanh series when u = f^2 < 1e-4 and per-node
// logarithms otherwise (computed only for CTAs that need them).  Mixed: the
// prologue recovers the pressure in FP64 and stages FP32 node data; pairs,
// sums and face lifts run in FP32; the log branch uses log1pf of the ratio;
// the geopotential is carried relative to each element's first node.
#pragma once
#include "volume_pipe.cuh"
#include "volume_tile.cuh"
#include "volume_ws.cuh"

namespace esdg_vol {

template <bool MIXED>
cudaError_t launch_volume_t(const EsdgGrid& g, const EsdgLGL& L, const EsdgPhys& P, int mode,
                            const EsdgVolArgs& a, cudaStream_t s) {
#define ESDG_CASE(NN)                                                          \
  case NN:                                                                     \
    if constexpr (!MIXED) {                                                    \
      return mode ? launch_pipe64<NN, 1>(g, P, L, a, s)                        \
                  : launch_pipe64<NN, 0>(g, P, L, a, s);                       \
    }                                                                          \
    if constexpr (MIXED) {                                                     \
      if (a.bg && a.bgq) return esdg_launch_volume_mixed_moving(g, L, P, mode, a, s); \
      if (a.bg) {                                                              \
        if constexpr (WsCfg<NN>::ON && Ws32<NN, 1>::SMEM <= ESDG_PIPE_SMEM_MAX) \
          return mode ? launch_ws32<NN, 1>(g, P, L, a, s)                      \
                      : launch_ws32<NN, 0>(g, P, L, a, s);                     \
        if constexpr (Pipe32<NN, 1>::SMEM <= ESDG_PIPE_SMEM_MAX)               \
          return mode ? launch_pipe32<NN, 1>(g, P, L, a, s)                    \
                      : launch_pipe32<NN, 0>(g, P, L, a, s);                   \
        return mode ? launch_one<NN, MIXED, 1, true>(g, P, L, a, s)            \
                    : launch_one<NN, MIXED, 0, true>(g, P, L, a, s);           \
      }                                                                        \
      return mode ? launch_one<NN, MIXED, 1, false>(g, P, L, a, s)             \
                  : launch_one<NN, MIXED, 0, false>(g, P, L, a, s);            \
    }
  switch (g.N) {
    ESDG_CASE(1)
    ESDG_CASE(2)
    ESDG_CASE(3)
    ESDG_CASE(4)
    ESDG_CASE(5)
    ESDG_CASE(6)
    ESDG_CASE(7)
    default:
      return cudaErrorInvalidValue;
  }
#undef ESDG_CASE
}

}  // namespace esdg_vol
