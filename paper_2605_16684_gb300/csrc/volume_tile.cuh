// volume_tile.cuh -- the per-tile volume kernel: one CTA per tile of EPB
// elements (k_volume), its persistent batched form over a device work table
// (k_volume_batch), and their launchers.  Used for the mixed path without a
// background or with a moving one, for tiles whose pipelined form exceeds
// shared memory, and as the autotuner's alternative batch variants.
#pragma once
#include "volume_pairs.cuh"

namespace esdg_vol {

// One tile: elements e0 .. e0 + EPB - 1 of one mesh, processed by a CTA of
// SH::THREADS threads with SH::SMEM bytes of shared memory at smraw.
template <int N, bool MIXED, int MODE, int BG, int EPB_ = 0>
__device__ __forceinline__ void volume_tile(const EsdgGrid& g, const EsdgPhys& P, const EsdgLGL& L,
                                            const EsdgVolArgs& a, int e0, unsigned char* smraw) {
  using SH = Shape<N, MIXED, BG, EPB_>;
  using R = typename SH::R;
  constexpr int Nq = SH::Nq, NP = SH::NP, NPEN = SH::NPEN, EPB = SH::EPB, NF = SH::NF;
  constexpr int T = SH::THREADS;
  R* sm = reinterpret_cast<R*>(smraw);
  const int E = g.E;
  const R* vg = reinterpret_cast<const R*>(a.vgeo);
  const double gm1 = P.gamma - 1.0;
  const float gm1f = esdg_d2f(gm1);

  // ---- prologue: primitives once per node -------------------------------
  int need_logs = 0;
  for (int idx = threadIdx.x; idx < EPB * NP; idx += T) {
    const int el = idx / NP, n = idx - el * NP, e = e0 + el;
    R* S = sm + (size_t)el * NF * NP;
    if (e < E) {
      const double* qe = a.q_in + (size_t)e * 5 * NP;
      const double q0 = qe[n], q1 = qe[NP + n], q2 = qe[2 * NP + n], q3 = qe[3 * NP + n],
                   q4 = qe[4 * NP + n];
      const double phi = a.vgeo64[((size_t)e * ESDG_NVGEO + 10) * NP + n];
      if constexpr (MIXED) {
        const float phh = vg[((size_t)e * ESDG_NVGEO + 10) * NP + n];
        if constexpr (BG == 2) {
          const double* bq = a.bgq + (size_t)e * 5 * NP + n;
          const float* bpe = a.bgp + (size_t)e * 4 * NP + n;
          const float* bu = a.bgu + (size_t)e * 3 * NP + n;
          const Prim32m o = prims32bgm(q0, q1, q2, q3, q4, phi, phh, gm1f, bq[0], bq[NP],
                                       bq[2 * NP], bq[3 * NP], bq[4 * NP], bpe[0], bpe[NP],
                                       bpe[2 * NP], bpe[3 * NP], bu[0], bu[NP], bu[2 * NP]);
#pragma unroll
          for (int k = 0; k < 7; k++) {
            S[k * NP + n] = o.s[k];
            S[(SH::F_BG + k) * NP + n] = o.bgf[k];
          }
#pragma unroll
          for (int k = 0; k < 3; k++) S[(SH::F_BG + 7 + k) * NP + n] = o.up[k];
        } else if constexpr (BG) {
          const double* bge = a.bg + (size_t)e * 3 * NP;
          const float* bpe = a.bgp + (size_t)e * 4 * NP;
          const Prim32 o = prims32bg(q0, q1, q2, q3, q4, phi, phh, gm1f, bge[n], bge[NP + n],
                                     bpe[n], bpe[NP + n], bpe[2 * NP + n], bpe[3 * NP + n]);
#pragma unroll
          for (int k = 0; k < 7; k++) {
            S[k * NP + n] = o.s[k];
            S[(SH::F_BG + k) * NP + n] = o.bgf[k];
          }
        } else {
          prims32<NP>(q0, q1, q2, q3, q4, phi, phh, gm1, S, n);
        }
      } else {
        prims64<NP>(q0, q1, q2, q3, q4, phi, gm1, S, n);
      }
#pragma unroll
      for (int k = 0; k < 9; k++)
        S[(SH::F_NH + k) * NP + n] = vg[((size_t)e * ESDG_NVGEO + k) * NP + n];
    } else {  // padding element: any valid state, results are discarded
      S[0 * NP + n] = (R)0.25;
      S[1 * NP + n] = (R)0.5;
      S[2 * NP + n] = (R)1;
      for (int k = 3; k < NF; k++) S[k * NP + n] = (R)0;
    }
  }
  __syncthreads();
  if constexpr (!MIXED) {
    for (int idx = threadIdx.x; idx < EPB * NP; idx += T) {
      const int el = idx / NP, n = idx - el * NP;
      if (out_of_series64<NP>(sm + (size_t)el * NF * NP, n)) need_logs = 1;
    }
    need_logs = __syncthreads_or(need_logs);
    if (need_logs) {
      for (int idx = threadIdx.x; idx < EPB * NP; idx += T) {
        const int el = idx / NP, n = idx - el * NP;
        R* S = sm + (size_t)el * NF * NP;
        S[SH::F_LR * NP + n] = log(4.0 * S[n]);
        S[SH::F_LB * NP + n] = log(2.0 * S[NP + n]);
      }
      __syncthreads();
    }
  } else {
    for (int idx = threadIdx.x; idx < EPB * NP; idx += T) {
      const int el = idx / NP, n = idx - el * NP;
      const R* S = sm + (size_t)el * NF * NP;
      const float r0 = S[0], rn = S[n], b0 = S[NP], bn = S[NP + n];
      // |f| < 0.14 keeps u < ESDG_LOG_EPS32 for every pair
      if (fabsf(rn - r0) > 0.13f * r0 || fabsf(bn - b0) > 0.13f * b0) need_logs = 1;
    }
    need_logs = __syncthreads_or(need_logs);
  }

  // ---- pair pass: one pencil per thread ---------------------------------
  const int tid = threadIdx.x;
  const bool active = tid < SH::PENCILS;
  const int el = active ? tid / (3 * NPEN) : 0;
  const int rr = tid - el * 3 * NPEN;
  const int d = active ? rr / NPEN : 0;
  const int pen = rr - d * NPEN;
  const int s = pen % Nq, t = pen / Nq;
  const int stride = (d == 0) ? 1 : ((d == 1) ? Nq : Nq * Nq);
  const int base = (d == 0) ? Nq * (s + Nq * t) : ((d == 1) ? (s + Nq * Nq * t) : (s + Nq * t));
  const int e = e0 + el;
  R acc[Nq][5];
#pragma unroll
  for (int i = 0; i < Nq; i++)
#pragma unroll
    for (int v = 0; v < 5; v++) acc[i][v] = (R)0;
  if constexpr (!MIXED)
    if (active && e < E) face_lift<true, N, R>(g, a, e, d, s + Nq * t, acc);
  if (active && e < E) {
    // mixed: the face terms and the element's reference geopotential are
    // fetched ahead of the pair pass and applied after it
    FaceTerms<R> ft{};
    R phi0 = (R)0;
    if constexpr (MIXED) {
      ft = face_fetch<N, R>(g, a, e, d, s + Nq * t);
      phi0 = esdg_d2f(a.vgeo64[((size_t)e * ESDG_NVGEO + 10) * NP]);
    }
    const R* S = sm + (size_t)el * NF * NP;
    const auto ce = [&] {
      if constexpr (MIXED) return esdg_d2f(0.5 * P.igm1);
      else return ce_series(0.5 * P.igm1);
    }();
    if (need_logs)
      pencil_pass<N, MIXED, true, BG>(S, d, base, stride, L, ce, acc);
    else
      pencil_pass<N, MIXED, false, BG>(S, d, base, stride, L, ce, acc);
    if constexpr (MIXED) {
      // restore the element's reference geopotential in the energy flux
#pragma unroll
      for (int i = 0; i < Nq; i++) acc[i][4] = fmaf(phi0, acc[i][0], acc[i][4]);
      face_add<N, R>(ft, acc);
    }
  }
  __syncthreads();
  if (active && e < E) {
    R* S = sm + (size_t)el * NF * NP;
#pragma unroll
    for (int i = 0; i < Nq; i++)
#pragma unroll
      for (int v = 0; v < 5; v++) S[(d * 5 + v) * NP + base + i * stride] = acc[i][v];
  }
  __syncthreads();

  // ---- epilogue: one thread per node -------------------------------------
  const bool rotating = (P.f0 != 0.0) || (P.beta != 0.0);
  bool bad = false;
  for (int idx = threadIdx.x; idx < EPB * NP; idx += T) {
    const int el2 = idx / NP, n = idx - el2 * NP, e2 = e0 + el2;
    if (e2 >= E) continue;
    const R* S = sm + (size_t)el2 * NF * NP;
    if constexpr (MIXED && MODE != 0) {
      const float iJf = vg[((size_t)e2 * ESDG_NVGEO + 9) * NP + n];
      float r32[5];
#pragma unroll
      for (int v = 0; v < 5; v++)
        r32[v] = -iJf * (S[v * NP + n] + S[(5 + v) * NP + n] + S[(10 + v) * NP + n]);
      const size_t qb = (size_t)e2 * 5 * NP + n;
      const double y = rotating ? a.x[((size_t)e2 * 3 + 1) * NP + n] : 0.0;
      float* dq = reinterpret_cast<float*>(a.dq);
      const float* rbg = BG == 2 ? a.rhs_bgm + qb : (BG ? a.rhs_bg + (size_t)e2 * 3 * NP + n : nullptr);
      bad |= stage32<NP, BG>(r32, rbg, P, y, a.q_in + qb, dq + qb, dq + qb, a.q_io + qb, a.rkA,
                             a.rkB, a.dt, BG == 2 ? a.bgq + qb : nullptr);
      continue;
    }
    // FP64 stage update: dt is folded into the -1/J scale (r then holds dt rhs)
    constexpr bool DT_IN_R = !MIXED && MODE != 0;
    R iJ = vg[((size_t)e2 * ESDG_NVGEO + 9) * NP + n];
    if constexpr (DT_IN_R) iJ *= a.dt;
    double r[5];
#pragma unroll
    for (int v = 0; v < 5; v++) {
      const R rv = -iJ * (S[v * NP + n] + S[(5 + v) * NP + n] + S[(10 + v) * NP + n]);
      if constexpr (MIXED) r[v] = esdg_f2d(rv);
      else r[v] = rv;
    }
    const size_t qb = (size_t)e2 * 5 * NP + n;
    if constexpr (BG == 2) {  // the moving background's own right-hand side
#pragma unroll
      for (int v = 0; v < 5; v++) r[v] += a.rhs_bgm[qb + (size_t)v * NP];
    } else if constexpr (BG) {  // the background's own momentum right-hand side
      r[1] += a.rhs_bg[((size_t)e2 * 3 + 0) * NP + n];
      r[2] += a.rhs_bg[((size_t)e2 * 3 + 1) * NP + n];
      r[3] += a.rhs_bg[((size_t)e2 * 3 + 2) * NP + n];
    }
    if (rotating) {
      const double y = a.x[((size_t)e2 * 3 + 1) * NP + n];
      double f = P.f0 + P.beta * (y - P.y0);
      if constexpr (DT_IN_R) f *= a.dt;
      // with a moving background its Coriolis force is part of its rhs
      const double my = BG == 2 ? a.q_in[qb + 2 * NP] - a.bgq[qb + 2 * NP] : a.q_in[qb + 2 * NP];
      const double mx = BG == 2 ? a.q_in[qb + NP] - a.bgq[qb + NP] : a.q_in[qb + NP];
      r[1] = fma(f, my, r[1]);
      r[2] = fma(-f, mx, r[2]);
    }
    if constexpr (MODE == 0) {
#pragma unroll
      for (int v = 0; v < 5; v++) a.rhs[qb + (size_t)v * NP] = r[v];
    } else {
      if constexpr (MIXED) {
        // handled above
      } else {
        double* dq = reinterpret_cast<double*>(a.dq);
#pragma unroll
        for (int v = 0; v < 5; v++) {
          // first stage (A = 0): the register is not read (see stage32)
          const double dv = a.rkA == 0.0 ? r[v] : fma(a.rkA, dq[qb + (size_t)v * NP], r[v]);
          dq[qb + (size_t)v * NP] = dv;
          const double qn = fma(a.rkB, dv, a.q_in[qb + (size_t)v * NP]);
          a.q_io[qb + (size_t)v * NP] = qn;
          bad |= esdg_bad_state(qn, v == 0);
        }
      }
    }
  }
  if (MODE != 0 && bad && a.status) *a.status = 1;
}

template <int N, bool MIXED, int MODE, int BG>
__global__ void __launch_bounds__(Shape<N, MIXED, BG>::THREADS)
    k_volume(EsdgGrid g, EsdgPhys P, EsdgLGL L, EsdgVolArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  volume_tile<N, MIXED, MODE, BG>(g, P, L, a, blockIdx.x * Shape<N, MIXED, BG>::EPB, smraw);
}

// Persistent batched volume kernel: CTAs stride over a device work table of
// (member, first element) tiles of meshes with the same N and precision and
// apply one LSRK stage to each (dt per member, stage coefficients per launch).
// The member descriptor of the current tile is staged in shared memory.
template <int N, bool MIXED, bool BG, int EPB_>
__global__ void __launch_bounds__(Shape<N, MIXED, BG, EPB_>::THREADS)
    k_volume_batch(const EsdgMember* __restrict__ members, const int2* __restrict__ tiles,
                   const int* __restrict__ ntiles, EsdgLGL L, double rkA, double rkB) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ EsdgMember mb;
  const int nt = *ntiles;
  for (int t = blockIdx.x; t < nt; t += gridDim.x) {
    const int2 tile = tiles[t];
    {
      const int* src = reinterpret_cast<const int*>(members + tile.x);
      int* dst = reinterpret_cast<int*>(&mb);
      for (int k = threadIdx.x; k < (int)(sizeof(EsdgMember) / sizeof(int)); k += blockDim.x)
        dst[k] = src[k];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      mb.a.rkA = rkA;
      mb.a.rkB = rkB;
    }
    __syncthreads();
    volume_tile<N, MIXED, 1, BG, EPB_>(mb.g, mb.P, L, mb.a, tile.y, smraw);
    __syncthreads();
  }
}

template <int N, bool MIXED, int MODE, int BG>
cudaError_t launch_one(const EsdgGrid& g, const EsdgPhys& P, const EsdgLGL& L,
                       const EsdgVolArgs& a, cudaStream_t s) {
  using SH = Shape<N, MIXED, BG>;
  static bool configured = false;  // one-time attribute set per instantiation
  if (!configured) {
    cudaError_t err = cudaFuncSetAttribute(k_volume<N, MIXED, MODE, BG>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)SH::SMEM);
    if (err != cudaSuccess) return err;
    configured = true;
  }
  const unsigned blocks = (unsigned)((g.E + SH::EPB - 1) / SH::EPB);
  if (blocks == 0) return cudaSuccess;
  k_volume<N, MIXED, MODE, BG><<<blocks, SH::THREADS, SH::SMEM, s>>>(g, P, L, a);
  return cudaGetLastError();
}

template <int N, bool MIXED, bool BG, int EPB_>
cudaError_t launch_batch_one(const EsdgMember* members, const int2* tiles, const int* ntiles,
                             int grid, const EsdgLGL& L, double A, double B, cudaStream_t s) {
  using SH = Shape<N, MIXED, BG, EPB_>;
  static bool configured = false;
  if (!configured) {
    cudaError_t err = cudaFuncSetAttribute(k_volume_batch<N, MIXED, BG, EPB_>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)SH::SMEM);
    if (err != cudaSuccess) return err;
    configured = true;
  }
  k_volume_batch<N, MIXED, BG, EPB_><<<grid, SH::THREADS, SH::SMEM, s>>>(members, tiles, ntiles, L,
                                                                          A, B);
  return cudaGetLastError();
}

template <int N, bool MIXED, bool BG, int EPB_>
int batch_occupancy() {
  using SH = Shape<N, MIXED, BG, EPB_>;
  int nb = 0;
  cudaFuncSetAttribute(k_volume_batch<N, MIXED, BG, EPB_>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)SH::SMEM);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_volume_batch<N, MIXED, BG, EPB_>,
                                                    SH::THREADS, SH::SMEM) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return nb > 0 ? nb : 1;
}

}  // namespace esdg_vol
